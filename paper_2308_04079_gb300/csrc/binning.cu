// binning.cu -- DuplicateWithKeys, SortByKeys and IdentifyTileRanges of Algorithm 2 (App. C).
//
// Result (both schedules): the instance array ordered as ONE stable sort of the keys
// (tile id << 32) | fp32 bits of depth, emitted in (Gaussian index, row-major tile) order,
// plus [start, end) per tile.
//
// GS_SORT_KEY64 -- the paper's schedule: emit 64-bit keys in Gaussian order, LSD radix sort of
//   the 32 + ceil(log2 tiles) significant bits (8-bit digits), ranges by neighbour compare.
// GS_SORT_TWO_PHASE -- the same order with far fewer passes over the instances: first a stable
//   LSD sort of the N Gaussians by fp32 depth bits (culled ones keyed 0xFFFFFFFF go last), then
//   emit each visible Gaussian's tiles in that order and stable-sort the instances by tile id
//   only.  Within a tile, instances then appear in (depth bits, Gaussian index) order, exactly
//   the order the 64-bit sort produces.
//
// Radix sort: one kernel per digit pass in the onesweep style (Merrill & Grimshaw's radix
// sorting, single-pass with decoupled look-back): every block claims a 4096-key chunk from an
// atomic counter (chunks are claimed in order, so a block only ever waits on chunks already
// held by running blocks), ranks its keys with warp-private shared-memory digit counters and
// __match_any_sync, publishes per-digit counts, resolves its global digit offsets by looking
// back over predecessor chunks (bounded spin), stages the keys in shared memory in local sorted
// order and writes them out coalesced.  Digit histograms of every pass are computed up front
// (fused into the kernel that produces the keys).
#include <type_traits>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr uint32_t kLbAgg = 0x40000000u;   // look-back word: aggregate of this chunk only
constexpr uint32_t kLbInc = 0x80000000u;   // look-back word: inclusive prefix up to this chunk
constexpr uint32_t kLbFlags = 0xC0000000u;
constexpr uint32_t kLbValue = 0x3FFFFFFFu;
constexpr int kLbWindow = 8;                // predecessors read per look-back round

constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanInc = 2ull << 62;
constexpr unsigned long long kScanFlags = 3ull << 62;
constexpr unsigned long long kScanValue = (1ull << 62) - 1;

template <typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int shift) {
    return (uint32_t)(k >> shift) & 0xFFu;
}

__device__ __forceinline__ void backoff(uint32_t spins) {
    if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Depth-key histograms (TWO_PHASE): key = fp32 bits of depth, culled -> 0xFFFFFFFF.
// Also zeroes the look-back rows the first depth pass uses.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_depth_hist(DepthHistArgs a) {
    __shared__ uint32_t s_hist[4][256];
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) (&s_hist[0][0])[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const int i = base + threadIdx.x;
        const bool valid = i < a.n;
        uint32_t key = 0xFFFFFFFFu;
        if (valid && a.radius[i] > 0) key = __float_as_uint(a.depth[i]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t d = valid ? (key >> (8 * p)) & 0xFFu : 0x100u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && (peers & lt) == 0) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
        }
        const uint32_t vis = __ballot_sync(0xffffffffu, valid && key != 0xFFFFFFFFu);
        if (lane == 0 && vis) atomicAdd(a.num_visible, (uint32_t)__popc(vis));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) {
        const uint32_t v = (&s_hist[0][0])[k];
        if (v) atomicAdd(&a.hist[k], v);
    }
    const int rows = (a.n + kSortTile - 1) / kSortTile;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)rows * 256; k += stride)
        a.lookback_first[k] = 0;
}

// ---------------------------------------------------------------------------------------
// One LSD digit pass (8 bits at `shift`), stable.
// ---------------------------------------------------------------------------------------
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(SortPassArgs<KeyT> a) {
    constexpr int ITEMS = SortTile<KeyT>::items;
    constexpr int TILE = SortTile<KeyT>::keys;
    constexpr int WARPS = kSortThreads / 32;
    __shared__ __align__(16) KeyT s_keys[TILE];
    __shared__ uint32_t s_vals[TILE];
    __shared__ uint32_t s_hist[WARPS][256];
    __shared__ uint32_t s_block_start[256];
    __shared__ uint32_t s_global[256];
    __shared__ uint32_t s_digit_off[256];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    uint32_t count = a.count_host;
    if (a.count_dev) count = min(count, *a.count_dev);
    const uint32_t chunks = (count + TILE - 1) / TILE;
    {
        uint32_t tot;
        s_digit_off[tid] = block_exclusive_scan<uint32_t>(a.hist[tid], s_scan, &tot);
    }
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(a.chunk_counter, 1u);
        for (int k = tid; k < WARPS * 256; k += kSortThreads) (&s_hist[0][0])[k] = 0;
        __syncthreads();
        const uint32_t chunk = s_chunk;
        if (chunk >= chunks) break;
        if (a.lookback_next) a.lookback_next[(size_t)chunk * 256 + tid] = 0;
        const uint32_t wbase = chunk * TILE + warp * 32 * ITEMS;

        KeyT key[ITEMS];
        uint32_t pos_local[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t pos = wbase + i * 32 + lane;
            if (pos < count) {
                if (a.keys_in) {
                    key[i] = a.keys_in[pos];
                } else {
                    key[i] = (KeyT)(a.radius_src[pos] > 0 ? __float_as_uint(a.depth_src[pos]) : 0xFFFFFFFFu);
                }
            } else {
                key[i] = ~KeyT(0);
            }
        }
        // Warp-level stable ranking: lanes with equal digits are ordered by lane, items by i.
        uint32_t* wh = s_hist[warp];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t d = digit_of(key[i], a.shift);
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t below = peers & lt;
            const uint32_t prev = wh[d];
            __syncwarp();
            if (below == 0) wh[d] = prev + (uint32_t)__popc(peers);
            __syncwarp();
            pos_local[i] = prev + (uint32_t)__popc(below);
        }
        __syncthreads();
        // Per digit (thread = digit): warp offsets, block count, block-local start.
        const uint32_t d = tid;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t cnt = s_hist[w][d];
            s_hist[w][d] = run;
            run += cnt;
        }
        const uint32_t block_cnt = run;
        {
            uint32_t tot;
            s_block_start[d] = block_exclusive_scan<uint32_t>(block_cnt, s_scan, &tot);
        }
        // Decoupled look-back over predecessor chunks for digit d, kLbWindow predecessors per
        // round of loads: chunks start together, so a one-at-a-time walk would serialise the
        // first wave of blocks into a chain of dependent loads.
        uint32_t* my = a.lookback + (size_t)chunk * 256 + d;
        uint32_t excl = 0;
        if (chunk == 0) {
            st_relaxed(my, kLbInc | block_cnt);
        } else {
            st_relaxed(my, kLbAgg | block_cnt);
            int j = (int)chunk - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                uint32_t v[kLbWindow];
#pragma unroll
                for (int w = 0; w < kLbWindow; ++w)
                    v[w] = (j - w >= 0) ? ld_relaxed(a.lookback + (size_t)(j - w) * 256 + d) : kLbInc;
                int used = 0;
                bool stop = false, wait = false;
#pragma unroll
                for (int w = 0; w < kLbWindow; ++w) {
                    if (stop || wait) continue;
                    const uint32_t f = v[w] & kLbFlags;
                    if (f == 0) { wait = true; continue; }
                    excl += v[w] & kLbValue;
                    ++used;
                    if (f == kLbInc) stop = true;
                }
                if (stop) break;
                j -= used;
                if (wait) {
                    if (++spins > kSpinLimit) {
                        atomicOr(&a.status->flags, kFlagTimeout);
                        break;
                    }
                    backoff(spins);
                }
            }
            st_relaxed(my, kLbInc | ((excl + block_cnt) & kLbValue));
        }
        s_global[d] = s_digit_off[d] + excl;
        __syncthreads();
        // Stage keys and values in local sorted order.
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t dd = digit_of(key[i], a.shift);
            const uint32_t p = s_block_start[dd] + s_hist[warp][dd] + pos_local[i];
            s_keys[p] = key[i];
            const uint32_t pos = wbase + i * 32 + lane;
            uint32_t v = 0;
            if (pos < count) v = a.vals_in ? a.vals_in[pos] : pos;
            s_vals[p] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < ITEMS; ++k) {
            const uint32_t s = tid + k * kSortThreads;
            const KeyT kk = s_keys[s];
            const uint32_t dd = digit_of(kk, a.shift);
            const uint32_t dest = s_global[dd] + (s - s_block_start[dd]);
            if (dest < count) {
                a.keys_out[dest] = kk;
                a.vals_out[dest] = s_vals[s];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Scan of tiles per Gaussian (in `order`) with chained look-back.  Per Gaussian it stores the
// exclusive instance offset and the tile rectangle, and adds the rectangle's four corners to a
// 2D difference grid over the tiles (+1 at (x0, y0) and (x1, y1), -1 at (x1, y0) and (x0, y1));
// its 2D prefix sum is the number of instances of every tile, from which k_tile_ranges derives
// the tile ranges and the digit histograms of the tile-id sort passes.  In KEY64 mode the depth
// digits of the four low passes are constant per Gaussian: their histograms are weighted by the
// Gaussian's tile count here.
// ---------------------------------------------------------------------------------------
template <bool KEY64>
__global__ void __launch_bounds__(kDupThreads) k_scan_tiles(ScanArgs a) {
    constexpr int PER = kDupChunk / kDupThreads;
    __shared__ uint32_t s_hist[KEY64 ? 4 : 1][256];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x;
    uint32_t count = (uint32_t)a.n;
    if (a.count_dev) count = min(count, *a.count_dev);
    const uint32_t chunks = (count + kDupChunk - 1) / kDupChunk;
    const CamK& c = a.cam;
    const int gw = c.tiles_x + 1;

    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(a.chunk_counter, 1u);
        if (KEY64)
            for (int k = tid; k < 4 * 256; k += kDupThreads) (&s_hist[0][0])[k] = 0;
        __syncthreads();
        const uint32_t chunk = s_chunk;
        if (chunk >= chunks) break;
        uint32_t tiles[PER];
        uint32_t gids[PER];
        int rad[PER];
        float4 mean[PER];
        uint32_t run = 0;
        // gather first (independent loads in flight together), then compute
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const uint32_t j = chunk * kDupChunk + tid * PER + k;
            uint32_t gid = j < count ? (a.order ? a.order[j] : j) : 0u;
            if (gid >= (uint32_t)a.n) gid = 0;   // only reachable after a timed-out sort
            gids[k] = gid;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const uint32_t j = chunk * kDupChunk + tid * PER + k;
            rad[k] = j < count ? a.radius[gids[k]] : 0;
            mean[k] = a.xy[gids[k]];
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const uint32_t j = chunk * kDupChunk + tid * PER + k;
            tiles[k] = 0;
            uint2 rect = make_uint2(0u, 0u);
            if (j < count) {
                const uint32_t gid = gids[k];
                const int r = rad[k];
                int x0, x1, y0, y1;
                if (r > 0 && tile_rect(mean[k], r, c, x0, x1, y0, y1)) {
                    tiles[k] = (uint32_t)((x1 - x0) * (y1 - y0));
                    rect = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)(x1 - x0) | ((uint32_t)(y1 - y0) << 16));
                    atomicAdd(&a.diff[y0 * gw + x0], 1);
                    atomicAdd(&a.diff[y0 * gw + x1], -1);
                    atomicAdd(&a.diff[y1 * gw + x0], -1);
                    atomicAdd(&a.diff[y1 * gw + x1], 1);
                    if (KEY64) {
                        const uint32_t db = __float_as_uint(a.depth[gid]);
#pragma unroll
                        for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][(db >> (8 * p)) & 0xFFu], tiles[k]);
                    }
                }
                a.rect[j] = rect;
            }
            run += tiles[k];
        }
        uint32_t block_total;
        const uint32_t texcl = block_exclusive_scan<uint32_t>(run, s_scan, &block_total);
        // Decoupled look-back by warp 0, 32 predecessors per round of loads.
        if (tid < 32) {
            unsigned long long* my = a.lookback + chunk;
            unsigned long long excl = 0;
            if (tid == 0) st_relaxed64(my, (chunk == 0 ? kScanInc : kScanAgg) | block_total);
            if (chunk > 0) {
                int j = (int)chunk - 1;
                uint32_t spins = 0;
                while (true) {
                    const int idx = j - tid;
                    const unsigned long long v = idx >= 0 ? ld_relaxed64(a.lookback + idx) : kScanInc;
                    const unsigned long long f = v & kScanFlags;
                    const uint32_t inc = __ballot_sync(0xffffffffu, f == kScanInc);
                    const uint32_t zero = __ballot_sync(0xffffffffu, f == 0);
                    const int first_inc = inc ? __ffs(inc) - 1 : 32;
                    const uint32_t upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
                    if (zero & upto) {   // a predecessor in front of the first prefix is not ready
                        if (++spins > kSpinLimit) {
                            if (tid == 0) atomicOr(&a.status->flags, kFlagTimeout);
                            break;
                        }
                        backoff(spins);
                        continue;
                    }
                    unsigned long long part = (tid <= first_inc) ? (v & kScanValue) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    excl += part;
                    if (first_inc < 32) break;
                    j -= 32;
                }
                if (tid == 0) st_relaxed64(my, kScanInc | ((excl + block_total) & kScanValue));
            }
            if (tid == 0) {
                s_base = excl;
                if (chunk == chunks - 1) {
                    const unsigned long long total = excl + block_total;
                    a.status->num_instances = (uint32_t)min(total, 0xFFFFFFFFull);
                    if (total > a.capacity) atomicOr(&a.status->flags, kFlagCapacity);
                }
            }
        }
        __syncthreads();
        unsigned long long off = s_base + texcl;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const uint32_t j = chunk * kDupChunk + tid * PER + k;
            if (j < count) a.start[j] = (uint32_t)min(off, 0xFFFFFFFFull);
            off += tiles[k];
        }
        if (KEY64) {
            __syncthreads();
            for (int k = tid; k < 4 * 256; k += kDupThreads) {
                const uint32_t v = (&s_hist[0][0])[k];
                if (v) atomicAdd(&a.hist[k], v);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// IdentifyTileRanges from instance counts (one block): 2D prefix sum of the difference grid
// gives the instances of every tile; their exclusive scan in tile-id order gives [start, end)
// (clamped to the capacity), exactly the ranges of the sorted instance array.  Also adds the
// digit histograms of the tile-id radix passes (tile ids are the key bits from key_shift on).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tile_ranges(TileRangesArgs a) {
    __shared__ uint32_t s_hist[kMaxKeyPasses][256];
    __shared__ uint32_t s_scan[33];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int TX = a.tiles_x, TY = a.tiles_y, gw = TX + 1;
    for (int k = tid; k < kMaxKeyPasses * 256; k += nt) (&s_hist[0][0])[k] = 0;
    // row-wise then column-wise inclusive prefix sums, in place
    for (int y = tid; y <= TY; y += nt) {
        int run = 0;
        for (int x = 0; x <= TX; ++x) { run += a.diff[y * gw + x]; a.diff[y * gw + x] = run; }
    }
    __syncthreads();
    for (int x = tid; x <= TX; x += nt) {
        int run = 0;
        for (int y = 0; y <= TY; ++y) { run += a.diff[y * gw + x]; a.diff[y * gw + x] = run; }
    }
    __syncthreads();
    const uint32_t T = (uint32_t)(TX * TY);
    const unsigned long long cap = a.capacity;
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < T; base += (uint32_t)nt) {
        const uint32_t t = base + tid;
        uint32_t cnt = 0;
        if (t < T) cnt = (uint32_t)a.diff[(t / TX) * gw + (t % TX)];
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<uint32_t>(cnt, s_scan, &tot);
        if (t < T) {
            const unsigned long long s0 = carry + ex, s1 = s0 + cnt;
            a.ranges[2 * t] = cnt ? (uint32_t)min(s0, cap) : 0u;       // empty tiles: [0, 0)
            a.ranges[2 * t + 1] = cnt ? (uint32_t)min(s1, cap) : 0u;
            if (cnt) {
                for (int p = 0; p < a.tile_passes; ++p) {
                    const int bit = a.key_shift + 8 * p;
                    const uint32_t d = bit >= 32 ? ((uint32_t)(((unsigned long long)t << 32) >> bit) & 0xFFu)
                                                 : ((t >> bit) & 0xFFu);
                    atomicAdd(&s_hist[p][d], cnt);
                }
            }
        }
        carry += tot;
    }
    __syncthreads();
    for (int k = tid; k < a.tile_passes * 256; k += nt) {
        const uint32_t v = (&s_hist[0][0])[k];
        if (v) atomicAdd(&a.hist[k], v);
    }
}

// ---------------------------------------------------------------------------------------
// DuplicateWithKeys, load-balanced over output slots: a block writes 2048 consecutive instances.
// Each thread finds the Gaussian of its first slot by binary search over the exclusive offsets
// and walks forward; the tile of slot `local` inside a w x h rectangle is (local % w, local / w)
// (quotient from a float reciprocal, corrected by one step).  Keys and values are staged in
// shared memory and written out coalesced.
// ---------------------------------------------------------------------------------------
template <bool KEY64>
__global__ void __launch_bounds__(kEmitThreads) k_emit(EmitArgs a) {
    using KeyT = typename std::conditional<KEY64, unsigned long long, uint32_t>::type;
    constexpr int PER = kEmitSlots / kEmitThreads;
    constexpr int WIN = kEmitSlots + 1;         // offsets of the Gaussians that can own the block's slots
    __shared__ KeyT s_key[kEmitSlots];
    __shared__ uint32_t s_val[kEmitSlots];
    __shared__ uint32_t s_start[WIN];
    __shared__ uint32_t s_j0;
    const int tid = threadIdx.x;
    const unsigned long long K = min((unsigned long long)a.status->num_instances, a.capacity);
    uint32_t count = (uint32_t)a.n;
    if (a.count_dev) count = min(count, *a.count_dev);
    const int TX = a.tiles_x;
    KeyT* keys_out = reinterpret_cast<KeyT*>(a.keys_out);
    for (unsigned long long k0 = (unsigned long long)blockIdx.x * kEmitSlots; k0 < K;
         k0 += (unsigned long long)gridDim.x * kEmitSlots) {
        if (tid == 0) {
            // last j with start[j] <= k0 (one global binary search per block)
            uint32_t lo = 0, hi = count - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (a.start[mid] <= k0) lo = mid;
                else hi = mid - 1;
            }
            s_j0 = lo;
        }
        __syncthreads();
        const uint32_t j0 = s_j0;
        // Window of offsets start[j0 .. j0 + WIN - 1]; entries past the end act as +infinity.
        for (int w = tid; w < WIN; w += kEmitThreads)
            s_start[w] = (j0 + w < count) ? a.start[j0 + w] : 0xFFFFFFFFu;
        __syncthreads();
        const unsigned long long first = k0 + (unsigned long long)tid * PER;
        if (first < K) {
            // last w with s_start[w] <= first, within the window (a Gaussian owning a slot has at
            // least one tile, so the owners of the block's 2048 slots start inside the window
            // unless Gaussians without tiles sit in between)
            int lo = 0, hi = WIN - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((unsigned long long)s_start[mid] <= first) lo = mid;
                else hi = mid - 1;
            }
            uint32_t j = j0 + (uint32_t)lo;
            if (lo == WIN - 1) {   // window exhausted: continue the search in global memory
                uint32_t glo = j, ghi = count - 1;
                while (glo < ghi) {
                    const uint32_t mid = (glo + ghi + 1) >> 1;
                    if (a.start[mid] <= first) glo = mid;
                    else ghi = mid - 1;
                }
                j = glo;
            }
            uint32_t st = a.start[j];
            uint32_t nxt = (j + 1 < count) ? a.start[j + 1] : 0xFFFFFFFFu;
            uint2 rect = a.rect[j];
            uint32_t gid = a.order ? a.order[j] : j;
            if (gid >= (uint32_t)a.n) gid = 0;
            float inv_w = 1.0f / (float)(rect.y & 0xFFFFu);
            uint32_t dbits = KEY64 ? __float_as_uint(a.depth[gid]) : 0u;
#pragma unroll 4
            for (int i = 0; i < PER; ++i) {
                const unsigned long long kk = first + i;
                if (kk >= K) break;
                while ((unsigned long long)nxt <= kk) {   // advance to the Gaussian owning slot kk
                    ++j;
                    st = nxt;
                    nxt = (j + 1 < count) ? a.start[j + 1] : 0xFFFFFFFFu;
                    rect = a.rect[j];
                    gid = a.order ? a.order[j] : j;
                    if (gid >= (uint32_t)a.n) gid = 0;
                    inv_w = 1.0f / (float)(rect.y & 0xFFFFu);
                    if (KEY64) dbits = __float_as_uint(a.depth[gid]);
                }
                const int w = (int)(rect.y & 0xFFFFu);
                const int local = (int)(kk - st);
                int qy = (int)(((float)local + 0.5f) * inv_w);
                int rx = local - qy * w;
                if (rx < 0) { --qy; rx += w; }
                if (rx >= w) { ++qy; rx -= w; }
                const uint32_t tile =
                    (uint32_t)(((int)(rect.x >> 16) + qy) * TX + (int)(rect.x & 0xFFFFu) + rx);
                const int slot = tid * PER + i;
                if (KEY64) s_key[slot] = (KeyT)(((unsigned long long)tile << 32) | dbits);
                else s_key[slot] = (KeyT)tile;
                s_val[slot] = gid;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int slot = i * kEmitThreads + tid;
            const unsigned long long kk = k0 + slot;
            if (kk < K) {
                keys_out[kk] = s_key[slot];
                a.vals_out[kk] = s_val[slot];
            }
        }
        __syncthreads();
    }
}

// Zero the look-back rows of the first instance-sort pass (row count depends on the
// device-side instance count).
__global__ void k_sort_prepare(SortPrepareArgs a) {
    const uint32_t count = min((unsigned long long)a.status->num_instances, a.capacity);
    const uint32_t rows = (count + a.tile_keys - 1) / a.tile_keys;
    const size_t total = (size_t)rows * 256;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
        a.lookback[k] = 0;
}

cudaError_t launch_depth_hist(const DepthHistArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    int grid = (a.n + 255) / 256;
    const int cap = persistent_grid((const void*)k_depth_hist, 256);
    if (grid > cap) grid = cap;
    k_depth_hist<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename KeyT>
static cudaError_t launch_onesweep_t(const SortPassArgs<KeyT>& a, int max_chunks, cudaStream_t s) {
    int grid = persistent_grid((const void*)k_onesweep<KeyT>, kSortThreads);
    if (max_chunks > 0 && grid > max_chunks) grid = max_chunks;
    k_onesweep<KeyT><<<grid, kSortThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_onesweep(const SortPassArgs<uint32_t>& a, int max_chunks, cudaStream_t s) {
    return launch_onesweep_t(a, max_chunks, s);
}

cudaError_t launch_onesweep(const SortPassArgs<unsigned long long>& a, int max_chunks, cudaStream_t s) {
    return launch_onesweep_t(a, max_chunks, s);
}

cudaError_t launch_scan_tiles(const ScanArgs& a, bool key64, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (key64) k_scan_tiles<true><<<persistent_grid((const void*)k_scan_tiles<true>, kDupThreads), kDupThreads, 0, s>>>(a);
    else k_scan_tiles<false><<<persistent_grid((const void*)k_scan_tiles<false>, kDupThreads), kDupThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const TileRangesArgs& a, cudaStream_t s) {
    k_tile_ranges<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_emit(const EmitArgs& a, bool key64, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (key64) k_emit<true><<<persistent_grid((const void*)k_emit<true>, kEmitThreads), kEmitThreads, 0, s>>>(a);
    else k_emit<false><<<persistent_grid((const void*)k_emit<false>, kEmitThreads), kEmitThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sort_prepare(const SortPrepareArgs& a, cudaStream_t s) {
    k_sort_prepare<<<persistent_grid((const void*)k_sort_prepare, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gs
