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
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr uint32_t kLbAgg = 0x40000000u;   // look-back word: aggregate of this chunk only
constexpr uint32_t kLbInc = 0x80000000u;   // look-back word: inclusive prefix up to this chunk
constexpr uint32_t kLbFlags = 0xC0000000u;
constexpr uint32_t kLbValue = 0x3FFFFFFFu;

constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanInc = 2ull << 62;
constexpr unsigned long long kScanFlags = 3ull << 62;
constexpr unsigned long long kScanValue = (1ull << 62) - 1;

template <typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int shift) {
    return (uint32_t)(k >> shift) & 0xFFu;
}

__device__ __forceinline__ uint32_t tile_of(uint32_t k) { return k; }
__device__ __forceinline__ uint32_t tile_of(unsigned long long k) { return (uint32_t)(k >> 32); }

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
__global__ void __launch_bounds__(kSortThreads) k_onesweep(SortPassArgs<KeyT> a) {
    constexpr int ITEMS = kSortItems;
    constexpr int TILE = kSortTile;
    constexpr int WARPS = kSortThreads / 32;
    __shared__ __align__(16) KeyT s_keys[TILE];
    __shared__ uint32_t s_hist[WARPS][256];
    __shared__ uint32_t s_block_start[256];
    __shared__ uint32_t s_global[256];
    __shared__ uint32_t s_digit_off[256];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk;
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys);

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
            const uint32_t c = s_hist[w][d];
            s_hist[w][d] = run;
            run += c;
        }
        const uint32_t block_cnt = run;
        {
            uint32_t tot;
            s_block_start[d] = block_exclusive_scan<uint32_t>(block_cnt, s_scan, &tot);
        }
        // Decoupled look-back over predecessor chunks for digit d.
        uint32_t* my = a.lookback + (size_t)chunk * 256 + d;
        uint32_t excl = 0;
        if (chunk == 0) {
            st_relaxed(my, kLbInc | block_cnt);
        } else {
            st_relaxed(my, kLbAgg | block_cnt);
            int j = (int)chunk - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const uint32_t v = ld_relaxed(a.lookback + (size_t)j * 256 + d);
                const uint32_t f = v & kLbFlags;
                if (f == 0) {
                    if (++spins > kSpinLimit) {
                        atomicOr(&a.status->flags, kFlagTimeout);
                        break;
                    }
                    backoff(spins);
                    continue;
                }
                excl += v & kLbValue;
                if (f == kLbInc) break;
                --j;
            }
            st_relaxed(my, kLbInc | ((excl + block_cnt) & kLbValue));
        }
        s_global[d] = s_digit_off[d] + excl;
        __syncthreads();
        // Stage keys in local sorted order.
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t dd = digit_of(key[i], a.shift);
            const uint32_t p = s_block_start[dd] + s_hist[warp][dd] + pos_local[i];
            s_keys[p] = key[i];
            pos_local[i] = p;
        }
        __syncthreads();
        uint32_t dst[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const uint32_t s = tid + k * kSortThreads;
            const KeyT kk = s_keys[s];
            const uint32_t dd = digit_of(kk, a.shift);
            const uint32_t dest = s_global[dd] + (s - s_block_start[dd]);
            dst[k] = dest;
            if (dest < count) a.keys_out[dest] = kk;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t pos = wbase + i * 32 + lane;
            uint32_t v = 0;
            if (pos < count) v = a.vals_in ? a.vals_in[pos] : pos;
            s_vals[pos_local[i]] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const uint32_t s = tid + k * kSortThreads;
            if (dst[k] < count) a.vals_out[dst[k]] = s_vals[s];
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------------------
// Fused exclusive scan of tiles-per-Gaussian + DuplicateWithKeys + key histograms.
// Chunks of kDupChunk Gaussians (in `order`), chained-scan look-back for the instance offset,
// then a load-balanced emission loop: each thread takes output slots and finds its Gaussian
// by binary search over the chunk's inclusive offsets.
// ---------------------------------------------------------------------------------------
template <bool KEY64>
__global__ void __launch_bounds__(kDupThreads) k_scan_duplicate(DupArgs a) {
    constexpr int PER = kDupChunk / kDupThreads;
    __shared__ uint32_t s_incl[kDupChunk];
    __shared__ uint32_t s_gid[kDupChunk];
    __shared__ int s_x0[kDupChunk];
    __shared__ int s_y0[kDupChunk];
    __shared__ int s_w[kDupChunk];
    __shared__ uint32_t s_hist[kMaxKeyPasses][256];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_base;

    const int tid = threadIdx.x;
    const uint32_t lt = lanemask_lt();
    uint32_t count = (uint32_t)a.n;
    if (a.count_dev) count = min(count, *a.count_dev);
    const uint32_t chunks = (count + kDupChunk - 1) / kDupChunk;
    const CamK& c = a.cam;

    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(a.chunk_counter, 1u);
        for (int k = tid; k < a.passes * 256; k += kDupThreads) (&s_hist[0][0])[k] = 0;
        __syncthreads();
        const uint32_t chunk = s_chunk;
        if (chunk >= chunks) break;

        uint32_t run = 0;
        uint32_t incl[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid * PER + k;
            const uint32_t j = chunk * kDupChunk + e;
            uint32_t tiles = 0;
            if (j < count) {
                uint32_t gid = a.order ? a.order[j] : j;
                if (gid >= (uint32_t)a.n) gid = 0;   // only reachable after a timed-out sort
                const int r = a.radius[gid];
                if (r > 0) {
                    const float4 m = a.xy[gid];
                    int x0, x1, y0, y1;
                    if (tile_rect(m, r, c, x0, x1, y0, y1)) {
                        tiles = (uint32_t)((x1 - x0) * (y1 - y0));
                        s_x0[e] = x0;
                        s_y0[e] = y0;
                        s_w[e] = x1 - x0;
                    }
                }
                s_gid[e] = gid;
            }
            run += tiles;
            incl[k] = run;
        }
        uint32_t block_total;
        const uint32_t texcl = block_exclusive_scan<uint32_t>(run, s_scan, &block_total);
#pragma unroll
        for (int k = 0; k < PER; ++k) s_incl[tid * PER + k] = texcl + incl[k];

        if (tid == 0) {
            unsigned long long* my = a.lookback + chunk;
            unsigned long long excl = 0;
            if (chunk == 0) {
                st_relaxed64(my, kScanInc | block_total);
            } else {
                st_relaxed64(my, kScanAgg | block_total);
                int j = (int)chunk - 1;
                uint32_t spins = 0;
                while (j >= 0) {
                    const unsigned long long v = ld_relaxed64(a.lookback + j);
                    const unsigned long long f = v & kScanFlags;
                    if (f == 0) {
                        if (++spins > kSpinLimit) {
                            atomicOr(&a.status->flags, kFlagTimeout);
                            break;
                        }
                        backoff(spins);
                        continue;
                    }
                    excl += v & kScanValue;
                    if (f == kScanInc) break;
                    --j;
                }
                st_relaxed64(my, kScanInc | ((excl + block_total) & kScanValue));
            }
            s_base = excl;
            if (chunk == chunks - 1) {
                const unsigned long long total = excl + block_total;
                a.status->num_instances = (uint32_t)min(total, 0xFFFFFFFFull);
                if (total > a.capacity) atomicOr(&a.status->flags, kFlagCapacity);
            }
        }
        __syncthreads();
        const unsigned long long base = s_base;

        for (uint32_t kb = 0; kb < block_total; kb += kDupThreads) {
            const uint32_t k = kb + tid;
            const bool valid = k < block_total && base + k < a.capacity;
            unsigned long long key = 0;
            if (valid) {
                // first e with s_incl[e] > k
                int lo = 0, hi = kDupChunk - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_incl[mid] > k) hi = mid;
                    else lo = mid + 1;
                }
                const int e = lo;
                const uint32_t local = k - (e > 0 ? s_incl[e - 1] : 0u);
                const int w = s_w[e];
                const int tx = s_x0[e] + (int)(local % (uint32_t)w);
                const int ty = s_y0[e] + (int)(local / (uint32_t)w);
                const uint32_t tile = (uint32_t)(ty * c.tiles_x + tx);
                const uint32_t gid = s_gid[e];
                const size_t out = (size_t)(base + k);
                if (KEY64) {
                    key = ((unsigned long long)tile << 32) | __float_as_uint(a.depth[gid]);
                    reinterpret_cast<unsigned long long*>(a.keys_out)[out] = key;
                } else {
                    key = tile;
                    reinterpret_cast<uint32_t*>(a.keys_out)[out] = tile;
                }
                a.vals_out[out] = gid;
            }
            for (int p = 0; p < a.passes; ++p) {
                const uint32_t d = valid ? (uint32_t)(key >> (8 * p)) & 0xFFu : 0x100u;
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                if (valid && (peers & lt) == 0) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        for (int k = tid; k < a.passes * 256; k += kDupThreads) {
            const uint32_t v = (&s_hist[0][0])[k];
            if (v) atomicAdd(&a.hist[k], v);
        }
        __syncthreads();
    }
}


// Zero the look-back rows of the first instance-sort pass (row count depends on the
// device-side instance count).
__global__ void k_sort_prepare(SortPrepareArgs a) {
    const uint32_t count = min((unsigned long long)a.status->num_instances, a.capacity);
    const uint32_t rows = (count + kSortTile - 1) / kSortTile;
    const size_t total = (size_t)rows * 256;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
        a.lookback[k] = 0;
}

// IdentifyTileRanges: one thread per sorted instance compares its tile id with its neighbours.
template <typename KeyT>
__global__ void k_ranges(RangesArgs<KeyT> a) {
    const uint32_t count = (uint32_t)min((unsigned long long)a.status->num_instances, a.capacity);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
        const uint32_t t = tile_of(a.keys[j]);
        if (t >= a.tiles) continue;   // only reachable after a timed-out sort
        if (j == 0 || tile_of(a.keys[j - 1]) != t) a.ranges[2 * t] = j;
        if (j + 1 == count || tile_of(a.keys[j + 1]) != t) a.ranges[2 * t + 1] = j + 1;
    }
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

cudaError_t launch_scan_duplicate(const DupArgs& a, bool key64, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (key64) {
        k_scan_duplicate<true><<<persistent_grid((const void*)k_scan_duplicate<true>, kDupThreads), kDupThreads, 0, s>>>(a);
    } else {
        k_scan_duplicate<false><<<persistent_grid((const void*)k_scan_duplicate<false>, kDupThreads), kDupThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort_prepare(const SortPrepareArgs& a, cudaStream_t s) {
    k_sort_prepare<<<persistent_grid((const void*)k_sort_prepare, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const RangesArgs<uint32_t>& a, cudaStream_t s) {
    k_ranges<uint32_t><<<persistent_grid((const void*)k_ranges<uint32_t>, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const RangesArgs<unsigned long long>& a, cudaStream_t s) {
    k_ranges<unsigned long long><<<persistent_grid((const void*)k_ranges<unsigned long long>, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gs
