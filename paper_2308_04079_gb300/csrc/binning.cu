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
//   each visible Gaussian's tiles in that order, stable-sorted by tile id only: for frames up to
//   255 tile columns by the row-segmented tile sort of tilesort.cu (the segment records sorted
//   by row, the instances placed by column), otherwise by emitting the instances and sorting
//   them with byte passes over the tile id.  Within a tile, instances then appear in (depth
//   bits, Gaussian index) order, exactly the order the 64-bit sort produces.
//
// Radix sort: one kernel per digit pass in the onesweep style (Merrill & Grimshaw's radix
// sorting, single-pass with decoupled look-back): every block claims a 4096-key chunk from an
// atomic counter (chunks are claimed in order, so a block only ever waits on chunks already
// held by running blocks), ranks its keys with warp-private shared-memory digit counters and
// __match_any_sync, publishes per-digit counts, resolves its global digit offsets by looking
// back over predecessor chunks (bounded spin), stages the keys in shared memory in local sorted
// order and writes them out coalesced.  Digit histograms of every pass are computed up front
// (fused into the kernel that produces the keys).
#include <algorithm>
#include <type_traits>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanInc = 2ull << 62;
constexpr unsigned long long kScanFlags = 3ull << 62;

template <typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int shift, uint32_t mask) {
    return (uint32_t)(k >> shift) & mask;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Depth-key histograms (TWO_PHASE): key = fp32 bits of depth, culled -> 0xFFFFFFFF.
// Also zeroes the look-back rows the first depth pass uses.
// ---------------------------------------------------------------------------------------
template <int MAXF>
__global__ void __launch_bounds__(256) k_depth_hist(const __grid_constant__ Multi<DepthHistArgs, MAXF> m) {
    // frame f owns blocks [base[f], base[f + 1])
    const int f = find_frame<MAXF>(m.base, m.frames, blockIdx.x);
    const DepthHistArgs& a = m.a[f];
    const int lblock = (int)(blockIdx.x - m.base[f]), nblocks = (int)(m.base[f + 1] - m.base[f]);
    __shared__ uint32_t s_hist[4][256];
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) (&s_hist[0][0])[k] = 0;
    __syncthreads();
    __shared__ uint32_t s_vis;
    if (threadIdx.x == 0) s_vis = 0;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int stride = nblocks * blockDim.x;
    uint32_t vis_count = 0;   // per warp (lane 0); one global atomic per block at the end
    for (int base = lblock * blockDim.x; base < a.n; base += stride) {
        const int i = base + threadIdx.x;
        const bool valid = i < a.n;
        uint32_t key = 0xFFFFFFFFu;
        if (valid && a.radius[i] > 0) key = __float_as_uint(a.depth[i]);
        // the two low bytes of the depth bits are spread (plain shared atomics rarely collide);
        // the two high bytes repeat across a warp (one atomic per distinct digit)
#pragma unroll
        for (int p = 0; p < 2; ++p)
            if (valid) atomicAdd(&s_hist[p][(key >> (8 * p)) & 0xFFu], 1u);
#pragma unroll
        for (int p = 2; p < 4; ++p) {
            const uint32_t d = valid ? (key >> (8 * p)) & 0xFFu : 0x100u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && (peers & lt) == 0) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
        }
        vis_count += (uint32_t)__popc(__ballot_sync(0xffffffffu, valid && key != 0xFFFFFFFFu));
    }
    __syncthreads();
    if (lane == 0 && vis_count) atomicAdd(&s_vis, vis_count);
    __syncthreads();
    if (threadIdx.x == 0 && s_vis) atomicAdd(a.num_visible, s_vis);
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) {
        const uint32_t v = (&s_hist[0][0])[k];
        if (v) atomicAdd(&a.hist[k], v);
    }
    const int rows = (a.n + kSortTile - 1) / kSortTile;
    for (long long k = (long long)lblock * blockDim.x + threadIdx.x; k < (long long)rows * 256; k += stride)
        a.lookback_first[k] = 0;
}

// ---------------------------------------------------------------------------------------
// One LSD digit pass (8 bits at `shift`), stable.
// ---------------------------------------------------------------------------------------
template <typename KeyT, int MAXF>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(const __grid_constant__ Multi<SortPassArgs<KeyT>, MAXF> m) {
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
    __shared__ uint32_t s_base[MAXF + 1];   // chunks of frames [0, f) (device-side counts)
    __shared__ int s_frame;                 // frame whose digit offsets s_digit_off holds
    // A batch reads its frame's arguments from a shared copy: loads through a pointer into the
    // parameter array would be generic loads, repeated after every global store.
    __shared__ __align__(16) SortPassArgs<KeyT> s_args;
    __shared__ int s_argf;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    if (tid < 32) {
        uint32_t c = 0;
        if (tid < m.frames) {
            const SortPassArgs<KeyT>& af = m.a[tid];
            uint32_t cnt = af.count_host;
            if (af.count_dev) cnt = min(cnt, *af.count_dev);
            c = (cnt + TILE - 1) / TILE;
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(c);
        if (tid < m.frames) s_base[tid + 1] = inc;
        if (tid == 0) {
            s_base[0] = 0;
            s_frame = -1;
            s_argf = -1;
        }
    }
    __syncthreads();
    const uint32_t total = s_base[m.frames];
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(m.a[0].chunk_counter, 1u);
        for (int k = tid; k < WARPS * 256; k += kSortThreads) (&s_hist[0][0])[k] = 0;
        __syncthreads();
        const uint32_t g = s_chunk;
        if (g >= total) break;
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_base[f + 1] <= g) ++f;
        auto body = [&](const SortPassArgs<KeyT>& a) {
        const uint32_t chunk = g - s_base[f];
        uint32_t count = a.count_host;
        if (a.count_dev) count = min(count, *a.count_dev);
        if (f != s_frame) {   // block-uniform: global digit offsets of this frame's pass
            uint32_t tot;
            s_digit_off[tid] = block_exclusive_scan<uint32_t>(a.hist[tid], s_scan, &tot);
            if (tid == 0) s_frame = f;
        }
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
            const uint32_t d = digit_of(key[i], a.shift, a.mask);
            // lanes holding the same digit: __match_any_sync costs more the more distinct
            // digits a warp holds, one ballot per digit bit costs the same for any keys; the
            // host asks for ballots (as many as the pass's digits have bits) on passes whose
            // digits are spread (the first tile pass)
            uint32_t peers;
            if (a.ballot_rank) {
                peers = 0xffffffffu;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (b < a.ballot_rank) {
                        const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                        peers &= ((d >> b) & 1u) ? bal : ~bal;
                    }
                }
            } else {
                peers = __match_any_sync(0xffffffffu, d);
            }
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
                    if (++spins > a.spin_limit) {
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
            const uint32_t dd = digit_of(key[i], a.shift, a.mask);
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
            const uint32_t dd = digit_of(kk, a.shift, a.mask);
            const uint32_t dest = s_global[dd] + (s - s_block_start[dd]);
            if (dest < count) {
                a.keys_out[dest] = kk;
                a.vals_out[dest] = s_vals[s];
            } else if (GS_DEBUG && chunk * (uint32_t)TILE + s < count) {   // a real key: padding sorts last
                debug_fail(a.status);
            }
        }
        };
        if constexpr (MAXF == 1) {
            body(m.a[0]);
        } else {
            if (f != s_argf) {   // block-uniform
                for (int k = tid; k < (int)(sizeof(SortPassArgs<KeyT>) / 4); k += kSortThreads)
                    reinterpret_cast<uint32_t*>(&s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f])[k];
                __syncthreads();
                if (tid == 0) s_argf = f;
            }
            body(s_args);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// DuplicateWithKeys.  Per Gaussian (in `order`): the 3-sigma tile rectangle, and in each of its
// rows the interval of tiles the splat can reach (reach_row).  Pass 1 counts every entry's
// non-empty rows (segments) and tiles, pass 2 scans those pairs, pass 3 writes one record per
// segment (first instance, first tile id, Gaussian id), pass 4 (k_emit) expands the records
// into keys and values.  The two-phase schedule runs passes 1-3 as one kernel (k_segments);
// KEY64 keeps them apart, its depth digits of the four low key passes being constant per
// Gaussian: their histograms are weighted by its tile count in pass 1.
// ---------------------------------------------------------------------------------------
// Look-back words carry (segments, instances) as two 31-bit fields, each saturated at 2^30
// (above any capacity), so sums over many chunks cannot carry from one field into the other.
constexpr unsigned long long kPairSat = 1ull << 30;
constexpr unsigned long long kField = 0x7FFFFFFFull;
constexpr int kLocalShift = 40;   // block-local packing: segments << 40 | instances (no overflow
                                  // for 2048 entries of at most 2^24 tiles and 2^12 rows each)

__device__ __forceinline__ unsigned long long pair_word(unsigned long long segs, unsigned long long tiles) {
    return (min(segs, kPairSat) << 31) | min(tiles, kPairSat);
}

__device__ __forceinline__ bool tile_row(const Reach& e, int rect_only, float u, float v, int ty, int tw_log2, int th,
                                         int x0, int x1, int& txa, int& txb) {
    if (rect_only) {
        txa = x0;
        txb = x1;
        return true;
    }
    return reach_row(e, u, v, ty, tw_log2, th, x0, x1, txa, txb);
}

// Rows of one splat are handled by a group of kRowLanes lanes (lane r of the group takes rows
// r, r + kRowLanes, ...), so that a warp's lanes stay busy whatever the mix of splat heights.
// A round gives each of the warp's 32 / kRowLanes groups the splat of one owner lane.
constexpr int kRowLanes = 8;
constexpr int kGroups = 32 / kRowLanes;

// Per-splat state a group needs, broadcast from the owner lane.
struct RowJob {
    Reach e;
    float u, v;
    int x0, x1, y0, rows;
};

__device__ __forceinline__ RowJob row_job(const Reach& e, float u, float v, uint32_t rx, uint32_t ry, int src) {
    RowJob j;
    j.e.tm = __shfl_sync(0xffffffffu, e.tm, src);
    j.e.ylim = __shfl_sync(0xffffffffu, e.ylim, src);
    j.e.ystar = __shfl_sync(0xffffffffu, e.ystar, src);
    j.e.inv11 = __shfl_sync(0xffffffffu, e.inv11, src);
    j.e.l21 = __shfl_sync(0xffffffffu, e.l21, src);
    j.e.l22 = __shfl_sync(0xffffffffu, e.l22, src);
    j.e.any = j.e.tm > 0.f;
    j.u = __shfl_sync(0xffffffffu, u, src);
    j.v = __shfl_sync(0xffffffffu, v, src);
    const uint32_t x = __shfl_sync(0xffffffffu, rx, src), y = __shfl_sync(0xffffffffu, ry, src);
    j.x0 = (int)(x & 0xFFFFu);
    j.x1 = (int)(x >> 16);
    j.y0 = (int)(y & 0xFFFFu);
    j.rows = (int)(y >> 16) - j.y0;
    return j;
}

// Per-frame split of entry units (kDupThreads entries each) from device-side entry counts,
// computed by warp 0 into s_ubase; returns the total number of units.
template <int MAXF>
__device__ __forceinline__ uint32_t unit_split(const Multi<ScanArgs, MAXF>& m, uint32_t* s_ubase) {
    if (threadIdx.x < 32) {
        uint32_t units = 0;
        if ((int)threadIdx.x < m.frames) {
            const ScanArgs& af = m.a[threadIdx.x];
            uint32_t cnt = (uint32_t)af.n;
            if (af.count_dev) cnt = min(cnt, *af.count_dev);
            units = (cnt + kDupThreads - 1) / kDupThreads;
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(units);
        if ((int)threadIdx.x < m.frames) s_ubase[threadIdx.x + 1] = inc;
        if (threadIdx.x == 0) s_ubase[0] = 0;
    }
    __syncthreads();
    return s_ubase[m.frames];
}

// The splat of entry j of the (depth-ordered) list: Gaussian id, rectangle and reach state.
struct EntrySplat {
    uint32_t gid;
    float4 mean;
    uint32_t rx, ry;   // rectangle columns / rows packed lo | hi << 16 (rows 0: none)
    Reach e;
};

__device__ __forceinline__ EntrySplat load_entry(const ScanArgs& a, uint32_t j, uint32_t count) {
    EntrySplat sp;
    uint32_t gid = j < count ? (a.order ? a.order[j] : j) : 0u;
    if (gid >= (uint32_t)a.n) {   // only reachable after a timed-out sort
        debug_fail(a.status);
        gid = 0;
    }
    sp.gid = gid;
    const int rad = j < count ? a.radius[gid] : 0;
    sp.mean = a.xy[gid];
    sp.rx = sp.ry = 0;
    int x0, x1, y0, y1;
    if (rad > 0 && tile_rect(sp.mean, rad, a.cam, x0, x1, y0, y1)) {
        sp.rx = (uint32_t)x0 | ((uint32_t)x1 << 16);
        sp.ry = (uint32_t)y0 | ((uint32_t)y1 << 16);
    }
    sp.e = reach_setup(a.conic[gid], a.tau[gid]);
    return sp;
}

// DuplicateWithKeys, pass 1: per entry, the number of non-empty tile rows (segments) and of
// reachable tiles, packed (segments << 32) | tiles into pairs[j].  KEY64: histograms of the
// four depth digits, weighted by the tile counts.
template <bool KEY64, int MAXF>
__global__ void __launch_bounds__(kDupThreads) k_count_tiles(const __grid_constant__ Multi<ScanArgs, MAXF> m) {
    constexpr int ROUNDS = 32 / kGroups;
    __shared__ uint32_t s_hist[KEY64 ? 4 : 1][256];
    __shared__ uint32_t s_ubase[MAXF + 1];
    __shared__ __align__(16) ScanArgs s_args;   // batches: the frame's arguments (see k_onesweep)
    __shared__ int s_argf;
    const int tid = threadIdx.x, lane = tid & 31, sub = lane % kRowLanes, grp = lane / kRowLanes;
    if (KEY64)
        for (int k = tid; k < 4 * 256; k += kDupThreads) (&s_hist[0][0])[k] = 0;
    if (tid == 0) s_argf = -1;
    const uint32_t total = unit_split(m, s_ubase);
    int hist_f = -1;   // frame whose depth histogram s_hist accumulates (KEY64)
    auto flush = [&](int hf) {
        __syncthreads();
        const ScanArgs& ah = m.a[hf];
        for (int k = tid; k < 4 * 256; k += kDupThreads) {
            const uint32_t v = (&s_hist[0][0])[k];
            if (v) atomicAdd(&ah.hist[k], v);
            (&s_hist[0][0])[k] = 0;
        }
        __syncthreads();
    };
    for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {   // block-uniform
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_ubase[f + 1] <= u) ++f;
        if (KEY64 && f != hist_f) {
            if (hist_f >= 0) flush(hist_f);
            hist_f = f;
        }
        auto body = [&](const ScanArgs& a) {
            uint32_t count = (uint32_t)a.n;
            if (a.count_dev) count = min(count, *a.count_dev);
            const uint32_t j = (u - s_ubase[f]) * kDupThreads + tid;
            const EntrySplat sp = load_entry(a, j, count);
            const int tw_log2 = a.cam.tile_w == 16 ? 4 : 3;
            uint32_t nseg = 0, ntile = 0;
            for (int r = 0; r < ROUNDS; ++r) {
                const RowJob jb = row_job(sp.e, sp.mean.x, sp.mean.y, sp.rx, sp.ry, r * kGroups + grp);
                uint32_t sg = 0, t = 0;
                for (int base = 0; __any_sync(0xffffffffu, base < jb.rows); base += kRowLanes) {
                    int txa, txb;
                    if (base + sub < jb.rows && tile_row(jb.e, a.rect_only, jb.u, jb.v, jb.y0 + base + sub, tw_log2,
                                                         a.cam.tile_h, jb.x0, jb.x1, txa, txb)) {
                        sg += 1;
                        t += (uint32_t)(txb - txa);
                    }
                }
#pragma unroll
                for (int o = 1; o < kRowLanes; o <<= 1) {
                    sg += __shfl_xor_sync(0xffffffffu, sg, o);
                    t += __shfl_xor_sync(0xffffffffu, t, o);
                }
                // owner lane r * kGroups + q takes the totals of group q
                const int from = (lane % kGroups) * kRowLanes;
                const uint32_t ts = __shfl_sync(0xffffffffu, sg, from), tt = __shfl_sync(0xffffffffu, t, from);
                if (lane / kGroups == r) {
                    nseg = ts;
                    ntile = tt;
                }
            }
            if (j < count) a.pairs[j] = ((unsigned long long)nseg << 32) | ntile;
            if (KEY64 && ntile) {
                const uint32_t db = __float_as_uint(a.depth[sp.gid]);
#pragma unroll
                for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][(db >> (8 * p)) & 0xFFu], ntile);
            }
        };
        if constexpr (MAXF == 1) {
            body(m.a[0]);
        } else {
            if (f != s_argf) {   // block-uniform
                __syncthreads();
                for (int k = tid; k < (int)(sizeof(ScanArgs) / 4); k += kDupThreads)
                    reinterpret_cast<uint32_t*>(&s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f])[k];
                __syncthreads();
                if (tid == 0) s_argf = f;
                __syncthreads();
            }
            body(s_args);
        }
    }
    if (KEY64 && hist_f >= 0) flush(hist_f);
}

// DuplicateWithKeys, pass 2: exclusive scan of the (segments, tiles) pairs in list order,
// chunks of kPairChunk entries chained by decoupled look-back; pairs[j] becomes
// (first segment << 32) | first instance (both clamped to the capacity).  The last chunk
// records the totals, flags a capacity overflow and closes the last segment.
template <int MAXF>
__global__ void __launch_bounds__(kDupThreads) k_scan_pairs(const __grid_constant__ Multi<ScanArgs, MAXF> m) {
    constexpr int PER = kPairChunk / kDupThreads;
    __shared__ unsigned long long s_scan[33];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_base_s, s_base_t;
    __shared__ uint32_t s_fbase[MAXF + 1];   // chunks of frames [0, f)
    const int tid = threadIdx.x;
    if (tid < 32) {
        uint32_t ch = 0;
        if (tid < m.frames) {
            const ScanArgs& af = m.a[tid];
            uint32_t cnt = (uint32_t)af.n;
            if (af.count_dev) cnt = min(cnt, *af.count_dev);
            ch = (cnt + kPairChunk - 1) / kPairChunk;
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(ch);
        if (tid < m.frames) s_fbase[tid + 1] = inc;
        if (tid == 0) s_fbase[0] = 0;
    }
    __syncthreads();
    const uint32_t total = s_fbase[m.frames];
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(m.a[0].chunk_counter, 1u);
        __syncthreads();
        const uint32_t g = s_chunk;
        if (g >= total) break;
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_fbase[f + 1] <= g) ++f;
        const ScanArgs& a = m.a[f];   // a few scalar loads per chunk
        unsigned long long* const pairs = a.pairs;
        unsigned long long* const lookback = a.lookback;
        const uint32_t chunk = g - s_fbase[f];
        const uint32_t chunks = s_fbase[f + 1] - s_fbase[f];
        uint32_t count = (uint32_t)a.n;
        if (a.count_dev) count = min(count, *a.count_dev);
        const unsigned long long cap = a.capacity;
        // this thread's PER consecutive entries
        const uint32_t j0 = chunk * kPairChunk + tid * PER;
        unsigned long long v[PER];
        unsigned long long run = 0;   // block-local packing: segments << kLocalShift | tiles
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const unsigned long long p = j0 + k < count ? pairs[j0 + k] : 0ull;
            v[k] = ((p >> 32) << kLocalShift) | (p & 0xFFFFFFFFull);
            run += v[k];
        }
        unsigned long long local_total;
        const unsigned long long excl = block_exclusive_scan<unsigned long long>(run, s_scan, &local_total);
        const unsigned long long blk_s = local_total >> kLocalShift;
        const unsigned long long blk_t = local_total & ((1ull << kLocalShift) - 1);
        if (tid < 32) {
            unsigned long long* my = lookback + chunk;
            unsigned long long ex_s = 0, ex_t = 0;
            if (tid == 0) st_relaxed64(my, (chunk == 0 ? kScanInc : kScanAgg) | pair_word(blk_s, blk_t));
            if (chunk > 0) {
                int jj = (int)chunk - 1;
                uint32_t spins = 0;
                while (true) {
                    const int idx = jj - tid;
                    const unsigned long long w = idx >= 0 ? ld_relaxed64(lookback + idx) : kScanInc;
                    const unsigned long long fl = w & kScanFlags;
                    const uint32_t inc = __ballot_sync(0xffffffffu, fl == kScanInc);
                    const uint32_t zero = __ballot_sync(0xffffffffu, fl == 0);
                    const int first_inc = inc ? __ffs(inc) - 1 : 32;
                    const uint32_t upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
                    if (zero & upto) {   // a predecessor in front of the first prefix is not ready
                        if (++spins > a.spin_limit) {
                            if (tid == 0) atomicOr(&a.status->flags, kFlagTimeout);
                            break;
                        }
                        backoff(spins);
                        continue;
                    }
                    const bool use = tid <= first_inc;
                    unsigned long long ps = use ? ((w >> 31) & kField) : 0ull;
                    unsigned long long pt = use ? (w & kField) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        ps += __shfl_xor_sync(0xffffffffu, ps, o);
                        pt += __shfl_xor_sync(0xffffffffu, pt, o);
                    }
                    ex_s = min(ex_s + ps, kPairSat);
                    ex_t = min(ex_t + pt, kPairSat);
                    if (first_inc < 32) break;
                    jj -= 32;
                }
                if (tid == 0) st_relaxed64(my, kScanInc | pair_word(ex_s + blk_s, ex_t + blk_t));
            }
            if (tid == 0) {
                s_base_s = ex_s;
                s_base_t = ex_t;
                if (chunk == chunks - 1) {
                    const unsigned long long segs = min(ex_s + blk_s, kPairSat);
                    const unsigned long long tiles = min(ex_t + blk_t, kPairSat);
                    a.status->num_instances = (uint32_t)tiles;
                    *a.num_segments = (uint32_t)segs;
                    if (tiles > cap) atomicOr(&a.status->flags, kFlagCapacity);
                    else a.seg_off[segs] = (uint32_t)tiles;   // end of the last segment
                }
            }
        }
        __syncthreads();
        unsigned long long ss = s_base_s + (excl >> kLocalShift);
        unsigned long long st = s_base_t + (excl & ((1ull << kLocalShift) - 1));
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (j0 + k < count) pairs[j0 + k] = (min(ss, cap) << 32) | min(st, cap);
            ss += v[k] >> kLocalShift;
            st += v[k] & ((1ull << kLocalShift) - 1);
        }
    }
}

// DuplicateWithKeys, pass 3: per entry, the segment records (first instance, first tile,
// Gaussian) of its non-empty rows in row order.
template <int MAXF>
__global__ void __launch_bounds__(kDupThreads) k_write_segments(const __grid_constant__ Multi<ScanArgs, MAXF> m) {
    constexpr int ROUNDS = 32 / kGroups;
    __shared__ uint32_t s_ubase[MAXF + 1];
    __shared__ __align__(16) ScanArgs s_args;
    __shared__ int s_argf;
    const int tid = threadIdx.x, lane = tid & 31, sub = lane % kRowLanes, grp = lane / kRowLanes;
    if (tid == 0) s_argf = -1;
    const uint32_t total = unit_split(m, s_ubase);
    for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {   // block-uniform
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_ubase[f + 1] <= u) ++f;
        auto body = [&](const ScanArgs& a) {
            uint32_t count = (uint32_t)a.n;
            if (a.count_dev) count = min(count, *a.count_dev);
            const uint32_t j = (u - s_ubase[f]) * kDupThreads + tid;
            const EntrySplat sp = load_entry(a, j, count);
            const unsigned long long base_pair = j < count ? a.pairs[j] : 0ull;
            const uint32_t seg0 = (uint32_t)(base_pair >> 32), off0 = (uint32_t)base_pair;
            const int tw_log2 = a.cam.tile_w == 16 ? 4 : 3;
            const uint32_t cap32 = (uint32_t)a.capacity;
            for (int r = 0; r < ROUNDS; ++r) {
                const int src = r * kGroups + grp;
                const RowJob jb = row_job(sp.e, sp.mean.x, sp.mean.y, sp.rx, sp.ry, src);
                const uint32_t gs0 = __shfl_sync(0xffffffffu, seg0, src);
                const uint32_t go0 = __shfl_sync(0xffffffffu, off0, src);
                const uint32_t sgid = __shfl_sync(0xffffffffu, sp.gid, src);
                uint32_t cs = 0, ct = 0;   // segments / tiles of the rows before this pass
                for (int base = 0; __any_sync(0xffffffffu, base < jb.rows); base += kRowLanes) {
                    const int ty = jb.y0 + base + sub;
                    int txa = 0, txb = 0;
                    const bool ok = base + sub < jb.rows && tile_row(jb.e, a.rect_only, jb.u, jb.v, ty, tw_log2,
                                                                     a.cam.tile_h, jb.x0, jb.x1, txa, txb);
                    const uint32_t len = ok ? (uint32_t)(txb - txa) : 0u;
                    uint32_t is = ok ? 1u : 0u, it = len;   // inclusive scans over the group's lanes
#pragma unroll
                    for (int d = 1; d < kRowLanes; d <<= 1) {
                        const uint32_t ns = __shfl_up_sync(0xffffffffu, is, d, kRowLanes);
                        const uint32_t nt = __shfl_up_sync(0xffffffffu, it, d, kRowLanes);
                        if (sub >= d) {
                            is += ns;
                            it += nt;
                        }
                    }
                    if (ok) {
                        const uint32_t seg = gs0 + cs + is - 1u;
                        if (seg < cap32) {
                            a.seg_off[seg] = min(go0 + ct + it - len, cap32);
                            a.seg_tile[seg] = (uint32_t)(ty * a.cam.tiles_x + txa);
                            a.seg_gid[seg] = sgid;
                        }
                    }
                    cs += __shfl_sync(0xffffffffu, is, kRowLanes - 1, kRowLanes);
                    ct += __shfl_sync(0xffffffffu, it, kRowLanes - 1, kRowLanes);
                }
            }
        };
        if constexpr (MAXF == 1) {
            body(m.a[0]);
        } else {
            if (f != s_argf) {   // block-uniform
                __syncthreads();
                for (int k = tid; k < (int)(sizeof(ScanArgs) / 4); k += kDupThreads)
                    reinterpret_cast<uint32_t*>(&s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f])[k];
                __syncthreads();
                if (tid == 0) s_argf = f;
                __syncthreads();
            }
            body(s_args);
        }
    }
}

// ---------------------------------------------------------------------------------------
// DuplicateWithKeys passes 1-3 in one kernel (the two-phase schedule).  A chunk of kDupThreads
// depth-ordered entries is claimed in order; the tile rows of its splats' rectangles are
// numbered in entry order and each thread evaluates one contiguous run of ceil(rows / 256)
// of them (so large and small splats load the block evenly; the thread finds the entry of its
// first row by a search and walks forward), keeping (first tile column, length) of the first
// kSegRowCap rows in shared memory; the block scan of the runs' (segments, instances) gives
// the chunk's totals and every run's offset in the chunk, a decoupled look-back over the
// predecessors (bounded spin) the chunk's global offsets, and each thread then writes the
// records of its run's non-empty rows in order (one block scan per chunk instead of one per
// 256 rows: config 3 binning 0.853 -> 0.830 ms).  Rows past kSegRowCap (chunks of very large
// splats) are evaluated a second time when their records are written.  For the row-segmented tile sort (row_passes > 0)
// the record is (row key, Gaussian) and the pass also counts the row digits the row passes
// sort on, in shared memory, added to the frame's histograms when the block leaves it.
// ---------------------------------------------------------------------------------------
constexpr int kSegRowCap = 4096;

template <int MAXF>
__global__ void __launch_bounds__(kDupThreads) k_segments(const __grid_constant__ Multi<ScanArgs, MAXF> m) {
    __shared__ uint32_t s_rowpre[kDupThreads + 1];   // first row of every entry's splat; [256] = rows
    __shared__ float s_rf[8][kDupThreads];           // per entry: reach state (6), screen mean (u, v)
    __shared__ uint32_t s_x01[kDupThreads], s_y0[kDupThreads], s_gid[kDupThreads];
    __shared__ uint32_t s_row[kSegRowCap];           // per row: first tile column | length << 16
    __shared__ unsigned long long s_scan[33];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_base_s, s_base_t;
    __shared__ uint32_t s_fbase[MAXF + 1];           // chunks of frames [0, f)
    __shared__ __align__(16) ScanArgs s_args;
    __shared__ int s_argf;
    __shared__ uint32_t s_rh[2][256];                // row-digit histograms (row-key records)
    const int tid = threadIdx.x;
    s_rh[0][tid] = 0;
    s_rh[1][tid] = 0;
    int rh_f = -1;                                   // frame whose row histograms s_rh holds
    auto flush_rows = [&](int hf) {                  // block-uniform
        __syncthreads();
        const ScanArgs& ah = m.a[hf];
        for (int p = 0; p < ah.row_passes; ++p) {
            const uint32_t v = s_rh[p][tid];
            if (v) atomicAdd(&ah.hist[p * 256 + tid], v);
        }
        s_rh[0][tid] = 0;
        s_rh[1][tid] = 0;
        __syncthreads();
    };
    if (tid < 32) {
        uint32_t ch = 0;
        if (tid < m.frames) {
            const ScanArgs& af = m.a[tid];
            uint32_t cnt = (uint32_t)af.n;
            if (af.count_dev) cnt = min(cnt, *af.count_dev);
            ch = (cnt + kDupThreads - 1) / kDupThreads;
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(ch);
        if (tid < m.frames) s_fbase[tid + 1] = inc;
        if (tid == 0) {
            s_fbase[0] = 0;
            s_argf = -1;
        }
    }
    __syncthreads();
    const uint32_t total = s_fbase[m.frames];
    constexpr unsigned long long kOne = 1ull << kLocalShift;   // one segment in the packed pair
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(m.a[0].chunk_counter, 1u);
        __syncthreads();
        const uint32_t g = s_chunk;
        if (g >= total) break;
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_fbase[f + 1] <= g) ++f;
        if (f != rh_f) {   // block-uniform: chunks are claimed in frame order
            if (rh_f >= 0) flush_rows(rh_f);
            rh_f = f;
        }
        auto body = [&](const ScanArgs& a) {
            uint32_t count = (uint32_t)a.n;
            if (a.count_dev) count = min(count, *a.count_dev);
            const uint32_t chunk = g - s_fbase[f];
            const uint32_t chunks = s_fbase[f + 1] - s_fbase[f];
            const unsigned long long cap = a.capacity;
            const int tw_log2 = a.cam.tile_w == 16 ? 4 : 3;
            const uint32_t tiles_x = (uint32_t)a.cam.tiles_x;

            // this thread's entry: splat state and rectangle rows
            {
                const EntrySplat sp = load_entry(a, chunk * kDupThreads + tid, count);
                s_rf[0][tid] = sp.e.tm;
                s_rf[1][tid] = sp.e.ylim;
                s_rf[2][tid] = sp.e.ystar;
                s_rf[3][tid] = sp.e.inv11;
                s_rf[4][tid] = sp.e.l21;
                s_rf[5][tid] = sp.e.l22;
                s_rf[6][tid] = sp.mean.x;
                s_rf[7][tid] = sp.mean.y;
                s_x01[tid] = sp.rx;
                s_y0[tid] = sp.ry & 0xFFFFu;
                s_gid[tid] = sp.gid;
                const uint32_t rows = (sp.ry >> 16) - (sp.ry & 0xFFFFu);   // 0 when culled
                unsigned long long tr;
                const unsigned long long ex = block_exclusive_scan<unsigned long long>(rows, s_scan, &tr);
                s_rowpre[tid] = (uint32_t)ex;
                if (tid == 0) s_rowpre[kDupThreads] = (uint32_t)tr;
            }
            __syncthreads();
            const uint32_t TR = s_rowpre[kDupThreads];
            // row fr of the chunk: its entry (the last whose first row is <= fr) and tile columns
            auto find_entry = [&](uint32_t fr) -> int {   // the last entry whose first row is <= fr
                int e = 0;
#pragma unroll
                for (int step = kDupThreads / 2; step > 0; step >>= 1)
                    if (s_rowpre[e + step] <= fr) e += step;
                return e;
            };
            auto eval_row = [&](uint32_t fr, int& e, int& ty, int& txa, int& txb) -> bool {
                Reach r;
                r.tm = s_rf[0][e];
                r.ylim = s_rf[1][e];
                r.ystar = s_rf[2][e];
                r.inv11 = s_rf[3][e];
                r.l21 = s_rf[4][e];
                r.l22 = s_rf[5][e];
                r.any = r.tm > 0.f;
                const uint32_t x01 = s_x01[e];
                ty = (int)s_y0[e] + (int)(fr - s_rowpre[e]);
                return tile_row(r, a.rect_only, s_rf[6][e], s_rf[7][e], ty, tw_log2, a.cam.tile_h,
                                (int)(x01 & 0xFFFFu), (int)(x01 >> 16), txa, txb);
            };

            // rows in contiguous runs, one run per thread; the chunk's (segments, instances)
            const uint32_t per = (TR + kDupThreads - 1) / kDupThreads;
            const uint32_t r0 = min(TR, (uint32_t)tid * per), r1 = min(TR, r0 + per);
            unsigned long long mine = 0;
            int ew = r0 < r1 ? find_entry(r0) : 0;   // entry of row fr, walked forward
#pragma unroll 2
            for (uint32_t fr = r0; fr < r1; ++fr) {
                while (s_rowpre[ew + 1] <= fr) ++ew;
                int e = ew, ty, txa = 0, txb = 0;
                const bool ok = eval_row(fr, e, ty, txa, txb);
                const uint32_t len = ok ? (uint32_t)(txb - txa) : 0u;
                if (fr < (uint32_t)kSegRowCap) s_row[fr] = ok ? ((uint32_t)txa | (len << 16)) : 0u;
                if (ok) mine += kOne | len;
            }
            unsigned long long local_total;
            const unsigned long long run_ex = block_exclusive_scan<unsigned long long>(mine, s_scan, &local_total);
            const unsigned long long blk_s = local_total >> kLocalShift;
            const unsigned long long blk_t = local_total & (kOne - 1);

            // global base of the chunk: decoupled look-back
            if (tid < 32) {
                unsigned long long* const lookback = a.lookback;
                unsigned long long* my = lookback + chunk;
                unsigned long long ex_s = 0, ex_t = 0;
                if (tid == 0) st_relaxed64(my, (chunk == 0 ? kScanInc : kScanAgg) | pair_word(blk_s, blk_t));
                if (chunk > 0) {
                    int jj = (int)chunk - 1;
                    uint32_t spins = 0;
                    while (true) {
                        const int idx = jj - tid;
                        const unsigned long long w = idx >= 0 ? ld_relaxed64(lookback + idx) : kScanInc;
                        const unsigned long long fl = w & kScanFlags;
                        const uint32_t inc = __ballot_sync(0xffffffffu, fl == kScanInc);
                        const uint32_t zero = __ballot_sync(0xffffffffu, fl == 0);
                        const int first_inc = inc ? __ffs(inc) - 1 : 32;
                        const uint32_t upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
                        if (zero & upto) {   // a predecessor in front of the first prefix is not ready
                            if (++spins > a.spin_limit) {
                                if (tid == 0) atomicOr(&a.status->flags, kFlagTimeout);
                                break;
                            }
                            backoff(spins);
                            continue;
                        }
                        const bool use = tid <= first_inc;
                        unsigned long long ps = use ? ((w >> 31) & kField) : 0ull;
                        unsigned long long pt = use ? (w & kField) : 0ull;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            ps += __shfl_xor_sync(0xffffffffu, ps, o);
                            pt += __shfl_xor_sync(0xffffffffu, pt, o);
                        }
                        ex_s = min(ex_s + ps, kPairSat);
                        ex_t = min(ex_t + pt, kPairSat);
                        if (first_inc < 32) break;
                        jj -= 32;
                    }
                    if (tid == 0) st_relaxed64(my, kScanInc | pair_word(ex_s + blk_s, ex_t + blk_t));
                }
                if (tid == 0) {
                    s_base_s = ex_s;
                    s_base_t = ex_t;
                    if (chunk == chunks - 1) {
                        const unsigned long long segs = min(ex_s + blk_s, kPairSat);
                        const unsigned long long tiles = min(ex_t + blk_t, kPairSat);
                        a.status->num_instances = (uint32_t)tiles;
                        *a.num_segments = (uint32_t)segs;
                        if (tiles > cap) atomicOr(&a.status->flags, kFlagCapacity);
                        else if (!a.row_passes) a.seg_off[segs] = (uint32_t)tiles;   // end of the last segment
                    }
                }
            }
            __syncthreads();
            const unsigned long long base_s = s_base_s, base_t = s_base_t;

            // segment records: each thread numbers the non-empty rows of its run from the run's
            // exclusive prefix (the runs are in row order, so the records are too)
            unsigned long long at = run_ex;
            ew = r0 < r1 ? find_entry(r0) : 0;
#pragma unroll 2
            for (uint32_t fr = r0; fr < r1; ++fr) {
                while (s_rowpre[ew + 1] <= fr) ++ew;
                int e = ew, ty = 0, txa = 0;
                uint32_t len = 0;
                {
                    if (fr < (uint32_t)kSegRowCap) {
                        const uint32_t w = s_row[fr];
                        len = w >> 16;
                        if (len) {
                            ty = (int)s_y0[e] + (int)(fr - s_rowpre[e]);
                            txa = (int)(w & 0xFFFFu);
                        }
                    } else {
                        int txb = 0;
                        if (eval_row(fr, e, ty, txa, txb)) len = (uint32_t)(txb - txa);
                    }
                }
                if (len) {
                    const unsigned long long seg = base_s + (at >> kLocalShift);
                    const unsigned long long off = base_t + (at & (kOne - 1));
                    at += kOne | len;
                    if (seg < cap) {
                        if (a.row_passes) {
                            a.seg_tile[seg] = row_key((uint32_t)ty, len, (uint32_t)txa);
                            atomicAdd(&s_rh[0][ty & 0xFF], 1u);
                            if (a.row_passes > 1) atomicAdd(&s_rh[1][(ty >> 8) & 0xFF], 1u);
                        } else {
                            a.seg_off[seg] = (uint32_t)min(off, cap);
                            a.seg_tile[seg] = (uint32_t)ty * tiles_x + (uint32_t)txa;
                        }
                        a.seg_gid[seg] = s_gid[e];
                    }
                }
            }
        };
        if constexpr (MAXF == 1) {
            body(m.a[0]);
        } else {
            if (f != s_argf) {   // block-uniform
                for (int k = tid; k < (int)(sizeof(ScanArgs) / 4); k += kDupThreads)
                    reinterpret_cast<uint32_t*>(&s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f])[k];
                __syncthreads();
                if (tid == 0) s_argf = f;
            }
            body(s_args);
        }
        __syncthreads();   // shared state is rewritten by the next chunk
    }
    if (rh_f >= 0) flush_rows(rh_f);
}

// ---------------------------------------------------------------------------------------
// DuplicateWithKeys, pass 4: a warp takes 32 consecutive segment records, whose outputs form
// one contiguous run; every lane finds the segment of each output position it writes by a
// 5-step search over the lanes' segment ends, so keys and values are written coalesced.  A
// block takes 256 records (one frame per block unit); the digit histograms of the tile-id
// radix passes (tile_digit_bits bits each) are accumulated in shared memory on the way.  Nothing is written after a
// capacity overflow or a timed-out scan.
// ---------------------------------------------------------------------------------------
template <bool KEY64, int MAXF>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const __grid_constant__ Multi<EmitArgs, MAXF> m) {
    using KeyT = typename std::conditional<KEY64, unsigned long long, uint32_t>::type;
    constexpr int UNIT = kEmitThreads;   // segment records per block unit
    __shared__ uint32_t s_ubase[MAXF + 1];   // block units of frames [0, f)
    __shared__ uint32_t s_hist[kMaxTilePasses][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 32) {
        uint32_t units = 0;
        if (tid < m.frames) {
            const EmitArgs& af = m.a[tid];
            const uint32_t S = *af.num_segments;
            if (blockIdx.x == 0) af.status->num_segments = S;
            // nothing is emitted for a frame after a capacity overflow or a timed-out scan
            if (!(af.status->flags & kFlagAbort)) units = (S + UNIT - 1) / UNIT;
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(units);
        if (tid < m.frames) s_ubase[tid + 1] = inc;
        if (tid == 0) s_ubase[0] = 0;
    }
    for (int k = tid; k < kMaxTilePasses * 256; k += kEmitThreads) (&s_hist[0][0])[k] = 0;
    __syncthreads();
    const uint32_t total = s_ubase[m.frames];
    int hist_f = -1;   // frame whose histograms s_hist accumulates
    auto flush = [&](int hf) {
        __syncthreads();
        const EmitArgs& ah = m.a[hf];
        for (int k = tid; k < ah.tile_passes * 256; k += kEmitThreads) {
            const uint32_t v = (&s_hist[0][0])[k];
            if (v) atomicAdd(&ah.hist[k], v);
        }
        for (int k = tid; k < kMaxTilePasses * 256; k += kEmitThreads) (&s_hist[0][0])[k] = 0;
        __syncthreads();
    };
    for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {   // block-uniform
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_ubase[f + 1] <= u) ++f;
        if (f != hist_f) {
            if (hist_f >= 0) flush(hist_f);
            hist_f = f;
        }
        const EmitArgs& a = m.a[f];
        const uint32_t K = a.status->num_instances;
        const uint32_t S = *a.num_segments;
        const int passes = a.tile_passes;
        const int wbits = a.tile_digit_bits;
        const uint32_t dmask = (1u << wbits) - 1u;
        KeyT* const keys_out = reinterpret_cast<KeyT*>(a.keys_out);
        uint32_t* const vals_out = a.vals_out;
        const uint32_t s0 = (u - s_ubase[f]) * UNIT + warp * 32u;
        if (s0 >= S) continue;   // warp-uniform
        const uint32_t sidx = s0 + (uint32_t)lane;
        const bool valid = sidx < S;
        const uint32_t beg = valid ? a.seg_off[sidx] : K;
        const uint32_t end = valid ? a.seg_off[sidx + 1] : 0xFFFFFFFFu;   // seg_off[S] = K
        const uint32_t tile0 = valid ? a.seg_tile[sidx] : 0u;
        uint32_t gid = valid ? a.seg_gid[sidx] : 0u;
        if (gid >= (uint32_t)a.n) gid = 0;
        uint32_t dbits = 0;
        if (KEY64 && valid) dbits = __float_as_uint(a.depth[gid]);
        const uint32_t out0 = __shfl_sync(0xffffffffu, beg, 0);
        const uint32_t last_lane = min(31u, S - 1u - s0);
        const uint32_t out1 = min(__shfl_sync(0xffffffffu, end, last_lane), K);
        // digits above the lowest of the tile ids [tile0, tile0 + len): constant over runs of
        // 256^p ids, so the segment's owner adds one count per run
        if (valid && end <= K && end > beg) {
            const uint32_t t_end = tile0 + (end - beg);
            for (int p = 1; p < passes; ++p) {
                const int sh = wbits * p;
                for (uint32_t t = tile0; t < t_end;) {
                    const uint32_t run_end = min(t_end, ((t >> sh) + 1u) << sh);
                    atomicAdd(&s_hist[p][(t >> sh) & dmask], run_end - t);
                    t = run_end;
                }
            }
        }
        for (uint32_t base = out0; base < out1; base += 32u) {   // warp-uniform trip count
            const uint32_t out = base + (uint32_t)lane;
            // segment of position out: the first lane whose segment ends after it
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, end, lo + step - 1);
                if (e <= out) lo += step;
            }
            const uint32_t sb = __shfl_sync(0xffffffffu, beg, lo);
            const uint32_t tile = __shfl_sync(0xffffffffu, tile0, lo) + (out - sb);
            const uint32_t g = __shfl_sync(0xffffffffu, gid, lo);
            const uint32_t db = __shfl_sync(0xffffffffu, dbits, lo);
            if (out < out1) {
                if (KEY64) keys_out[out] = (KeyT)(((unsigned long long)tile << 32) | db);
                else keys_out[out] = (KeyT)tile;
                vals_out[out] = g;
                // lowest tile-id digit: consecutive outputs mostly hold consecutive tiles
                if (passes > 0) atomicAdd(&s_hist[0][tile & dmask], 1u);
            }
        }
    }
    if (hist_f >= 0) flush(hist_f);
}

// IdentifyTileRanges (App. C): after the sort, a tile's range starts where its id differs
// from the previous key's and ends where the next key's differs (ranges were zeroed, so empty
// tiles keep [0, 0)).
template <bool KEY64, int MAXF>
__global__ void __launch_bounds__(256) k_ranges(const __grid_constant__ Multi<RangesArgs, MAXF> m) {
    using KeyT = typename std::conditional<KEY64, unsigned long long, uint32_t>::type;
    constexpr uint32_t UNIT = 1024;   // positions per unit
    __shared__ uint32_t s_ubase[MAXF + 1];
    const int tid = threadIdx.x;
    if (tid < 32) {
        uint32_t units = 0;
        if (tid < m.frames) {
            const RangesArgs& af = m.a[tid];
            if (!(af.status->flags & kFlagAbort))
                units = (uint32_t)((min((unsigned long long)af.status->num_instances, af.capacity) + UNIT - 1) / UNIT);
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(units);
        if (tid < m.frames) s_ubase[tid + 1] = inc;
        if (tid == 0) s_ubase[0] = 0;
    }
    __syncthreads();
    const uint32_t total = s_ubase[m.frames];
    for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {   // block-uniform
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_ubase[f + 1] <= u) ++f;
        const RangesArgs& a = m.a[f];
        const uint32_t K = (uint32_t)min((unsigned long long)a.status->num_instances, a.capacity);
        const KeyT* const keys = reinterpret_cast<const KeyT*>(a.keys);
        uint32_t* const ranges = a.ranges;
        const uint32_t tiles = (uint32_t)a.tiles;
        for (uint32_t i = (u - s_ubase[f]) * UNIT + tid; i < min(K, (u - s_ubase[f] + 1) * UNIT); i += 256) {
            const uint32_t t = (uint32_t)(KEY64 ? (keys[i] >> 32) : keys[i]);
            const uint32_t tp = i > 0 ? (uint32_t)(KEY64 ? (keys[i - 1] >> 32) : keys[i - 1]) : 0xFFFFFFFFu;
            if (t != tp) {
                if (t < tiles) ranges[2 * t] = i;
                if (i > 0 && tp < tiles) ranges[2 * tp + 1] = i;
            }
            if (i + 1 == K && t < tiles) ranges[2 * t + 1] = K;
        }
    }
}

// The same for uint32 tile ids, HBM-friendly: a thread takes two quads of keys per unit, each
// with one 16-byte load, plus the key in front of the quad (an L1 hit: the neighbouring
// thread's quad).
template <int MAXF>
__global__ void __launch_bounds__(256) k_ranges32(const __grid_constant__ Multi<RangesArgs, MAXF> m) {
    constexpr uint32_t QUADS = 2;
    constexpr uint32_t UNIT = 256 * QUADS * 4;   // positions per unit
    __shared__ uint32_t s_ubase[MAXF + 1];
    const int tid = threadIdx.x;
    if (tid < 32) {
        uint32_t units = 0;
        if (tid < m.frames) {
            const RangesArgs& af = m.a[tid];
            if (!(af.status->flags & kFlagAbort))
                units = (uint32_t)((min((unsigned long long)af.status->num_instances, af.capacity) + UNIT - 1) / UNIT);
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(units);
        if (tid < m.frames) s_ubase[tid + 1] = inc;
        if (tid == 0) s_ubase[0] = 0;
    }
    __syncthreads();
    const uint32_t total = s_ubase[m.frames];
    for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {   // block-uniform
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_ubase[f + 1] <= u) ++f;
        const RangesArgs& a = m.a[f];
        const uint32_t K = (uint32_t)min((unsigned long long)a.status->num_instances, a.capacity);
        const uint32_t* const keys = reinterpret_cast<const uint32_t*>(a.keys);
        uint32_t* const ranges = a.ranges;
        const uint32_t tiles = (uint32_t)a.tiles;
        uint32_t k[QUADS][4], prev[QUADS], i0[QUADS];
#pragma unroll
        for (uint32_t h = 0; h < QUADS; ++h) {
            i0[h] = ((u - s_ubase[f]) * (UNIT / 4) + h * 256 + (uint32_t)tid) * 4;
            if (i0[h] + 4 <= K) {
                const uint4 q = reinterpret_cast<const uint4*>(keys)[i0[h] / 4];
                k[h][0] = q.x; k[h][1] = q.y; k[h][2] = q.z; k[h][3] = q.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) k[h][e] = i0[h] + e < K ? keys[i0[h] + e] : 0xFFFFFFFFu;
            }
            prev[h] = (i0[h] > 0 && i0[h] <= K) ? keys[i0[h] - 1] : 0xFFFFFFFFu;
        }
#pragma unroll
        for (uint32_t h = 0; h < QUADS; ++h) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t i = i0[h] + e;
                if (i >= K) break;
                const uint32_t t = k[h][e];
                const uint32_t tp = e == 0 ? (i > 0 ? prev[h] : 0xFFFFFFFFu) : k[h][e - 1];
                if (t != tp) {
                    if (t < tiles) ranges[2 * t] = i;
                    if (i > 0 && tp < tiles) ranges[2 * tp + 1] = i;
                }
                if (i + 1 == K && t < tiles) ranges[2 * t + 1] = K;
            }
        }
    }
}

// Zero the look-back rows of the first pass of the instance sort, or of the row sort of the
// segment records (row count depends on a device-side count).
template <int MAXF>
__global__ void k_sort_prepare(const __grid_constant__ Multi<SortPrepareArgs, MAXF> m) {
    for (int f = 0; f < m.frames; ++f) {
        const SortPrepareArgs& a = m.a[f];
        const uint32_t count =
            min((unsigned long long)(a.count_dev ? *a.count_dev : a.status->num_instances), a.capacity);
        const size_t stride = (size_t)gridDim.x * blockDim.x;
        const uint32_t rows = (count + a.tile_keys - 1) / a.tile_keys;
        const size_t total = (size_t)rows * 256;
        for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride) a.lookback[k] = 0;
        if (a.lookback2) {
            const size_t total2 = (size_t)((count + a.tile_keys2 - 1) / a.tile_keys2) * 256;
            for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total2; k += stride) a.lookback2[k] = 0;
        }
    }
}

template <int MAXF>
cudaError_t launch_depth_hist(Multi<DepthHistArgs, MAXF>& m, cudaStream_t s) {
    // blocks per frame: 8 keys per thread, at most a persistent grid each
    const int cap = persistent_grid((const void*)k_depth_hist<MAXF>, 256);
    m.base[0] = 0;
    for (int f = 0; f < m.frames; ++f) {
        const int b = std::min(std::max((m.a[f].n + 2047) / 2048, 1), cap);
        m.base[f + 1] = m.base[f] + (uint32_t)(m.a[f].n > 0 ? b : 0);
    }
    if (m.base[m.frames] == 0) return cudaSuccess;
    k_depth_hist<MAXF><<<m.base[m.frames], 256, 0, s>>>(m);
    return cudaGetLastError();
}

template <typename KeyT, int MAXF>
cudaError_t launch_onesweep(const Multi<SortPassArgs<KeyT>, MAXF>& m, int max_chunks, cudaStream_t s) {
    int grid = persistent_grid((const void*)k_onesweep<KeyT, MAXF>, kSortThreads);
    if (max_chunks > 0 && grid > max_chunks) grid = max_chunks;
    k_onesweep<KeyT, MAXF><<<grid, kSortThreads, 0, s>>>(m);
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_scan_tiles(const Multi<ScanArgs, MAXF>& m, bool key64, cudaStream_t s) {
    if (!key64) {   // the two-phase schedule: counting, scan and segment records in one pass
        k_segments<MAXF><<<persistent_grid((const void*)k_segments<MAXF>, kDupThreads), kDupThreads, 0, s>>>(m);
        return cudaGetLastError();
    }
    // KEY64: count, scan and write the segment records in three passes
    k_count_tiles<true, MAXF><<<persistent_grid((const void*)k_count_tiles<true, MAXF>, kDupThreads), kDupThreads, 0,
                                s>>>(m);
    k_scan_pairs<MAXF><<<persistent_grid((const void*)k_scan_pairs<MAXF>, kDupThreads), kDupThreads, 0, s>>>(m);
    k_write_segments<MAXF><<<persistent_grid((const void*)k_write_segments<MAXF>, kDupThreads), kDupThreads, 0, s>>>(
        m);
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_ranges(const Multi<RangesArgs, MAXF>& m, bool key64, cudaStream_t s) {
    if (key64)
        k_ranges<true, MAXF><<<persistent_grid((const void*)k_ranges<true, MAXF>, 256), 256, 0, s>>>(m);
    else
        k_ranges32<MAXF><<<persistent_grid((const void*)k_ranges32<MAXF>, 256), 256, 0, s>>>(m);
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_emit(const Multi<EmitArgs, MAXF>& m, bool key64, cudaStream_t s) {
    if (key64)
        k_emit<true, MAXF><<<persistent_grid((const void*)k_emit<true, MAXF>, kEmitThreads), kEmitThreads, 0, s>>>(m);
    else
        k_emit<false, MAXF><<<persistent_grid((const void*)k_emit<false, MAXF>, kEmitThreads), kEmitThreads, 0, s>>>(m);
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_sort_prepare(const Multi<SortPrepareArgs, MAXF>& m, cudaStream_t s) {
    k_sort_prepare<MAXF><<<persistent_grid((const void*)k_sort_prepare<MAXF>, 256), 256, 0, s>>>(m);
    return cudaGetLastError();
}

// Zeroes every frame's regions of a batch (one launch instead of one memset per region).
__global__ void __launch_bounds__(256) k_clear(const __grid_constant__ Multi<ClearArgs, kMaxFrames> m) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int f = 0; f < m.frames; ++f) {
        for (int r = 0; r < kClearRegions; ++r) {
            uint32_t* p = m.a[f].ptr[r];
            const unsigned long long w = m.a[f].words[r];
            if (!p || !w) continue;
            if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
                uint4* p4 = reinterpret_cast<uint4*>(p);
                const unsigned long long w4 = w / 4;
                for (unsigned long long k = t0; k < w4; k += stride) p4[k] = make_uint4(0u, 0u, 0u, 0u);
                for (unsigned long long k = 4 * w4 + t0; k < w; k += stride) p[k] = 0u;
            } else {
                for (unsigned long long k = t0; k < w; k += stride) p[k] = 0u;
            }
        }
    }
}

cudaError_t launch_clear(const Multi<ClearArgs, kMaxFrames>& m, cudaStream_t s) {
    unsigned long long words = 0;   // blocks for the largest region (16 bytes per thread), at most one wave
    for (int f = 0; f < m.frames; ++f)
        for (int r = 0; r < kClearRegions; ++r) words = std::max(words, m.a[f].ptr[r] ? m.a[f].words[r] : 0ull);
    const unsigned long long want = (words / 4 + 255) / 256;
    const int grid = (int)std::max(1ull, std::min(want, (unsigned long long)persistent_grid((const void*)k_clear, 256)));
    k_clear<<<grid, 256, 0, s>>>(m);
    return cudaGetLastError();
}

#define GS_INSTANTIATE_BINNING(F)                                                                           \
    template cudaError_t launch_depth_hist<F>(Multi<DepthHistArgs, F>&, cudaStream_t);                        \
    template cudaError_t launch_onesweep<uint32_t, F>(const Multi<SortPassArgs<uint32_t>, F>&, int, cudaStream_t); \
    template cudaError_t launch_onesweep<unsigned long long, F>(const Multi<SortPassArgs<unsigned long long>, F>&, \
                                                                int, cudaStream_t);                           \
    template cudaError_t launch_scan_tiles<F>(const Multi<ScanArgs, F>&, bool, cudaStream_t);                  \
    template cudaError_t launch_ranges<F>(const Multi<RangesArgs, F>&, bool, cudaStream_t);                    \
    template cudaError_t launch_emit<F>(const Multi<EmitArgs, F>&, bool, cudaStream_t);                        \
    template cudaError_t launch_sort_prepare<F>(const Multi<SortPrepareArgs, F>&, cudaStream_t);

GS_INSTANTIATE_BINNING(1)
GS_INSTANTIATE_BINNING(kMaxFrames)

}  // namespace gs
