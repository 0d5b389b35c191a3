// tilesort.cu -- SortByKeys and IdentifyTileRanges of Algorithm 2 (App. C) for the two-phase
// schedule, as a row-segmented tile sort.
//
// After the depth sort, the segment pass emits every visible splat's reachable tiles as one
// record per tile row it touches (row, first column, length), in depth order.  The instance
// order the paper's single sort of (tile id << 32 | depth) produces is, tile by tile, the depth
// order of the splats reaching the tile.  Here:
//   1. the records are stable-sorted by row (k_onesweep on the row bytes of the row key):
//      9M records instead of 28M instances on the 1080p frame;
//   2. k_col_count, per chunk of kColChunk row-sorted records: per-tile instance counts (a
//      difference array over the chunk's rows in shared memory, added to the frame's tile
//      counts) and, per column, the counts of the chunk's last row, published with a decoupled
//      look-back that runs inside a row (the chunk where the row starts ends it);
//   3. k_tile_scan: exclusive scan of the tile counts = the [start, end) range of every tile;
//   4. k_col_scatter, per chunk: the records' instances, expanded in rounds of kRound, ranked
//      stably by column (one ballot per digit bit, per-warp counters), staged in shared
//      memory in column order and written to start(tile) + (the row's instances of that column
//      in earlier chunks and rounds) + rank: every instance goes straight to its final slot.
// Within a tile, instances keep the record order, which is the depth order: the result is
// identical to the instance radix sort (and to the KEY64 schedule).
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr int kColThreads = 256;
constexpr int kColWarps = kColThreads / 32;
constexpr int kColPer = kColChunk / kColThreads;    // records per thread
constexpr int kColDiff = 2048;                      // tiles of one count window
constexpr int kRound = 4096;                        // instances ranked per round
constexpr int kRoundPer = kRound / kColThreads;     // instances per thread and round

__device__ __forceinline__ uint32_t rk_row(uint32_t g) { return g >> kRowKeyRowShift; }
__device__ __forceinline__ uint32_t rk_len(uint32_t g) { return (g >> 8) & 0x1FFu; }
__device__ __forceinline__ uint32_t rk_col(uint32_t g) { return g & 0xFFu; }

// Shared-memory index with one word of padding per 32: a thread's run of 8 or 16 consecutive
// entries and a warp's 32 consecutive entries are both free of bank conflicts.
__device__ __forceinline__ uint32_t pad32(uint32_t k) { return k + (k >> 5); }

// Chunks per frame from the device-side segment counts, scanned into s_base (warp 0).
template <int MAXF>
__device__ __forceinline__ uint32_t chunk_split(const Multi<ColArgs, MAXF>& m, uint32_t* s_base) {
    if (threadIdx.x < 32) {
        uint32_t c = 0;
        if ((int)threadIdx.x < m.frames) {
            const ColArgs& af = m.a[threadIdx.x];
            const uint32_t S = (uint32_t)min((unsigned long long)*af.num_segments, af.capacity);
            c = (S + kColChunk - 1) / kColChunk;
        }
        const uint32_t inc = warp_inclusive_scan<uint32_t>(c);
        if ((int)threadIdx.x < m.frames) s_base[threadIdx.x + 1] = inc;
        if (threadIdx.x == 0) s_base[0] = 0;
    }
    __syncthreads();
    return s_base[m.frames];
}

// Runs body(args) for frame f: straight from the parameter bank for a single frame, from a
// shared copy for a batch (loads through a pointer into the parameter array would be generic).
template <int MAXF, typename Body>
__device__ __forceinline__ void with_args(const Multi<ColArgs, MAXF>& m, int f, ColArgs* s_args, int* s_argf,
                                          Body&& body) {
    if constexpr (MAXF == 1) {
        body(m.a[0]);
    } else {
        if (f != *s_argf) {   // block-uniform
            __syncthreads();
            for (int k = threadIdx.x; k < (int)(sizeof(ColArgs) / 4); k += blockDim.x)
                reinterpret_cast<uint32_t*>(s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f])[k];
            __syncthreads();
            if (threadIdx.x == 0) *s_argf = f;
        }
        body(*s_args);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Per chunk of row-sorted records: tile counts, and the column counts of its last row with
// a look-back inside that row.
// ---------------------------------------------------------------------------------------
template <int MAXF>
__global__ void __launch_bounds__(kColThreads, 6) k_col_count(const __grid_constant__ Multi<ColArgs, MAXF> m) {
    __shared__ uint32_t s_diff[kColDiff + 1 + (kColDiff + 1) / 32 + 1];   // padded difference array
    __shared__ uint32_t s_base[MAXF + 1];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk, s_ra, s_rb;
    __shared__ int s_cont, s_skip;
    __shared__ __align__(16) ColArgs s_args;
    __shared__ int s_argf;
    const int tid = threadIdx.x;
    if (tid == 0) s_argf = -1;
    const uint32_t total = chunk_split(m, s_base);
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(m.a[0].chunk_counter, 1u);
        __syncthreads();
        const uint32_t g = s_chunk;
        if (g >= total) break;
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_base[f + 1] <= g) ++f;
        with_args(m, f, &s_args, &s_argf, [&](const ColArgs& a) {
            const uint32_t chunk = g - s_base[f];
            const uint32_t S = (uint32_t)min((unsigned long long)*a.num_segments, a.capacity);
            const uint32_t j0 = chunk * kColChunk;
            const uint32_t mcnt = min((uint32_t)kColChunk, S - j0);
            const uint32_t tx = (uint32_t)a.tiles_x, tiles = (uint32_t)a.tiles;
            uint32_t gk[kColPer];
#pragma unroll
            for (int i = 0; i < kColPer; ++i) {
                const uint32_t j = (uint32_t)(i * kColThreads + tid);
                gk[i] = j < mcnt ? a.geom[j0 + j] : 0xFFFFFFFFu;   // row 0x7FFF: in no window
            }
            // rows of the first and last record, and whether the previous chunk ends in the
            // first one, from the loaded records (thread 0 adds the one in front)
            if (tid == 0) {
                const uint32_t prev = chunk > 0 ? a.geom[j0 - 1] : 0xFFFFFFFFu;
                s_skip = (a.status->flags & kFlagAbort) != 0;
                s_ra = rk_row(gk[0]);
                s_cont = chunk > 0 && rk_row(prev) == rk_row(gk[0]);
            }
#pragma unroll
            for (int i = 0; i < kColPer; ++i)
                if ((uint32_t)(i * kColThreads + tid) == mcnt - 1) s_rb = rk_row(gk[i]);
            __syncthreads();
            if (s_skip) return;   // block-uniform
            const uint32_t ra = s_ra, rb = s_rb;
            const uint32_t rpw = kColDiff / tx;   // rows per window (>= 8)
            uint32_t last = 0;                    // thread c < tx: this chunk's count of (rb, c)
            for (uint32_t wr = ra; wr <= rb; wr += rpw) {   // block-uniform
                const uint32_t nrows = min(rpw, rb - wr + 1);
                const uint32_t W = nrows * tx;
                for (uint32_t k = tid; k <= W; k += kColThreads) s_diff[pad32(k)] = 0;
                __syncthreads();
#pragma unroll
                for (int i = 0; i < kColPer; ++i) {
                    const uint32_t r = rk_row(gk[i]), c = rk_col(gk[i]), len = rk_len(gk[i]);
                    if (r >= wr && r - wr < nrows && c + len <= tx) {
                        const uint32_t b = (r - wr) * tx + c;
                        atomicAdd(&s_diff[pad32(b)], 1u);
                        atomicAdd(&s_diff[pad32(b + len)], 0xFFFFFFFFu);
                    }
                }
                __syncthreads();
                // counts = inclusive prefix of the differences; thread t takes [8 t, 8 t + 8)
                constexpr int PER = kColDiff / kColThreads;
                uint32_t v[PER];
                uint32_t sum = 0;
#pragma unroll
                for (int e = 0; e < PER; ++e) {
                    const uint32_t k = (uint32_t)tid * PER + e;
                    v[e] = k < W ? s_diff[pad32(k)] : 0u;
                    sum += v[e];
                }
                uint32_t tot;
                uint32_t run = block_exclusive_scan<uint32_t>(sum, s_scan, &tot);
#pragma unroll
                for (int e = 0; e < PER; ++e) {
                    const uint32_t k = (uint32_t)tid * PER + e;
                    run += v[e];
                    if (k < W) {
                        if (run && wr * tx + k < tiles) atomicAdd(&a.tile_cnt[wr * tx + k], run);
                        s_diff[pad32(k)] = run;
                    }
                }
                __syncthreads();
                if (rb - wr < nrows && (uint32_t)tid < tx) last = s_diff[pad32((rb - wr) * tx + tid)];
                __syncthreads();
            }
            // the last row's column counts, inclusive of the row's earlier chunks
            if ((uint32_t)tid < tx) {
                uint32_t* my = a.lookback + (size_t)chunk * 256 + tid;
                if (!(s_cont && ra == rb)) {   // the row starts in this chunk
                    st_relaxed(my, kLbInc | last);
                } else {
                    st_relaxed(my, kLbAgg | last);
                    uint32_t excl = 0;
                    int j = (int)chunk - 1;
                    uint32_t spins = 0;
                    while (j >= 0) {
                        uint32_t v[kLbWindow];
#pragma unroll
                        for (int w = 0; w < kLbWindow; ++w)
                            v[w] = (j - w >= 0) ? ld_relaxed(a.lookback + (size_t)(j - w) * 256 + tid) : kLbInc;
                        int used = 0;
                        bool stop = false, wait = false;
#pragma unroll
                        for (int w = 0; w < kLbWindow; ++w) {
                            if (stop || wait) continue;
                            const uint32_t fl = v[w] & kLbFlags;
                            if (fl == 0) { wait = true; continue; }
                            excl += v[w] & kLbValue;
                            ++used;
                            if (fl == kLbInc) stop = true;
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
                    st_relaxed(my, kLbInc | ((excl + last) & kLbValue));
                }
            }
        });
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Tile ranges: one block per frame scans its tile counts; empty tiles get [0, 0).  Nothing is
// kept (all ranges empty) after a capacity overflow or a timed-out pass, or if the counts do
// not add up to the instance count.
// ---------------------------------------------------------------------------------------
template <int MAXF>
__global__ void __launch_bounds__(1024) k_tile_scan(const __grid_constant__ Multi<ColArgs, MAXF> m) {
    constexpr int PER = 4;
    __shared__ uint32_t s_scan[33];
    const ColArgs& a = m.a[blockIdx.x];
    const int tid = threadIdx.x;
    const uint32_t tiles = (uint32_t)a.tiles;
    const uint32_t K = a.status->num_instances;
    bool dead = (a.status->flags & kFlagAbort) != 0;
    uint32_t carry = 0;
    for (int pass = 0; pass < 2; ++pass) {   // the second pass clears the ranges if the total is wrong
        carry = 0;
        for (uint32_t t0 = 0; t0 < tiles; t0 += 1024 * PER) {   // block-uniform
            uint32_t v[PER], sum = 0;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const uint32_t t = t0 + (uint32_t)tid * PER + e;
                v[e] = (!dead && t < tiles) ? a.tile_cnt[t] : 0u;
                sum += v[e];
            }
            uint32_t tot;
            uint32_t run = carry + block_exclusive_scan<uint32_t>(sum, s_scan, &tot);
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const uint32_t t = t0 + (uint32_t)tid * PER + e;
                if (t < tiles)   // empty tiles get [0, 0), as in the radix schedule
                    *reinterpret_cast<uint2*>(a.ranges + 2 * t) = v[e] ? make_uint2(run, run + v[e]) : make_uint2(0u, 0u);
                run += v[e];
            }
            carry += tot;
        }
        if (dead || carry == K) break;
        dead = true;   // the tile counts do not add up to the instance count
        if (tid == 0) atomicOr(&a.status->flags, kFlagInternal);
    }
    if (tid == 0) a.status->num_segments = *a.num_segments;
}

// ---------------------------------------------------------------------------------------
// Column pass: per chunk, per run of records of one row, rounds of kRound instances.
// ---------------------------------------------------------------------------------------
// 5 blocks per SM (51 registers, 44.7 KB of shared memory each): config 3 binning 0.865 ->
// 0.854 ms against 4 blocks at 64 registers.
template <int MAXF>
__global__ void __launch_bounds__(kColThreads, 5) k_col_scatter(const __grid_constant__ Multi<ColArgs, MAXF> m) {
    __shared__ uint32_t s_offx[kColChunk + 1];        // first instance of the record in the chunk << 8 | column
    __shared__ uint16_t s_row[kColChunk];
    __shared__ uint32_t s_item[kRound + kRound / 32];  // column | record << 8 (padded), then staged Gaussians
    __shared__ uint8_t s_col[kRound];                  // column of each staged instance
    __shared__ uint32_t s_hist[kColWarps][256];
    __shared__ uint32_t s_bstart[256], s_gbase[256], s_dst[256];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk;
    __shared__ uint32_t s_base[MAXF + 1];
    __shared__ int s_skip, s_cont;
    __shared__ __align__(16) ColArgs s_args;
    __shared__ int s_argf;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    if (tid == 0) s_argf = -1;
    const uint32_t total = chunk_split(m, s_base);
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(m.a[0].chunk_counter, 1u);
        __syncthreads();
        const uint32_t g = s_chunk;
        if (g >= total) break;
        int f = 0;
        if (MAXF > 1)
            while (f + 1 < m.frames && s_base[f + 1] <= g) ++f;
        with_args(m, f, &s_args, &s_argf, [&](const ColArgs& a) {
            const uint32_t chunk = g - s_base[f];
            const uint32_t S = (uint32_t)min((unsigned long long)*a.num_segments, a.capacity);
            const uint32_t j0 = chunk * kColChunk;
            const uint32_t mcnt = min((uint32_t)kColChunk, S - j0);
            const uint32_t tx = (uint32_t)a.tiles_x, tiles = (uint32_t)a.tiles;
            const uint32_t K = (uint32_t)min((unsigned long long)a.status->num_instances, a.capacity);
            constexpr uint32_t sent = 255u;   // digit of the padding items (columns are <= 254)
            if (tid == 0) {
                s_skip = (a.status->flags & kFlagAbort) != 0;
                s_cont = chunk > 0 && rk_row(a.geom[j0 - 1]) == rk_row(a.geom[j0]);
            }
            // thread t: records [8 t, 8 t + 8) of the chunk; their first instances by a block scan
            uint32_t gk[kColPer];
            const uint32_t jt = (uint32_t)tid * kColPer;
            if (jt + kColPer <= mcnt) {
                const uint4* src = reinterpret_cast<const uint4*>(a.geom + j0 + jt);
                const uint4 x = src[0], y = src[1];
                gk[0] = x.x; gk[1] = x.y; gk[2] = x.z; gk[3] = x.w;
                gk[4] = y.x; gk[5] = y.y; gk[6] = y.z; gk[7] = y.w;
            } else {
#pragma unroll
                for (int e = 0; e < kColPer; ++e) gk[e] = jt + e < mcnt ? a.geom[j0 + jt + e] : 0u;
            }
            uint32_t sum = 0;
#pragma unroll
            for (int e = 0; e < kColPer; ++e) sum += rk_len(gk[e]);
            uint32_t tot;
            uint32_t run = block_exclusive_scan<uint32_t>(sum, s_scan, &tot);
#pragma unroll
            for (int e = 0; e < kColPer; ++e) {
                s_offx[jt + e] = run << 8 | rk_col(gk[e]);
                s_row[jt + e] = (uint16_t)rk_row(gk[e]);
                run += rk_len(gk[e]);
            }
            if (tid == kColThreads - 1) s_offx[kColChunk] = run << 8;
            __syncthreads();
            if (s_skip) return;   // block-uniform
            uint32_t ja = 0;
            while (ja < mcnt) {   // block-uniform: every thread finds the same run [ja, jb) of one row
                const uint32_t r = s_row[ja];
                uint32_t lo = ja + 1, hi = mcnt;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_row[mid] <= r) lo = mid + 1;
                    else hi = mid;
                }
                const uint32_t jb = lo;
                const uint32_t I0 = s_offx[ja] >> 8, I1 = s_offx[jb] >> 8;
                // column c's next destination: its tile's start, plus the row's instances of c
                // in earlier chunks (the inclusive count of the previous chunk, same row)
                if ((uint32_t)tid < tx) {
                    const uint32_t t = r * tx + (uint32_t)tid;
                    uint32_t b = t < tiles ? a.ranges[2 * t] : 0u;
                    if (ja == 0 && s_cont) b += a.lookback[(size_t)(chunk - 1) * 256 + tid] & kLbValue;
                    s_gbase[tid] = b;
                }
                for (uint32_t R0 = I0; R0 < I1; R0 += kRound) {   // block-uniform
                    const uint32_t n = min((uint32_t)kRound, I1 - R0);
                    for (int k = tid; k < kColWarps * 256; k += kColThreads) (&s_hist[0][0])[k] = 0;
                    // thread t expands instances [16 t, 16 t + 16) of the round: record by a
                    // search for the first, then a walk
                    {
                        const uint32_t q0 = (uint32_t)tid * kRoundPer;
                        if (q0 < n) {
                            const uint32_t q = R0 + q0;
                            uint32_t l = ja, h = jb;   // off(l) <= q < off(h)
                            while (h - l > 1) {
                                const uint32_t mid = (l + h) >> 1;
                                if ((s_offx[mid] >> 8) <= q) l = mid;
                                else h = mid;
                            }
                            uint32_t j = l;
                            uint32_t jstart = s_offx[j] >> 8, jnext = s_offx[j + 1] >> 8;
#pragma unroll 4
                            for (int i = 0; i < kRoundPer; ++i) {
                                const uint32_t qq = q0 + (uint32_t)i;
                                if (qq >= n) break;
                                const uint32_t qa = R0 + qq;
                                while (jnext <= qa) {   // ends at jb: off(jb) = I1 > qa
                                    ++j;
                                    jstart = jnext;
                                    jnext = s_offx[j + 1] >> 8;
                                }
                                const uint32_t c = (s_offx[j] & 0xFFu) + (qa - jstart);
                                s_item[pad32(qq)] = (c & 0xFFu) | (j << 8);
                            }
                        }
                    }
                    __syncthreads();
                    // rank by column: warps in order, then items, then lanes (= instance order)
                    uint32_t it[kRoundPer], pos[kRoundPer];
                    uint32_t* wh = s_hist[warp];
                    const uint32_t wbase = (uint32_t)warp * (kRound / kColWarps);
#pragma unroll
                    for (int i = 0; i < kRoundPer; ++i) {
                        pos[i] = 0;
                        it[i] = sent;
                        if (wbase + (uint32_t)i * 32 >= n) continue;   // warp-uniform
                        const uint32_t qq = wbase + (uint32_t)i * 32 + (uint32_t)lane;
                        if (qq < n) it[i] = s_item[pad32(qq)];
                        const uint32_t d = it[i] & 0xFFu;
                        uint32_t peers = 0xffffffffu;
#pragma unroll
                        for (int b = 0; b < 8; ++b) {   // all 8 bits: no branch per bit
                            const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                            peers &= ((d >> b) & 1u) ? bal : ~bal;
                        }
                        const uint32_t below = peers & lt;
                        const uint32_t prev = wh[d];
                        __syncwarp();
                        if (below == 0) wh[d] = prev + (uint32_t)__popc(peers);
                        __syncwarp();
                        pos[i] = prev + (uint32_t)__popc(below);
                    }
                    __syncthreads();
                    // per column (thread = digit): warp offsets, block start, destination base
                    {
                        const uint32_t d = (uint32_t)tid;
                        uint32_t cnt = 0;
#pragma unroll
                        for (int w = 0; w < kColWarps; ++w) {
                            const uint32_t c = s_hist[w][d];
                            s_hist[w][d] = cnt;
                            cnt += c;
                        }
                        uint32_t rt;
                        const uint32_t bs = block_exclusive_scan<uint32_t>(cnt, s_scan, &rt);
                        s_bstart[d] = bs;
                        if (d < tx) {
                            const uint32_t gb = s_gbase[d];
                            s_dst[d] = gb - bs;
                            s_gbase[d] = gb + cnt;
                        }
                    }
                    __syncthreads();
                    // stage the Gaussians in column order
#pragma unroll
                    for (int i = 0; i < kRoundPer; ++i) {
                        const uint32_t d = it[i] & 0xFFu;
                        if (d == sent) continue;
                        const uint32_t p = s_bstart[d] + s_hist[warp][d] + pos[i];
                        s_item[p] = a.gid[j0 + (it[i] >> 8)];
                        s_col[p] = (uint8_t)d;
                    }
                    __syncthreads();
                    const uint32_t rbase = r * tx;
#pragma unroll 4
                    for (uint32_t s = (uint32_t)tid; s < n; s += kColThreads) {
                        const uint32_t d = s_col[s];
                        const uint32_t dest = s_dst[d] + s;
                        if (dest < K) {
                            a.keys_out[dest] = rbase + d;
                            a.vals_out[dest] = s_item[s];
                        } else {
                            debug_fail(a.status);
                        }
                    }
                    __syncthreads();
                }
                ja = jb;
            }
        });
        __syncthreads();
    }
}

template <int MAXF>
cudaError_t launch_col_count(const Multi<ColArgs, MAXF>& m, cudaStream_t s) {
    k_col_count<MAXF><<<persistent_grid((const void*)k_col_count<MAXF>, kColThreads), kColThreads, 0, s>>>(m);
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_tile_scan(const Multi<ColArgs, MAXF>& m, cudaStream_t s) {
    k_tile_scan<MAXF><<<m.frames, 1024, 0, s>>>(m);
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_col_scatter(const Multi<ColArgs, MAXF>& m, cudaStream_t s) {
    k_col_scatter<MAXF><<<persistent_grid((const void*)k_col_scatter<MAXF>, kColThreads), kColThreads, 0, s>>>(m);
    return cudaGetLastError();
}

#define GS_INSTANTIATE_TILESORT(F)                                                          \
    template cudaError_t launch_col_count<F>(const Multi<ColArgs, F>&, cudaStream_t);     \
    template cudaError_t launch_tile_scan<F>(const Multi<ColArgs, F>&, cudaStream_t);     \
    template cudaError_t launch_col_scatter<F>(const Multi<ColArgs, F>&, cudaStream_t);

GS_INSTANTIATE_TILESORT(1)
GS_INSTANTIATE_TILESORT(kMaxFrames)

}  // namespace gs
