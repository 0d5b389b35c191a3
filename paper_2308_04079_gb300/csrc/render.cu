// render.cu -- per-tile blending (Algorithm 2, BlendInOrder) and its backward pass (Sec. 6).
//
// One thread block per tile; TPR = 4 threads per tile row, each owning PX = tile_w / TPR pixels
// of that row (columns c, c + TPR, ...).  The block stages batches of the tile's depth-sorted Gaussians in
// shared memory; a staged splat carries its offset from the tile's first pixel centre, the
// Cholesky factor of its conic pre-scaled to log2 units, log2 of its opacity and its skip
// threshold (see Staged), so that for a pixel at offset d:
//   p = l11' dx + l21' dy, q = l22' dy, s = p^2 + q^2 = -log2(e) power,  o exp(power) = 2^(lo - s)
// and "alpha < 1/255" is the single comparison s > thr with thr = lo - log2(1/255).  Pixels of
// one row share dy, q and q^2, and p advances by TPR l11' from one owned pixel to the next, so a
// skipped (pixel, splat) pair costs three instructions and no exp.
//
// Forward (eq. front-to-back, App. C): a = min(0.99, o exp(power)); skip a < 1/255; stop before
//   T (1 - a) < 1e-4; C += a T c; T *= 1 - a.  The tile stops as soon as all its pixels are done
//   (checked once per batch with __syncthreads_count).  Writes C + T bg, T and the 1-based list
//   position of the last blended Gaussian.  The staging thread of a splat also computes, per
//   warp (a band of 8 tile rows), whether the splat can reach alpha_min anywhere in the band
//   (band_mask), and a warp skips the splats that cannot; for every 32 splats a warp ORs into
//   its contribution bits (one bit per instance of the frame) those that some pixel of the
//   warp blended.
// Backward: the tile's list is walked back to front from the largest last position in the tile,
//   each warp visiting only the splats its contribution bits name (it blends exactly the
//   forward's pairs); each pixel only processes positions below its own last position, recovers
//   T_i = T_{i+1} / (1 - a_i) from the stored final T, and keeps R . dL/dC, the projection of
//   the colour behind the current Gaussian (normalised by the transmittance in front of it; R
//   starts at bg) on the pixel's dL/dC, which is all the recurrence needs:
//     dL/dc_i = a_i T_i dL/dC,  dL/da_i = T_i (c_i - R_{i+1}) . dL/dC,  R_i = a_i c_i + (1 - a_i) R_{i+1}.
//   Through a = o G (zero when clamped), with g = Sigma'^-1 d = L (p, q) (L the Cholesky factor
//   of the conic, (p, q) = L^T d): d(power)/d(mean) = g and d(power)/d(Sigma') = g g^T / 2.  The
//   mean and Sigma' sums are kept in the whitened frame of L: sum dL/dpower (p, q) and
//   (1/2) sum dL/dpower (p, q)(p, q)^T =: K; the per-Gaussian stage maps them back with the same
//   stored L (dL/dmean2D = L (p, q) sums, dL/dSigma' = L K L^T contracted without forming it).
//   In pixel coordinates the three entries of dL/dSigma' of an elongated splat are all dominated
//   by its minor axis and their major-axis part, which the scale along the long axis needs, is
//   lost to cancellation in fp32 sums over many pixels; in the whitened frame every direction of
//   the splat has the same scale.  A thread sums its pixels' terms (mean, Sigma', opacity,
//   colour); when more than kDirectLanes (24) lanes of a warp contributed, the warp sums its
//   lanes with a transposed reduce-scatter (warp_reduce9) and nine lanes add the nine totals
//   with one atomic instruction each, otherwise every contributing lane adds its own sums (two
//   float4 atomics and one scalar).
//
// Limited-BW (cfg.grad_limit = N > 0, the ablation of Sec. 7.3): the forward pass also records
// the number of blended splats of every pixel (COUNT); the backward pass (LIMIT) keeps the
// recurrences over all of them but adds gradients only for the N front-most, i.e. it skips the
// gradient terms of the first (count - N) blended splats it meets from the back.
//
// The forward and the backward evaluate a (pixel, splat) pair with the same staging and the same
// operation sequence (stage_splat, splat_row, splat_s), so their skip and clamp decisions agree
// bit for bit.
//
// Block order: block b of a frame renders tile order[b], the frame's tiles by decreasing list
// length (k_tile_order, run at the end of the binning stage).  The work of a tile grows with its
// list and varies by a factor of several across a frame; blocks start roughly in index order, so
// in row-major order the longest tiles (the frame's centre) could start late and finish alone.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

// sqrt(log2(e) / 2): scales the Cholesky factor so that p^2 + q^2 = -log2(e) power.
constexpr float kScaleLog2 = 0.84932180028801907f;
// 1 / kScaleLog2 = sqrt(2 ln 2): scaled p, q back to the whitened frame of the unscaled factor.
constexpr float kUnscale = 1.1774100225154747f;
// (1/2) / kScaleLog2^2 = ln 2: scaled (p, q)(p, q)^T sums to K = (1/2) sum dL/dpower (p, q)(p, q)^T.
constexpr float kLn2 = 0.69314718055994531f;
// At most this many contributing lanes add their own sums instead of a warp reduction (measured
// on the 3M-Gaussian 1080p frame: 24 beats 6, 12, 16, 20 and 32).
constexpr int kDirectLanes = 24;

struct Staged {
    float4 a;   // (ox, oy, thr, lo): tile-relative offset, skip threshold, log2(opacity)
    float4 b;   // (l11', l21', l22', 1/o)
};

__device__ __forceinline__ void stage_splat(float4 m, float4 L, int x0, int y0, float log2_amin, Staged& s) {
    const float ox = tile_offset(x0, m.x, m.z);
    const float oy = tile_offset(y0, m.y, m.w);
    const float lo = __log2f(L.w);
    const float thr = __fsub_rn(lo, log2_amin);
    s.a = make_float4(ox, oy, thr, lo);
    s.b = make_float4(__fmul_rn(L.x, kScaleLog2), __fmul_rn(L.y, kScaleLog2), __fmul_rn(L.z, kScaleLog2),
                      __frcp_rn(L.w));
}

// Minimum of s = (l11 x + l21 y)^2 + (l22 y)^2 (the staged splat's scaled quadratic form) over
// the rectangle [xa, xb] x [ya, yb] of pixel-centre offsets: 0 when the splat centre is inside,
// else the smallest of the four edge minima (each a one-dimensional convex quadratic).
__device__ __forceinline__ float rect_min_s(const Staged& st, float xa, float xb, float ya, float yb) {
    const float l11 = st.b.x, l21 = st.b.y, l22 = st.b.z;
    if (xa <= 0.f && 0.f <= xb && ya <= 0.f && 0.f <= yb) return 0.f;
    const float i11 = 1.0f / l11, A = fmaf(l21, l21, l22 * l22), iA = 1.0f / A;
    auto at = [&](float x, float y) { const float p = fmaf(l11, x, l21 * y), q = l22 * y; return fmaf(p, p, q * q); };
    float m = 3.0e38f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float y = e ? yb : ya;                          // horizontal edge: x* = -l21 y / l11
        m = fminf(m, at(fminf(fmaxf(-l21 * y * i11, xa), xb), y));
        const float x = e ? xb : xa;                          // vertical edge: y* = -l11 l21 x / A
        m = fminf(m, at(x, fminf(fmaxf(-l11 * l21 * x * iA, ya), yb)));
    }
    return m;
}

// Warps of a render block (bit w) whose band of tile rows [w rows_per_warp, (w + 1) rows_per_warp)
// holds a point where the staged splat reaches alpha_min: the minimum of its quadratic form over
// the band's rectangle (continuous, so it covers every pixel centre) within a small margin of the
// threshold.  A cleared bit proves no pixel of that warp blends the splat.
__device__ __forceinline__ uint32_t band_mask(const Staged& st, int tile_w, int tile_h, int rows_per_warp) {
    const float thr = st.a.z;
    if (!(thr > 0.f)) return 0u;
    const float lim = fmaf(thr, 1.0009765625f, 0.0009765625f);   // thr (1 + 2^-10) + 2^-10
    uint32_t m = 0;
    for (int w = 0; w * rows_per_warp < tile_h; ++w) {
        const float ya = st.a.y + (float)(w * rows_per_warp), yb = ya + (float)(rows_per_warp - 1);
        if (rect_min_s(st, st.a.x, st.a.x + (float)(tile_w - 1), ya, yb) <= lim) m |= 1u << w;
    }
    return m;
}

// 32 bits of a contribution bit array ending at bit `hi` (bit 31 = bit hi, bit 0 = bit hi - 31;
// bits below 0 read as 0).
__device__ __forceinline__ uint32_t bits_window(const uint32_t* w, uint32_t hi) {
    const uint32_t word = hi >> 5, sh = hi & 31u;
    const uint32_t top = w[word] << (31u - sh);
    const uint32_t low = (sh < 31u && word > 0) ? (w[word - 1] >> (sh + 1u)) : 0u;
    return top | low;
}

// Sum over the warp of the 9 accumulators v[0..8] by a transposed reduce-scatter: each round
// halves the values a lane keeps (it sends the half its partner keeps and adds the half it
// receives), 12 shuffles instead of 45.  Afterwards the total of accumulator slot(lane) is in
// the even lanes of each pair (slot < 0: padding); see reduce_slot.
__device__ __forceinline__ float warp_reduce9(const float (&v)[9], int lane) {
    float a[5];
    const bool h16 = lane & 16;
#pragma unroll
    for (int i = 0; i < 5; ++i) {   // lanes 0-15 keep v[0..4], lanes 16-31 keep v[5..8] (+ padding)
        const float lo = v[i], hi = i < 4 ? v[5 + i] : 0.f;
        a[i] = (h16 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h16 ? lo : hi, 16);
    }
    float b[3];
    const bool h8 = lane & 8;
#pragma unroll
    for (int i = 0; i < 3; ++i) {   // keep a[0..2] or a[3..4] (+ padding)
        const float lo = a[i], hi = i < 2 ? a[3 + i] : 0.f;
        b[i] = (h8 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h8 ? lo : hi, 8);
    }
    float c[2];
    const bool h4 = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // keep b[0..1] or b[2] (+ padding)
        const float lo = b[i], hi = i < 1 ? b[2] : 0.f;
        c[i] = (h4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h4 ? lo : hi, 4);
    }
    const bool h2 = lane & 2;
    float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h2 ? c[0] : c[1], 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

// Accumulator slot whose warp total warp_reduce9 leaves in `lane` (-1: padding).
__device__ __forceinline__ int reduce_slot(int lane) {
    const int base = (lane & 16) ? 5 : 0;   // values kept after the first round
    int l3[3];
    if (lane & 8) { l3[0] = base + 3; l3[1] = base + 4; l3[2] = -1; }
    else { l3[0] = base; l3[1] = base + 1; l3[2] = base + 2; }
    int l2[2];
    if (lane & 4) { l2[0] = l3[2]; l2[1] = -1; }
    else { l2[0] = l3[0]; l2[1] = l3[1]; }
    const int slot = (lane & 2) ? l2[1] : l2[0];
    return slot > 8 ? -1 : slot;
}

// Per (thread row, splat): p at the thread's first pixel, its step to the next owned pixel
// (`step` columns to the right), q, q^2.
__device__ __forceinline__ void splat_row(const Staged& s, float lyf, float c0f, float step, float& p0, float& dp,
                                          float& q, float& qq) {
    const float dy = __fadd_rn(lyf, s.a.y);
    const float dx0 = __fadd_rn(c0f, s.a.x);
    q = __fmul_rn(s.b.z, dy);
    qq = __fmul_rn(q, q);
    p0 = __fmaf_rn(s.b.y, dy, __fmul_rn(s.b.x, dx0));
    dp = __fmul_rn(step, s.b.x);
}

// s = p^2 + q^2 at the thread's j-th pixel.
__device__ __forceinline__ float splat_s(float p0, float dp, float qq, int j, float& p) {
    p = __fmaf_rn((float)j, dp, p0);
    return __fmaf_rn(p, p, qq);
}

constexpr int kOrderThreads = 1024;
constexpr int kOrderWarps = kOrderThreads / 32;
constexpr int kOrderBuckets = 128;   // = 4 per lane of the scan warp

// Bucket of a tile's list length: four per octave (the leading bit and the two below it),
// longer lists in higher buckets; lengths below 2^30 reach bucket 120 at most.
__device__ __forceinline__ int order_bucket(uint32_t len) {
    if (len == 0) return 0;
    const int e = 31 - __clz(len);
    const uint32_t frac = e >= 2 ? (len >> (e - 2)) & 3u : (len << (2 - e)) & 3u;
    return min(kOrderBuckets - 1, 1 + 4 * e + (int)frac);
}

// One block per frame: a stable counting sort of the tiles by decreasing bucket.  Warp w takes
// a contiguous range of tiles: it counts its range per bucket (its own row of s_pos), a scan over
// buckets (in decreasing order) and warps turns the counts into first positions, and each warp
// places its range in tile order.
template <int MAXF>
__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const __grid_constant__ Multi<TileOrderArgs, MAXF> m) {
    __shared__ uint32_t s_pos[kOrderWarps][kOrderBuckets];
    __shared__ uint32_t s_tot[kOrderBuckets];
    const TileOrderArgs& a = m.a[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = a.tiles;
    const int per = ((tiles + kOrderThreads - 1) / kOrderThreads) * 32;   // tiles per warp, a multiple of 32
    const int t_lo = min(tiles, warp * per), t_hi = min(tiles, t_lo + per);
    for (int b = lane; b < kOrderBuckets; b += 32) s_pos[warp][b] = 0;
    __syncwarp();
    for (int t = t_lo + lane; t < t_hi; t += 32) atomicAdd(&s_pos[warp][order_bucket(a.ranges[2 * t + 1] - a.ranges[2 * t])], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBuckets) {
        uint32_t sum = 0;
        for (int w = 0; w < kOrderWarps; ++w) sum += s_pos[w][threadIdx.x];
        s_tot[threadIdx.x] = sum;
    }
    __syncthreads();
    if (warp == 0) {   // lane l: buckets 127 - 4l, ..., 124 - 4l
        uint32_t c[4], sum = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) { c[e] = s_tot[kOrderBuckets - 1 - 4 * lane - e]; sum += c[e]; }
        uint32_t run = warp_inclusive_scan<uint32_t>(sum) - sum;
#pragma unroll
        for (int e = 0; e < 4; ++e) { s_tot[kOrderBuckets - 1 - 4 * lane - e] = run; run += c[e]; }
    }
    __syncthreads();
    if (threadIdx.x < kOrderBuckets) {
        uint32_t run = s_tot[threadIdx.x];
        for (int w = 0; w < kOrderWarps; ++w) { const uint32_t c = s_pos[w][threadIdx.x]; s_pos[w][threadIdx.x] = run; run += c; }
    }
    __syncthreads();
    for (int t0 = t_lo; t0 < t_hi; t0 += 32) {   // warp-uniform
        const int t = t0 + lane;
        const int b = t < t_hi ? order_bucket(a.ranges[2 * t + 1] - a.ranges[2 * t]) : -1;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (b >= 0) a.order[s_pos[warp][b] + rank] = (uint32_t)t;
        __syncwarp();
        if (b >= 0 && rank == 0) s_pos[warp][b] += __popc(peers);
        __syncwarp();
    }
}

// Forward pass of the tile order[block_slot] of a frame with ntiles tiles.
template <int PX, int TPR, bool COUNT>
__device__ __forceinline__ void forward_tile(const RenderFwdArgs& a, uint32_t block_slot, uint32_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Staged* s_sp = reinterpret_cast<Staged*>(smem_raw);
    float4* s_rgb = reinterpret_cast<float4*>(smem_raw + sizeof(Staged) * a.batch);
    uint32_t* s_band = reinterpret_cast<uint32_t*>(smem_raw + (sizeof(Staged) + sizeof(float4)) * a.batch);
    const CamK& c = a.cam;
    const uint32_t tile_id = a.order[block_slot];
    if (tile_id >= ntiles) {   // an order not written by gs_bin_sort
        if (threadIdx.x == 0) debug_fail(a.status);
        return;
    }
    const int tile = (int)tile_id;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int nthreads = blockDim.x;
    const int ly = threadIdx.x / TPR, c0 = threadIdx.x % TPR;   // TPR threads per tile row
    const int x0 = tx * c.tile_w, y0 = ty * c.tile_h;
    const int py = y0 + ly;
    const float lyf = (float)ly, c0f = (float)c0;
    const int warp = threadIdx.x >> 5;
    const uint32_t start = a.ranges[2 * tile];
    uint32_t end = a.ranges[2 * tile + 1];
    if (GS_DEBUG && (end < start || end > a.capacity)) {   // a range outside the instance lists
        if (threadIdx.x == 0) debug_fail(a.status);
        end = start;
    }
    const int lane = threadIdx.x & 31;
    uint32_t* const wbits = a.contrib + (size_t)(threadIdx.x >> 5) * a.contrib_words;
    const float amax = a.cfg.alpha_max, tmin = a.cfg.T_min;
    const float log2_amin = __log2f(a.cfg.alpha_min);
    // what the loops read, in registers
    const int batch = a.batch, n = a.n, tile_w = c.tile_w, tile_h = c.tile_h;
    const uint32_t* const vals = a.vals;
    const float4* const xy = a.xy;
    const float4* const conic = a.conic_opacity;
    const float4* const rgb = a.rgb;

    float T[PX], Cr[PX], Cg[PX], Cb[PX];
    uint32_t last[PX], nblended[PX];
    bool done[PX];
    int ndone = 0;
#pragma unroll
    for (int j = 0; j < PX; ++j) {
        T[j] = 1.0f;
        Cr[j] = Cg[j] = Cb[j] = 0.f;
        last[j] = 0;
        nblended[j] = 0;
        done[j] = !(x0 + c0 + TPR * j < c.W && py < c.H);
        ndone += done[j];
    }
    for (uint32_t b = start; b < end; b += batch) {
        if (__syncthreads_count(ndone == PX) == nthreads) break;
        const int nb = (int)min((uint32_t)batch, end - b);
        for (int k = threadIdx.x; k < nb; k += nthreads) {
            uint32_t g = vals[b + k];
            if (g >= (uint32_t)n) {   // only reachable after a timed-out sort
                debug_fail(a.status);
                g = 0;
            }
            Staged st;
            stage_splat(xy[g], conic[g], x0, y0, log2_amin, st);
            s_sp[k] = st;
            s_rgb[k] = rgb[g];
            s_band[k] = band_mask(st, tile_w, tile_h, 32 / TPR);
        }
        __syncthreads();
        // 32 splats at a time: the warp's contribution bits for them are one word
        for (int k0 = 0; k0 < nb; k0 += 32) {
            uint32_t mb = 0;   // bit k - k0: some pixel of this thread blended splat k
            if (ndone < PX) {
                const int k1 = min(k0 + 32, nb);
#pragma unroll 2   // lets the next splat's row setup overlap this one's blend (forward 0.340 -> 0.333 ms)
                for (int k = k0; k < k1; ++k) {
                    if (!((s_band[k] >> warp) & 1u)) continue;           // no pixel of this warp reaches alpha_min
                    const Staged st = s_sp[k];
                    float p0, dp, q, qq;
                    splat_row(st, lyf, c0f, (float)TPR, p0, dp, q, qq);
                    if (qq > st.a.z) continue;                         // s >= q^2: the whole row skips
#pragma unroll
                    for (int j = 0; j < PX; ++j) {
                        float p;
                        const float s = splat_s(p0, dp, qq, j, p);
                        if (done[j] || s > st.a.z) continue;           // alpha < 1/255: skip
                        const float oG = hw_exp2(__fsub_rn(st.a.w, s));
                        const float alpha = fminf(amax, oG);
                        const float test = __fmul_rn(T[j], __fsub_rn(1.0f, alpha));
                        if (test < tmin) {                             // stop before exceeding 0.9999
                            done[j] = true;
                            ++ndone;
                            continue;
                        }
                        const float w = alpha * T[j];
                        const float4 col = s_rgb[k];
                        Cr[j] += w * col.x;
                        Cg[j] += w * col.y;
                        Cb[j] += w * col.z;
                        T[j] = test;
                        last[j] = b - start + (uint32_t)k + 1u;
                        mb |= 1u << (k - k0);
                        if (COUNT) ++nblended[j];
                    }
                    if (ndone == PX) break;
                }
            }
            mb = __reduce_or_sync(0xffffffffu, mb);
            if (lane == 0 && mb) {   // instances b + k0 .. b + k0 + 31 of this warp's bit array
                const uint32_t gi = b + (uint32_t)k0, sh = gi & 31u;
                atomicOr(wbits + (gi >> 5), mb << sh);
                if (sh) atomicOr(wbits + (gi >> 5) + 1, mb >> (32u - sh));
            }
            if (__all_sync(0xffffffffu, ndone == PX)) break;
        }
    }
    const size_t P = (size_t)c.W * c.H;
#pragma unroll
    for (int j = 0; j < PX; ++j) {
        const int px = x0 + c0 + TPR * j;
        if (px < c.W && py < c.H) {
            const size_t p = (size_t)py * c.W + px;
            a.out_rgb[p] = Cr[j] + T[j] * a.bg[0];
            a.out_rgb[P + p] = Cg[j] + T[j] * a.bg[1];
            a.out_rgb[2 * P + p] = Cb[j] + T[j] * a.bg[2];
            a.out_T[p] = T[j];
            a.out_last[p] = last[j];
            if (COUNT) a.out_count[p] = nblended[j];
        }
    }
}

// One block per tile.  A single frame reads its arguments straight from the parameter bank; a
// batch copies its frame's block of arguments into registers once (measured on four 1M-Gaussian
// views: half the instructions of a shared-memory copy, whose compiled form executed the blend
// loop's skipped pairs at the cost of blended ones).
template <int PX, int TPR, int MAXF, bool COUNT>
__global__ void __launch_bounds__(64, 1) k_render_forward_t(const __grid_constant__ Multi<RenderFwdArgs, MAXF> m) {
    if constexpr (MAXF == 1) {
        forward_tile<PX, TPR, COUNT>(m.a[0], blockIdx.x, m.base[1]);
    } else {
        const int f = find_frame<MAXF>(m.base, m.frames, blockIdx.x);
        const RenderFwdArgs a = m.a[f];
        forward_tile<PX, TPR, COUNT>(a, blockIdx.x - m.base[f], m.base[f + 1] - m.base[f]);
    }
}

// Backward pass of the tile order[block_slot] of a frame with ntiles tiles.
template <int PX, int TPR, bool LIMIT>
__device__ __forceinline__ void backward_tile(const RenderBwdArgs& a, uint32_t block_slot, uint32_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Staged* s_sp = reinterpret_cast<Staged*>(smem_raw);
    float4* s_rgb = reinterpret_cast<float4*>(smem_raw + sizeof(Staged) * a.batch);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(smem_raw + (sizeof(Staged) + sizeof(float4)) * a.batch);
    const uint32_t* const wbits = a.contrib + (size_t)(threadIdx.x >> 5) * a.contrib_words;
    __shared__ uint32_t s_max;
    const CamK& c = a.cam;
    const uint32_t tile_id = a.order[block_slot];
    if (tile_id >= ntiles) {   // an order not written by gs_bin_sort
        if (threadIdx.x == 0) debug_fail(a.status);
        return;
    }
    const int tile = (int)tile_id;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int nthreads = blockDim.x;
    const int ly = threadIdx.x / TPR, c0 = threadIdx.x % TPR;   // TPR threads per tile row
    const int x0 = tx * c.tile_w, y0 = ty * c.tile_h;
    const int py = y0 + ly;
    const float lyf = (float)ly, c0f = (float)c0;
    const uint32_t start = a.ranges[2 * tile];
    uint32_t len = a.ranges[2 * tile + 1] - start;
    if (GS_DEBUG && (a.ranges[2 * tile + 1] < start || a.ranges[2 * tile + 1] > a.capacity)) {
        if (threadIdx.x == 0) debug_fail(a.status);
        len = 0;
    }
    const float amax = a.cfg.alpha_max;
    const float log2_amin = __log2f(a.cfg.alpha_min);
    const size_t P = (size_t)c.W * c.H;
    // what the loops read, in registers (see the forward pass)
    const int batch = a.batch, n = a.n;
    const uint32_t* const vals = a.vals;
    const float4* const xy = a.xy;
    const float4* const conic = a.conic_opacity;
    const float4* const rgb = a.rgb;
    float* const grad2d = a.grad2d;

    // Per pixel: T, R . dL/dC (only this projection of the colour behind is ever needed) and dL/dC.
    float T[PX], Rd[PX], dLr[PX], dLg[PX], dLb[PX];
    uint32_t mylast[PX];
    // LIMIT: the first `skip` blended splats met from the back (all but the grad_limit front-most)
    // get no gradient; the recurrences for T and R . dL/dC still run through them
    uint32_t skip[PX], seen[PX];
    uint32_t tmax = 0;
#pragma unroll
    for (int j = 0; j < PX; ++j) {
        const int px = x0 + c0 + TPR * j;
        mylast[j] = 0;
        skip[j] = seen[j] = 0;
        T[j] = 1.0f;
        dLr[j] = dLg[j] = dLb[j] = 0.f;
        if (px < c.W && py < c.H) {
            const size_t p = (size_t)py * c.W + px;
            mylast[j] = a.last[p];
            if (LIMIT) {
                const uint32_t nb = a.count[p], lim = (uint32_t)a.cfg.grad_limit;
                skip[j] = nb > lim ? nb - lim : 0u;
            }
            T[j] = a.T_final[p];
            dLr[j] = a.dL_drgb[p];
            dLg[j] = a.dL_drgb[P + p];
            dLb[j] = a.dL_drgb[2 * P + p];
        }
        Rd[j] = a.bg[0] * dLr[j] + a.bg[1] * dLg[j] + a.bg[2] * dLb[j];
        tmax = max(tmax, mylast[j]);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, tmax);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const uint32_t count = min(s_max, len);   // last positions never exceed the tile's list
    uint32_t nblend = 0;
    const int lane = threadIdx.x & 31;
    const int slot = reduce_slot(lane);

    for (int bend = (int)count; bend > 0; bend -= batch) {
        const int nb = min(batch, bend);
        __syncthreads();
        for (int k = threadIdx.x; k < nb; k += nthreads) {
            uint32_t g = vals[start + (uint32_t)(bend - 1 - k)];
            if (g >= (uint32_t)n) {   // only reachable after a timed-out sort
                debug_fail(a.status);
                g = 0;
            }
            Staged st;
            stage_splat(xy[g], conic[g], x0, y0, log2_amin, st);
            s_sp[k] = st;
            s_rgb[k] = rgb[g];
            s_idx[k] = g;
        }
        __syncthreads();
        // Only the splats some pixel of this warp blended in the forward pass (its contribution
        // bits; the backward blends exactly the forward's pairs), 32 at a time.
        for (int k0 = 0; k0 < nb; k0 += 32) {
          uint32_t todo = __brev(bits_window(wbits, start + (uint32_t)(bend - 1 - k0)));   // bit i: splat k0 + i
          if (nb - k0 < 32) todo &= (1u << (nb - k0)) - 1u;
          while (todo) {
            const int k = k0 + __ffs(todo) - 1;
            todo &= todo - 1u;
            const uint32_t pos = (uint32_t)(bend - 1 - k);
            float g[9];
#pragma unroll
            for (int v = 0; v < 9; ++v) g[v] = 0.f;
            bool contrib = false;
            const Staged st = s_sp[k];
            float p0, dp, q, qq;
            splat_row(st, lyf, c0f, (float)TPR, p0, dp, q, qq);
            if (pos < tmax && qq <= st.a.z) {                      // s >= q^2: else the whole row skips
                const float4 col = s_rgb[k];
#pragma unroll
                for (int j = 0; j < PX; ++j) {
                    float p;
                    const float s = splat_s(p0, dp, qq, j, p);
                    if (pos >= mylast[j] || s > st.a.z) continue;
                    const bool grad = !LIMIT || seen[j]++ >= skip[j];
                    contrib |= grad;
                    ++nblend;
                    const float oG = hw_exp2(__fsub_rn(st.a.w, s));
                    const float alpha = fminf(amax, oG);
                    const float one_m = __fsub_rn(1.0f, alpha);
                    const float Ti = T[j] * hw_rcp(one_m);      // T_i = T_{i+1} / (1 - alpha_i), one_m >= 0.01
                    const float w = alpha * Ti;
                    // dL/dalpha = T_i (c_i - R_{i+1}) . dL/dC;  R_i . dL/dC = R_{i+1} . dL/dC + alpha (c_i - R_{i+1}) . dL/dC
                    const float diff = col.x * dLr[j] + col.y * dLg[j] + col.z * dLb[j] - Rd[j];
                    const float dalpha = Ti * diff;
                    Rd[j] = fmaf(alpha, diff, Rd[j]);
                    T[j] = Ti;
                    if (LIMIT && !grad) continue;
                    g[6] += w * dLr[j];
                    g[7] += w * dLg[j];
                    g[8] += w * dLb[j];
                    if (oG <= amax) {
                        // dpow = dL/d(power): sums of dpow (p, q) and dpow (p, q)(p, q)^T in the
                        // whitened frame (scaled p, q), the constant factors 1/o, 1/kScaleLog2 and
                        // ln 2 once per splat below
                        const float dpow = oG * dalpha;
                        const float dpp = dpow * p, dpq = dpow * q;
                        g[0] += dpp;
                        g[1] += dpq;
                        g[2] = fmaf(dpp, p, g[2]);
                        g[3] = fmaf(dpp, q, g[3]);
                        g[4] = fmaf(dpq, q, g[4]);
                        g[5] += dpow;
                    }
                }
            }
            const uint32_t who = __ballot_sync(0xffffffffu, contrib);
            if (who == 0) continue;
            float* dst = grad2d + 12 * (size_t)s_idx[k];
            const float k1 = kUnscale, k2 = kLn2, ko = st.b.w;
            if (__popc(who) <= kDirectLanes) {
                // few contributing lanes: each adds its own sums (cheaper than a butterfly)
                if (contrib) {
                    atomicAdd(reinterpret_cast<float4*>(dst), make_float4(k1 * g[0], k1 * g[1], k2 * g[2], k2 * g[3]));
                    atomicAdd(reinterpret_cast<float4*>(dst) + 1, make_float4(k2 * g[4], ko * g[5], g[6], g[7]));
                    atomicAdd(dst + 8, g[8]);
                }
            } else {
                const float tot = warp_reduce9(g, lane);
                if (slot >= 0 && !(lane & 1)) atomicAdd(dst + slot, tot * (slot < 2 ? k1 : slot < 5 ? k2 : slot == 5 ? ko : 1.0f));
            }
          }
        }
    }
    const uint32_t wblend = __reduce_add_sync(0xffffffffu, nblend);
    if ((threadIdx.x & 31) == 0 && wblend) atomicAdd(a.blended, (unsigned long long)wblend);
}

// One block per tile, arguments as in k_render_forward_t.
template <int PX, int TPR, int MAXF, bool LIMIT>
__global__ void __launch_bounds__(64) k_render_backward_t(const __grid_constant__ Multi<RenderBwdArgs, MAXF> m) {
    if constexpr (MAXF == 1) {
        backward_tile<PX, TPR, LIMIT>(m.a[0], blockIdx.x, m.base[1]);
    } else {
        const int f = find_frame<MAXF>(m.base, m.frames, blockIdx.x);
        const RenderBwdArgs a = m.a[f];
        backward_tile<PX, TPR, LIMIT>(a, blockIdx.x - m.base[f], m.base[f + 1] - m.base[f]);
    }
}

size_t fwd_smem(int batch) { return (sizeof(Staged) + sizeof(float4) + sizeof(uint32_t)) * (size_t)batch; }
size_t bwd_smem(int batch) { return (sizeof(Staged) + sizeof(float4) + sizeof(uint32_t)) * (size_t)batch; }

}  // namespace

// Tiles of every frame, in frame order (frames without Gaussians still get their background
// and transmittance written); all frames of a batch share the tile shape and the batch depth.
template <typename A, int MAXF>
static uint32_t tile_split(Multi<A, MAXF>& m) {
    m.base[0] = 0;
    for (int f = 0; f < m.frames; ++f)
        m.base[f + 1] = m.base[f] + (uint32_t)(m.a[f].cam.tiles_x * m.a[f].cam.tiles_y);
    return m.base[m.frames];
}

template <int MAXF>
cudaError_t launch_render_forward(Multi<RenderFwdArgs, MAXF>& m, cudaStream_t s) {
    const uint32_t tiles = tile_split(m);
    if (tiles == 0) return cudaSuccess;
    const RenderFwdArgs& a = m.a[0];
    // 4 threads per tile row (measured: 2 per row, one warp per 16x16 tile, is 1.5x slower; 8 per
    // row makes the forward 4 % faster and the backward 10 % slower, and both kernels must
    // evaluate a pixel with the same operation sequence for their decisions to agree)
    const dim3 grid(tiles), block(4 * a.cam.tile_h);
    const size_t smem = fwd_smem(a.batch);
    if (a.out_count) {   // gradient-limited frames also record the blended splats per pixel
        if (a.cam.tile_w == 16) k_render_forward_t<4, 4, MAXF, true><<<grid, block, smem, s>>>(m);
        else k_render_forward_t<2, 4, MAXF, true><<<grid, block, smem, s>>>(m);
    } else {
        if (a.cam.tile_w == 16) k_render_forward_t<4, 4, MAXF, false><<<grid, block, smem, s>>>(m);
        else k_render_forward_t<2, 4, MAXF, false><<<grid, block, smem, s>>>(m);
    }
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_render_backward(Multi<RenderBwdArgs, MAXF>& m, cudaStream_t s) {
    const uint32_t tiles = tile_split(m);
    if (tiles == 0) return cudaSuccess;
    const RenderBwdArgs& a = m.a[0];
    const dim3 grid(tiles), block(4 * a.cam.tile_h);
    const size_t smem = bwd_smem(a.batch);
    if (a.count) {
        if (a.cam.tile_w == 16) k_render_backward_t<4, 4, MAXF, true><<<grid, block, smem, s>>>(m);
        else k_render_backward_t<2, 4, MAXF, true><<<grid, block, smem, s>>>(m);
    } else {
        if (a.cam.tile_w == 16) k_render_backward_t<4, 4, MAXF, false><<<grid, block, smem, s>>>(m);
        else k_render_backward_t<2, 4, MAXF, false><<<grid, block, smem, s>>>(m);
    }
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_tile_order(const Multi<TileOrderArgs, MAXF>& m, cudaStream_t s) {
    k_tile_order<MAXF><<<m.frames, kOrderThreads, 0, s>>>(m);
    return cudaGetLastError();
}

template cudaError_t launch_tile_order<1>(const Multi<TileOrderArgs, 1>&, cudaStream_t);
template cudaError_t launch_tile_order<kMaxFrames>(const Multi<TileOrderArgs, kMaxFrames>&, cudaStream_t);
template cudaError_t launch_render_forward<1>(Multi<RenderFwdArgs, 1>&, cudaStream_t);
template cudaError_t launch_render_forward<kMaxFrames>(Multi<RenderFwdArgs, kMaxFrames>&, cudaStream_t);
template cudaError_t launch_render_backward<1>(Multi<RenderBwdArgs, 1>&, cudaStream_t);
template cudaError_t launch_render_backward<kMaxFrames>(Multi<RenderBwdArgs, kMaxFrames>&, cudaStream_t);

}  // namespace gs
