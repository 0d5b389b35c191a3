// render.cu -- per-tile blending (Algorithm 2, BlendInOrder) and its backward pass (Sec. 6).
//
// One thread block per tile, one thread per pixel.  The block stages batches of the tile's
// depth-sorted Gaussians (screen mean, conic + opacity, colour) in shared memory; every pixel
// then walks the batch.
//
// Forward (eq. front-to-back, App. C): a = min(0.99, o exp(power)); skip a < 1/255; stop before
//   T (1 - a) < 1e-4; C += a T c; T *= 1 - a.  The tile stops as soon as all its pixels are done
//   (checked once per batch with __syncthreads_count).  Writes C + T bg, T and the 1-based list
//   position of the last blended Gaussian.
// Backward: the tile's list is walked back to front from the largest last position in the tile;
//   each pixel only processes positions below its own last position, recovers
//   T_i = T_{i+1} / (1 - a_i) from the stored final T, and keeps R, the colour behind the current
//   Gaussian normalised by the transmittance in front of it (R starts at bg):
//     dL/dc_i = a_i T_i dL/dC,  dL/da_i = T_i (c_i - R_{i+1}) . dL/dC,  R_i = a_i c_i + (1 - a_i) R_{i+1}.
//   Through a = o G (zero when clamped) and power = -d^T Sigma'^-1 d / 2 it yields
//   dL/d(mean2D, Sigma', opacity, colour) per pixel; these are summed over the warp with
//   shuffles and added to the per-Gaussian accumulators with vector atomics.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

__global__ void __launch_bounds__(kMaxTilePixels) k_render_forward(RenderFwdArgs a) {
    __shared__ float2 s_off[kMaxTilePixels];
    __shared__ float4 s_co[kMaxTilePixels];
    __shared__ float4 s_rgb[kMaxTilePixels];
    const CamK& c = a.cam;
    const int tile = blockIdx.x;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int npx = blockDim.x;
    const int lx = threadIdx.x % c.tile_w, ly = threadIdx.x / c.tile_w;
    const int px = tx * c.tile_w + lx, py = ty * c.tile_h + ly;
    const bool inside = px < c.W && py < c.H;
    const float lxf = (float)lx, lyf = (float)ly;
    const int x0 = tx * c.tile_w, y0 = ty * c.tile_h;
    const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
    const float amin = a.cfg.alpha_min, amax = a.cfg.alpha_max, tmin = a.cfg.T_min;

    float T = 1.0f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t b = start; b < end; b += a.batch) {
        if (__syncthreads_count(done) == npx) break;
        const uint32_t j = b + threadIdx.x;
        if ((int)threadIdx.x < a.batch && j < end) {
            uint32_t g = a.vals[j];
            if (g >= (uint32_t)a.n) g = 0;   // only reachable after a timed-out sort
            const float4 m = a.xy[g];
            s_off[threadIdx.x] = make_float2(tile_offset(x0, m.x, m.z), tile_offset(y0, m.y, m.w));
            s_co[threadIdx.x] = a.conic_opacity[g];
            s_rgb[threadIdx.x] = a.rgb[g];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)a.batch, end - b);
        if (!done) {
            for (int k = 0; k < nb; ++k) {
                float G, oG, pp, qq;
                const float4 co = s_co[k];
                const float2 o = s_off[k];
                const float dx = __fadd_rn(lxf, o.x), dy = __fadd_rn(lyf, o.y);
                const float power = splat_power(dx, dy, co, pp, qq);
                const float alpha = splat_alpha(power, co.w, amax, G, oG);
                if (alpha < amin) continue;
                const float test = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                if (test < tmin) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                const float4 col = s_rgb[k];
                Cr += w * col.x;
                Cg += w * col.y;
                Cb += w * col.z;
                T = test;
                last = b - start + (uint32_t)k + 1u;
            }
        }
    }
    if (inside) {
        const size_t P = (size_t)c.W * c.H;
        const size_t p = (size_t)py * c.W + px;
        a.out_rgb[p] = Cr + T * a.bg[0];
        a.out_rgb[P + p] = Cg + T * a.bg[1];
        a.out_rgb[2 * P + p] = Cb + T * a.bg[2];
        a.out_T[p] = T;
        a.out_last[p] = last;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kMaxTilePixels) k_render_backward(RenderBwdArgs a) {
    __shared__ uint32_t s_idx[kMaxTilePixels];
    __shared__ float2 s_off[kMaxTilePixels];
    __shared__ float4 s_co[kMaxTilePixels];
    __shared__ float4 s_rgb[kMaxTilePixels];
    __shared__ uint32_t s_max;
    const CamK& c = a.cam;
    const int tile = blockIdx.x;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int lx = threadIdx.x % c.tile_w, ly = threadIdx.x / c.tile_w;
    const int px = tx * c.tile_w + lx, py = ty * c.tile_h + ly;
    const bool inside = px < c.W && py < c.H;
    const float lxf = (float)lx, lyf = (float)ly;
    const int x0 = tx * c.tile_w, y0 = ty * c.tile_h;
    const uint32_t start = a.ranges[2 * tile], len = a.ranges[2 * tile + 1] - start;
    const float amin = a.cfg.alpha_min, amax = a.cfg.alpha_max;
    const size_t P = (size_t)c.W * c.H;
    const size_t p = (size_t)py * c.W + px;

    uint32_t my_last = 0;
    float T = 1.0f, dLr = 0.f, dLg = 0.f, dLb = 0.f;
    if (inside) {
        my_last = a.last[p];
        T = a.T_final[p];
        dLr = a.dL_drgb[p];
        dLg = a.dL_drgb[P + p];
        dLb = a.dL_drgb[2 * P + p];
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, my_last);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const uint32_t count = min(s_max, len);   // last positions never exceed the tile's list

    float Rr = a.bg[0], Rg = a.bg[1], Rb = a.bg[2];
    for (int bend = (int)count; bend > 0; bend -= a.batch) {
        const int bstart = max(bend - a.batch, 0);
        const int nb = bend - bstart;
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            uint32_t g = a.vals[start + (uint32_t)(bend - 1 - (int)threadIdx.x)];
            if (g >= (uint32_t)a.n) g = 0;   // only reachable after a timed-out sort
            s_idx[threadIdx.x] = g;
            const float4 m = a.xy[g];
            s_off[threadIdx.x] = make_float2(tile_offset(x0, m.x, m.z), tile_offset(y0, m.y, m.w));
            s_co[threadIdx.x] = a.conic_opacity[g];
            s_rgb[threadIdx.x] = a.rgb[g];
        }
        __syncthreads();
        for (int k = 0; k < nb; ++k) {
            const uint32_t pos = (uint32_t)(bend - 1 - k);
            float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_o = 0.f, g_r = 0.f, g_g = 0.f, g_bl = 0.f;
            bool contrib = false;
            if (pos < my_last) {
                float G, oG, pp, qq;
                const float4 co = s_co[k];
                const float2 o = s_off[k];
                const float dx = __fadd_rn(lxf, o.x), dy = __fadd_rn(lyf, o.y);
                const float power = splat_power(dx, dy, co, pp, qq);
                const float alpha = splat_alpha(power, co.w, amax, G, oG);
                if (alpha >= amin) {
                    contrib = true;
                    const float one_m = __fsub_rn(1.0f, alpha);
                    const float Ti = T / one_m;
                    const float w = alpha * Ti;
                    const float4 col = s_rgb[k];
                    g_r = w * dLr;
                    g_g = w * dLg;
                    g_bl = w * dLb;
                    const float dalpha = Ti * ((col.x - Rr) * dLr + (col.y - Rg) * dLg + (col.z - Rb) * dLb);
                    Rr = alpha * col.x + one_m * Rr;
                    Rg = alpha * col.y + one_m * Rg;
                    Rb = alpha * col.z + one_m * Rb;
                    T = Ti;
                    if (oG <= amax) {
                        g_o = G * dalpha;
                        const float dpow = oG * dalpha;
                        // With g = Q d = L (p, q): d(power)/d(mean) = g and
                        // d(power)/d(Sigma') = g g^T / 2 (from d(Q) = -Q d(Sigma') Q).  Accumulating
                        // dL/dSigma' here, instead of dL/dconic followed by -Q G Q per Gaussian,
                        // avoids the cancellation of that product for elongated splats.
                        const float gx = co.x * pp, gy = co.y * pp + co.z * qq;
                        const float h = 0.5f * dpow;
                        g_u = gx * dpow;
                        g_v = gy * dpow;
                        g_a = h * gx * gx;
                        g_b = h * gx * gy;
                        g_c = h * gy * gy;
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                g_u = warp_sum(g_u);
                g_v = warp_sum(g_v);
                g_a = warp_sum(g_a);
                g_b = warp_sum(g_b);
                g_c = warp_sum(g_c);
                g_o = warp_sum(g_o);
                g_r = warp_sum(g_r);
                g_g = warp_sum(g_g);
                g_bl = warp_sum(g_bl);
                if ((threadIdx.x & 31) == 0) {
                    float4* acc = reinterpret_cast<float4*>(a.grad2d) + 3 * (size_t)s_idx[k];
                    atomicAdd(acc, make_float4(g_u, g_v, g_a, g_b));
                    atomicAdd(acc + 1, make_float4(g_c, g_o, g_r, g_g));
                    atomicAdd(reinterpret_cast<float*>(acc + 2), g_bl);
                }
            }
        }
    }
}

cudaError_t launch_render_forward(const RenderFwdArgs& a, int tiles, int threads, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_render_forward<<<tiles, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const RenderBwdArgs& a, int tiles, int threads, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_render_backward<<<tiles, threads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gs
