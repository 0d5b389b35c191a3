// preprocess.cu -- per-Gaussian forward (Algorithm 2: CullGaussian + ScreenspaceGaussians)
// and backward (chain rule of App. A) kernels, one thread per Gaussian.
//
// Forward, per Gaussian (Sec. 4, Sec. 6):
//   t = W mu + t_w; reject z <= near, |x/z| > guard tan_x, |y/z| > guard tan_y;
//   R = R(q / |q|) (eq. quat), M = R diag(s), Sigma = M M^T;
//   Sigma' = J W Sigma W^T J^T (eq. volume-render) evaluated as V V^T with V = (J W) M, so the
//   determinant comes from the cross product |v0 x v1|^2 (no cancellation), plus 0.3 I;
//   conic = Sigma'^-1 (stored as its Cholesky factor); radius = ceil(3 sqrt(lambda_max));
//   mean2D = (fx x/z + cx, fy y/z + cy) in double-float;
//   tile rectangle (culled when empty); rgb = max(0, sum_k c_k Y_k((mu - C)/|mu - C|)).
// Backward: the same quantities recomputed, then dL/dSigma' = L K L^T (K accumulated per pixel by
//   the tile traversal in the whitened frame of the conic's Cholesky factor L) -> dL/dV = 2 H V
//   -> dL/dM = (J W)^T dL/dV -> (s, R) -> q_hat -> q (normalisation Jacobian);
//   dL/d(J W) -> dL/dJ -> dL/dt; dL/dmean2D -> dL/dt; dL/dt -> dL/dmu = W^T dL/dt;
//   dL/drgb (clamp mask) -> dL/dSH = Y dL/drgb and -> dL/d dir -> dL/dmu.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

struct Proj {
    float tx, ty, tz;     // camera-space mean (rounded)
    float xz, yz;         // x/z, y/z (rounded)
    DF u, v;              // screen mean, double-float
    float qn[4];          // normalised quaternion
    float qinv;           // 1 / |q|
    float R[9];           // R(q_hat)
    float M[9];           // R diag(s)
    float T2[6];          // J W (2 x 3)
    float V[6];           // J W M (2 x 3)
    float A, B, C;        // Sigma' with dilation
    float det;
};

__device__ __forceinline__ void rot_from_quat(const float* q, float* R) {
    const float r = q[0], i = q[1], j = q[2], k = q[3];
    R[0] = 1.f - 2.f * (j * j + k * k); R[1] = 2.f * (i * j - r * k);       R[2] = 2.f * (i * k + r * j);
    R[3] = 2.f * (i * j + r * k);       R[4] = 1.f - 2.f * (i * i + k * k); R[5] = 2.f * (j * k - r * i);
    R[6] = 2.f * (i * k - r * j);       R[7] = 2.f * (j * k + r * i);       R[8] = 1.f - 2.f * (i * i + j * j);
}

// Camera-space mean, guard-band test and screen mean.  The mean is carried in double-float
// (compensated dot product and division) so that u, v and the depth are accurate to about
// 1e-12 relative: fp32 alone would leave errors of ~1e-4 px at the far side of a 1080p image.
// Returns false when rejected.
__device__ __forceinline__ bool project_mean(const float* mu, const CamK& c, Proj& p) {
    const DF x = dot3_plus(c.R, mu, c.t[0]);
    const DF y = dot3_plus(c.R + 3, mu, c.t[1]);
    const DF z = dot3_plus(c.R + 6, mu, c.t[2]);
    p.tx = x.hi;
    p.ty = y.hi;
    p.tz = z.hi;
    if (!(p.tz > c.near_z) || !isfinite(p.tz)) return false;
    const DF xz = df_div(x, z), yz = df_div(y, z);
    p.xz = xz.hi;
    p.yz = yz.hi;
    if (fabsf(p.xz) > c.lim_x || fabsf(p.yz) > c.lim_y) return false;
    p.u = df_mul_add(c.fx, xz, c.cx);
    p.v = df_mul_add(c.fy, yz, c.cy);
    return true;
}

// Covariance projection; requires project_mean first.
__device__ __forceinline__ void project_cov(const float* s, const float4 q, const CamK& c, float dilation,
                                            Proj& p) {
    const float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    p.qinv = rsqrtf(qq);
    p.qn[0] = q.x * p.qinv; p.qn[1] = q.y * p.qinv; p.qn[2] = q.z * p.qinv; p.qn[3] = q.w * p.qinv;
    rot_from_quat(p.qn, p.R);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) p.M[3 * r + k] = p.R[3 * r + k] * s[k];
    // J W: row0 = fx/z (W0 - x/z W2), row1 = fy/z (W1 - y/z W2)
    const float fz = c.fx / p.tz, gz = c.fy / p.tz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p.T2[k] = fz * (c.R[k] - p.xz * c.R[6 + k]);
        p.T2[3 + k] = gz * (c.R[3 + k] - p.yz * c.R[6 + k]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            p.V[3 * r + k] = p.T2[3 * r] * p.M[k] + p.T2[3 * r + 1] * p.M[3 + k] + p.T2[3 * r + 2] * p.M[6 + k];
    const float a = p.V[0] * p.V[0] + p.V[1] * p.V[1] + p.V[2] * p.V[2];
    const float b = p.V[0] * p.V[3] + p.V[1] * p.V[4] + p.V[2] * p.V[5];
    const float cc = p.V[3] * p.V[3] + p.V[4] * p.V[4] + p.V[5] * p.V[5];
    // det(V V^T) = |v0 x v1|^2 (Cauchy-Binet)
    const float cx = p.V[1] * p.V[5] - p.V[2] * p.V[4];
    const float cy = p.V[2] * p.V[3] - p.V[0] * p.V[5];
    const float cz = p.V[0] * p.V[4] - p.V[1] * p.V[3];
    const float det_raw = cx * cx + cy * cy + cz * cz;
    p.A = a + dilation;
    p.B = b;
    p.C = cc + dilation;
    p.det = det_raw + dilation * (a + cc) + dilation * dilation;
}

__device__ __forceinline__ bool finite3(const float* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

// SH coefficients of one Gaussian, [D][3] floats.  VEC: the row starts 16-byte aligned and its
// stride is a multiple of 4 floats, so it is read as float4 (rounded up to whole float4s, which
// stays inside the row).
template <int D, bool VEC>
__device__ __forceinline__ void load_sh(const float* __restrict__ sh, float (&f)[4 * ((3 * D + 3) / 4)]) {
    constexpr int N4 = (3 * D + 3) / 4;
    if (VEC) {
        const float4* p = reinterpret_cast<const float4*>(sh);
#pragma unroll
        for (int k = 0; k < N4; ++k) {
            const float4 v = p[k];
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3 * D; ++k) f[k] = sh[k];
    }
}

// 256-bit global accesses of 8 floats (PTX ld/st.global.v8.f32; p 32-byte aligned).  A thread's
// SH gradient row written as 32-byte stores fills each 32-byte sector with one store instead of
// two 16-byte halves from separate instructions: the per-Gaussian backward on the 3M-Gaussian
// frame 0.303 -> 0.249 ms.  (The same loads of the SH rows made the forward preprocess slower.)
__device__ __forceinline__ void st_v8(float* p, const float (&v)[8]) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ void ld_v8(const float* p, float (&v)[8]) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
}

}  // namespace

// 6 blocks of 256 per SM (40 registers): config 3 (3M Gaussians) 0.157 -> 0.148 ms against the
// 48-register build at 5 blocks; streaming or L2-only loads of the SH rows were slower (0.194,
// 0.175 ms) and also slowed the backward, which re-reads the rows that stay in L2.
template <int DEG, bool VEC, int MAXF, bool ISO>
__global__ void __launch_bounds__(256, 6) k_preprocess_t(const __grid_constant__ Multi<PreprocessArgs, MAXF> m) {
    constexpr int D = (DEG + 1) * (DEG + 1);
    const int f = find_frame<MAXF>(m.base, m.frames, blockIdx.x);   // frame f owns blocks [base[f], base[f+1])
    // a batch reads its frame's arguments from a shared copy (generic loads otherwise)
    __shared__ __align__(16) PreprocessArgs s_args;
    if (MAXF > 1) {
        for (int k = threadIdx.x; k < (int)(sizeof(PreprocessArgs) / 4); k += blockDim.x)
            reinterpret_cast<uint32_t*>(&s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f])[k];
        __syncthreads();
    }
    const PreprocessArgs& a = MAXF == 1 ? m.a[0] : s_args;
    const int i = (int)(blockIdx.x - m.base[f]) * blockDim.x + threadIdx.x;
    bool visible = false;
    if (i < a.n) {
        const CamK& c = a.cam;
        const float mu[3] = {a.means[3 * i], a.means[3 * i + 1], a.means[3 * i + 2]};
        // ISO (the isotropic ablation of Sec. 7.3): one scale for all axes and no rotation
        const float s0 = ISO ? a.scales[i] : a.scales[3 * i];
        const float s[3] = {s0, ISO ? s0 : a.scales[3 * i + 1], ISO ? s0 : a.scales[3 * i + 2]};
        const float4 q = ISO ? make_float4(1.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(a.quats)[i];
        const float o = a.opacities[i];
        const bool finite = finite3(mu) && finite3(s) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) &&
                            isfinite(q.w) && isfinite(o);
        int radius = 0;
        float4 xy = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 rgb = make_float4(0.f, 0.f, 0.f, 0.f);
        float depth = 0.f;
        Proj p;
        if (!finite) {
            atomicAdd(&a.status->num_nonfinite, 1u);
        } else if (project_mean(mu, c, p) && (q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w) > 0.f) {
            project_cov(s, q, c, a.cfg.dilation, p);
            if (p.det > 0.f) {
                // Cholesky factor of the conic (see splat_power).
                co = make_float4(sqrtf(p.C / p.det), -p.B / sqrtf(p.C * p.det), 1.0f / sqrtf(p.C), o);
                const float m = 0.5f * (p.A + p.C);
                const float h = 0.5f * (p.A - p.C);
                const float lam = m + sqrtf(h * h + p.B * p.B);
                const float rr = a.cfg.extent * sqrtf(lam);
                radius = rr >= (float)a.cfg.radius_max ? a.cfg.radius_max : (int)ceilf(rr);
                xy = make_float4(p.u.hi, p.v.hi, p.u.lo, p.v.lo);
                int x0, x1, y0, y1;
                if (!tile_rect(xy, radius, c, x0, x1, y0, y1)) radius = 0;
                depth = p.tz;
            }
        }
        if (radius > 0) {
            // View-dependent colour from the SH coefficients.
            float dx = mu[0] - c.campos[0], dy = mu[1] - c.campos[1], dz = mu[2] - c.campos[2];
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv; dy *= inv; dz *= inv;
            float Y[16];
            sh_basis(DEG, dx, dy, dz, Y);
            float f[4 * ((3 * D + 3) / 4)];
            load_sh<D, VEC>(a.sh + (size_t)i * a.sh_stride * 3, f);
            float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                r += f[3 * k] * Y[k];
                g += f[3 * k + 1] * Y[k];
                b += f[3 * k + 2] * Y[k];
            }
            if (!(isfinite(r) && isfinite(g) && isfinite(b))) {
                atomicAdd(&a.status->num_nonfinite, 1u);
                radius = 0;
            } else {
                const uint32_t mask = (r < 0.f ? 1u : 0u) | (g < 0.f ? 2u : 0u) | (b < 0.f ? 4u : 0u);
                rgb = make_float4(fmaxf(r, 0.f), fmaxf(g, 0.f), fmaxf(b, 0.f), __uint_as_float(mask));
            }
        }
        visible = radius > 0;
        a.xy[i] = xy;
        a.depth[i] = depth;
        a.conic_opacity[i] = co;
        a.rgb[i] = rgb;
        a.radius[i] = radius;
        // alpha >= alpha_min  <=>  d^T Q d <= 2 ln(o / alpha_min): the level the binning
        // stage intersects with each tile row (reach_setup).
        a.tau[i] = visible ? 2.0f * (logf(o) - logf(a.cfg.alpha_min)) : 0.0f;
    }
    const uint32_t vis = __ballot_sync(0xffffffffu, visible);
    if ((threadIdx.x & 31) == 0 && vis) atomicAdd(&a.status->num_visible, (uint32_t)__popc(vis));
}

// Gradient of one Gaussian from one view, added into the accumulators (the Gaussian's
// parameters and SH coefficients are loaded once for all views of a batch).
template <int DEG>
struct BwdAcc {
    static constexpr int D = (DEG + 1) * (DEG + 1);
    static constexpr int NF = 4 * ((3 * D + 3) / 4);
    float gm[3], gs[3], gq[4], go, du, dv;
    float gsh[NF];
};

template <int DEG>
__device__ __forceinline__ void bwd_view(const PreprocessBwdArgs& a, int i, const float mu[3], const float s[3],
                                         float4 q, const float* f, BwdAcc<DEG>& acc) {
    constexpr int D = BwdAcc<DEG>::D;
    const CamK& c = a.cam;
    const float4 g0 = reinterpret_cast<const float4*>(a.grad2d)[3 * i];       // P Q K00 K01
    const float4 g1 = reinterpret_cast<const float4*>(a.grad2d)[3 * i + 1];   // K11 do dr dg
    const float g2 = a.grad2d[12 * i + 8];                                    // db(rgb)
    const float4 L = a.conic[i];                                              // (l11, l21, l22, o)
    Proj p;
    project_mean(mu, c, p);
    project_cov(s, q, c, a.cfg.dilation, p);
    // The tile traversal summed dL/dpower (p, q) and K = (1/2) dL/dpower (p, q)(p, q)^T in the
    // whitened frame (p, q) = L^T d of the conic's Cholesky factor L; with g = Sigma'^-1 d = L (p, q):
    // dL/dmean2D = L (P, Q) and dL/dSigma' = L K L^T =: H.
    const float du = L.x * g0.x, dv = fmaf(L.y, g0.x, L.z * g0.y);
    const float K00 = g0.z, K01 = g0.w, K11 = g1.x;
    // Sigma'_raw = V V^T: dL/dV = 2 H V = 2 L (K (L^T V)), never forming H (whose pixel-frame
    // entries lose the long axis of an elongated splat to cancellation).
    float dV[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float w0 = fmaf(L.x, p.V[k], L.y * p.V[3 + k]), w1 = L.z * p.V[3 + k];   // L^T V
        const float z0 = fmaf(K00, w0, K01 * w1), z1 = fmaf(K01, w0, K11 * w1);         // K L^T V
        dV[k] = 2.f * (L.x * z0);
        dV[3 + k] = 2.f * fmaf(L.y, z0, L.z * z1);
    }
    // V = T2 M: dL/dM = T2^T dV, dL/dT2 = dV M^T.
    float dM[9], dT2[6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) dM[3 * r + k] = p.T2[r] * dV[k] + p.T2[3 + r] * dV[3 + k];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dT2[3 * r + k] = dV[3 * r] * p.M[3 * k] + dV[3 * r + 1] * p.M[3 * k + 1] + dV[3 * r + 2] * p.M[3 * k + 2];
    // M = R diag(s).
    float dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.gs[k] += dM[k] * p.R[k] + dM[3 + k] * p.R[3 + k] + dM[6 + k] * p.R[6 + k];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) dR[3 * r + k] = dM[3 * r + k] * s[k];
    // R(q_hat), eq. quat.
    const float qr = p.qn[0], qi = p.qn[1], qj = p.qn[2], qk = p.qn[3];
    float dq[4];
    dq[0] = 2.f * (-qk * dR[1] + qj * dR[2] + qk * dR[3] - qi * dR[5] - qj * dR[6] + qi * dR[7]);
    dq[1] = 2.f * (qj * dR[1] + qk * dR[2] + qj * dR[3] - 2.f * qi * dR[4] - qr * dR[5] + qk * dR[6] + qr * dR[7] -
                   2.f * qi * dR[8]);
    dq[2] = 2.f * (-2.f * qj * dR[0] + qi * dR[1] + qr * dR[2] + qi * dR[3] + qk * dR[5] - qr * dR[6] + qk * dR[7] -
                   2.f * qj * dR[8]);
    dq[3] = 2.f * (-2.f * qk * dR[0] - qr * dR[1] + qi * dR[2] + qr * dR[3] - 2.f * qk * dR[4] + qj * dR[5] +
                   qi * dR[6] + qj * dR[7]);
    const float proj = dq[0] * qr + dq[1] * qi + dq[2] * qj + dq[3] * qk;
    acc.gq[0] += (dq[0] - qr * proj) * p.qinv;
    acc.gq[1] += (dq[1] - qi * proj) * p.qinv;
    acc.gq[2] += (dq[2] - qj * proj) * p.qinv;
    acc.gq[3] += (dq[3] - qk * proj) * p.qinv;
    // T2 = J W with J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]].
    float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dJ00 += dT2[k] * c.R[k];
        dJ02 += dT2[k] * c.R[6 + k];
        dJ11 += dT2[3 + k] * c.R[3 + k];
        dJ12 += dT2[3 + k] * c.R[6 + k];
    }
    const float iz = 1.0f / p.tz, iz2 = iz * iz;
    const float fx = c.fx, fy = c.fy;
    const float dt0 = du * fx * iz - dJ02 * fx * iz2;
    const float dt1 = dv * fy * iz - dJ12 * fy * iz2;
    const float dt2 = -du * fx * p.xz * iz - dv * fy * p.yz * iz - dJ00 * fx * iz2 + dJ02 * 2.f * fx * p.xz * iz2 -
                      dJ11 * fy * iz2 + dJ12 * 2.f * fy * p.yz * iz2;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.gm[k] += c.R[k] * dt0 + c.R[3 + k] * dt1 + c.R[6 + k] * dt2;

    // Colour: dL/dSH and the view-direction term.
    const float4 rgbm = a.rgb[i];
    const uint32_t mask = __float_as_uint(rgbm.w);
    const float dr = (mask & 1u) ? 0.f : g1.z;
    const float dg = (mask & 2u) ? 0.f : g1.w;
    const float dbl = (mask & 4u) ? 0.f : g2;
    float ex = mu[0] - c.campos[0], ey = mu[1] - c.campos[1], ez = mu[2] - c.campos[2];
    const float ninv = rsqrtf(ex * ex + ey * ey + ez * ez);
    ex *= ninv; ey *= ninv; ez *= ninv;
    float Y[16];
    float3 dY[16];
    sh_basis(DEG, ex, ey, ez, Y);
    sh_basis_grad(DEG, ex, ey, ez, dY);
    float ddx = 0.f, ddy = 0.f, ddz = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float w = f[3 * k] * dr + f[3 * k + 1] * dg + f[3 * k + 2] * dbl;
        ddx += w * dY[k].x;
        ddy += w * dY[k].y;
        ddz += w * dY[k].z;
        acc.gsh[3 * k] += Y[k] * dr;
        acc.gsh[3 * k + 1] += Y[k] * dg;
        acc.gsh[3 * k + 2] += Y[k] * dbl;
    }
    const float dp = ddx * ex + ddy * ey + ddz * ez;
    acc.gm[0] += (ddx - ex * dp) * ninv;
    acc.gm[1] += (ddy - ey * dp) * ninv;
    acc.gm[2] += (ddz - ez * dp) * ninv;
    acc.go += g1.y;
    acc.du += du;
    acc.dv += dv;
}

// One thread per Gaussian of a group of frames that render the same Gaussians (views of one
// scene): the gradients of all the group's views are summed in registers and written once
// (or added to the output when accumulating).  Group g owns blocks [block_base[g],
// block_base[g+1]) and frames [frame_begin[g], frame_begin[g+1]).
template <int DEG, bool VEC, int MAXF, bool ISO>
__global__ void __launch_bounds__(256) k_preprocess_backward_t(const __grid_constant__ BwdPlan<MAXF> m) {
    constexpr int D = (DEG + 1) * (DEG + 1);
    constexpr int NF = BwdAcc<DEG>::NF;
    const int g = find_frame<MAXF>(m.block_base, m.groups, blockIdx.x);
    const int f0 = m.frame_begin[g], f1 = m.frame_begin[g + 1];
    // a batch reads its group's arguments from a shared copy (generic loads otherwise)
    __shared__ __align__(16) PreprocessBwdArgs s_args[MAXF > 1 ? MAXF : 1];
    if (MAXF > 1) {
        const int words = (int)(sizeof(PreprocessBwdArgs) / 4) * (f1 - f0);
        for (int k = threadIdx.x; k < words; k += blockDim.x)
            reinterpret_cast<uint32_t*>(s_args)[k] = reinterpret_cast<const uint32_t*>(&m.a[f0])[k];
        __syncthreads();
    }
    const PreprocessBwdArgs& a = MAXF == 1 ? m.a[0] : s_args[0];   // Gaussians and outputs shared by the group
    const int i = (int)(blockIdx.x - m.block_base[g]) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float* gsh = a.g_sh + (size_t)i * a.sh_stride * 3;
    const int row = a.sh_stride * 3;   // floats per Gaussian in the SH buffers
    BwdAcc<DEG> acc;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.gm[k] = acc.gs[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.gq[k] = 0.f;
    acc.go = acc.du = acc.dv = 0.f;
#pragma unroll
    for (int k = 0; k < NF; ++k) acc.gsh[k] = 0.f;
    bool any = false;
    float mu[3], s[3], f[NF];
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    const int nv = MAXF == 1 ? 1 : f1 - f0;   // a single frame: straight-line code
    for (int k = 0; k < nv; ++k) {
        const PreprocessBwdArgs& av = MAXF == 1 ? m.a[0] : s_args[k];
        if (av.radius[i] <= 0) continue;
        if (!any) {
            any = true;
            mu[0] = a.means[3 * i]; mu[1] = a.means[3 * i + 1]; mu[2] = a.means[3 * i + 2];
            if (ISO) {   // one scale for all axes, no rotation
                s[0] = s[1] = s[2] = a.scales[i];
                q = make_float4(1.f, 0.f, 0.f, 0.f);
            } else {
                s[0] = a.scales[3 * i]; s[1] = a.scales[3 * i + 1]; s[2] = a.scales[3 * i + 2];
                q = reinterpret_cast<const float4*>(a.quats)[i];
            }
            load_sh<D, VEC>(a.sh + (size_t)i * row, f);
        }
        bwd_view<DEG>(av, i, mu, s, q, f, acc);
    }
    if (!any && a.accumulate) return;   // no view saw it: nothing to add
    if (VEC && NF % 8 == 0 && row % 8 == 0 && (reinterpret_cast<uintptr_t>(gsh) & 31u) == 0) {
#pragma unroll
        for (int k = 0; k < NF / 8; ++k) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = acc.gsh[8 * k + e];
            if (a.accumulate) {
                float o[8];
                ld_v8(gsh + 8 * k, o);
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] += o[e];
            }
            st_v8(gsh + 8 * k, v);
        }
        if (!a.accumulate) {
            const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int k = NF; k < row; k += 8) st_v8(gsh + k, z);
        }
    } else if (VEC) {
        float4* g4 = reinterpret_cast<float4*>(gsh);
#pragma unroll
        for (int k = 0; k < NF / 4; ++k) {
            float4 v = make_float4(acc.gsh[4 * k], acc.gsh[4 * k + 1], acc.gsh[4 * k + 2], acc.gsh[4 * k + 3]);
            if (a.accumulate) {
                const float4 o4 = g4[k];
                v = make_float4(o4.x + v.x, o4.y + v.y, o4.z + v.z, o4.w + v.w);
            }
            g4[k] = v;
        }
        if (!a.accumulate)
            for (int k = NF / 4; k < row / 4; ++k) g4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
        for (int k = 0; k < 3 * D; ++k) {
            if (a.accumulate) gsh[k] += acc.gsh[k];
            else gsh[k] = acc.gsh[k];
        }
        if (!a.accumulate)
            for (int k = 3 * D; k < row; ++k) gsh[k] = 0.f;
    }
    const float4 gq = make_float4(acc.gq[0], acc.gq[1], acc.gq[2], acc.gq[3]);
    // ISO: dL/ds is the sum over the axes; there is no rotation gradient
    const float gs_iso = acc.gs[0] + acc.gs[1] + acc.gs[2];
    if (a.accumulate) {
        for (int k = 0; k < 3; ++k) a.g_means[3 * i + k] += acc.gm[k];
        if (ISO) {
            a.g_scales[i] += gs_iso;
        } else {
            for (int k = 0; k < 3; ++k) a.g_scales[3 * i + k] += acc.gs[k];
            const float4 o4 = reinterpret_cast<float4*>(a.g_quats)[i];
            reinterpret_cast<float4*>(a.g_quats)[i] = make_float4(o4.x + gq.x, o4.y + gq.y, o4.z + gq.z, o4.w + gq.w);
        }
        a.g_opacities[i] += acc.go;
        if (a.g_mean2d) { a.g_mean2d[2 * i] += acc.du; a.g_mean2d[2 * i + 1] += acc.dv; }
    } else {
        for (int k = 0; k < 3; ++k) a.g_means[3 * i + k] = acc.gm[k];
        if (ISO) {
            a.g_scales[i] = gs_iso;
        } else {
            for (int k = 0; k < 3; ++k) a.g_scales[3 * i + k] = acc.gs[k];
            reinterpret_cast<float4*>(a.g_quats)[i] = gq;
        }
        a.g_opacities[i] = acc.go;
        if (a.g_mean2d) { a.g_mean2d[2 * i] = acc.du; a.g_mean2d[2 * i + 1] = acc.dv; }
    }
}

int persistent_grid(const void* kernel, int threads) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

namespace {

// SH rows can be read and written as float4 when every row starts 16-byte aligned.
bool sh_vectorisable(const float* sh, int sh_stride, const float* gsh = nullptr) {
    const bool base = reinterpret_cast<uintptr_t>(sh) % 16 == 0 &&
                      (gsh == nullptr || reinterpret_cast<uintptr_t>(gsh) % 16 == 0);
    return base && (3 * sh_stride) % 4 == 0;
}

template <int DEG, int MAXF>
void preprocess_deg(const Multi<PreprocessArgs, MAXF>& m, bool vec, cudaStream_t s) {
    const dim3 grid(m.base[m.frames]);
    if (m.a[0].cfg.isotropic) {
        if (vec) k_preprocess_t<DEG, true, MAXF, true><<<grid, 256, 0, s>>>(m);
        else k_preprocess_t<DEG, false, MAXF, true><<<grid, 256, 0, s>>>(m);
    } else {
        if (vec) k_preprocess_t<DEG, true, MAXF, false><<<grid, 256, 0, s>>>(m);
        else k_preprocess_t<DEG, false, MAXF, false><<<grid, 256, 0, s>>>(m);
    }
}

template <int DEG, int MAXF>
void preprocess_bwd_deg(const BwdPlan<MAXF>& m, bool vec, cudaStream_t s) {
    const dim3 grid(m.block_base[m.groups]);
    if (m.a[0].cfg.isotropic) {
        if (vec) k_preprocess_backward_t<DEG, true, MAXF, true><<<grid, 256, 0, s>>>(m);
        else k_preprocess_backward_t<DEG, false, MAXF, true><<<grid, 256, 0, s>>>(m);
    } else {
        if (vec) k_preprocess_backward_t<DEG, true, MAXF, false><<<grid, 256, 0, s>>>(m);
        else k_preprocess_backward_t<DEG, false, MAXF, false><<<grid, 256, 0, s>>>(m);
    }
}

}  // namespace

// Frames of one launch share the SH degree and the SH row alignment; the caller groups them.
template <int MAXF>
cudaError_t launch_preprocess(Multi<PreprocessArgs, MAXF>& m, cudaStream_t s) {
    m.base[0] = 0;
    for (int f = 0; f < m.frames; ++f) m.base[f + 1] = m.base[f] + (uint32_t)((m.a[f].n + 255) / 256);
    if (m.base[m.frames] == 0) return cudaSuccess;
    const PreprocessArgs& a = m.a[0];
    const bool vec = sh_vectorisable(a.sh, a.sh_stride);
    switch (a.sh_degree) {
        case 0: preprocess_deg<0>(m, vec, s); break;
        case 1: preprocess_deg<1>(m, vec, s); break;
        case 2: preprocess_deg<2>(m, vec, s); break;
        default: preprocess_deg<3>(m, vec, s); break;
    }
    return cudaGetLastError();
}

template <int MAXF>
cudaError_t launch_preprocess_backward(BwdPlan<MAXF>& m, cudaStream_t s) {
    m.block_base[0] = 0;
    for (int g = 0; g < m.groups; ++g)
        m.block_base[g + 1] = m.block_base[g] + (uint32_t)((m.a[m.frame_begin[g]].n + 255) / 256);
    if (m.block_base[m.groups] == 0) return cudaSuccess;
    const PreprocessBwdArgs& a = m.a[0];
    const bool vec = sh_vectorisable(a.sh, a.sh_stride, a.g_sh);
    switch (a.sh_degree) {
        case 0: preprocess_bwd_deg<0>(m, vec, s); break;
        case 1: preprocess_bwd_deg<1>(m, vec, s); break;
        case 2: preprocess_bwd_deg<2>(m, vec, s); break;
        default: preprocess_bwd_deg<3>(m, vec, s); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_preprocess<1>(Multi<PreprocessArgs, 1>&, cudaStream_t);
template cudaError_t launch_preprocess<kMaxFrames>(Multi<PreprocessArgs, kMaxFrames>&, cudaStream_t);
template cudaError_t launch_preprocess_backward<1>(BwdPlan<1>&, cudaStream_t);
template cudaError_t launch_preprocess_backward<kMaxFrames>(BwdPlan<kMaxFrames>&, cudaStream_t);

}  // namespace gs
