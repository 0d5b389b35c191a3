// gs_device.cuh -- device-side helpers shared by the rasterizer kernels (sm_103a).
//
// Kernel-side camera / constants, the tile rectangle rule, the exact fp32 evaluation of a
// splat's alpha (used identically by the forward and the backward kernels so that their
// skip / clamp decisions agree bit for bit), the real SH basis of bands 0..3 and small
// warp/block primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

// Kernel-side camera: the gs_camera fields plus values derived once on the host.
struct CamK {
    int W, H;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float near_z;
    float campos[3];   // camera centre in world space, -R^T t
    float lim_x, lim_y;  // guard * tan(fov_x / 2), guard * tan(fov_y / 2)
    int tile_w, tile_h, tiles_x, tiles_y;
};

struct CfgK {
    float alpha_min, alpha_max, T_min, dilation, extent;
    int radius_max;
    int grad_limit;   // > 0: gradients for the grad_limit front-most blended splats of a pixel only
    int isotropic;    // 1: one scale per Gaussian, no rotation
};

constexpr int kRadiusMax = 1 << 24;   // screen radius clamp (pixels)

// Status-block flags (gs_device_status.flags).
constexpr uint32_t kFlagCapacity = 1u;
constexpr uint32_t kFlagTimeout = 2u;
constexpr uint32_t kFlagInternal = 4u;   // a consistency check failed (see GS_ERR_INTERNAL)
// Any of these: the later binning kernels write nothing.
constexpr uint32_t kFlagAbort = kFlagCapacity | kFlagTimeout | kFlagInternal;

// Upper bound on polling iterations of a device spin-wait when the caller gives none (the
// binning kernels take cfg.spin_limit); the waiting thread then sets kFlagTimeout and gives up
// (results invalid, no hang).
constexpr uint32_t kSpinLimit = GS_DEFAULT_SPIN_LIMIT;

// GS_DEBUG builds (libgs_gb300_debug.so) add bounds checks on instance and range indices that a
// correct run never fails; a failed check sets kFlagInternal (GS_ERR_INTERNAL) in the status
// block and the access is skipped or clamped, so the kernel neither traps nor reads or writes
// out of bounds.  Release builds keep the clamps without reporting.
#ifndef GS_DEBUG
#define GS_DEBUG 0
#endif
// A check that fails after a capacity overflow or a timed-out wait reports nothing: the data
// it looked at were never produced, and the status block already says why.
__device__ __forceinline__ void debug_fail(gs_device_status* st) {
    if (GS_DEBUG && st && !(*reinterpret_cast<volatile const uint32_t*>(&st->flags) & (kFlagCapacity | kFlagTimeout)))
        atomicOr(&st->flags, kFlagInternal);
}

// 2^x with the hardware approximation (PTX ex2.approx.ftz.f32), the one transcendental of the
// blend; a subnormal result flushes to zero, which never matters there (o G below 1/255 is
// skipped before it is used).  The forward and the backward both evaluate alpha with it, and the
// ex2 throughput microbenchmark measures it.
__device__ __forceinline__ float hw_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x with the hardware approximation (PTX rcp.approx.ftz.f32); the render backward divides only
// by 1 - alpha >= 0.01.
__device__ __forceinline__ float hw_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// Exponent of the 2D Gaussian at offset d = pixel centre - mean:
//   power = -(1/2) d^T Q d,  Q = Sigma'^-1 = [[a, b], [b, c]] (the conic),
// evaluated through the lower Cholesky factor Q = L L^T, L = [[l11, 0], [l21, l22]]:
//   p = l11 dx + l21 dy,  q = l22 dy,  power = -(p^2 + q^2) / 2.
// This is the same quadratic form as -(a dx^2 + c dy^2)/2 - b dx dy, but its fp32 rounding
// error grows like sqrt(lambda_max / lambda_min) of Sigma' instead of lambda_max / lambda_min
// (the expanded form cancels along the major axis of elongated splats).  With
// Sigma' = [[A, B], [B, C]] and D = det Sigma': l11 = sqrt(C / D), l21 = -B / sqrt(C D),
// l22 = 1 / sqrt(C).  Written with explicit round-to-nearest intrinsics so that the forward
// and backward kernels evaluate it with the same operation sequence.
__device__ __forceinline__ float splat_power(float dx, float dy, float4 L, float& p, float& q) {
    p = __fmaf_rn(L.y, dy, __fmul_rn(L.x, dx));
    q = __fmul_rn(L.z, dy);
    return __fmul_rn(-0.5f, __fmaf_rn(p, p, __fmul_rn(q, q)));
}

// Offset of a tile's first pixel centre from a splat mean stored as an unevaluated sum
// m = hi + lo (the preprocess stores u and v that way): (x0 + 0.5 - hi) - lo.  The first difference is exact
// whenever the mean is near the tile (Sterbenz), so a pixel's offset lx + o is accurate to a
// few units in the last place of the offset itself rather than of the absolute coordinate.
__device__ __forceinline__ float tile_offset(int x0, float hi, float lo) {
    return __fsub_rn(__fsub_rn((float)x0 + 0.5f, hi), lo);
}

// ---- double-float (unevaluated sum of two fp32) arithmetic, error-free transforms --------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// r . m + t in double-float (compensated dot product).
__device__ __forceinline__ DF dot3_plus(const float* r, const float* m, float t) {
    DF acc = two_prod(r[0], m[0]);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        const DF p = two_prod(r[k], m[k]);
        const DF s = two_sum(acc.hi, p.hi);
        acc = {s.hi, __fadd_rn(__fadd_rn(s.lo, acc.lo), p.lo)};
    }
    const DF s = two_sum(acc.hi, t);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, acc.lo));
}

// a / b in double-float.
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    float r = __fmaf_rn(-q1, b.hi, a.hi);
    r = __fadd_rn(r, a.lo);
    r = __fmaf_rn(-q1, b.lo, r);
    const float q2 = __fdiv_rn(r, b.hi);
    return fast_two_sum(q1, q2);
}

// f * q + c in double-float.
__device__ __forceinline__ DF df_mul_add(float f, DF q, float c) {
    DF p = two_prod(f, q.hi);
    p.lo = __fmaf_rn(f, q.lo, p.lo);
    const DF s = two_sum(p.hi, c);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, p.lo));
}

// floor(hi + lo) for a normalised double-float.
__device__ __forceinline__ int df_floor(float hi, float lo) {
    const float f = floorf(hi);
    return (int)f - ((f == hi && lo < 0.f) ? 1 : 0);
}

// Tile rectangle [x0, x1) x [y0, y1) of a splat with screen mean (u, v) and integer radius r:
// x0 = floor((u - r) / tile_w), x1 = floor((u + r) / tile_w) + 1, clamped to the tile grid.
// r is an integer, so floor((u -/+ r) / tile) = floor_div(floor(u) -/+ r, tile) exactly.
// The mean is the double-float m = (u_hi, v_hi, u_lo, v_lo).
__device__ __forceinline__ bool tile_rect(float4 m, int r, const CamK& c, int& x0, int& x1, int& y0, int& y1) {
    const int fu = df_floor(m.x, m.z), fv = df_floor(m.y, m.w);
    x0 = clampi(floor_div(fu - r, c.tile_w), 0, c.tiles_x);
    x1 = clampi(floor_div(fu + r, c.tile_w) + 1, 0, c.tiles_x);
    y0 = clampi(floor_div(fv - r, c.tile_h), 0, c.tiles_y);
    y1 = clampi(floor_div(fv + r, c.tile_h) + 1, 0, c.tiles_y);
    return x0 < x1 && y0 < y1;
}

// ---- tiles a splat can reach ---------------------------------------------------------------
// A pixel at offset d from the mean is blended only if o exp(-d^T Q d / 2) >= alpha_min, i.e.
// d^T Q d <= tau = 2 ln(o / alpha_min) (Q = Sigma'^-1 = L L^T).  Inside the 3-sigma tile rectangle
// only tiles holding such a pixel are instantiated; every other tile would skip the splat at
// every pixel, so the image and the gradients are those of the full rectangle.  Per tile row,
// the pixel centres of the row form a band of offsets y in [ya, yb]; the ellipse d^T Q d <= tau
// restricted to the band spans x in [xa, xb], where the right end x(y) = (sqrt(tau - (l22 y)^2) -
// l21 y) / l11 is concave in y and is largest at the band-clamped y of the ellipse's rightmost
// point (symmetrically for the left end).  tau is widened by 2^-10 (relative and absolute) and
// the interval by 0.01 px so that rounding never drops a tile the per-pixel test keeps.  Only
// correctly rounded operations are used, in a fixed order, so the rule is reproducible
// bit for bit.
struct Reach {
    float tm, ylim, ystar, inv11, l21, l22;
    bool any;
};

__device__ __forceinline__ Reach reach_setup(float4 L, float tau) {
    Reach e;
    e.l21 = L.y;
    e.l22 = L.z;
    e.tm = __fadd_rn(__fmul_rn(tau, 1.0f + 0.0009765625f), 0.0009765625f);
    e.any = e.tm > 0.f;
    e.inv11 = __fdiv_rn(1.0f, L.x);
    const float sq = __fsqrt_rn(e.tm);
    e.ylim = __fdiv_rn(sq, e.l22);
    const float a = __fmul_rn(L.x, e.l22);
    const float qi00 = __fdiv_rn(__fadd_rn(__fmul_rn(e.l21, e.l21), __fmul_rn(e.l22, e.l22)), __fmul_rn(a, a));
    const float qi01 = __fdiv_rn(-e.l21, __fmul_rn(a, e.l22));
    e.ystar = __fmul_rn(qi01, __fsqrt_rn(__fdiv_rn(e.tm, qi00)));
    return e;
}

__device__ __forceinline__ float reach_x(const Reach& e, float y, float sgn) {
    const float q = __fmul_rn(e.l22, y);
    const float h = __fsqrt_rn(fmaxf(__fsub_rn(e.tm, __fmul_rn(q, q)), 0.0f));
    return __fmul_rn(__fsub_rn(__fmul_rn(sgn, h), __fmul_rn(e.l21, y)), e.inv11);
}

// Tiles [txa, txb) of tile row ty (inside the rectangle columns [x0, x1)) that the splat with
// screen mean (u, v) can reach; false when none.  Tile widths are powers of two (tw_log2).
__device__ __forceinline__ bool reach_row(const Reach& e, float u, float v, int ty, int tw_log2, int th, int x0,
                                          int x1, int& txa, int& txb) {
    if (!e.any) return false;
    float ya = __fsub_rn(__fadd_rn((float)(ty * th), 0.5f), v);
    float yb = __fsub_rn(__fsub_rn((float)(ty * th + th), 0.5f), v);
    ya = fmaxf(ya, -e.ylim);
    yb = fminf(yb, e.ylim);
    if (ya > yb) return false;
    const float yr = fminf(fmaxf(e.ystar, ya), yb);
    const float yl = fminf(fmaxf(-e.ystar, ya), yb);
    const float xb = __fadd_rn(reach_x(e, yr, 1.0f), 0.01f);
    const float xa = __fsub_rn(reach_x(e, yl, -1.0f), 0.01f);
    // pixel columns px with px + 0.5 - u in [xa, xb]
    const float fa = ceilf(__fsub_rn(__fadd_rn(u, xa), 0.5f));
    const float fb = floorf(__fsub_rn(__fadd_rn(u, xb), 0.5f));
    const float lim = 1048576.0f;
    const int pa = (int)fminf(fmaxf(fa, -lim), lim), pb = (int)fminf(fmaxf(fb, -lim), lim);
    if (pb < pa) return false;
    txa = max(x0, pa >> tw_log2);          // arithmetic shift: floor division
    txb = min(x1, (pb >> tw_log2) + 1);
    return txa < txb;
}

// alpha = min(alpha_max, o * G), G = exp(power).  Returns o * G (unclamped) in oG.
__device__ __forceinline__ float splat_alpha(float power, float o, float alpha_max, float& G, float& oG) {
    G = __expf(power);
    oG = __fmul_rn(o, G);
    return fminf(alpha_max, oG);
}

// Real spherical harmonics, bands 0..3, Condon-Shortley phase, unit direction (x, y, z),
// coefficient index k = l^2 + l + m:
//   Y0 = 1/(2 sqrt(pi));  Y1..3 = sqrt(3/(4 pi)) (-y, z, -x);
//   Y4..8 = sqrt(15/pi)/2 xy, -sqrt(15/pi)/2 yz, sqrt(5/pi)/4 (3z^2-1), -sqrt(15/pi)/2 xz,
//           sqrt(15/pi)/4 (x^2-y^2);
//   Y9..15 = -sqrt(35/(2pi))/4 y(3x^2-y^2), sqrt(105/pi)/2 xyz, -sqrt(21/(2pi))/4 y(5z^2-1),
//            sqrt(7/pi)/4 z(5z^2-3), -sqrt(21/(2pi))/4 x(5z^2-1), sqrt(105/pi)/4 z(x^2-y^2),
//            -sqrt(35/(2pi))/4 x(x^2-3y^2).
struct SH {
    static constexpr float C0 = 0.28209479177387814f;
    static constexpr float C1 = 0.4886025119029199f;
    static constexpr float C2a = 1.0925484305920792f;
    static constexpr float C2b = 0.31539156525252005f;
    static constexpr float C2c = 0.5462742152960396f;
    static constexpr float C3a = 0.5900435899266435f;
    static constexpr float C3b = 2.890611442640554f;
    static constexpr float C3c = 0.4570457994644658f;
    static constexpr float C3d = 0.3731763325901154f;
    static constexpr float C3e = 1.445305721320277f;
};

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
    Y[0] = SH::C0;
    if (deg < 1) return;
    Y[1] = -SH::C1 * y;
    Y[2] = SH::C1 * z;
    Y[3] = -SH::C1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH::C2a * x * y;
    Y[5] = -SH::C2a * y * z;
    Y[6] = SH::C2b * (3.0f * zz - 1.0f);
    Y[7] = -SH::C2a * x * z;
    Y[8] = SH::C2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -SH::C3a * y * (3.0f * xx - yy);
    Y[10] = SH::C3b * x * y * z;
    Y[11] = -SH::C3c * y * (5.0f * zz - 1.0f);
    Y[12] = SH::C3d * z * (5.0f * zz - 3.0f);
    Y[13] = -SH::C3c * x * (5.0f * zz - 1.0f);
    Y[14] = SH::C3e * z * (xx - yy);
    Y[15] = -SH::C3a * x * (xx - 3.0f * yy);
}

// Gradient of the polynomials above w.r.t. (x, y, z): dY[k] = (dYk/dx, dYk/dy, dYk/dz).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float3* dY) {
    dY[0] = make_float3(0.f, 0.f, 0.f);
    if (deg < 1) return;
    dY[1] = make_float3(0.f, -SH::C1, 0.f);
    dY[2] = make_float3(0.f, 0.f, SH::C1);
    dY[3] = make_float3(-SH::C1, 0.f, 0.f);
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[4] = make_float3(SH::C2a * y, SH::C2a * x, 0.f);
    dY[5] = make_float3(0.f, -SH::C2a * z, -SH::C2a * y);
    dY[6] = make_float3(0.f, 0.f, 6.0f * SH::C2b * z);
    dY[7] = make_float3(-SH::C2a * z, 0.f, -SH::C2a * x);
    dY[8] = make_float3(2.0f * SH::C2c * x, -2.0f * SH::C2c * y, 0.f);
    if (deg < 3) return;
    dY[9] = make_float3(-6.0f * SH::C3a * x * y, -3.0f * SH::C3a * (xx - yy), 0.f);
    dY[10] = make_float3(SH::C3b * y * z, SH::C3b * x * z, SH::C3b * x * y);
    dY[11] = make_float3(0.f, -SH::C3c * (5.0f * zz - 1.0f), -10.0f * SH::C3c * y * z);
    dY[12] = make_float3(0.f, 0.f, SH::C3d * (15.0f * zz - 3.0f));
    dY[13] = make_float3(-SH::C3c * (5.0f * zz - 1.0f), 0.f, -10.0f * SH::C3c * x * z);
    dY[14] = make_float3(2.0f * SH::C3e * x * z, -2.0f * SH::C3e * y * z, SH::C3e * (xx - yy));
    dY[15] = make_float3(-3.0f * SH::C3a * (xx - yy), 6.0f * SH::C3a * x * y, 0.f);
}

// ---- warp / block primitives ---------------------------------------------------------

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x a multiple of 32, <= 1024).
// scratch: >= 33 elements of shared memory.  Returns the exclusive prefix; *total gets the sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* scratch, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? scratch[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < nw) scratch[lane] = wi - w;
        if (lane == nw - 1) scratch[32] = wi;
    }
    __syncthreads();
    T r = inc - v + scratch[warp];
    *total = scratch[32];
    __syncthreads();
    return r;
}

}  // namespace gs
