// loss.cu -- the training loss of Sec. 5.1: L = (1 - lambda) L1 + lambda (1 - SSIM), and its
// gradient with respect to the rendered image.
//
// SSIM (Wang et al. 2004) per channel with an 11x11 Gaussian window (sigma 1.5, normalised),
// C1 = 0.01^2, C2 = 0.03^2, zero padding outside the image ("same" size), averaged over all
// pixels and channels; L1 is the mean absolute difference.  With the window moments at pixel p
//   mx = w*x, my = w*y, Exx = w*x^2, Eyy = w*y^2, Exy = w*(x y)   (w* = windowed sum)
//   A1 = 2 mx my + C1, A2 = 2 (Exy - mx my) + C2, B1 = mx^2 + my^2 + C1,
//   B2 = Exx - mx^2 + Eyy - my^2 + C2, S = A1 A2 / (B1 B2),
// the derivative of S(p) with respect to the image x at q is
//   w(p - q) [dS/dmx(p) + 2 x(q) dS/dExx(p) + y(q) dS/dExy(p)],
//   dS/dmx = 2 my (A2 - A1) / (B1 B2) - 2 mx S (B2 - B1) / (B1 B2),
//   dS/dExx = -S / B2,  dS/dExy = 2 A1 / (B1 B2),
// so dSSIM/dx = (w * a) + 2 x (w * b) + y (w * c) with the coefficient maps a, b, c of
// dS/dmx, dS/dExx, dS/dExy (w is symmetric).  Pass 1 computes the moments, S, L1 and the
// coefficient maps; pass 2 windows the coefficient maps and forms dL/dx.  Both passes are
// separable 11-tap convolutions on 32x32 output tiles (the three channels in turn), staged with
// their halo in shared memory; a thread computes consecutive outputs of each 1-D window from
// registers, reading each input once for all of them.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

constexpr int kWin = 11, kHalf = 5;
constexpr int kTile = 32;
constexpr int kIn = kTile + 2 * kHalf;   // 42
constexpr int kRowsPer = 4;              // output rows per thread in the vertical passes (256 threads)
constexpr int kColsPer = 2;              // output columns per thread in the horizontal passes
static_assert(kTile * kTile == 256 * kRowsPer, "one row group per thread");

// Normalised 1-D Gaussian window, sigma 1.5 (the 2-D window is its outer product), computed by
// every block into shared memory.
__device__ __forceinline__ void load_window(float* w) {
    if (threadIdx.x < kWin) {
        double sum = 0.0;
        for (int k = 0; k < kWin; ++k) sum += exp(-(double)((k - kHalf) * (k - kHalf)) / (2.0 * 1.5 * 1.5));
        const int t = (int)threadIdx.x - kHalf;
        w[threadIdx.x] = (float)(exp(-(double)(t * t) / (2.0 * 1.5 * 1.5)) / sum);
    }
}

struct LossArgs {
    const float* img;     // [3, H, W]
    const float* target;  // [3, H, W]
    int W, H;
    float lambda;
    float* coef;          // [3 channels][3 maps][H * W]: dS/dmx, dS/dExx, dS/dExy
    double* partial;      // [blocks][2]: sums of S and |x - y| of every tile
    unsigned int* done;   // block counter of pass 1 (zeroed)
    float* out_loss;      // [3]: L, L1, mean SSIM
    float* dL_dimg;       // [3, H, W]
};

__device__ __forceinline__ float load0(const float* p, int W, int H, int x, int y) {
    return (x >= 0 && x < W && y >= 0 && y < H) ? p[(size_t)y * W + x] : 0.f;
}

// Pass 1: window moments, SSIM, L1 and the coefficient maps of one 32x32 tile, all channels.
__global__ void __launch_bounds__(256) k_ssim_forward(LossArgs a) {
    __shared__ float s_x[kIn][kIn + 1], s_y[kIn][kIn + 1];
    __shared__ float s_h[5][kIn][kTile + 1];   // horizontally windowed x, y, x^2, y^2, x y
    __shared__ double s_red[2][8];
    __shared__ float c_win[kWin];
    load_window(c_win);
    const int tid = threadIdx.x;
    const int bx = blockIdx.x * kTile, by = blockIdx.y * kTile;
    const size_t P = (size_t)a.W * a.H;
    __syncthreads();
    float w[kWin];   // the window in registers
#pragma unroll
    for (int t = 0; t < kWin; ++t) w[t] = c_win[t];
    // per-thread sums of at most 3 x 4 terms in [-1, 1] and [0, 1] stay in fp32; blocks and the
    // grid sum in fp64
    float sum_s = 0.f, sum_l1 = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
    const float* x = a.img + ch * P;
    const float* y = a.target + ch * P;
    __syncthreads();   // the previous channel's reads of s_x, s_y and s_h are done
    for (int k = tid; k < kIn * kIn; k += blockDim.x) {
        const int r = k / kIn, cc = k % kIn;
        s_x[r][cc] = load0(x, a.W, a.H, bx + cc - kHalf, by + r - kHalf);
        s_y[r][cc] = load0(y, a.W, a.H, bx + cc - kHalf, by + r - kHalf);
    }
    __syncthreads();
    // horizontal windows: a thread takes kColsPer consecutive columns of one row, reading the
    // kColsPer + 10 inputs they need once
    for (int k = tid; k < kIn * (kTile / kColsPer); k += blockDim.x) {
        const int r = k / (kTile / kColsPer), c0 = (k % (kTile / kColsPer)) * kColsPer;
        float h[5][kColsPer];
#pragma unroll
        for (int mm = 0; mm < 5; ++mm)
#pragma unroll
            for (int j = 0; j < kColsPer; ++j) h[mm][j] = 0.f;
#pragma unroll
        for (int cc = 0; cc < kColsPer + kWin - 1; ++cc) {
            const float xv = s_x[r][c0 + cc], yv = s_y[r][c0 + cc];
            const float xx = xv * xv, yy = yv * yv, xy = xv * yv;
#pragma unroll
            for (int j = 0; j < kColsPer; ++j)
                if (cc - j >= 0 && cc - j < kWin) {
                    const float wt = w[cc - j];
                    h[0][j] += wt * xv;
                    h[1][j] += wt * yv;
                    h[2][j] += wt * xx;
                    h[3][j] += wt * yy;
                    h[4][j] += wt * xy;
                }
        }
#pragma unroll
        for (int mm = 0; mm < 5; ++mm)
#pragma unroll
            for (int j = 0; j < kColsPer; ++j) s_h[mm][r][c0 + j] = h[mm][j];
    }
    __syncthreads();
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    // vertical windows: a thread takes kRowsPer consecutive rows of one column, reading the
    // kRowsPer + 10 rows they need once per map
    {
        const int cc = tid % kTile, r0 = (tid / kTile) * kRowsPer;
        float mom[5][kRowsPer];
#pragma unroll
        for (int mm = 0; mm < 5; ++mm) {
#pragma unroll
            for (int j = 0; j < kRowsPer; ++j) mom[mm][j] = 0.f;
#pragma unroll
            for (int rr = 0; rr < kRowsPer + kWin - 1; ++rr) {
                const float v = s_h[mm][r0 + rr][cc];
#pragma unroll
                for (int j = 0; j < kRowsPer; ++j)
                    if (rr - j >= 0 && rr - j < kWin) mom[mm][j] += w[rr - j] * v;
            }
        }
#pragma unroll
        for (int j = 0; j < kRowsPer; ++j) {
            const int r = r0 + j;
            const int px = bx + cc, py = by + r;
            if (px >= a.W || py >= a.H) continue;
            const float mx = mom[0][j], my = mom[1][j], exx = mom[2][j], eyy = mom[3][j], exy = mom[4][j];
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * (exy - mx * my) + C2;
            const float B1 = mx * mx + my * my + C1, B2 = (exx - mx * mx) + (eyy - my * my) + C2;
            const float inv = 1.f / (B1 * B2);
            const float S = A1 * A2 * inv;
            const size_t q = (size_t)py * a.W + px;
            float* coef = a.coef + (size_t)ch * 3 * P;
            coef[q] = 2.f * my * (A2 - A1) * inv - 2.f * mx * S * (B2 - B1) * inv;
            coef[P + q] = -S / B2;
            coef[2 * P + q] = 2.f * A1 * inv;
            sum_s += S;
            sum_l1 += fabsf(s_x[r + kHalf][cc + kHalf] - s_y[r + kHalf][cc + kHalf]);
        }
    }
    }
    // block sums (fixed order), then the last block adds the tiles in index order
    double d_s = sum_s, d_l1 = sum_l1;
    for (int o = 16; o > 0; o >>= 1) {
        d_s += __shfl_xor_sync(0xffffffffu, d_s, o);
        d_l1 += __shfl_xor_sync(0xffffffffu, d_l1, o);
    }
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = d_s;
        s_red[1][tid >> 5] = d_l1;
    }
    __syncthreads();
    const int blocks = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    __shared__ bool s_last;
    if (tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += s_red[0][w]; s1 += s_red[1][w]; }
        a.partial[2 * bid] = s0;
        a.partial[2 * bid + 1] = s1;
        __threadfence();
        s_last = atomicAdd(a.done, 1u) == (unsigned)(blocks - 1);
    }
    __syncthreads();
    if (s_last) {   // the last block: its threads sum the tiles' partials in a fixed order
        __threadfence();
        double p0 = 0.0, p1 = 0.0;
        for (int b = tid; b < blocks; b += blockDim.x) {
            p0 += __ldcg(a.partial + 2 * b);
            p1 += __ldcg(a.partial + 2 * b + 1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            p0 += __shfl_xor_sync(0xffffffffu, p0, o);
            p1 += __shfl_xor_sync(0xffffffffu, p1, o);
        }
        __syncthreads();
        if ((tid & 31) == 0) {
            s_red[0][tid >> 5] = p0;
            s_red[1][tid >> 5] = p1;
        }
        __syncthreads();
    }
    if (s_last && tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            s0 += s_red[0][k];
            s1 += s_red[1][k];
        }
        const double n = 3.0 * (double)P;
        const double ssim = s0 / n, l1 = s1 / n;
        a.out_loss[0] = (float)((1.0 - a.lambda) * l1 + a.lambda * (1.0 - ssim));
        a.out_loss[1] = (float)l1;
        a.out_loss[2] = (float)ssim;
    }
}

// Pass 2: dL/dx = (1 - lambda) sign(x - y) / N - lambda / N [(w * a) + 2 x (w * b) + y (w * c)].
__global__ void __launch_bounds__(256) k_ssim_backward(LossArgs a) {
    __shared__ float s_c[3][kIn][kIn + 1];
    __shared__ float s_h[3][kIn][kTile + 1];
    __shared__ float c_win[kWin];
    load_window(c_win);
    const int tid = threadIdx.x;
    const int bx = blockIdx.x * kTile, by = blockIdx.y * kTile;
    const size_t P = (size_t)a.W * a.H;
    const float invN = 1.0f / (3.0f * (float)P);
    __syncthreads();
    float w[kWin];   // the window in registers
#pragma unroll
    for (int t = 0; t < kWin; ++t) w[t] = c_win[t];
    for (int ch = 0; ch < 3; ++ch) {
    const float* coef = a.coef + (size_t)ch * 3 * P;
    __syncthreads();   // the previous channel's reads of s_c and s_h are done
    for (int k = tid; k < kIn * kIn; k += blockDim.x) {
        const int r = k / kIn, cc = k % kIn;
#pragma unroll
        for (int mmap = 0; mmap < 3; ++mmap)
            s_c[mmap][r][cc] = load0(coef + mmap * P, a.W, a.H, bx + cc - kHalf, by + r - kHalf);
    }
    __syncthreads();
    for (int k = tid; k < kIn * (kTile / kColsPer); k += blockDim.x) {
        const int r = k / (kTile / kColsPer), c0 = (k % (kTile / kColsPer)) * kColsPer;
        float h[3][kColsPer];
#pragma unroll
        for (int mm = 0; mm < 3; ++mm)
#pragma unroll
            for (int j = 0; j < kColsPer; ++j) h[mm][j] = 0.f;
#pragma unroll
        for (int cc = 0; cc < kColsPer + kWin - 1; ++cc) {
#pragma unroll
            for (int mm = 0; mm < 3; ++mm) {
                const float v = s_c[mm][r][c0 + cc];
#pragma unroll
                for (int j = 0; j < kColsPer; ++j)
                    if (cc - j >= 0 && cc - j < kWin) h[mm][j] += w[cc - j] * v;
            }
        }
#pragma unroll
        for (int mm = 0; mm < 3; ++mm)
#pragma unroll
            for (int j = 0; j < kColsPer; ++j) s_h[mm][r][c0 + j] = h[mm][j];
    }
    __syncthreads();
        {
            const int cc = tid % kTile, r0 = (tid / kTile) * kRowsPer;
            float acc[3][kRowsPer];
#pragma unroll
            for (int mm = 0; mm < 3; ++mm) {
#pragma unroll
                for (int j = 0; j < kRowsPer; ++j) acc[mm][j] = 0.f;
#pragma unroll
                for (int rr = 0; rr < kRowsPer + kWin - 1; ++rr) {
                    const float v = s_h[mm][r0 + rr][cc];
#pragma unroll
                    for (int j = 0; j < kRowsPer; ++j)
                        if (rr - j >= 0 && rr - j < kWin) acc[mm][j] += w[rr - j] * v;
                }
            }
#pragma unroll
            for (int j = 0; j < kRowsPer; ++j) {
                const int r = r0 + j;
                const int px = bx + cc, py = by + r;
                if (px >= a.W || py >= a.H) continue;
                const size_t q = (size_t)py * a.W + px;
                const float xv = a.img[ch * P + q], yv = a.target[ch * P + q];
                const float d = xv - yv;
                const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                const float dssim = acc[0][j] + 2.f * xv * acc[1][j] + yv * acc[2][j];
                a.dL_dimg[ch * P + q] = (1.f - a.lambda) * invN * sgn - a.lambda * invN * dssim;
            }
        }
    }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" size_t gs_loss_workspace_size(int width, int height) {
    if (width <= 0 || height <= 0 || width > 32768 || height > 32768) return 0;
    const size_t P = (size_t)width * height;
    const size_t blocks = (size_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
    return 256 + ((9 * P * sizeof(float) + 255) / 256) * 256 + blocks * 2 * sizeof(double);
}

extern "C" gs_status gs_loss_l1_dssim(const float* img, const float* target, int width, int height, float lambda,
                                     void* ws, size_t ws_bytes, float* out_loss, float* dL_dimg, cudaStream_t s) {
    const size_t need = gs_loss_workspace_size(width, height);
    if (!need || !img || !target || !ws || !out_loss || !dL_dimg || ws_bytes < need) return GS_ERR_INVALID_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % 256) return GS_ERR_INVALID_ARG;
    const size_t P = (size_t)width * height;
    char* base = static_cast<char*>(ws);
    LossArgs a;
    a.img = img;
    a.target = target;
    a.W = width;
    a.H = height;
    a.lambda = lambda;
    a.done = reinterpret_cast<unsigned int*>(base);
    a.coef = reinterpret_cast<float*>(base + 256);
    a.partial = reinterpret_cast<double*>(base + 256 + ((9 * P * sizeof(float) + 255) / 256) * 256);
    a.out_loss = out_loss;
    a.dL_dimg = dL_dimg;
    if (cudaMemsetAsync(a.done, 0, sizeof(unsigned int), s) != cudaSuccess) return GS_ERR_CUDA;
    const dim3 grid((width + kTile - 1) / kTile, (height + kTile - 1) / kTile);
    k_ssim_forward<<<grid, 256, 0, s>>>(a);
    k_ssim_backward<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
