// peaks.cu -- throughput microbenchmarks that anchor the roofline of the issue-bound render
// kernels, whose work per (pixel, splat) pair is FP32 fused multiply-adds plus one 2^x: the
// measured FP32 FMA rate (2 flops per lane per instruction) and the rate of the render's 2^x
// instruction (hw_exp2, PTX ex2.approx.ftz.f32) on this GPU.
//
// Every thread runs kChains independent dependency chains, kUnroll steps per loop trip, so each
// SM sub-partition always has ready instructions despite the pipeline latency.  The chains'
// sum is stored only under a condition that the arithmetic can never meet (the inputs keep
// every value finite and non-negative), which keeps all of them live without memory traffic.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

constexpr int kPeakThreads = 1024;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(int iters, float b, float c, float* sink) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s < 0.f) sink[blockIdx.x] = s;   // b, c >= 0: never taken
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(int iters, float* sink) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)((threadIdx.x + k) & 255) * (1.0f / 256.0f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = hw_exp2(-a[k]);   // stays in (0.5, 1]
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s < 0.f) sink[blockIdx.x] = s;   // never taken
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_peak_fma(int blocks, int iters, float* sink, cudaStream_t s) {
    if (blocks <= 0 || iters <= 0 || !sink) return GS_ERR_INVALID_ARG;
    k_peak_fma<<<blocks, kPeakThreads, 0, s>>>(iters, 0.999f, 1e-4f, sink);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status gs_peak_ex2(int blocks, int iters, float* sink, cudaStream_t s) {
    if (blocks <= 0 || iters <= 0 || !sink) return GS_ERR_INVALID_ARG;
    k_peak_ex2<<<blocks, kPeakThreads, 0, s>>>(iters, sink);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" unsigned long long gs_peak_ops(int blocks, int iters) {
    return (unsigned long long)blocks * kPeakThreads * (unsigned long long)iters * kUnroll * kChains;
}
