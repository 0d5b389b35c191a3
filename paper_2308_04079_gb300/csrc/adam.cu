// adam.cu -- the parameter update of Algorithm 1 (Adam on the gradients of the loss), fused
// with the activations of Sec. 5.1: opacity = sigmoid(raw), scale = exp(raw).
//
// Per parameter tensor (a group): the rasterizer's gradient g is with respect to the activated
// value a = act(raw), so the raw gradient is g a (exp) or g a (1 - a) (sigmoid), then Adam
// (Kingma & Ba) with bias correction:
//   m = b1 m + (1 - b1) g_raw,  v = b2 v + (1 - b2) g_raw^2,
//   raw -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
// and the activated value of the updated raw parameter is written for the next forward pass.
// One launch covers every group; the work is HBM-bound (each element read and written once).
#include <cmath>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

struct AdamGroupK {
    float* param;
    const float* grad;
    float* m;
    float* v;
    float* activated;          // nullable: act(param) after the update
    unsigned long long n;
    float lr;
    int activation;            // GS_ACT_*
};

constexpr int kMaxGroups = 8;

constexpr int kAdamChunk = 1024;   // elements per block unit: 256 threads x 4

struct AdamArgs {
    int groups;
    unsigned long long base[kMaxGroups + 1];   // block-unit prefix of the groups
    AdamGroupK g[kMaxGroups];
    float b1, b2, eps, c1, c2;                 // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__device__ __forceinline__ float activate(float raw, int act) {
    if (act == GS_ACT_EXP) return expf(raw);
    if (act == GS_ACT_SIGMOID) return 1.0f / (1.0f + expf(-raw));
    return raw;
}

struct AdamConsts {
    float b1, b2, eps, c1, c2, lr;
    int act;
};

__device__ __forceinline__ float adam_one(const AdamConsts& k, float raw, float g, float& m, float& v, float& act_out) {
    if (k.act != GS_ACT_NONE) {
        const float a = activate(raw, k.act);
        g *= k.act == GS_ACT_EXP ? a : a * (1.0f - a);
    }
    m = k.b1 * m + (1.0f - k.b1) * g;
    v = k.b2 * v + (1.0f - k.b2) * g * g;
    const float nraw = raw - k.lr * (m / k.c1) / (sqrtf(v / k.c2) + k.eps);
    act_out = activate(nraw, k.act);
    return nraw;
}

// Block unit u of group k covers elements [(u - base[k]) * kAdamChunk, + kAdamChunk); each
// thread takes 4 consecutive elements, as one 16-byte access when the group allows it.
__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamArgs a) {
    const unsigned long long total = a.base[a.groups];
    for (unsigned long long u = blockIdx.x; u < total; u += gridDim.x) {   // block-uniform
        int k = 0;
        while (k + 1 < a.groups && a.base[k + 1] <= u) ++k;
        const AdamGroupK& gr = a.g[k];
        float* const param = gr.param;
        const float* const grad = gr.grad;
        float* const mm = gr.m;
        float* const vv = gr.v;
        float* const activated = gr.activated;
        const unsigned long long n = gr.n;
        const AdamConsts c{a.b1, a.b2, a.eps, a.c1, a.c2, gr.lr, gr.activation};
        const unsigned long long j = (u - a.base[k]) * kAdamChunk + 4ull * threadIdx.x;
        const bool vec = ((reinterpret_cast<uintptr_t>(param) | reinterpret_cast<uintptr_t>(grad) |
                           reinterpret_cast<uintptr_t>(mm) | reinterpret_cast<uintptr_t>(vv) |
                           reinterpret_cast<uintptr_t>(activated)) & 15) == 0;
        if (vec && j + 4 <= n) {
            float4 p = *reinterpret_cast<const float4*>(param + j);
            const float4 g = *reinterpret_cast<const float4*>(grad + j);
            float4 m = *reinterpret_cast<const float4*>(mm + j);
            float4 v = *reinterpret_cast<const float4*>(vv + j);
            float4 act;
            p.x = adam_one(c, p.x, g.x, m.x, v.x, act.x);
            p.y = adam_one(c, p.y, g.y, m.y, v.y, act.y);
            p.z = adam_one(c, p.z, g.z, m.z, v.z, act.z);
            p.w = adam_one(c, p.w, g.w, m.w, v.w, act.w);
            *reinterpret_cast<float4*>(param + j) = p;
            *reinterpret_cast<float4*>(mm + j) = m;
            *reinterpret_cast<float4*>(vv + j) = v;
            if (activated) *reinterpret_cast<float4*>(activated + j) = act;
        } else {
            for (unsigned long long e = j; e < j + 4 && e < n; ++e) {
                float m = mm[e], v = vv[e], act;
                param[e] = adam_one(c, param[e], grad[e], m, v, act);
                mm[e] = m;
                vv[e] = v;
                if (activated) activated[e] = act;
            }
        }
    }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_adam_step(const gs_adam_group* groups, int count, float beta1, float beta2, float eps,
                                 int step, cudaStream_t s) {
    if (!groups || count < 1 || count > kMaxGroups || step < 1) return GS_ERR_INVALID_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f)) return GS_ERR_INVALID_ARG;
    AdamArgs a;
    a.groups = count;
    a.base[0] = 0;
    for (int k = 0; k < count; ++k) {
        const gs_adam_group& g = groups[k];
        if (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v)) return GS_ERR_INVALID_ARG;
        if (g.activation != GS_ACT_NONE && g.activation != GS_ACT_EXP && g.activation != GS_ACT_SIGMOID)
            return GS_ERR_INVALID_ARG;
        a.g[k] = AdamGroupK{g.param, g.grad, g.m, g.v, g.activated, g.n, g.lr, g.activation};
        a.base[k + 1] = a.base[k] + (g.n + kAdamChunk - 1) / kAdamChunk;
    }
    a.b1 = beta1;
    a.b2 = beta2;
    a.eps = eps;
    a.c1 = (float)(1.0 - std::pow((double)beta1, step));
    a.c2 = (float)(1.0 - std::pow((double)beta2, step));
    if (a.base[count] == 0) return GS_OK;
    const unsigned long long blocks = a.base[count];
    const int cap = persistent_grid((const void*)k_adam, 256) * 8;
    k_adam<<<(int)(blocks < (unsigned long long)cap ? blocks : cap), 256, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
