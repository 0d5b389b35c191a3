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

struct AdamArgs {
    int groups;
    unsigned long long base[kMaxGroups + 1];   // element prefix of the groups
    AdamGroupK g[kMaxGroups];
    float b1, b2, eps, c1, c2;                 // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__device__ __forceinline__ float activate(float raw, int act) {
    if (act == GS_ACT_EXP) return expf(raw);
    if (act == GS_ACT_SIGMOID) return 1.0f / (1.0f + expf(-raw));
    return raw;
}

__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamArgs a) {
    const unsigned long long total = a.base[a.groups];
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        int k = 0;
        while (k + 1 < a.groups && a.base[k + 1] <= i) ++k;
        const AdamGroupK& gr = a.g[k];
        const unsigned long long j = i - a.base[k];
        const float raw = gr.param[j];
        float g = gr.grad[j];
        if (gr.activation != GS_ACT_NONE) {
            const float act = activate(raw, gr.activation);
            g *= gr.activation == GS_ACT_EXP ? act : act * (1.0f - act);
        }
        const float m = a.b1 * gr.m[j] + (1.0f - a.b1) * g;
        const float v = a.b2 * gr.v[j] + (1.0f - a.b2) * g * g;
        gr.m[j] = m;
        gr.v[j] = v;
        const float upd = gr.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
        const float nraw = raw - upd;
        gr.param[j] = nraw;
        if (gr.activated) gr.activated[j] = activate(nraw, gr.activation);
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
        a.base[k + 1] = a.base[k] + g.n;
    }
    a.b1 = beta1;
    a.b2 = beta2;
    a.eps = eps;
    a.c1 = (float)(1.0 - std::pow((double)beta1, step));
    a.c2 = (float)(1.0 - std::pow((double)beta2, step));
    if (a.base[count] == 0) return GS_OK;
    const unsigned long long blocks = (a.base[count] + 255) / 256;
    const int cap = persistent_grid((const void*)k_adam, 256) * 4;
    k_adam<<<(int)(blocks < (unsigned long long)cap ? blocks : cap), 256, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
