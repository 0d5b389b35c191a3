// density.cu -- adaptive density control of Sec. 5.2 (the refinement step of Algorithm 1):
// view-space gradient statistics, then one pass that prunes, clones and splits, and the
// periodic opacity reset.
//
// The refinement is a stream compaction with expansion: Gaussian i yields c_i in {0, 1, 2}
// output rows (pruned 0, kept 1, cloned 2 = original + copy, split 2 = two children), written
// in source order at the exclusive prefix sum of c.  k_densify does it in one pass over the
// parameters: each block takes the next chunk of 256 Gaussians (chunks are claimed in order
// from a counter, so every predecessor is running or done), decides its rows, publishes the
// chunk's count, finds its output base by a decoupled look-back over the predecessors
// (bounded spin), and copies the 15 arrays (5 parameter tensors and their two Adam moments)
// row by row with coalesced accesses.  HBM-bound: each surviving row is read once and each
// output row written once.
//
// Decisions are taken in fp32 in the raw parameter domains, with thresholds transformed on the
// host in double and rounded to fp32 once: opacity = sigmoid(raw) < epsilon  <=>
// raw < logit(epsilon); max scale = exp(max raw) > tau_S  <=>  max raw > ln(tau_S).
#include <cmath>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

constexpr int kDensChunk = 256;     // Gaussians per chunk (one per thread)
constexpr int kArrays = 15;         // 5 parameter tensors x (value, first moment, second moment)
constexpr int kParamMeans = 0, kParamLogScales = 1, kParamOpacity = 3;

constexpr unsigned long long kDAgg = 1ull << 62;
constexpr unsigned long long kDInc = 2ull << 62;
constexpr unsigned long long kDFlags = 3ull << 62;
constexpr unsigned long long kDValue = (1ull << 62) - 1;

enum : uint8_t { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

struct DensifyArgs {
    int n, capacity;
    int width[5];                         // floats per row of each parameter tensor
    const float* src[kArrays];            // [tensor + 5 * kind], kind 0 value, 1 m, 2 v
    float* dst[kArrays];
    const float* accum;
    const float* count;
    const float* max_radius;
    const float* normals;                 // [n, 2, 3]
    float* out_accum;
    float* out_count;
    float* out_max_radius;
    float* act_scales;                    // nullable: exp(out log_scales)
    float* act_opacities;                 // nullable: sigmoid(out logit_opacities)
    float grad_thr, logit_thr, ln_split, ln_world, max_screen, ln_phi;
    unsigned long long* lookback;         // per chunk, zeroed before the launch
    uint32_t* chunk_counter;              // zeroed before the launch
    uint32_t* result;                     // [0] output rows, [1] flags
};

// the activations of Sec. 5.1, as the Adam kernel applies them
__device__ __forceinline__ float sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ void spin_backoff(uint32_t spins) {
    if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
}

// Copy one array of the chunk: element e of the source rows [0, rows) goes to output row
// base + off[r] (and + 1 for clone / split), transformed by the row's decision.
template <int KIND, int PARAM>
__device__ __forceinline__ void copy_rows(const DensifyArgs& a, int w, const float* __restrict__ src,
                                          float* __restrict__ dst, int rows, unsigned long long base,
                                          const uint8_t* s_code, const uint32_t* s_off, const float* s_mu) {
    const int total = rows * w;
    const unsigned long long cap = (unsigned long long)a.capacity;
    for (int e0 = threadIdx.x; e0 < total; e0 += 4 * kDensChunk) {
        float val[4];
        int r[4], col[4];
        uint8_t code[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = e0 + k * kDensChunk;
            r[k] = e / w;
            col[k] = e - r[k] * w;
            code[k] = e < total ? s_code[r[k]] : kPrune;
            val[k] = code[k] != kPrune ? src[e] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (code[k] == kPrune) continue;
            float v0 = val[k], v1 = 0.f;
            if (KIND == 0) {
                v1 = val[k];
                if (code[k] == kSplit) {
                    if (PARAM == kParamMeans) {
                        v0 = s_mu[r[k] * 6 + col[k]];
                        v1 = s_mu[r[k] * 6 + 3 + col[k]];
                    } else if (PARAM == kParamLogScales) {
                        v0 = v1 = val[k] - a.ln_phi;
                    }
                }
            } else if (code[k] == kSplit) {
                v0 = 0.f;
            }
            const unsigned long long o = base + s_off[r[k]];
            const bool two = code[k] >= kClone;
            if (o < cap) dst[o * w + col[k]] = v0;
            if (two && o + 1 < cap) dst[(o + 1) * w + col[k]] = v1;
            if (KIND == 0 && PARAM == kParamLogScales && a.act_scales) {
                if (o < cap) a.act_scales[o * w + col[k]] = expf(v0);
                if (two && o + 1 < cap) a.act_scales[(o + 1) * w + col[k]] = expf(v1);
            }
            if (KIND == 0 && PARAM == kParamOpacity && a.act_opacities) {
                if (o < cap) a.act_opacities[o] = sigmoid(v0);
                if (two && o + 1 < cap) a.act_opacities[o + 1] = sigmoid(v1);
            }
        }
    }
}

template <int KIND>
__device__ __forceinline__ void copy_kind(const DensifyArgs& a, size_t row0, int rows, unsigned long long base,
                                          const uint8_t* s_code, const uint32_t* s_off, const float* s_mu) {
#define GS_COPY(P)                                                                                           \
    if (a.width[P] > 0)                                                                                      \
        copy_rows<KIND, P>(a, a.width[P], a.src[P + 5 * KIND] + row0 * a.width[P], a.dst[P + 5 * KIND], rows, \
                           base, s_code, s_off, s_mu);
    GS_COPY(0)
    GS_COPY(1)
    GS_COPY(2)
    GS_COPY(3)
    GS_COPY(4)
#undef GS_COPY
}

__global__ void __launch_bounds__(kDensChunk) k_densify(const __grid_constant__ DensifyArgs a) {
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_off[kDensChunk];
    __shared__ uint8_t s_code[kDensChunk];
    __shared__ float s_mu[kDensChunk * 6];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x;
    const uint32_t chunks = (uint32_t)((a.n + kDensChunk - 1) / kDensChunk);
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(a.chunk_counter, 1u);
        __syncthreads();
        const uint32_t chunk = s_chunk;
        if (chunk >= chunks) break;
        const size_t row0 = (size_t)chunk * kDensChunk;
        const int rows = min(kDensChunk, a.n - (int)row0);
        const size_t i = row0 + tid;

        // decision of Gaussian i (Algorithm 1: prune, then clone or split)
        uint8_t code = kPrune;
        float ls[3] = {0.f, 0.f, 0.f};
        if (tid < rows) {
            const float* lsp = a.src[kParamLogScales] + 3 * i;
            ls[0] = lsp[0];
            ls[1] = lsp[1];
            ls[2] = lsp[2];
            const float smax = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
            bool prune = a.src[3][i] < a.logit_thr || smax > a.ln_world;
            if (a.max_screen > 0.f) prune = prune || a.max_radius[i] > a.max_screen;
            const float cnt = a.count[i];
            const bool dens = !prune && cnt > 0.f && __fdiv_rn(a.accum[i], cnt) > a.grad_thr;
            code = prune ? kPrune : (!dens ? kKeep : (smax > a.ln_split ? kSplit : kClone));
        }
        const uint32_t c = code == kPrune ? 0u : (code == kKeep ? 1u : 2u);
        uint32_t block_total;
        const uint32_t excl = block_exclusive_scan<uint32_t>(c, s_scan, &block_total);
        s_off[tid] = excl;
        s_code[tid] = code;

        if (code == kSplit) {
            // children: mu + R(q / |q|) diag(exp(raw scale)) z, z the two given draws
            const float* q = a.src[2] + 4 * i;
            const float qr = q[0], qi = q[1], qj = q[2], qk = q[3];
            const float nn = qr * qr + qi * qi + qj * qj + qk * qk;
            float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
            if (nn > 0.f) {
                const float inv = __fdiv_rn(1.0f, __fsqrt_rn(nn));
                const float r = qr * inv, x = qi * inv, y = qj * inv, z = qk * inv;
                R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - r * z); R[2] = 2.f * (x * z + r * y);
                R[3] = 2.f * (x * y + r * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - r * x);
                R[6] = 2.f * (x * z - r * y); R[7] = 2.f * (y * z + r * x); R[8] = 1.f - 2.f * (x * x + y * y);
            }
            const float s0 = expf(ls[0]), s1 = expf(ls[1]), s2 = expf(ls[2]);
            const float* mu = a.src[kParamMeans] + 3 * i;
            const float* zz = a.normals + 6 * i;
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                const float d0 = s0 * zz[3 * ch], d1 = s1 * zz[3 * ch + 1], d2 = s2 * zz[3 * ch + 2];
#pragma unroll
                for (int row = 0; row < 3; ++row)
                    s_mu[tid * 6 + 3 * ch + row] = mu[row] + (R[3 * row] * d0 + R[3 * row + 1] * d1 + R[3 * row + 2] * d2);
            }
        }

        // output base of the chunk: decoupled look-back over the predecessors
        if (tid < 32) {
            unsigned long long* my = a.lookback + chunk;
            unsigned long long ex = 0;
            if (tid == 0) st_relaxed64(my, (chunk == 0 ? kDInc : kDAgg) | block_total);
            if (chunk > 0) {
                int jj = (int)chunk - 1;
                uint32_t spins = 0;
                while (true) {
                    const int idx = jj - tid;
                    const unsigned long long w = idx >= 0 ? ld_relaxed64(a.lookback + idx) : kDInc;
                    const unsigned long long fl = w & kDFlags;
                    const uint32_t inc = __ballot_sync(0xffffffffu, fl == kDInc);
                    const uint32_t zero = __ballot_sync(0xffffffffu, fl == 0);
                    const int first_inc = inc ? __ffs(inc) - 1 : 32;
                    const uint32_t upto = first_inc >= 31 ? 0xffffffffu : ((2u << first_inc) - 1u);
                    if (zero & upto) {   // a predecessor in front of the first prefix is not ready
                        if (++spins > kSpinLimit) {
                            if (tid == 0) atomicOr(a.result + 1, kFlagTimeout);
                            break;
                        }
                        spin_backoff(spins);
                        continue;
                    }
                    unsigned long long part = tid <= first_inc ? (w & kDValue) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    ex += part;
                    if (first_inc < 32) break;
                    jj -= 32;
                }
                if (tid == 0) st_relaxed64(my, kDInc | (ex + block_total));
            }
            if (tid == 0) {
                s_base = ex;
                if (chunk == chunks - 1) {
                    const unsigned long long total = ex + block_total;
                    a.result[0] = (uint32_t)total;
                    if (total > (unsigned long long)a.capacity) atomicOr(a.result + 1, kFlagCapacity);
                }
            }
        }
        __syncthreads();
        const unsigned long long base = s_base;
        copy_kind<0>(a, row0, rows, base, s_code, s_off, s_mu);
        copy_kind<1>(a, row0, rows, base, s_code, s_off, s_mu);
        copy_kind<2>(a, row0, rows, base, s_code, s_off, s_mu);
        // statistics of the output rows restart at zero
        for (uint32_t k = tid; k < block_total; k += kDensChunk) {
            const unsigned long long o = base + k;
            if (o >= (unsigned long long)a.capacity) break;
            if (a.out_accum) a.out_accum[o] = 0.f;
            if (a.out_count) a.out_count[o] = 0.f;
            if (a.out_max_radius) a.out_max_radius[o] = 0.f;
        }
        __syncthreads();   // shared state is rewritten by the next chunk
    }
}

// One view's statistics: for Gaussians not culled in it, accum += |dL/d(u, v)| in normalised
// device coordinates (pixel gradient scaled by W / 2, H / 2), count += 1, and the largest
// screen radius.
__global__ void __launch_bounds__(256) k_density_stats(int n, const int* __restrict__ radius,
                                                       const float2* __restrict__ grad, float hw, float hh,
                                                       float* __restrict__ accum, float* __restrict__ count,
                                                       float* __restrict__ max_radius) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = radius[i];
        if (r <= 0) continue;
        const float2 g = grad[i];
        const float gx = g.x * hw, gy = g.y * hh;
        accum[i] += __fsqrt_rn(gx * gx + gy * gy);
        count[i] += 1.f;
        if (max_radius) max_radius[i] = fmaxf(max_radius[i], (float)r);
    }
}

// opacity <- min(opacity, max) in the raw domain; the opacity moments restart at zero.
__global__ void __launch_bounds__(256) k_opacity_reset(int n, float cap, float* __restrict__ raw,
                                                       float* __restrict__ m, float* __restrict__ v,
                                                       float* __restrict__ opacity) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float r = fminf(raw[i], cap);
        raw[i] = r;
        if (opacity) opacity[i] = sigmoid(r);
        if (m) m[i] = 0.f;
        if (v) v[i] = 0.f;
    }
}

size_t densify_lookback_bytes(int n) {
    const size_t chunks = ((size_t)n + kDensChunk - 1) / kDensChunk;
    return (chunks * sizeof(unsigned long long) + 255) / 256 * 256;
}

bool valid_arrays(const gs_param_arrays* p, int sh_floats) {
    return p && p->means && p->log_scales && p->quats && p->logit_opacities && (sh_floats == 0 || p->sh);
}

int grid_for(int n, int threads) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = ((long long)n + threads - 1) / threads;
    const long long cap = (long long)sms * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_density_stats(const gs_frame* f, const float* mean2d_grad, float* grad_accum,
                                      float* grad_count, float* max_radius, cudaStream_t s) {
    if (!f || !f->ws || f->n < 0) return GS_ERR_INVALID_ARG;
    gs_layout L;
    if (gs_workspace_layout(f->n, f->cam.width, f->cam.height, f->capacity, &f->cfg, &L) != GS_OK ||
        f->ws_bytes < L.total_bytes)
        return GS_ERR_INVALID_ARG;
    if (f->n == 0) return GS_OK;
    if (!mean2d_grad || !grad_accum || !grad_count) return GS_ERR_INVALID_ARG;
    const int* radius = reinterpret_cast<const int*>(static_cast<const char*>(f->ws) + L.radius);
    k_density_stats<<<grid_for(f->n, 256), 256, 0, s>>>(f->n, radius, reinterpret_cast<const float2*>(mean2d_grad),
                                                        0.5f * f->cam.width, 0.5f * f->cam.height, grad_accum,
                                                        grad_count, max_radius);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" size_t gs_densify_scratch_size(int n) {
    if (n < 0) return 0;
    return densify_lookback_bytes(n) + 256;
}

extern "C" gs_status gs_densify(const gs_density_config* dc, int n, int sh_floats, const gs_param_arrays* params,
                                const gs_param_arrays* adam_m, const gs_param_arrays* adam_v,
                                const float* grad_accum, const float* grad_count, const float* max_radius,
                                const float* normals, const gs_param_arrays* out_params,
                                const gs_param_arrays* out_m, const gs_param_arrays* out_v, float* out_grad_accum,
                                float* out_grad_count, float* out_max_radius, float* out_scales,
                                float* out_opacities, int out_capacity, uint32_t* result, void* scratch,
                                size_t scratch_bytes, cudaStream_t s) {
    if (!dc || n < 0 || sh_floats < 0 || out_capacity < 0 || !result) return GS_ERR_INVALID_ARG;
    if (!(dc->grad_threshold >= 0.f) || !(dc->min_opacity > 0.f && dc->min_opacity < 1.f) ||
        !(dc->split_scale > 0.f) || !(dc->split_factor > 0.f) || !std::isfinite(dc->grad_threshold) ||
        !std::isfinite(dc->split_scale) || !std::isfinite(dc->split_factor) || std::isnan(dc->max_world_scale) ||
        std::isnan(dc->max_screen_radius))
        return GS_ERR_INVALID_ARG;
    if ((long long)n * 2 > (long long)kDValue) return GS_ERR_INVALID_ARG;
    if (cudaMemsetAsync(result, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    if (n == 0) return GS_OK;
    if (!scratch || scratch_bytes < gs_densify_scratch_size(n) || (reinterpret_cast<uintptr_t>(scratch) & 255))
        return GS_ERR_INVALID_ARG;
    if (!valid_arrays(params, sh_floats) || !valid_arrays(adam_m, sh_floats) || !valid_arrays(adam_v, sh_floats) ||
        !grad_accum || !grad_count || !normals || (dc->max_screen_radius > 0.f && !max_radius))
        return GS_ERR_INVALID_ARG;
    if (out_capacity > 0 && (!valid_arrays(out_params, sh_floats) || !valid_arrays(out_m, sh_floats) ||
                             !valid_arrays(out_v, sh_floats)))
        return GS_ERR_INVALID_ARG;

    DensifyArgs a{};
    a.n = n;
    a.capacity = out_capacity;
    const int widths[5] = {3, 3, 4, 1, sh_floats};
    const gs_param_arrays* in[3] = {params, adam_m, adam_v};
    const gs_param_arrays* out[3] = {out_params, out_m, out_v};
    for (int kind = 0; kind < 3; ++kind) {
        const gs_param_arrays* p = in[kind];
        const float* srcs[5] = {p->means, p->log_scales, p->quats, p->logit_opacities, p->sh};
        for (int t = 0; t < 5; ++t) a.src[t + 5 * kind] = srcs[t];
        if (out_capacity > 0) {
            const gs_param_arrays* q = out[kind];
            float* dsts[5] = {q->means, q->log_scales, q->quats, q->logit_opacities, q->sh};
            for (int t = 0; t < 5; ++t) a.dst[t + 5 * kind] = dsts[t];
        }
    }
    for (int t = 0; t < 5; ++t) a.width[t] = widths[t];
    a.accum = grad_accum;
    a.count = grad_count;
    a.max_radius = max_radius;
    a.normals = normals;
    a.out_accum = out_capacity > 0 ? out_grad_accum : nullptr;
    a.out_count = out_capacity > 0 ? out_grad_count : nullptr;
    a.out_max_radius = out_capacity > 0 ? out_max_radius : nullptr;
    a.act_scales = out_capacity > 0 ? out_scales : nullptr;
    a.act_opacities = out_capacity > 0 ? out_opacities : nullptr;
    const double eps = dc->min_opacity;
    a.grad_thr = dc->grad_threshold;
    a.logit_thr = (float)std::log(eps / (1.0 - eps));
    a.ln_split = (float)std::log((double)dc->split_scale);
    a.ln_world = dc->max_world_scale > 0.f ? (float)std::log((double)dc->max_world_scale) : INFINITY;
    a.max_screen = dc->max_screen_radius > 0.f ? dc->max_screen_radius : 0.f;
    a.ln_phi = (float)std::log((double)dc->split_factor);
    char* sc = static_cast<char*>(scratch);
    a.lookback = reinterpret_cast<unsigned long long*>(sc);
    a.chunk_counter = reinterpret_cast<uint32_t*>(sc + densify_lookback_bytes(n));
    a.result = result;
    if (cudaMemsetAsync(scratch, 0, gs_densify_scratch_size(n), s) != cudaSuccess) return GS_ERR_CUDA;
    const int chunks = (n + kDensChunk - 1) / kDensChunk;
    const int cap = persistent_grid((const void*)k_densify, kDensChunk);
    k_densify<<<chunks < cap ? chunks : cap, kDensChunk, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status gs_opacity_reset(float* logit_opacities, float* adam_m, float* adam_v, float* opacities,
                                      int n, float max_opacity, cudaStream_t s) {
    if (n < 0 || !(max_opacity > 0.f && max_opacity < 1.f)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!logit_opacities) return GS_ERR_INVALID_ARG;
    const double p = max_opacity;
    const float cap = (float)std::log(p / (1.0 - p));
    k_opacity_reset<<<grid_for(n, 256), 256, 0, s>>>(n, cap, logit_opacities, adam_m, adam_v, opacities);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
