// density.cu -- adaptive density control of Sec. 5.2 (the refinement step of Algorithm 1):
// view-space gradient statistics, then one pass that prunes, clones and splits, and the
// periodic opacity reset.
//
// The refinement is a stream compaction with expansion: Gaussian i yields c_i in {0, 1, 2}
// output rows (pruned 0, kept 1, cloned 2 = original + copy, split 2 = two children), written
// in source order at the exclusive prefix sum of c.  Two kernels:
//   k_densify_plan  one thread per Gaussian, chunks of 256 claimed in order from a counter (so
//                   every predecessor is running or done): decision, block scan, decoupled
//                   look-back (bounded spin) for the chunk's output base; writes each source's
//                   output row and decision (plan), the split children's means, and zeroes the
//                   output statistics;
//   k_densify_copy  one block per (tensor, row range): stages the range's source rows in
//                   shared memory with 16-byte loads (rows that are pruned are not read), then
//                   writes the range's output rows, which are contiguous, with coalesced stores.
// HBM-bound: each surviving row is read once and each output row written once.
//
// Decisions are taken in fp32 in the raw parameter domains, with thresholds transformed on the
// host in double and rounded to fp32 once: opacity = sigmoid(raw) < epsilon  <=>
// raw < logit(epsilon); max scale = exp(max raw) > tau_S  <=>  max raw > ln(tau_S).
#include <cmath>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

constexpr int kPlanThreads = 256;
constexpr int kPlanPer = 4;                               // consecutive Gaussians per plan thread
constexpr int kDensChunk = kPlanThreads * kPlanPer;       // Gaussians per plan chunk
constexpr int kParamMeans = 0, kParamLogScales = 1, kParamOpacity = 3;

constexpr unsigned long long kDAgg = 1ull << 62;
constexpr unsigned long long kDInc = 2ull << 62;
constexpr unsigned long long kDFlags = 3ull << 62;
constexpr unsigned long long kDValue = (1ull << 62) - 1;

enum : uint8_t { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

constexpr uint32_t kOffMask = (1u << 30) - 1;   // plan word: output row | decision << 30

struct PlanArgs {
    int n, capacity;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* logit_opacities;
    const float* accum;
    const float* count;
    const float* max_radius;
    const float* normals;                 // [n, 2, 3]
    float* out_means;
    float* out_accum;
    float* out_count;
    float* out_max_radius;
    float grad_thr, logit_thr, ln_split, ln_world, max_screen;
    uint32_t* plan;                       // [n + 1]; plan[n] = total output rows
    unsigned long long* lookback;         // per chunk, zeroed before the launch
    uint32_t* chunk_counter;              // zeroed before the launch
    uint32_t* result;                     // [0] output rows, [1] flags
};

// One tensor of the copy: rows of w floats, processed in ranges of `rows` source rows.
struct CopyTensor {
    const float* src;
    float* dst;
    float* act;                           // nullable activated output (log scales, opacities)
    int w, rows, kind, param;             // kind 0 value, 1 / 2 Adam moments
};

constexpr int kCopyTensors = 15;
constexpr int kTileFloats = 6144;         // staged source floats per block (24 KB)
constexpr int kCopyThreads = 256;

struct CopyArgs {
    int n, capacity, tensors;
    unsigned int unit_base[kCopyTensors + 1];
    CopyTensor t[kCopyTensors];
    const uint32_t* plan;
    float ln_phi;
};

// the activations of Sec. 5.1, as the Adam kernel applies them
__device__ __forceinline__ float sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ void spin_backoff(uint32_t spins) {
    if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
}

// Decision of Gaussian i (Algorithm 1: prune, then clone or split); ls receives its raw scales.
__device__ __forceinline__ uint8_t decide(const PlanArgs& a, size_t i, float* ls) {
    const float* lsp = a.log_scales + 3 * i;
    ls[0] = lsp[0];
    ls[1] = lsp[1];
    ls[2] = lsp[2];
    const float smax = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
    bool prune = a.logit_opacities[i] < a.logit_thr || smax > a.ln_world;
    if (a.max_screen > 0.f) prune = prune || a.max_radius[i] > a.max_screen;
    const float cnt = a.count[i];
    const bool dens = !prune && cnt > 0.f && __fdiv_rn(a.accum[i], cnt) > a.grad_thr;
    return prune ? kPrune : (!dens ? kKeep : (smax > a.ln_split ? kSplit : kClone));
}

// Split children of Gaussian i at output rows o, o + 1 (those below the capacity):
// mu + R(q / |q|) diag(exp(raw scale)) z, z the two given draws.
__device__ __forceinline__ void split_means(const PlanArgs& a, size_t i, const float* ls, unsigned long long o,
                                            unsigned long long cap) {
    const float* q = a.quats + 4 * i;
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
    const float* mu = a.means + 3 * i;
    const float* zz = a.normals + 6 * i;
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
        if (o + ch >= cap) break;
        const float d0 = s0 * zz[3 * ch], d1 = s1 * zz[3 * ch + 1], d2 = s2 * zz[3 * ch + 2];
#pragma unroll
        for (int row = 0; row < 3; ++row)
            a.out_means[3 * (o + ch) + row] = mu[row] + (R[3 * row] * d0 + R[3 * row + 1] * d1 + R[3 * row + 2] * d2);
    }
}

__global__ void __launch_bounds__(kPlanThreads) k_densify_plan(const __grid_constant__ PlanArgs a) {
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x;
    const uint32_t chunks = (uint32_t)((a.n + kDensChunk - 1) / kDensChunk);
    const unsigned long long cap = (unsigned long long)a.capacity;
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(a.chunk_counter, 1u);
        __syncthreads();
        const uint32_t chunk = s_chunk;
        if (chunk >= chunks) break;
        // this thread's kPlanPer consecutive Gaussians
        const size_t i0 = (size_t)chunk * kDensChunk + (size_t)tid * kPlanPer;
        uint8_t code[kPlanPer];
        float ls[kPlanPer][3];
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < kPlanPer; ++k) {
            code[k] = kPrune;
            if (i0 + k < (size_t)a.n) code[k] = decide(a, i0 + k, ls[k]);
            mine += code[k] == kPrune ? 0u : (code[k] == kKeep ? 1u : 2u);
        }
        uint32_t block_total;
        const uint32_t excl = block_exclusive_scan<uint32_t>(mine, s_scan, &block_total);

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
                    a.plan[a.n] = (uint32_t)total;
                    if (total > cap) atomicOr(a.result + 1, kFlagCapacity);
                }
            }
        }
        __syncthreads();
        const unsigned long long base = s_base;
        unsigned long long o = base + excl;
#pragma unroll
        for (int k = 0; k < kPlanPer; ++k) {
            const size_t i = i0 + k;
            if (i >= (size_t)a.n) break;
            a.plan[i] = (uint32_t)o | ((uint32_t)code[k] << 30);
            if (code[k] == kSplit && o < cap) split_means(a, i, ls[k], o, cap);
            o += code[k] == kPrune ? 0u : (code[k] == kKeep ? 1u : 2u);
        }
        // statistics of the output rows restart at zero
        for (uint32_t k = tid; k < block_total; k += kPlanThreads) {
            const unsigned long long oo = base + k;
            if (oo >= cap) break;
            if (a.out_accum) a.out_accum[oo] = 0.f;
            if (a.out_count) a.out_count[oo] = 0.f;
            if (a.out_max_radius) a.out_max_radius[oo] = 0.f;
        }
        __syncthreads();   // s_chunk / s_base are rewritten by the next chunk
    }
}

// Copy of one (tensor, source row range): W floats per row (compile-time, or 0 = runtime w).
template <int W>
__device__ __forceinline__ void copy_unit(const CopyArgs& a, const CopyTensor& t, int row0, int rows,
                                          float* s_tile, uint16_t* s_inv, uint8_t* s_code) {
    const int w = W > 0 ? W : t.w;
    const int tid = threadIdx.x;
    const uint32_t out_begin = a.plan[row0] & kOffMask;
    const uint32_t out_end = a.plan[row0 + rows] & kOffMask;   // plan[n] holds the total
    // decisions and the inverse map output row -> (source row, child)
    for (int r = tid; r < rows; r += kCopyThreads) {
        const uint32_t p = a.plan[row0 + r];
        const uint8_t code = (uint8_t)(p >> 30);
        s_code[r] = code;
        if (code != kPrune) {
            const uint32_t l = (p & kOffMask) - out_begin;
            s_inv[l] = (uint16_t)(r << 1);
            if (code >= kClone) s_inv[l + 1] = (uint16_t)((r << 1) | 1);
        }
    }
    __syncthreads();
    // stage the source rows (16-byte loads when aligned; float4s of pruned rows only are skipped)
    const int total = rows * w;
    const float* src = t.src + (size_t)row0 * w;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        constexpr int kQ = kTileFloats / 4 / kCopyThreads;
        float4 buf[kQ];
        const int quads = total >> 2;
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
            const int q = tid + k * kCopyThreads;
            buf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < quads) {
                const int ra = (4 * q) / w, rb = (4 * q + 3) / w;
                bool need = false;
                for (int r = ra; r <= rb; ++r) need |= s_code[r] != kPrune;
                if (need) buf[k] = reinterpret_cast<const float4*>(src)[q];
            }
        }
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
            const int q = tid + k * kCopyThreads;
            if (q < quads) reinterpret_cast<float4*>(s_tile)[q] = buf[k];
        }
        for (int e = 4 * quads + tid; e < total; e += kCopyThreads) s_tile[e] = src[e];
    } else {
        for (int e = tid; e < total; e += kCopyThreads) s_tile[e] = src[e];
    }
    __syncthreads();
    // write the contiguous output rows [out_begin, out_end)
    const unsigned long long cap = (unsigned long long)a.capacity;
    const int outs = (int)min((unsigned long long)(out_end - out_begin),
                              cap > out_begin ? cap - out_begin : 0ull);   // rows below the capacity
    const bool split_from_plan = t.kind == 0 && t.param == kParamMeans;    // written by the plan kernel
    if (W > 0 && W % 4 == 0) {
        // rows of whole 16-byte vectors: one vector per thread and step (tile and dst aligned)
        constexpr int V = W > 0 && W % 4 == 0 ? W / 4 : 1;
        const float4* tile4 = reinterpret_cast<const float4*>(s_tile);
        float4* dst4 = reinterpret_cast<float4*>(t.dst) + (size_t)out_begin * V;
        const int total4 = outs * V;
        for (int j = tid; j < total4; j += kCopyThreads) {
            const int ol = j / V;
            const int c4 = j - ol * V;
            const uint32_t e = s_inv[ol];
            const int r = (int)(e >> 1);
            const uint8_t code = s_code[r];
            float4 v = tile4[r * V + c4];
            if (t.kind != 0 && (code == kSplit || (e & 1))) v = make_float4(0.f, 0.f, 0.f, 0.f);
            dst4[j] = v;
        }
    } else if (W == 1 || W == 3) {
        // one output row per thread and step
        float* dst = t.dst + (size_t)out_begin * W;
        float* act = t.act ? t.act + (size_t)out_begin * W : nullptr;
        for (int ol = tid; ol < outs; ol += kCopyThreads) {
            const uint32_t e = s_inv[ol];
            const int r = (int)(e >> 1);
            const uint8_t code = s_code[r];
            if (t.kind == 0 && code == kSplit && split_from_plan) continue;
#pragma unroll
            for (int c = 0; c < (W > 0 ? W : 1); ++c) {
                float v = s_tile[r * W + c];
                if (t.kind == 0) {
                    if (code == kSplit && t.param == kParamLogScales) v -= a.ln_phi;
                    if (act) act[ol * W + c] = t.param == kParamOpacity ? sigmoid(v) : expf(v);
                } else if (code == kSplit || (e & 1)) {
                    v = 0.f;   // moments restart at zero for the clone's copy and both split children
                }
                dst[ol * W + c] = v;
            }
        }
    } else {
        // any width: one element per thread and step
        const int ototal = outs * w;
        float* dst = t.dst + (size_t)out_begin * w;
        for (int j = tid; j < ototal; j += kCopyThreads) {
            const int ol = j / w;
            const int col = j - ol * w;
            const uint32_t e = s_inv[ol];
            const int r = (int)(e >> 1);
            const uint8_t code = s_code[r];
            float v = s_tile[r * w + col];
            if (t.kind == 0) {
                if (code == kSplit && split_from_plan) continue;
                if (code == kSplit && t.param == kParamLogScales) v -= a.ln_phi;
                if (t.act) t.act[(size_t)out_begin * w + j] = t.param == kParamOpacity ? sigmoid(v) : expf(v);
            } else if (code == kSplit || (e & 1)) {
                v = 0.f;
            }
            dst[j] = v;
        }
    }
}

__global__ void __launch_bounds__(kCopyThreads, 5) k_densify_copy(const __grid_constant__ CopyArgs a) {
    __shared__ __align__(16) float s_tile[kTileFloats];
    __shared__ uint16_t s_inv[2 * 2048];
    __shared__ uint8_t s_code[2048];
    const unsigned int u = blockIdx.x;
    int k = 0;
    while (k + 1 < a.tensors && a.unit_base[k + 1] <= u) ++k;
    const CopyTensor& t = a.t[k];
    const int row0 = (int)(u - a.unit_base[k]) * t.rows;
    const int rows = min(t.rows, a.n - row0);
    // compile-time widths: opacity 1, means / log-scales 3, quaternions 4, SH of degree 1 and 3
    // (12, 48 floats); 16-byte stores need an aligned destination
    const bool vec = (reinterpret_cast<uintptr_t>(t.dst) & 15) == 0;
    switch (t.w) {
        case 1: copy_unit<1>(a, t, row0, rows, s_tile, s_inv, s_code); break;
        case 3: copy_unit<3>(a, t, row0, rows, s_tile, s_inv, s_code); break;
        case 4:
            if (vec) copy_unit<4>(a, t, row0, rows, s_tile, s_inv, s_code);
            else copy_unit<0>(a, t, row0, rows, s_tile, s_inv, s_code);
            break;
        case 12:
            if (vec) copy_unit<12>(a, t, row0, rows, s_tile, s_inv, s_code);
            else copy_unit<0>(a, t, row0, rows, s_tile, s_inv, s_code);
            break;
        case 48:
            if (vec) copy_unit<48>(a, t, row0, rows, s_tile, s_inv, s_code);
            else copy_unit<0>(a, t, row0, rows, s_tile, s_inv, s_code);
            break;
        default: copy_unit<0>(a, t, row0, rows, s_tile, s_inv, s_code); break;
    }
}

// source rows per copy range: the largest power of two with rows * w <= kTileFloats, at most 2048
int copy_rows_for(int w) {
    int r = 2048;
    while (r > 1 && r * w > kTileFloats) r >>= 1;
    return r;
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

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// scratch: [look-back words of the plan chunks][chunk counter][plan words (n + 1)]; the first
// two parts are zeroed before every call
size_t densify_zeroed_bytes(int n) {
    const size_t chunks = ((size_t)n + kDensChunk - 1) / kDensChunk;
    return round256(chunks * sizeof(unsigned long long)) + 256;
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
    return densify_zeroed_bytes(n) + round256(((size_t)n + 1) * sizeof(uint32_t));
}

extern "C" gs_status gs_densify(const gs_density_config* dc, int n, int sh_floats, const gs_param_arrays* params,
                                const gs_param_arrays* adam_m, const gs_param_arrays* adam_v,
                                const float* grad_accum, const float* grad_count, const float* max_radius,
                                const float* normals, const gs_param_arrays* out_params,
                                const gs_param_arrays* out_m, const gs_param_arrays* out_v, float* out_grad_accum,
                                float* out_grad_count, float* out_max_radius, float* out_scales,
                                float* out_opacities, int out_capacity, uint32_t* result, void* scratch,
                                size_t scratch_bytes, cudaStream_t s) {
    if (!dc || n < 0 || sh_floats < 0 || sh_floats > kTileFloats / 32 || out_capacity < 0 || !result)
        return GS_ERR_INVALID_ARG;
    if (!(dc->grad_threshold >= 0.f) || !(dc->min_opacity > 0.f && dc->min_opacity < 1.f) ||
        !(dc->split_scale > 0.f) || !(dc->split_factor > 0.f) || !std::isfinite(dc->grad_threshold) ||
        !std::isfinite(dc->split_scale) || !std::isfinite(dc->split_factor) || std::isnan(dc->max_world_scale) ||
        std::isnan(dc->max_screen_radius))
        return GS_ERR_INVALID_ARG;
    if ((long long)n * 2 > (long long)kOffMask) return GS_ERR_INVALID_ARG;   // output rows fit the plan word
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

    char* sc = static_cast<char*>(scratch);
    const size_t zeroed = densify_zeroed_bytes(n);
    PlanArgs p{};
    p.n = n;
    p.capacity = out_capacity;
    p.means = params->means;
    p.log_scales = params->log_scales;
    p.quats = params->quats;
    p.logit_opacities = params->logit_opacities;
    p.accum = grad_accum;
    p.count = grad_count;
    p.max_radius = max_radius;
    p.normals = normals;
    p.out_means = out_capacity > 0 ? out_params->means : nullptr;
    p.out_accum = out_capacity > 0 ? out_grad_accum : nullptr;
    p.out_count = out_capacity > 0 ? out_grad_count : nullptr;
    p.out_max_radius = out_capacity > 0 ? out_max_radius : nullptr;
    const double eps = dc->min_opacity;
    p.grad_thr = dc->grad_threshold;
    p.logit_thr = (float)std::log(eps / (1.0 - eps));
    p.ln_split = (float)std::log((double)dc->split_scale);
    p.ln_world = dc->max_world_scale > 0.f ? (float)std::log((double)dc->max_world_scale) : INFINITY;
    p.max_screen = dc->max_screen_radius > 0.f ? dc->max_screen_radius : 0.f;
    p.lookback = reinterpret_cast<unsigned long long*>(sc);
    p.chunk_counter = reinterpret_cast<uint32_t*>(sc + zeroed - 256);
    p.plan = reinterpret_cast<uint32_t*>(sc + zeroed);
    p.result = result;
    if (cudaMemsetAsync(scratch, 0, zeroed, s) != cudaSuccess) return GS_ERR_CUDA;
    const int chunks = (n + kDensChunk - 1) / kDensChunk;
    const int pcap = persistent_grid((const void*)k_densify_plan, kPlanThreads);
    k_densify_plan<<<chunks < pcap ? chunks : pcap, kPlanThreads, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    if (out_capacity == 0) return GS_OK;

    CopyArgs c{};
    c.n = n;
    c.capacity = out_capacity;
    c.plan = p.plan;
    c.ln_phi = (float)std::log((double)dc->split_factor);
    const int widths[5] = {3, 3, 4, 1, sh_floats};
    const gs_param_arrays* in[3] = {params, adam_m, adam_v};
    const gs_param_arrays* out[3] = {out_params, out_m, out_v};
    unsigned long long units = 0;
    int k = 0;
    for (int kind = 0; kind < 3; ++kind) {
        const float* srcs[5] = {in[kind]->means, in[kind]->log_scales, in[kind]->quats, in[kind]->logit_opacities,
                                in[kind]->sh};
        float* dsts[5] = {out[kind]->means, out[kind]->log_scales, out[kind]->quats, out[kind]->logit_opacities,
                          out[kind]->sh};
        for (int t = 0; t < 5; ++t) {
            if (widths[t] == 0) continue;
            CopyTensor& ct = c.t[k];
            ct.src = srcs[t];
            ct.dst = dsts[t];
            ct.act = nullptr;
            if (kind == 0 && t == kParamLogScales) ct.act = out_scales;
            if (kind == 0 && t == kParamOpacity) ct.act = out_opacities;
            ct.w = widths[t];
            ct.rows = copy_rows_for(widths[t]);
            ct.kind = kind;
            ct.param = t;
            c.unit_base[k] = (unsigned int)units;
            units += ((unsigned long long)n + ct.rows - 1) / ct.rows;
            ++k;
        }
    }
    c.tensors = k;
    c.unit_base[k] = (unsigned int)units;
    k_densify_copy<<<(unsigned int)units, kCopyThreads, 0, s>>>(c);
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
