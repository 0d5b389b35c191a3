// gs_api.cu -- host side of the C ABI declared in include/gs.h: argument validation, the
// workspace layout, and the launch sequence of each stage of Algorithm 2.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "gs.h"
#include "gs_kernels.h"

using namespace gs;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int bits_for(uint32_t v) {
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

struct Layout {
    size_t control, xy, depth, conic, rgb, radius, tau;
    size_t gkey[2], gval[2];
    size_t scan_lb, sort_lb[2];
    size_t ikey[2], ival[2];
    size_t ranges, grad2d, total;
    size_t diff, diff_count;
    size_t sort_lb_rows, scan_lb_rows;
    int tiles_x, tiles_y, tiles, key_passes, depth_passes;
};

bool valid_cfg(const gs_raster_config* c) {
    if (!c) return false;
    const bool shape_ok = (c->tile_w == 16 && c->tile_h == 16) || (c->tile_w == 16 && c->tile_h == 8) ||
                          (c->tile_w == 8 && c->tile_h == 8);
    if (!shape_ok) return false;
    if (c->batch_depth < 1 || c->batch_depth > c->tile_w * c->tile_h) return false;
    if (c->sort_mode != GS_SORT_TWO_PHASE && c->sort_mode != GS_SORT_KEY64) return false;
    if (c->tile_rule != GS_TILES_REACH && c->tile_rule != GS_TILES_RECT) return false;
    if (!(c->alpha_min > 0.f && c->alpha_min < c->alpha_max && c->alpha_max < 1.f)) return false;
    if (!(c->T_min > 0.f && c->T_min < 1.f) || !(c->dilation >= 0.f) || !(c->guard > 0.f) || !(c->extent > 0.f))
        return false;
    return true;
}

bool make_layout(int n, int W, int H, uint64_t cap, const gs_raster_config* cfg, Layout* L) {
    if (n < 0 || W <= 0 || H <= 0 || W > 32768 || H > 32768 || !valid_cfg(cfg)) return false;
    if (cap > (1ull << 30) - 1) return false;
    std::memset(L, 0, sizeof(*L));
    L->tiles_x = (W + cfg->tile_w - 1) / cfg->tile_w;
    L->tiles_y = (H + cfg->tile_h - 1) / cfg->tile_h;
    L->tiles = L->tiles_x * L->tiles_y;
    const int tile_bits = bits_for((uint32_t)(L->tiles - 1));
    if (cfg->sort_mode == GS_SORT_KEY64) {
        L->key_passes = (32 + tile_bits + 7) / 8;
        L->depth_passes = 0;
    } else {
        L->key_passes = (tile_bits + 7) / 8;
        L->depth_passes = kDepthPasses;
    }
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t cc = (size_t)(cap > 0 ? cap : 1);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L->control = take(sizeof(Control));
    L->xy = take(nn * sizeof(float4));
    L->depth = take(nn * sizeof(float));
    L->conic = take(nn * sizeof(float4));
    L->rgb = take(nn * sizeof(float4));
    L->radius = take(nn * sizeof(int));
    L->tau = take(nn * sizeof(float));
    for (int k = 0; k < 2; ++k) { L->gkey[k] = take(nn * 4); L->gval[k] = take(nn * 4); }
    L->diff_count = (size_t)(L->tiles_x + 1) * (L->tiles_y + 1);
    L->diff = take(L->diff_count * sizeof(int));
    L->scan_lb_rows = (nn + kDupChunk - 1) / kDupChunk;
    L->scan_lb = take(L->scan_lb_rows * sizeof(unsigned long long));
    const size_t rows_n = (nn + kSortTile - 1) / kSortTile, rows_c = (cc + kSortTileMin - 1) / kSortTileMin;
    L->sort_lb_rows = rows_n > rows_c ? rows_n : rows_c;
    for (int k = 0; k < 2; ++k) L->sort_lb[k] = take(L->sort_lb_rows * 256 * sizeof(uint32_t));
    // ikey[1] / ival[1] also hold the segment records between the scan and the emit kernel:
    // first tiles and offsets (capacity + 1 entries) in ikey[1], Gaussian ids in ival[1].
    for (int k = 0; k < 2; ++k) { L->ikey[k] = take(cc * 8 + 16); L->ival[k] = take(cc * 4); }
    L->ranges = take((size_t)L->tiles * 2 * sizeof(uint32_t));
    L->grad2d = take(nn * 12 * sizeof(float));
    L->total = off;
    return true;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

bool valid_frame(const gs_frame* f, Layout* L) {
    if (!f || !f->ws) return false;
    if (reinterpret_cast<uintptr_t>(f->ws) % kAlign) return false;
    const gs_camera& c = f->cam;
    if (!(c.fx > 0.f && c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy) || !(c.near_z > 0.f)) return false;
    for (int k = 0; k < 9; ++k) if (!std::isfinite(c.R[k])) return false;
    for (int k = 0; k < 3; ++k) if (!std::isfinite(c.t[k])) return false;
    if (!make_layout(f->n, c.width, c.height, f->capacity, &f->cfg, L)) return false;
    return f->ws_bytes >= L->total;
}

bool valid_gaussians(const gs_frame* f, const gs_gaussians* g) {
    if (!g || g->n != f->n) return false;
    if (g->sh_degree < 0 || g->sh_degree > 3) return false;
    if (g->sh_stride < (g->sh_degree + 1) * (g->sh_degree + 1)) return false;
    if (g->n > 0) {
        if (!g->means || !g->scales || !g->quats || !g->opacities || !g->sh) return false;
        if (reinterpret_cast<uintptr_t>(g->quats) % 16) return false;
        if (reinterpret_cast<uintptr_t>(g->means) % 4 || reinterpret_cast<uintptr_t>(g->scales) % 4 ||
            reinterpret_cast<uintptr_t>(g->opacities) % 4 || reinterpret_cast<uintptr_t>(g->sh) % 4)
            return false;
    }
    return true;
}

CamK cam_k(const gs_frame* f, const Layout& L) {
    const gs_camera& c = f->cam;
    CamK k;
    k.W = c.width; k.H = c.height;
    k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy;
    for (int i = 0; i < 9; ++i) k.R[i] = c.R[i];
    for (int i = 0; i < 3; ++i) k.t[i] = c.t[i];
    k.near_z = c.near_z;
    for (int r = 0; r < 3; ++r)
        k.campos[r] = (float)-((double)c.R[r] * c.t[0] + (double)c.R[3 + r] * c.t[1] + (double)c.R[6 + r] * c.t[2]);
    k.lim_x = (float)((double)f->cfg.guard * (0.5 * c.width / (double)c.fx));
    k.lim_y = (float)((double)f->cfg.guard * (0.5 * c.height / (double)c.fy));
    k.tile_w = f->cfg.tile_w; k.tile_h = f->cfg.tile_h;
    k.tiles_x = L.tiles_x; k.tiles_y = L.tiles_y;
    return k;
}

CfgK cfg_k(const gs_raster_config& c) {
    CfgK k;
    k.alpha_min = c.alpha_min; k.alpha_max = c.alpha_max; k.T_min = c.T_min;
    k.dilation = c.dilation; k.extent = c.extent; k.radius_max = kRadiusMax;
    return k;
}

gs_status ok(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

size_t keys_sorted_off(const Layout& L) { return L.ikey[L.key_passes % 2]; }
size_t vals_sorted_off(const Layout& L) { return L.ival[L.key_passes % 2]; }

template <typename KeyT>
gs_status run_key_sort(const gs_frame* f, const Layout& L, Control* ctl, cudaStream_t s) {
    void* ws = f->ws;
    gs_device_status* st = &ctl->status;
    SortPrepareArgs pa{at<uint32_t>(ws, L.sort_lb[0]), SortTile<KeyT>::keys, st, (unsigned long long)f->capacity};
    if (launch_sort_prepare(pa, s) != cudaSuccess) return GS_ERR_CUDA;
    for (int p = 0; p < L.key_passes; ++p) {
        SortPassArgs<KeyT> a;
        a.keys_in = at<KeyT>(ws, L.ikey[p % 2]);
        a.vals_in = at<uint32_t>(ws, L.ival[p % 2]);
        a.depth_src = nullptr;
        a.radius_src = nullptr;
        a.keys_out = at<KeyT>(ws, L.ikey[(p + 1) % 2]);
        a.vals_out = at<uint32_t>(ws, L.ival[(p + 1) % 2]);
        a.count_dev = &st->num_instances;
        a.count_host = (uint32_t)f->capacity;
        a.shift = 8 * p;
        a.hist = ctl->hist_keys[p];
        a.lookback = at<uint32_t>(ws, L.sort_lb[p % 2]);
        a.lookback_next = (p + 1 < L.key_passes) ? at<uint32_t>(ws, L.sort_lb[(p + 1) % 2]) : nullptr;
        a.chunk_counter = &ctl->counters[8 + p];
        a.status = st;
        if (launch_onesweep(a, 0, s) != cudaSuccess) return GS_ERR_CUDA;
    }
    return GS_OK;
}

}  // namespace

extern "C" {

void gs_default_config(gs_raster_config* cfg) {
    if (!cfg) return;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->batch_depth = 128;
    cfg->sort_mode = GS_SORT_TWO_PHASE;
    cfg->alpha_min = 1.0f / 255.0f;
    cfg->alpha_max = 0.99f;
    cfg->T_min = 1e-4f;
    cfg->dilation = 0.3f;
    cfg->guard = 1.3f;
    cfg->extent = 3.0f;
    cfg->tile_rule = GS_TILES_REACH;
}

size_t gs_workspace_size(int n, int width, int height, uint64_t capacity, const gs_raster_config* cfg) {
    Layout L;
    if (!make_layout(n, width, height, capacity, cfg, &L)) return 0;
    return L.total;
}

gs_status gs_workspace_layout(int n, int width, int height, uint64_t capacity, const gs_raster_config* cfg,
                              gs_layout* out) {
    Layout L;
    if (!out || !make_layout(n, width, height, capacity, cfg, &L)) return GS_ERR_INVALID_ARG;
    out->xy = L.xy;
    out->depth = L.depth;
    out->conic_opacity = L.conic;
    out->rgb = L.rgb;
    out->radius = L.radius;
    out->tau = L.tau;
    out->vals_sorted = vals_sorted_off(L);
    out->keys_sorted = keys_sorted_off(L);
    out->ranges = L.ranges;
    out->grad2d = L.grad2d;
    out->status = L.control + offsetof(Control, status);
    out->total_bytes = L.total;
    out->tiles_x = L.tiles_x;
    out->tiles_y = L.tiles_y;
    out->key_passes = L.key_passes;
    out->depth_passes = L.depth_passes;
    return GS_OK;
}

gs_status gs_preprocess(const gs_frame* f, const gs_gaussians* g, cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !valid_gaussians(f, g)) return GS_ERR_INVALID_ARG;
    void* ws = f->ws;
    Control* ctl = at<Control>(ws, L.control);
    if (cudaMemsetAsync(&ctl->status, 0, sizeof(gs_device_status), s) != cudaSuccess) return GS_ERR_CUDA;
    if (f->n == 0) return GS_OK;
    PreprocessArgs a;
    a.n = f->n;
    a.means = g->means; a.scales = g->scales; a.quats = g->quats; a.opacities = g->opacities; a.sh = g->sh;
    a.sh_degree = g->sh_degree; a.sh_stride = g->sh_stride;
    a.cam = cam_k(f, L);
    a.cfg = cfg_k(f->cfg);
    a.xy = at<float4>(ws, L.xy);
    a.depth = at<float>(ws, L.depth);
    a.conic_opacity = at<float4>(ws, L.conic);
    a.rgb = at<float4>(ws, L.rgb);
    a.radius = at<int>(ws, L.radius);
    a.tau = at<float>(ws, L.tau);
    a.status = &ctl->status;
    return ok(launch_preprocess(a, s));
}

gs_status gs_bin_sort(const gs_frame* f, cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L)) return GS_ERR_INVALID_ARG;
    void* ws = f->ws;
    Control* ctl = at<Control>(ws, L.control);
    gs_device_status* st = &ctl->status;
    // flags + num_instances, then every counter and histogram
    if (cudaMemsetAsync(st, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(&ctl->counters[0], 0, sizeof(Control) - offsetof(Control, counters), s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaMemsetAsync(at<char>(ws, L.diff), 0, L.diff_count * sizeof(int), s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(at<char>(ws, L.scan_lb), 0, L.scan_lb_rows * sizeof(unsigned long long), s) != cudaSuccess)
        return GS_ERR_CUDA;
    const CamK cam = cam_k(f, L);
    const bool key64 = f->cfg.sort_mode == GS_SORT_KEY64;

    ScanArgs d;
    d.n = f->n;
    d.xy = at<float4>(ws, L.xy);
    d.conic = at<float4>(ws, L.conic);
    d.tau = at<float>(ws, L.tau);
    d.radius = at<int>(ws, L.radius);
    d.depth = at<float>(ws, L.depth);
    d.cam = cam;
    d.seg_tile = at<uint32_t>(ws, L.ikey[1]);
    d.seg_off = d.seg_tile + (f->capacity > 0 ? f->capacity : 1);
    d.seg_gid = at<uint32_t>(ws, L.ival[1]);
    d.num_segments = &ctl->counters[30];
    d.rect_only = f->cfg.tile_rule == GS_TILES_RECT;
    d.diff = at<int>(ws, L.diff);
    d.capacity = f->capacity;
    d.hist = &ctl->hist_keys[0][0];
    d.lookback = at<unsigned long long>(ws, L.scan_lb);
    d.chunk_counter = &ctl->counters[0];
    d.status = st;

    if (!key64) {
        // Phase 1: stable sort of all Gaussians by fp32 depth bits (culled ones last).
        if (f->n > 0) {
            DepthHistArgs h{f->n, at<float>(ws, L.depth), at<int>(ws, L.radius), &ctl->hist_depth[0][0],
                            at<uint32_t>(ws, L.sort_lb[0]), &ctl->counters[31]};
            if (launch_depth_hist(h, s) != cudaSuccess) return GS_ERR_CUDA;
            const int chunks = (f->n + kSortTile - 1) / kSortTile;
            for (int p = 0; p < kDepthPasses; ++p) {
                SortPassArgs<uint32_t> a;
                a.keys_in = p == 0 ? nullptr : at<uint32_t>(ws, L.gkey[(p + 1) % 2]);
                a.vals_in = p == 0 ? nullptr : at<uint32_t>(ws, L.gval[(p + 1) % 2]);
                a.depth_src = at<float>(ws, L.depth);
                a.radius_src = at<int>(ws, L.radius);
                a.keys_out = at<uint32_t>(ws, L.gkey[p % 2]);
                a.vals_out = at<uint32_t>(ws, L.gval[p % 2]);
                a.count_dev = nullptr;
                a.count_host = (uint32_t)f->n;
                a.shift = 8 * p;
                a.hist = ctl->hist_depth[p];
                a.lookback = at<uint32_t>(ws, L.sort_lb[p % 2]);
                a.lookback_next = (p + 1 < kDepthPasses) ? at<uint32_t>(ws, L.sort_lb[(p + 1) % 2]) : nullptr;
                a.chunk_counter = &ctl->counters[1 + p];
                a.status = st;
                if (launch_onesweep(a, chunks, s) != cudaSuccess) return GS_ERR_CUDA;
            }
        }
        d.order = at<uint32_t>(ws, L.gval[(kDepthPasses - 1) % 2]);
        d.count_dev = &ctl->counters[31];
    } else {
        d.order = nullptr;
        d.count_dev = nullptr;
    }
    if (launch_scan_tiles(d, key64, s) != cudaSuccess) return GS_ERR_CUDA;
    TileRangesArgs tr;
    tr.diff = at<int>(ws, L.diff);
    tr.tiles_x = L.tiles_x;
    tr.tiles_y = L.tiles_y;
    tr.ranges = at<uint32_t>(ws, L.ranges);
    tr.tile_passes = key64 ? L.key_passes - 4 : L.key_passes;
    tr.key_shift = key64 ? 32 : 0;
    tr.hist = key64 ? &ctl->hist_keys[4][0] : &ctl->hist_keys[0][0];
    tr.capacity = f->capacity;
    if (launch_tile_ranges(tr, s) != cudaSuccess) return GS_ERR_CUDA;
    EmitArgs e;
    e.n = f->n;
    e.seg_off = d.seg_off;
    e.seg_tile = d.seg_tile;
    e.seg_gid = d.seg_gid;
    e.num_segments = d.num_segments;
    e.depth = d.depth;
    e.keys_out = at<void>(ws, L.ikey[0]);
    e.vals_out = at<uint32_t>(ws, L.ival[0]);
    e.capacity = f->capacity;
    e.status = st;
    if (launch_emit(e, key64, s) != cudaSuccess) return GS_ERR_CUDA;
    if (key64) return run_key_sort<unsigned long long>(f, L, ctl, s);
    return run_key_sort<uint32_t>(f, L, ctl, s);
}

gs_status gs_render_forward(const gs_frame* f, const float bg[3], float* out_rgb, float* out_T, uint32_t* out_last,
                            cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !bg || !out_rgb || !out_T || !out_last) return GS_ERR_INVALID_ARG;
    void* ws = f->ws;
    RenderFwdArgs a;
    a.n = f->n;
    a.cam = cam_k(f, L);
    a.cfg = cfg_k(f->cfg);
    for (int k = 0; k < 3; ++k) a.bg[k] = bg[k];
    a.batch = f->cfg.batch_depth;
    a.ranges = at<uint32_t>(ws, L.ranges);
    a.vals = at<uint32_t>(ws, vals_sorted_off(L));
    a.xy = at<float4>(ws, L.xy);
    a.conic_opacity = at<float4>(ws, L.conic);
    a.rgb = at<float4>(ws, L.rgb);
    a.out_rgb = out_rgb;
    a.out_T = out_T;
    a.out_last = out_last;
    return ok(launch_render_forward(a, L.tiles, s));
}

gs_status gs_render_backward_tiles(const gs_frame* f, const float bg[3], const float* dL_drgb, const float* T,
                                   const uint32_t* last, cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !bg || !dL_drgb || !T || !last) return GS_ERR_INVALID_ARG;
    if (f->n == 0) return GS_OK;
    void* ws = f->ws;
    float* grad2d = at<float>(ws, L.grad2d);
    if (cudaMemsetAsync(grad2d, 0, (size_t)f->n * 12 * sizeof(float), s) != cudaSuccess) return GS_ERR_CUDA;
    gs_device_status* st = &at<Control>(ws, L.control)->status;
    if (cudaMemsetAsync(&st->blended_pairs, 0, sizeof(st->blended_pairs), s) != cudaSuccess) return GS_ERR_CUDA;
    RenderBwdArgs a;
    a.n = f->n;
    a.cam = cam_k(f, L);
    a.cfg = cfg_k(f->cfg);
    for (int k = 0; k < 3; ++k) a.bg[k] = bg[k];
    a.batch = f->cfg.batch_depth;
    a.ranges = at<uint32_t>(ws, L.ranges);
    a.vals = at<uint32_t>(ws, vals_sorted_off(L));
    a.xy = at<float4>(ws, L.xy);
    a.conic_opacity = at<float4>(ws, L.conic);
    a.rgb = at<float4>(ws, L.rgb);
    a.dL_drgb = dL_drgb;
    a.T_final = T;
    a.last = last;
    a.grad2d = grad2d;
    a.blended = reinterpret_cast<unsigned long long*>(&st->blended_pairs);
    return ok(launch_render_backward(a, L.tiles, s));
}

gs_status gs_render_backward_gaussians(const gs_frame* f, const gs_gaussians* g, const gs_gradients* gr,
                                       int accumulate, cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !valid_gaussians(f, g) || !gr) return GS_ERR_INVALID_ARG;
    if (f->n > 0 && (!gr->means || !gr->scales || !gr->quats || !gr->opacities || !gr->sh)) return GS_ERR_INVALID_ARG;
    if (f->n > 0 && reinterpret_cast<uintptr_t>(gr->quats) % 16) return GS_ERR_INVALID_ARG;
    if (f->n == 0) return GS_OK;
    void* ws = f->ws;
    PreprocessBwdArgs b;
    b.n = f->n;
    b.means = g->means; b.scales = g->scales; b.quats = g->quats; b.opacities = g->opacities; b.sh = g->sh;
    b.sh_degree = g->sh_degree; b.sh_stride = g->sh_stride;
    b.cam = cam_k(f, L);
    b.cfg = cfg_k(f->cfg);
    b.grad2d = at<float>(ws, L.grad2d);
    b.rgb = at<float4>(ws, L.rgb);
    b.radius = at<int>(ws, L.radius);
    b.g_means = gr->means; b.g_scales = gr->scales; b.g_quats = gr->quats; b.g_opacities = gr->opacities;
    b.g_sh = gr->sh; b.g_mean2d = gr->mean2d;
    b.accumulate = accumulate;
    return ok(launch_preprocess_backward(b, s));
}

gs_status gs_render_backward(const gs_frame* f, const gs_gaussians* g, const float bg[3], const float* dL_drgb,
                             const float* T, const uint32_t* last, const gs_gradients* gr, int accumulate,
                             cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !valid_gaussians(f, g) || !bg || !dL_drgb || !T || !last || !gr) return GS_ERR_INVALID_ARG;
    if (f->n > 0 && (!gr->means || !gr->scales || !gr->quats || !gr->opacities || !gr->sh)) return GS_ERR_INVALID_ARG;
    if (f->n > 0 && reinterpret_cast<uintptr_t>(gr->quats) % 16) return GS_ERR_INVALID_ARG;
    const gs_status st = gs_render_backward_tiles(f, bg, dL_drgb, T, last, s);
    if (st != GS_OK) return st;
    return gs_render_backward_gaussians(f, g, gr, accumulate, s);
}

gs_status gs_read_status(const gs_frame* f, gs_device_status* out, cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !out) return GS_ERR_INVALID_ARG;
    Control* ctl = at<Control>(f->ws, L.control);
    if (cudaMemcpyAsync(out, &ctl->status, sizeof(gs_device_status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    if (out->flags & kFlagTimeout) return GS_ERR_TIMEOUT;
    if (out->flags & kFlagCapacity) return GS_ERR_CAPACITY;
    if (out->num_nonfinite) return GS_ERR_NUMERIC;
    return GS_OK;
}

const char* gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CAPACITY: return "instance capacity exceeded";
        case GS_ERR_TIMEOUT: return "device spin-wait timed out";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_NUMERIC: return "non-finite inputs culled";
    }
    return "unknown status";
}

}  // extern "C"
