// gs_api.cu -- host side of the C ABI declared in include/gs.h: argument validation, the
// workspace layout, and the launch sequence of each stage of Algorithm 2.
#include <algorithm>
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
    size_t pairs, scan_lb, sort_lb[2];
    size_t ikey[2], ival[2];
    size_t ranges, tile_order, grad2d, pix_count, contrib, contrib_words, total;
    size_t sort_lb_rows, scan_lb_rows;
    size_t tile_cnt, col_lb, col_lb_rows;
    int tiles_x, tiles_y, tiles, key_passes, depth_passes, tile_passes, tile_digit_bits;
    bool row_sort;             // row-segmented tile sort (two-phase, tiles_x <= kRowSortMaxCols)
    int row_passes;
};

// Warps of a render block: 4 threads per tile row.
int render_warps(int tile_h) { return (4 * tile_h + 31) / 32; }

bool valid_cfg(const gs_raster_config* c) {
    if (!c) return false;
    const bool shape_ok = (c->tile_w == 16 && c->tile_h == 16) || (c->tile_w == 16 && c->tile_h == 8) ||
                          (c->tile_w == 8 && c->tile_h == 8);
    if (!shape_ok) return false;
    if (c->batch_depth < 1 || c->batch_depth > c->tile_w * c->tile_h) return false;
    if (c->sort_mode != GS_SORT_TWO_PHASE && c->sort_mode != GS_SORT_KEY64) return false;
    if (c->tile_rule != GS_TILES_REACH && c->tile_rule != GS_TILES_RECT) return false;
    if (c->grad_limit < 0 || (c->isotropic != 0 && c->isotropic != 1)) return false;
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
    // tile ids take ceil(bits / 8) radix passes of 8-bit digits (measured faster on 1080p
    // frames than equal-width digits: 8 + 5 bits beat 7 + 6)
    const int tile_bits = bits_for((uint32_t)(L->tiles - 1));
    L->tile_passes = (tile_bits + 7) / 8;
    L->tile_digit_bits = L->tile_passes ? 8 : 0;
    if (cfg->sort_mode == GS_SORT_KEY64) {
        L->key_passes = 4 + L->tile_passes;
        L->depth_passes = 0;
    } else {
        L->key_passes = L->tile_passes;
        L->depth_passes = kDepthPasses;
    }
    // Two-phase frames up to kRowSortMaxCols tile columns sort the segment records by row
    // (one byte pass per 8 row bits) and then place the instances by column in one pass.
    L->row_sort = cfg->sort_mode == GS_SORT_TWO_PHASE && L->tiles_x <= kRowSortMaxCols;
    if (L->row_sort) {
        L->row_passes = L->tiles_y > 256 ? 2 : 1;
        L->key_passes = L->row_passes + 1;
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
    L->pairs = take(nn * sizeof(unsigned long long));
    // one look-back word per chunk of the segment pass (kDupThreads entries; the KEY64
    // schedule's scan takes kPairChunk entries per word and needs fewer)
    L->scan_lb_rows = (nn + kDupThreads - 1) / kDupThreads;
    L->scan_lb = take(L->scan_lb_rows * sizeof(unsigned long long));
    const size_t rows_n = (nn + kSortTile - 1) / kSortTile, rows_c = (cc + kSortTileMin - 1) / kSortTileMin;
    L->sort_lb_rows = rows_n > rows_c ? rows_n : rows_c;
    for (int k = 0; k < 2; ++k) L->sort_lb[k] = take(L->sort_lb_rows * 256 * sizeof(uint32_t));
    // ikey[1] / ival[1] also hold the segment records between the scan and the emit kernel:
    // first tiles and offsets (capacity + 1 entries) in ikey[1], Gaussian ids in ival[1].
    for (int k = 0; k < 2; ++k) { L->ikey[k] = take(cc * 8 + 16); L->ival[k] = take(cc * 4); }
    L->ranges = take((size_t)L->tiles * 2 * sizeof(uint32_t));
    L->tile_order = take((size_t)L->tiles * sizeof(uint32_t));
    L->tile_cnt = take((size_t)L->tiles * sizeof(uint32_t));
    // column-count look-back rows, one per chunk of row-sorted segment records
    L->col_lb_rows = L->row_sort ? (cc + kColChunk - 1) / kColChunk : 0;
    L->col_lb = L->row_sort ? take(L->col_lb_rows * 256 * sizeof(uint32_t)) : 0;
    L->grad2d = take(nn * 12 * sizeof(float));
    // blended splats per pixel, written by the forward pass when gradients are limited
    L->pix_count = cfg->grad_limit > 0 ? take((size_t)W * H * sizeof(uint32_t)) : 0;
    // contribution bits: per warp of a tile block, one bit per instance, set by the forward pass
    // when some pixel of the warp blended that instance (the backward pass visits only those)
    L->contrib_words = (cc + 31) / 32 + 2;
    L->contrib = take((size_t)render_warps(cfg->tile_h) * L->contrib_words * sizeof(uint32_t));
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
        const bool iso = f->cfg.isotropic != 0;
        if (!g->means || !g->scales || (!iso && !g->quats) || !g->opacities || !g->sh) return false;
        if (!iso && reinterpret_cast<uintptr_t>(g->quats) % 16) return false;
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
    k.grad_limit = c.grad_limit; k.isotropic = c.isotropic;
    return k;
}

gs_status ok(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

// Optional per-launch timing of the binning stage (gs_bin_sort_timed): while a timer is active
// on the calling host thread, an event is recorded on the stream after every launch.
struct PhaseTimer {
    static constexpr int kMax = 32;
    cudaEvent_t ev[kMax + 1];   // ev[0]: before the first launch
    const char* name[kMax];
    int n = 0;
};
thread_local PhaseTimer* t_phase = nullptr;

void phase(const char* name, cudaStream_t s) {
    PhaseTimer* t = t_phase;
    if (!t || t->n >= PhaseTimer::kMax) return;
    t->name[t->n] = name;
    cudaEventRecord(t->ev[++t->n], s);
}

size_t keys_sorted_off(const Layout& L) { return L.ikey[L.key_passes % 2]; }
size_t vals_sorted_off(const Layout& L) { return L.ival[L.key_passes % 2]; }

// ---- stage implementations over a set of frames (a batch; a single frame is a batch of 1) ----

// Frames of one call, validated, with their layouts.
template <int MAXF>
struct FrameSet {
    int count = 0;
    const gs_frame* f[MAXF];
    Layout L[MAXF];
};

bool same_shape(const gs_raster_config& a, const gs_raster_config& b) {
    return a.tile_w == b.tile_w && a.tile_h == b.tile_h && a.batch_depth == b.batch_depth &&
           a.sort_mode == b.sort_mode && a.tile_rule == b.tile_rule && (a.grad_limit > 0) == (b.grad_limit > 0) &&
           a.isotropic == b.isotropic;
}

template <int MAXF>
bool collect(const gs_frame* frames, int views, FrameSet<MAXF>* fs) {
    if (!frames || views < 1 || views > MAXF) return false;
    fs->count = views;
    for (int v = 0; v < views; ++v) {
        fs->f[v] = &frames[v];
        if (!valid_frame(&frames[v], &fs->L[v])) return false;
        if (!same_shape(frames[v].cfg, frames[0].cfg)) return false;
    }
    return true;
}

template <int MAXF>
Control* control_of(const FrameSet<MAXF>& fs, int v) {
    return at<Control>(fs.f[v]->ws, fs.L[v].control);
}

// SH rows can be read and written as float4 when every row starts 16-byte aligned (the same
// rule the kernels' launchers apply to the first frame of a launch).
bool sh_vec(const float* sh, int sh_stride, const float* gsh = nullptr) {
    const bool base = reinterpret_cast<uintptr_t>(sh) % 16 == 0 &&
                      (gsh == nullptr || reinterpret_cast<uintptr_t>(gsh) % 16 == 0);
    return base && (3 * sh_stride) % 4 == 0;
}

// Zeroes, per frame, the regions [ptr, ptr + words): cudaMemsetAsync for one frame, one kernel
// for a batch.
template <int MAXF>
gs_status clear_regions(const FrameSet<MAXF>& fs, const ClearArgs* regions, cudaStream_t s) {
    // one region: a memset; several: one kernel for all of them (each memset is an operation
    // of its own on the stream)
    int nonempty = 0;
    for (int v = 0; v < fs.count; ++v)
        for (int r = 0; r < kClearRegions; ++r) nonempty += regions[v].ptr[r] && regions[v].words[r];
    if (nonempty <= 1) {
        for (int v = 0; v < fs.count; ++v)
            for (int r = 0; r < kClearRegions; ++r)
                if (regions[v].ptr[r] && regions[v].words[r] &&
                    cudaMemsetAsync(regions[v].ptr[r], 0, regions[v].words[r] * 4, s) != cudaSuccess)
                    return GS_ERR_CUDA;
        return GS_OK;
    }
    Multi<ClearArgs, kMaxFrames> m;
    m.frames = fs.count;
    for (int v = 0; v < fs.count; ++v) m.a[v] = regions[v];
    return ok(launch_clear(m, s));
}

template <int MAXF>
gs_status preprocess_impl(const FrameSet<MAXF>& fs, const gs_gaussians* g, cudaStream_t s) {
    ClearArgs clr[MAXF];
    for (int v = 0; v < fs.count; ++v) {
        clr[v] = ClearArgs{};
        clr[v].ptr[0] = reinterpret_cast<uint32_t*>(&control_of(fs, v)->status);
        clr[v].words[0] = sizeof(gs_device_status) / 4;
    }
    gs_status st = clear_regions(fs, clr, s);
    if (st != GS_OK) return st;
    // one launch per (SH degree, SH row alignment) class of frames
    bool done[MAXF] = {};
    for (int v0 = 0; v0 < fs.count; ++v0) {
        if (done[v0]) continue;
        Multi<PreprocessArgs, MAXF> m;
        m.frames = 0;
        for (int v = v0; v < fs.count; ++v) {
            if (done[v] || g[v].sh_degree != g[v0].sh_degree ||
                sh_vec(g[v].sh, g[v].sh_stride) != sh_vec(g[v0].sh, g[v0].sh_stride))
                continue;
            done[v] = true;
            const gs_frame* f = fs.f[v];
            const Layout& L = fs.L[v];
            void* ws = f->ws;
            PreprocessArgs& a = m.a[m.frames++];
            a.n = f->n;
            a.means = g[v].means; a.scales = g[v].scales; a.quats = g[v].quats; a.opacities = g[v].opacities;
            a.sh = g[v].sh;
            a.sh_degree = g[v].sh_degree; a.sh_stride = g[v].sh_stride;
            a.cam = cam_k(f, L);
            a.cfg = cfg_k(f->cfg);
            a.xy = at<float4>(ws, L.xy);
            a.depth = at<float>(ws, L.depth);
            a.conic_opacity = at<float4>(ws, L.conic);
            a.rgb = at<float4>(ws, L.rgb);
            a.radius = at<int>(ws, L.radius);
            a.tau = at<float>(ws, L.tau);
            a.status = &control_of(fs, v)->status;
        }
        if (launch_preprocess(m, s) != cudaSuccess) return GS_ERR_CUDA;
    }
    return GS_OK;
}

template <typename KeyT, int MAXF>
gs_status key_sort(const FrameSet<MAXF>& fs, cudaStream_t s) {
    Multi<SortPrepareArgs, MAXF> pm;
    pm.frames = fs.count;
    int max_passes = 0;
    for (int v = 0; v < fs.count; ++v) {
        Control* ctl = control_of(fs, v);
        pm.a[v] = SortPrepareArgs{at<uint32_t>(fs.f[v]->ws, fs.L[v].sort_lb[0]), SortTile<KeyT>::keys, &ctl->status,
                                  (unsigned long long)fs.f[v]->capacity};
        max_passes = std::max(max_passes, fs.L[v].key_passes);
    }
    if (launch_sort_prepare(pm, s) != cudaSuccess) return GS_ERR_CUDA;
    phase("sort prepare", s);
    Control* ctl0 = control_of(fs, 0);
    for (int p = 0; p < max_passes; ++p) {
        Multi<SortPassArgs<KeyT>, MAXF> m;
        m.frames = fs.count;
        for (int v = 0; v < fs.count; ++v) {
            const Layout& L = fs.L[v];
            void* ws = fs.f[v]->ws;
            Control* ctl = control_of(fs, v);
            SortPassArgs<KeyT>& a = m.a[v];
            const bool live = p < L.key_passes;   // frames with fewer tile bits sort fewer passes
            a.keys_in = at<KeyT>(ws, L.ikey[p % 2]);
            a.vals_in = at<uint32_t>(ws, L.ival[p % 2]);
            a.depth_src = nullptr;
            a.radius_src = nullptr;
            a.keys_out = at<KeyT>(ws, L.ikey[(p + 1) % 2]);
            a.vals_out = at<uint32_t>(ws, L.ival[(p + 1) % 2]);
            a.count_dev = &ctl->status.num_instances;
            a.count_host = live ? (uint32_t)fs.f[v]->capacity : 0u;
            // KEY64: four 8-bit depth digits, then the tile-id digits from bit 32
            const bool depth_digit = sizeof(KeyT) == 8 && p < 4;
            const int tp = sizeof(KeyT) == 8 ? p - 4 : p;
            a.shift = depth_digit ? 8 * p : (sizeof(KeyT) == 8 ? 32 : 0) + tp * L.tile_digit_bits;
            a.mask = depth_digit ? 0xFFu : (1u << L.tile_digit_bits) - 1u;
            a.ballot_rank = tp == 0 ? 8 : 0;   // lowest tile-id byte: spread digits
            a.hist = ctl->hist_keys[p < kMaxKeyPasses ? p : 0];
            a.lookback = at<uint32_t>(ws, L.sort_lb[p % 2]);
            a.lookback_next = (p + 1 < L.key_passes) ? at<uint32_t>(ws, L.sort_lb[(p + 1) % 2]) : nullptr;
            a.chunk_counter = &ctl0->counters[8 + p];
            a.status = &ctl->status;
            a.spin_limit = fs.f[v]->cfg.spin_limit;
        }
        if (launch_onesweep(m, 0, s) != cudaSuccess) return GS_ERR_CUDA;
        phase("instance radix pass", s);
    }
    return GS_OK;
}

// Instance radix sort: the segment records expanded into (tile id, Gaussian) instances (KEY64:
// (tile id << 32 | depth bits)), sorted by key, ranges by neighbour comparison.
template <int MAXF>
gs_status tiles_by_radix(const FrameSet<MAXF>& fs, bool key64, cudaStream_t s) {
    Multi<RangesArgs, MAXF> tr;
    tr.frames = fs.count;
    Multi<EmitArgs, MAXF> e;
    e.frames = fs.count;
    for (int v = 0; v < fs.count; ++v) {
        const gs_frame* f = fs.f[v];
        const Layout& L = fs.L[v];
        void* ws = f->ws;
        Control* ctl = control_of(fs, v);
        RangesArgs& t = tr.a[v];
        t.keys = at<void>(ws, keys_sorted_off(L));
        t.ranges = at<uint32_t>(ws, L.ranges);
        t.tiles = L.tiles;
        t.capacity = f->capacity;
        t.status = &ctl->status;
        EmitArgs& a = e.a[v];
        a.tile_passes = L.tile_passes;
        a.tile_digit_bits = L.tile_digit_bits;
        a.hist = key64 ? &ctl->hist_keys[4][0] : &ctl->hist_keys[0][0];
        a.n = f->n;
        a.seg_tile = at<uint32_t>(ws, L.ikey[1]);
        a.seg_off = a.seg_tile + (f->capacity > 0 ? f->capacity : 1);
        a.seg_gid = at<uint32_t>(ws, L.ival[1]);
        a.num_segments = &ctl->counters[30];
        a.depth = at<float>(ws, L.depth);
        a.keys_out = at<void>(ws, L.ikey[0]);
        a.vals_out = at<uint32_t>(ws, L.ival[0]);
        a.capacity = f->capacity;
        a.status = &ctl->status;
    }
    if (launch_emit(e, key64, s) != cudaSuccess) return GS_ERR_CUDA;
    phase("emit instances", s);
    const gs_status st = key64 ? key_sort<unsigned long long>(fs, s) : key_sort<uint32_t>(fs, s);
    if (st != GS_OK) return st;
    const gs_status r = ok(launch_ranges(tr, key64, s));
    phase("tile ranges", s);
    return r;
}

// Row-segmented tile sort: the segment records sorted by row, then every instance placed by
// its column within the row (tilesort.cu).
template <int MAXF>
gs_status tiles_by_rows(const FrameSet<MAXF>& fs, cudaStream_t s) {
    Multi<SortPrepareArgs, MAXF> pm;
    pm.frames = fs.count;
    int max_passes = 0;
    for (int v = 0; v < fs.count; ++v) {
        const Layout& L = fs.L[v];
        void* ws = fs.f[v]->ws;
        Control* ctl = control_of(fs, v);
        pm.a[v] = SortPrepareArgs{at<uint32_t>(ws, L.sort_lb[0]), kSortTile, &ctl->status,
                                  (unsigned long long)fs.f[v]->capacity, &ctl->counters[30],
                                  at<uint32_t>(ws, L.col_lb), kColChunk};
        max_passes = std::max(max_passes, L.row_passes);
    }
    if (launch_sort_prepare(pm, s) != cudaSuccess) return GS_ERR_CUDA;
    phase("sort prepare", s);
    Control* ctl0 = control_of(fs, 0);
    for (int p = 0; p < max_passes; ++p) {
        Multi<SortPassArgs<uint32_t>, MAXF> m;
        m.frames = fs.count;
        for (int v = 0; v < fs.count; ++v) {
            const Layout& L = fs.L[v];
            void* ws = fs.f[v]->ws;
            Control* ctl = control_of(fs, v);
            SortPassArgs<uint32_t>& a = m.a[v];
            const bool live = p < L.row_passes;
            a.keys_in = at<uint32_t>(ws, L.ikey[p % 2]);
            a.vals_in = at<uint32_t>(ws, L.ival[p % 2]);
            a.depth_src = nullptr;
            a.radius_src = nullptr;
            a.keys_out = at<uint32_t>(ws, L.ikey[(p + 1) % 2]);
            a.vals_out = at<uint32_t>(ws, L.ival[(p + 1) % 2]);
            a.count_dev = &ctl->counters[30];
            a.count_host = live ? (uint32_t)fs.f[v]->capacity : 0u;
            a.shift = kRowKeyRowShift + 8 * p;
            a.mask = 0xFFu;
            a.ballot_rank = 0;   // rows repeat across a warp's records
            a.hist = ctl->hist_keys[p];
            a.lookback = at<uint32_t>(ws, L.sort_lb[p % 2]);
            a.lookback_next = (p + 1 < L.row_passes) ? at<uint32_t>(ws, L.sort_lb[(p + 1) % 2]) : nullptr;
            a.chunk_counter = &ctl0->counters[8 + p];
            a.status = &ctl->status;
            a.spin_limit = fs.f[v]->cfg.spin_limit;
        }
        if (launch_onesweep(m, 0, s) != cudaSuccess) return GS_ERR_CUDA;
        phase("row radix pass", s);
    }
    Multi<ColArgs, MAXF> c;
    c.frames = fs.count;
    for (int v = 0; v < fs.count; ++v) {
        const Layout& L = fs.L[v];
        void* ws = fs.f[v]->ws;
        Control* ctl = control_of(fs, v);
        ColArgs& a = c.a[v];
        const int rp = L.row_passes;
        a.geom = at<uint32_t>(ws, L.ikey[rp % 2]);
        a.gid = at<uint32_t>(ws, L.ival[rp % 2]);
        a.num_segments = &ctl->counters[30];
        a.capacity = fs.f[v]->capacity;
        a.tiles_x = L.tiles_x;
        a.tiles = L.tiles;
        a.tile_cnt = at<uint32_t>(ws, L.tile_cnt);
        a.lookback = at<uint32_t>(ws, L.col_lb);
        a.ranges = at<uint32_t>(ws, L.ranges);
        a.keys_out = at<uint32_t>(ws, L.ikey[(rp + 1) % 2]);   // = keys_sorted_off (key_passes = rp + 1)
        a.vals_out = at<uint32_t>(ws, L.ival[(rp + 1) % 2]);
        a.chunk_counter = &ctl0->counters[16];
        a.status = &ctl->status;
        a.spin_limit = fs.f[v]->cfg.spin_limit;
    }
    if (launch_col_count(c, s) != cudaSuccess) return GS_ERR_CUDA;
    phase("column count", s);
    if (launch_tile_scan(c, s) != cudaSuccess) return GS_ERR_CUDA;
    phase("tile scan", s);
    for (int v = 0; v < fs.count; ++v) c.a[v].chunk_counter = &ctl0->counters[17];
    const gs_status r = ok(launch_col_scatter(c, s));
    phase("column pass", s);
    return r;
}

template <int MAXF>
gs_status bin_sort_impl(const FrameSet<MAXF>& fs, cudaStream_t s) {
    const bool key64 = fs.f[0]->cfg.sort_mode == GS_SORT_KEY64;
    ClearArgs clr[MAXF];
    for (int v = 0; v < fs.count; ++v) {
        const Layout& L = fs.L[v];
        void* ws = fs.f[v]->ws;
        Control* ctl = control_of(fs, v);
        clr[v] = ClearArgs{};
        // flags + num_instances, every counter and histogram, the tile ranges, the scan look-back
        clr[v].ptr[0] = reinterpret_cast<uint32_t*>(&ctl->status);
        clr[v].words[0] = 2;
        clr[v].ptr[1] = &ctl->counters[0];
        clr[v].words[1] = (sizeof(Control) - offsetof(Control, counters)) / 4;
        // the radix schedule leaves empty tiles' ranges as zeroed; the row sort writes every
        // range and needs its tile counts zeroed
        clr[v].ptr[2] = at<uint32_t>(ws, L.row_sort ? L.tile_cnt : L.ranges);
        clr[v].words[2] = (unsigned long long)L.tiles * (L.row_sort ? 1 : 2);
        clr[v].ptr[3] = at<uint32_t>(ws, L.scan_lb);
        clr[v].words[3] = L.scan_lb_rows * 2;
    }
    gs_status st = clear_regions(fs, clr, s);
    if (st != GS_OK) return st;
    phase("clear", s);
    Control* ctl0 = control_of(fs, 0);

    Multi<ScanArgs, MAXF> d;
    d.frames = fs.count;
    if (!key64) {
        // Phase 1: stable sort of every frame's Gaussians by fp32 depth bits (culled ones last).
        Multi<DepthHistArgs, MAXF> h;
        h.frames = fs.count;
        int chunks = 0;
        for (int v = 0; v < fs.count; ++v) {
            const Layout& L = fs.L[v];
            void* ws = fs.f[v]->ws;
            Control* ctl = control_of(fs, v);
            h.a[v] = DepthHistArgs{fs.f[v]->n, at<float>(ws, L.depth), at<int>(ws, L.radius), &ctl->hist_depth[0][0],
                                   at<uint32_t>(ws, L.sort_lb[0]), &ctl->counters[31]};
            chunks += (fs.f[v]->n + kSortTile - 1) / kSortTile;
        }
        if (launch_depth_hist(h, s) != cudaSuccess) return GS_ERR_CUDA;
        phase("depth histogram", s);
        for (int p = 0; p < kDepthPasses; ++p) {
            Multi<SortPassArgs<uint32_t>, MAXF> m;
            m.frames = fs.count;
            for (int v = 0; v < fs.count; ++v) {
                const Layout& L = fs.L[v];
                void* ws = fs.f[v]->ws;
                Control* ctl = control_of(fs, v);
                SortPassArgs<uint32_t>& a = m.a[v];
                a.keys_in = p == 0 ? nullptr : at<uint32_t>(ws, L.gkey[(p + 1) % 2]);
                a.vals_in = p == 0 ? nullptr : at<uint32_t>(ws, L.gval[(p + 1) % 2]);
                a.depth_src = at<float>(ws, L.depth);
                a.radius_src = at<int>(ws, L.radius);
                a.keys_out = at<uint32_t>(ws, L.gkey[p % 2]);
                a.vals_out = at<uint32_t>(ws, L.gval[p % 2]);
                a.count_dev = nullptr;
                a.count_host = (uint32_t)fs.f[v]->n;
                a.shift = 8 * p;
                a.mask = 0xFFu;
                a.ballot_rank = 0;
                a.hist = ctl->hist_depth[p];
                a.lookback = at<uint32_t>(ws, L.sort_lb[p % 2]);
                a.lookback_next = (p + 1 < kDepthPasses) ? at<uint32_t>(ws, L.sort_lb[(p + 1) % 2]) : nullptr;
                a.chunk_counter = &ctl0->counters[1 + p];
                a.status = &ctl->status;
                a.spin_limit = fs.f[v]->cfg.spin_limit;
            }
            if (chunks > 0 && launch_onesweep(m, chunks, s) != cudaSuccess) return GS_ERR_CUDA;
            phase("depth radix pass", s);
        }
    }
    for (int v = 0; v < fs.count; ++v) {
        const gs_frame* f = fs.f[v];
        const Layout& L = fs.L[v];
        void* ws = f->ws;
        Control* ctl = control_of(fs, v);
        ScanArgs& a = d.a[v];
        a.n = f->n;
        a.order = key64 ? nullptr : at<uint32_t>(ws, L.gval[(kDepthPasses - 1) % 2]);
        a.count_dev = key64 ? nullptr : &ctl->counters[31];
        a.xy = at<float4>(ws, L.xy);
        a.conic = at<float4>(ws, L.conic);
        a.tau = at<float>(ws, L.tau);
        a.rect_only = f->cfg.tile_rule == GS_TILES_RECT;
        a.radius = at<int>(ws, L.radius);
        a.depth = at<float>(ws, L.depth);
        a.cam = cam_k(f, L);
        if (L.row_sort) {   // (row key, Gaussian) records, the input of the first row pass
            a.seg_tile = at<uint32_t>(ws, L.ikey[0]);
            a.seg_off = nullptr;
            a.seg_gid = at<uint32_t>(ws, L.ival[0]);
            a.row_passes = L.row_passes;
        } else {
            a.seg_tile = at<uint32_t>(ws, L.ikey[1]);
            a.seg_off = a.seg_tile + (f->capacity > 0 ? f->capacity : 1);
            a.seg_gid = at<uint32_t>(ws, L.ival[1]);
            a.row_passes = 0;
        }
        a.num_segments = &ctl->counters[30];
        a.capacity = f->capacity;
        a.hist = &ctl->hist_keys[0][0];
        a.pairs = at<unsigned long long>(ws, L.pairs);
        a.lookback = at<unsigned long long>(ws, L.scan_lb);
        a.chunk_counter = &ctl0->counters[0];
        a.status = &ctl->status;
        a.spin_limit = fs.f[v]->cfg.spin_limit;
    }
    if (launch_scan_tiles(d, key64, s) != cudaSuccess) return GS_ERR_CUDA;
    phase(key64 ? "tile count, scan and segment write" : "segment pass", s);
    FrameSet<MAXF> radix, rows;
    for (int v = 0; v < fs.count; ++v) {
        FrameSet<MAXF>& g = fs.L[v].row_sort ? rows : radix;
        g.f[g.count] = fs.f[v];
        g.L[g.count] = fs.L[v];
        ++g.count;
    }
    if (radix.count) {
        st = tiles_by_radix(radix, key64, s);
        if (st != GS_OK) return st;
    }
    if (rows.count) {
        st = tiles_by_rows(rows, s);
        if (st != GS_OK) return st;
    }
    // the render passes' block order: every frame's tiles by decreasing list length
    Multi<TileOrderArgs, MAXF> o;
    o.frames = fs.count;
    for (int v = 0; v < fs.count; ++v)
        o.a[v] = TileOrderArgs{at<uint32_t>(fs.f[v]->ws, fs.L[v].ranges), at<uint32_t>(fs.f[v]->ws, fs.L[v].tile_order),
                               fs.L[v].tiles};
    st = ok(launch_tile_order(o, s));
    phase("tile order", s);
    return st;
}

template <int MAXF>
gs_status render_forward_impl(const FrameSet<MAXF>& fs, const float* bg, float* const* out_rgb,
                              float* const* out_T, uint32_t* const* out_last, cudaStream_t s) {
    ClearArgs clr[MAXF];
    Multi<RenderFwdArgs, MAXF> m;
    m.frames = fs.count;
    for (int v = 0; v < fs.count; ++v) {
        const gs_frame* f = fs.f[v];
        const Layout& L = fs.L[v];
        void* ws = f->ws;
        RenderFwdArgs& a = m.a[v];
        a.n = f->n;
        a.cam = cam_k(f, L);
        a.cfg = cfg_k(f->cfg);
        for (int k = 0; k < 3; ++k) a.bg[k] = bg[3 * v + k];
        a.batch = f->cfg.batch_depth;
        a.ranges = at<uint32_t>(ws, L.ranges);
        a.vals = at<uint32_t>(ws, vals_sorted_off(L));
        a.xy = at<float4>(ws, L.xy);
        a.conic_opacity = at<float4>(ws, L.conic);
        a.rgb = at<float4>(ws, L.rgb);
        a.out_rgb = out_rgb[v];
        a.out_T = out_T[v];
        a.out_last = out_last[v];
        a.out_count = f->cfg.grad_limit > 0 ? at<uint32_t>(ws, L.pix_count) : nullptr;
        a.capacity = f->capacity;
        a.status = &control_of(fs, v)->status;
        a.contrib = at<uint32_t>(ws, L.contrib);
        a.contrib_words = (uint32_t)L.contrib_words;
        a.order = at<uint32_t>(ws, L.tile_order);
        clr[v] = ClearArgs{};
        clr[v].ptr[0] = a.contrib;
        clr[v].words[0] = (unsigned long long)render_warps(f->cfg.tile_h) * L.contrib_words;
    }
    gs_status st = clear_regions(fs, clr, s);
    if (st != GS_OK) return st;
    return ok(launch_render_forward(m, s));
}

template <int MAXF>
gs_status render_backward_tiles_impl(const FrameSet<MAXF>& fs, const float* bg, const float* const* dL_drgb,
                                     const float* const* T, const uint32_t* const* last, cudaStream_t s) {
    ClearArgs clr[MAXF];
    Multi<RenderBwdArgs, MAXF> m;
    m.frames = fs.count;
    for (int v = 0; v < fs.count; ++v) {
        const gs_frame* f = fs.f[v];
        const Layout& L = fs.L[v];
        void* ws = f->ws;
        gs_device_status* st = &control_of(fs, v)->status;
        clr[v] = ClearArgs{};
        clr[v].ptr[0] = at<uint32_t>(ws, L.grad2d);
        clr[v].words[0] = (unsigned long long)f->n * 12;
        clr[v].ptr[1] = reinterpret_cast<uint32_t*>(&st->blended_pairs);
        clr[v].words[1] = 2;
        RenderBwdArgs& a = m.a[v];
        a.n = f->n;
        a.cam = cam_k(f, L);
        a.cfg = cfg_k(f->cfg);
        for (int k = 0; k < 3; ++k) a.bg[k] = bg[3 * v + k];
        a.batch = f->cfg.batch_depth;
        a.ranges = at<uint32_t>(ws, L.ranges);
        a.vals = at<uint32_t>(ws, vals_sorted_off(L));
        a.xy = at<float4>(ws, L.xy);
        a.conic_opacity = at<float4>(ws, L.conic);
        a.rgb = at<float4>(ws, L.rgb);
        a.dL_drgb = dL_drgb[v];
        a.T_final = T[v];
        a.last = last[v];
        a.count = f->cfg.grad_limit > 0 ? at<uint32_t>(ws, L.pix_count) : nullptr;
        a.grad2d = at<float>(ws, L.grad2d);
        a.blended = reinterpret_cast<unsigned long long*>(&st->blended_pairs);
        a.capacity = f->capacity;
        a.status = st;
        a.contrib = at<uint32_t>(ws, L.contrib);
        a.contrib_words = (uint32_t)L.contrib_words;
        a.order = at<uint32_t>(ws, L.tile_order);
    }
    gs_status st = clear_regions(fs, clr, s);
    if (st != GS_OK) return st;
    return ok(launch_render_backward(m, s));
}

bool same_gaussians(const gs_gaussians& a, const gs_gaussians& b) {
    return a.means == b.means && a.scales == b.scales && a.quats == b.quats && a.opacities == b.opacities &&
           a.sh == b.sh && a.n == b.n && a.sh_degree == b.sh_degree && a.sh_stride == b.sh_stride;
}

bool same_gradients(const gs_gradients& a, const gs_gradients& b) {
    return a.means == b.means && a.scales == b.scales && a.quats == b.quats && a.opacities == b.opacities &&
           a.sh == b.sh && a.mean2d == b.mean2d;
}

bool gradients_overlap(const gs_gradients& a, const gs_gradients& b) {
    return a.means == b.means || a.scales == b.scales || (a.quats && a.quats == b.quats) ||
           a.opacities == b.opacities || a.sh == b.sh || (a.mean2d && a.mean2d == b.mean2d);
}

// Groups the frames by the Gaussians they render: a group's gradients are summed into its
// outputs in one pass.  Frames of different groups must not share a gradient buffer.
template <int MAXF>
bool group_frames(int count, const gs_gaussians* g, const gs_gradients* gr, int* group_of, int* first, int* groups) {
    *groups = 0;
    for (int v = 0; v < count; ++v) {
        group_of[v] = -1;
        for (int k = 0; k < *groups; ++k) {
            const int u = first[k];
            if (same_gaussians(g[u], g[v]) && same_gradients(gr[u], gr[v])) { group_of[v] = k; break; }
            if (gradients_overlap(gr[u], gr[v])) return false;
        }
        if (group_of[v] < 0) { first[*groups] = v; group_of[v] = (*groups)++; }
    }
    return true;
}

template <int MAXF>
gs_status render_backward_gaussians_impl(const FrameSet<MAXF>& fs, const gs_gaussians* g, const gs_gradients* gr,
                                         int accumulate, cudaStream_t s) {
    int group_of[MAXF], first[MAXF], groups = 0;
    if (!group_frames<MAXF>(fs.count, g, gr, group_of, first, &groups)) return GS_ERR_INVALID_ARG;
    // one launch per (SH degree, SH row alignment) class of groups
    bool done[MAXF] = {};
    for (int k0 = 0; k0 < groups; ++k0) {
        if (done[k0]) continue;
        const gs_gaussians& g0 = g[first[k0]];
        const gs_gradients& r0 = gr[first[k0]];
        const bool vec0 = sh_vec(g0.sh, g0.sh_stride, r0.sh);
        BwdPlan<MAXF> m;
        m.groups = 0;
        int nf = 0;
        for (int k = k0; k < groups; ++k) {
            const gs_gaussians& gk = g[first[k]];
            const gs_gradients& rk = gr[first[k]];
            if (done[k] || gk.sh_degree != g0.sh_degree || sh_vec(gk.sh, gk.sh_stride, rk.sh) != vec0) continue;
            done[k] = true;
            if (gk.n == 0) continue;
            m.frame_begin[m.groups] = nf;
            for (int v = 0; v < fs.count; ++v) {
                if (group_of[v] != k) continue;
                const gs_frame* f = fs.f[v];
                const Layout& L = fs.L[v];
                void* ws = f->ws;
                PreprocessBwdArgs& b = m.a[nf++];
                b.n = f->n;
                b.means = gk.means; b.scales = gk.scales; b.quats = gk.quats; b.opacities = gk.opacities;
                b.sh = gk.sh;
                b.sh_degree = gk.sh_degree; b.sh_stride = gk.sh_stride;
                b.cam = cam_k(f, L);
                b.cfg = cfg_k(f->cfg);
                b.grad2d = at<float>(ws, L.grad2d);
                b.conic = at<float4>(ws, L.conic);
                b.rgb = at<float4>(ws, L.rgb);
                b.radius = at<int>(ws, L.radius);
                b.g_means = rk.means; b.g_scales = rk.scales; b.g_quats = rk.quats; b.g_opacities = rk.opacities;
                b.g_sh = rk.sh; b.g_mean2d = rk.mean2d;
                b.accumulate = accumulate;
            }
            m.frame_begin[++m.groups] = nf;
        }
        if (m.groups > 0 && launch_preprocess_backward(m, s) != cudaSuccess) return GS_ERR_CUDA;
    }
    return GS_OK;
}

bool valid_gradients(const gs_frame* f, const gs_gradients* gr) {
    if (!gr) return false;
    const bool iso = f->cfg.isotropic != 0;
    if (f->n > 0 && (!gr->means || !gr->scales || (!iso && !gr->quats) || !gr->opacities || !gr->sh)) return false;
    if (f->n > 0 && !iso && reinterpret_cast<uintptr_t>(gr->quats) % 16) return false;
    return true;
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
    cfg->grad_limit = 0;
    cfg->isotropic = 0;
    cfg->spin_limit = GS_DEFAULT_SPIN_LIMIT;
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
    out->tile_order = L.tile_order;
    return GS_OK;
}

gs_status gs_preprocess(const gs_frame* f, const gs_gaussians* g, cudaStream_t s) {
    FrameSet<1> fs;
    if (!collect(f, 1, &fs) || !valid_gaussians(f, g)) return GS_ERR_INVALID_ARG;
    return preprocess_impl(fs, g, s);
}

gs_status gs_bin_sort(const gs_frame* f, cudaStream_t s) {
    FrameSet<1> fs;
    if (!collect(f, 1, &fs)) return GS_ERR_INVALID_ARG;
    return bin_sort_impl(fs, s);
}

gs_status gs_render_forward(const gs_frame* f, const float bg[3], float* out_rgb, float* out_T, uint32_t* out_last,
                            cudaStream_t s) {
    FrameSet<1> fs;
    if (!collect(f, 1, &fs) || !bg || !out_rgb || !out_T || !out_last) return GS_ERR_INVALID_ARG;
    return render_forward_impl(fs, bg, &out_rgb, &out_T, &out_last, s);
}

gs_status gs_render_backward_tiles(const gs_frame* f, const float bg[3], const float* dL_drgb, const float* T,
                                   const uint32_t* last, cudaStream_t s) {
    FrameSet<1> fs;
    if (!collect(f, 1, &fs) || !bg || !dL_drgb || !T || !last) return GS_ERR_INVALID_ARG;
    if (f->n == 0) return GS_OK;
    return render_backward_tiles_impl(fs, bg, &dL_drgb, &T, &last, s);
}

gs_status gs_render_backward_gaussians(const gs_frame* f, const gs_gaussians* g, const gs_gradients* gr,
                                       int accumulate, cudaStream_t s) {
    FrameSet<1> fs;
    if (!collect(f, 1, &fs) || !valid_gaussians(f, g) || !valid_gradients(f, gr)) return GS_ERR_INVALID_ARG;
    if (f->n == 0) return GS_OK;
    return render_backward_gaussians_impl(fs, g, gr, accumulate, s);
}

gs_status gs_render_backward(const gs_frame* f, const gs_gaussians* g, const float bg[3], const float* dL_drgb,
                             const float* T, const uint32_t* last, const gs_gradients* gr, int accumulate,
                             cudaStream_t s) {
    FrameSet<1> fs;
    if (!collect(f, 1, &fs) || !valid_gaussians(f, g) || !bg || !dL_drgb || !T || !last || !valid_gradients(f, gr))
        return GS_ERR_INVALID_ARG;
    if (f->n == 0) return GS_OK;
    const gs_status st = render_backward_tiles_impl(fs, bg, &dL_drgb, &T, &last, s);
    if (st != GS_OK) return st;
    return render_backward_gaussians_impl(fs, g, gr, accumulate, s);
}

// ---- batches ----------------------------------------------------------------------------

gs_status gs_batch_preprocess(const gs_frame* frames, const gs_gaussians* g, int views, cudaStream_t s) {
    if (views == 1) return gs_preprocess(frames, g, s);
    FrameSet<kMaxFrames> fs;
    if (!g || !collect(frames, views, &fs)) return GS_ERR_INVALID_ARG;
    for (int v = 0; v < views; ++v)
        if (!valid_gaussians(&frames[v], &g[v])) return GS_ERR_INVALID_ARG;
    return preprocess_impl(fs, g, s);
}

gs_status gs_batch_bin_sort(const gs_frame* frames, int views, cudaStream_t s) {
    if (views == 1) return gs_bin_sort(frames, s);
    FrameSet<kMaxFrames> fs;
    if (!collect(frames, views, &fs)) return GS_ERR_INVALID_ARG;
    return bin_sort_impl(fs, s);
}

gs_status gs_batch_render_forward(const gs_frame* frames, int views, const float* bg, float* const* out_rgb,
                                  float* const* out_T, uint32_t* const* out_last, cudaStream_t s) {
    if (!bg || !out_rgb || !out_T || !out_last) return GS_ERR_INVALID_ARG;
    if (views == 1) return gs_render_forward(frames, bg, out_rgb[0], out_T[0], out_last[0], s);
    FrameSet<kMaxFrames> fs;
    if (!collect(frames, views, &fs)) return GS_ERR_INVALID_ARG;
    for (int v = 0; v < views; ++v)
        if (!out_rgb[v] || !out_T[v] || !out_last[v]) return GS_ERR_INVALID_ARG;
    return render_forward_impl(fs, bg, out_rgb, out_T, out_last, s);
}

gs_status gs_batch_render_backward(const gs_frame* frames, const gs_gaussians* g, int views, const float* bg,
                                   const float* const* dL_drgb, const float* const* T, const uint32_t* const* last,
                                   const gs_gradients* grads, int accumulate, cudaStream_t s) {
    if (!g || !bg || !dL_drgb || !T || !last || !grads) return GS_ERR_INVALID_ARG;
    if (views == 1) return gs_render_backward(frames, g, bg, dL_drgb[0], T[0], last[0], grads, accumulate, s);
    FrameSet<kMaxFrames> fs;
    if (!collect(frames, views, &fs)) return GS_ERR_INVALID_ARG;
    for (int v = 0; v < views; ++v)
        if (!valid_gaussians(&frames[v], &g[v]) || !dL_drgb[v] || !T[v] || !last[v] ||
            !valid_gradients(&frames[v], &grads[v]))
            return GS_ERR_INVALID_ARG;
    int group_of[kMaxFrames], first[kMaxFrames], groups = 0;
    if (!group_frames<kMaxFrames>(views, g, grads, group_of, first, &groups)) return GS_ERR_INVALID_ARG;
    const gs_status st = render_backward_tiles_impl(fs, bg, dL_drgb, T, last, s);
    if (st != GS_OK) return st;
    return render_backward_gaussians_impl(fs, g, grads, accumulate, s);
}

gs_status gs_bin_sort_timed(const gs_frame* f, float* ms, const char** names, int cap, int* count, cudaStream_t s) {
    if (!ms || !names || !count || cap <= 0) return GS_ERR_INVALID_ARG;
    *count = 0;
    PhaseTimer t;
    int made = 0;
    gs_status st = GS_OK;
    for (; made <= PhaseTimer::kMax; ++made)
        if (cudaEventCreate(&t.ev[made]) != cudaSuccess) { st = GS_ERR_CUDA; break; }
    if (st == GS_OK && cudaEventRecord(t.ev[0], s) != cudaSuccess) st = GS_ERR_CUDA;
    if (st == GS_OK) {
        t_phase = &t;
        st = gs_bin_sort(f, s);
        t_phase = nullptr;
    }
    if (st == GS_OK && cudaEventSynchronize(t.ev[t.n]) != cudaSuccess) st = GS_ERR_CUDA;
    if (st == GS_OK) {
        const int n = t.n < cap ? t.n : cap;
        for (int i = 0; i < n; ++i) {
            if (cudaEventElapsedTime(&ms[i], t.ev[i], t.ev[i + 1]) != cudaSuccess) st = GS_ERR_CUDA;
            names[i] = t.name[i];
        }
        *count = n;
    }
    for (int i = 0; i < made; ++i) cudaEventDestroy(t.ev[i]);
    return st;
}

gs_status gs_read_status(const gs_frame* f, gs_device_status* out, cudaStream_t s) {
    Layout L;
    if (!valid_frame(f, &L) || !out) return GS_ERR_INVALID_ARG;
    Control* ctl = at<Control>(f->ws, L.control);
    if (cudaMemcpyAsync(out, &ctl->status, sizeof(gs_device_status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    if (out->flags & kFlagInternal) return GS_ERR_INTERNAL;
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
        case GS_ERR_INTERNAL: return "device-side consistency check failed";
    }
    return "unknown status";
}

}  // extern "C"
