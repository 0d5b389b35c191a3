// gs_kernels.h -- kernel argument blocks and launch constants shared by the kernel files and
// the host-side C ABI implementation (gs_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"
#include "gs_device.cuh"

namespace gs {

// Decoupled look-back words of the radix passes and the column count: a 30-bit count with
// a flag saying whether it covers this chunk only or every chunk up to it.
constexpr uint32_t kLbAgg = 0x40000000u;
constexpr uint32_t kLbInc = 0x80000000u;
constexpr uint32_t kLbFlags = 0xC0000000u;
constexpr uint32_t kLbValue = 0x3FFFFFFFu;
constexpr int kLbWindow = 8;                // predecessors read per look-back round

// Bounded spin-waits poll at full rate for a while, then sleep between polls.
__device__ __forceinline__ void backoff(uint32_t spins) {
    if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
}

// Radix sort: 256 threads, 8-bit digits; 16 keys per thread for 32-bit keys, 12 for 64-bit keys
// (keys and values of a chunk are staged in shared memory, which must stay below 48 KB).
constexpr int kSortThreads = 256;
template <typename KeyT>
struct SortTile {
    static constexpr int items = sizeof(KeyT) == 8 ? 12 : 16;
    static constexpr int keys = kSortThreads * items;
};
constexpr int kSortTile = SortTile<uint32_t>::keys;            // 4096
constexpr int kSortTileMin = SortTile<unsigned long long>::keys; // 3072
constexpr int kMaxKeyPasses = 8;
constexpr int kMaxTilePasses = 3;   // tile ids below 2^24
constexpr int kDepthPasses = 4;

// Tiles per Gaussian: 256 threads, one list entry per thread; the scan of the per-entry
// (segments, tiles) pairs takes chunks of 2048 entries.
constexpr int kDupThreads = 256;
constexpr int kPairChunk = 2048;
// Instance emission: 256 threads, one warp per 32 segment records.
constexpr int kEmitThreads = 256;

// Render: one block per tile, 4 threads per tile row, each owning tile_w / 4 pixels.

// Batches: one launch per stage serves up to kMaxFrames frames (views of one scene, or of
// several scenes).  A kernel receives the argument blocks of all its frames by value; frame f
// owns the work units [base[f], base[f + 1]) (blocks, tiles or Gaussians) when the split is
// known on the host, otherwise the kernel derives it from device-side counts.  A single frame
// is a batch of one (MAXF = 1).
constexpr int kMaxFrames = 32;

template <typename A, int MAXF>
struct Multi {
    int frames;
    uint32_t base[MAXF + 1];
    A a[MAXF];
};

// Frame owning work unit g of a host-side split (frames <= 32: a linear walk).
template <int MAXF>
__device__ __forceinline__ int find_frame(const uint32_t* base, int frames, uint32_t g) {
    if (MAXF == 1) return 0;
    int f = 0;
    while (f + 1 < frames && base[f + 1] <= g) ++f;
    return f;
}

// Control block at the start of the workspace.
struct Control {
    gs_device_status status;
    uint32_t counters[32];                      // chunk-claim counters: [0] scan, [1..4] depth, [8..15] keys
                                                // (or rows), [16] column count, [17] column pass;
                                                // [30] segment records, [31] visible Gaussians
                                                // counted by the binning stage
    uint32_t hist_depth[kDepthPasses][256];     // digit histograms, depth sort
    uint32_t hist_keys[kMaxKeyPasses][256];     // digit histograms, instance sort
};

struct PreprocessArgs {
    int n;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacities;
    const float* sh;
    int sh_degree, sh_stride;
    CamK cam;
    CfgK cfg;
    float4* xy;               // (u_hi, v_hi, u_lo, v_lo): screen mean as a double-float
    float* depth;
    float4* conic_opacity;
    float4* rgb;
    int* radius;
    float* tau;               // alpha-threshold level 2 ln(o / alpha_min) (reach_setup)
    gs_device_status* status;
};

struct PreprocessBwdArgs {
    int n;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacities;
    const float* sh;
    int sh_degree, sh_stride;
    CamK cam;
    CfgK cfg;
    const float* grad2d;     // [n, 12]
    const float4* conic;     // (l11, l21, l22, o): the conic's Cholesky factor the tile kernels used
    const float4* rgb;
    const int* radius;
    float* g_means;
    float* g_scales;
    float* g_quats;
    float* g_opacities;
    float* g_sh;
    float* g_mean2d;
    int accumulate;
};

// Per-Gaussian backward of a batch: frames grouped by the Gaussians they render (group g =
// frames [frame_begin[g], frame_begin[g + 1]), all with the same Gaussians, gradient outputs
// and accumulate flag); group g owns blocks [block_base[g], block_base[g + 1]).
template <int MAXF>
struct BwdPlan {
    int groups;
    uint32_t block_base[MAXF + 1];
    int frame_begin[MAXF + 1];
    PreprocessBwdArgs a[MAXF];
};

// Zeroing of up to kClearRegions buffers per frame in one launch (batches).
constexpr int kClearRegions = 4;
struct ClearArgs {
    uint32_t* ptr[kClearRegions];
    unsigned long long words[kClearRegions];
};

struct DepthHistArgs {
    int n;
    const float* depth;
    const int* radius;
    uint32_t* hist;            // [4][256]
    uint32_t* lookback_first;  // rows for the first depth pass
    uint32_t* num_visible;     // count of radius > 0 (zeroed)
};

template <typename KeyT>
struct SortPassArgs {
    const KeyT* keys_in;       // null: keys from (depth_src, radius_src), values = index
    const uint32_t* vals_in;
    const float* depth_src;
    const int* radius_src;
    KeyT* keys_out;
    uint32_t* vals_out;
    const uint32_t* count_dev; // null: count_host
    uint32_t count_host;       // element count bound (capacity)
    int shift;                 // digit = (key >> shift) & mask
    uint32_t mask;
    int ballot_rank;           // > 0: rank digits with that many ballots (every digit below
                               // 2^ballot_rank; spread digits), 0: with match_any
    const uint32_t* hist;      // [256] digit counts of this pass
    uint32_t* lookback;        // [chunks][256], zeroed
    uint32_t* lookback_next;   // rows to zero for the next pass, or null
    uint32_t* chunk_counter;   // zeroed
    gs_device_status* status;
    uint32_t spin_limit;       // look-back polls before giving up (kFlagTimeout)
};

struct ScanArgs {
    const uint32_t* order;     // depth-sorted Gaussian ids (TWO_PHASE) or null (identity)
    const uint32_t* count_dev; // number of entries of `order` to use, or null (n)
    int n;
    const float4* xy;
    const float4* conic;       // (l11, l21, l22, o)
    const float* tau;          // alpha-threshold level per Gaussian
    int rect_only;             // 1: every tile of the 3-sigma rectangle (GS_TILES_RECT)
    unsigned long long* pairs; // [entries] (segments << 32 | tiles), then their exclusive prefix
    const int* radius;
    const float* depth;
    CamK cam;
    uint32_t* seg_off;         // [capacity + 1] first instance of every segment; [S] = K
    uint32_t* seg_tile;        // [capacity] first tile id of every segment (row_passes > 0: row key)
    uint32_t* seg_gid;         // [capacity] Gaussian of every segment
    int row_passes;            // > 0: row-segmented tile sort (row_key records, no seg_off, digit
                               // histograms of the row's row_passes bytes into hist)
    uint32_t* num_segments;
    unsigned long long capacity;
    uint32_t* hist;            // [4][256] depth-digit histograms (KEY64), row digits (row_passes > 0)
    unsigned long long* lookback;  // [entries / kDupThreads], zeroed
    uint32_t* chunk_counter;
    gs_device_status* status;
    uint32_t spin_limit;       // look-back polls before giving up (kFlagTimeout)
};

// Tile ranges from the sorted keys (uint32 tile ids, or 64-bit keys with the tile id high).
struct RangesArgs {
    const void* keys;
    uint32_t* ranges;          // [2 * tiles], zeroed
    int tiles;
    unsigned long long capacity;
    const gs_device_status* status;
};

struct EmitArgs {
    int n;
    const uint32_t* seg_off;
    const uint32_t* seg_tile;
    const uint32_t* seg_gid;
    const uint32_t* num_segments;
    const float* depth;
    void* keys_out;
    uint32_t* vals_out;
    uint32_t* hist;            // [tile_passes][256] digit histograms of the tile-id radix passes
    int tile_passes;
    int tile_digit_bits;       // bits per tile-id digit (<= 8)
    unsigned long long capacity;
    gs_device_status* status;  // num_segments is reported here
};

struct SortPrepareArgs {
    uint32_t* lookback;
    int tile_keys;             // keys per chunk of the pass that follows
    const gs_device_status* status;
    unsigned long long capacity;
    const uint32_t* count_dev; // keys of that pass; null: the instance count
    uint32_t* lookback2;       // optional second table (256 words per row), or null
    int tile_keys2;            // keys per row of the second table
};

// Row-segmented tile sort (TWO_PHASE, tiles_x <= kRowSortMaxCols).  A segment record is one
// splat's run of reachable tiles in one tile row, as the key
//   row_key = row << 17 | length << 8 | first column
// (row < 4096, length <= 255, column <= 254).  The records, emitted in depth order, are
// stable-sorted by row (1 or 2 byte passes of k_onesweep over the segments, not the instances);
// then per chunk of kSortTile row-sorted records: per-tile instance counts and, per column,
// the counts of the chunk's last row (look-back inside a row); a scan of the tile counts gives
// the ranges; the column pass expands the records into instances and stable-ranks them by
// column within their row, writing each to its final slot.
constexpr int kRowSortMaxCols = 255;
constexpr int kColChunk = 2048;   // row-sorted records per chunk of the count and column passes
constexpr int kRowKeyRowShift = 17;
__host__ __device__ constexpr uint32_t row_key(uint32_t row, uint32_t len, uint32_t col) {
    return row << kRowKeyRowShift | len << 8 | col;
}

struct ColArgs {
    const uint32_t* geom;          // [S] row-sorted row keys
    const uint32_t* gid;           // [S] their Gaussians
    const uint32_t* num_segments;  // S (device)
    unsigned long long capacity;
    int tiles_x, tiles;
    uint32_t* tile_cnt;            // [tiles] instances per tile (zeroed; the count pass adds)
    uint32_t* lookback;            // [chunks][256] per column: counts of a chunk's last row
                                   // (inclusive within the row), zeroed before the count pass
    uint32_t* ranges;              // [2 * tiles]
    uint32_t* keys_out;            // [K] tile id per instance
    uint32_t* vals_out;            // [K] Gaussian per instance
    uint32_t* chunk_counter;       // zeroed
    gs_device_status* status;
    uint32_t spin_limit;           // look-back polls before giving up (kFlagTimeout)
};

struct RenderFwdArgs {
    int n;
    CamK cam;
    CfgK cfg;
    float bg[3];
    int batch;
    const uint32_t* ranges;
    const uint32_t* vals;
    const float4* xy;
    const float4* conic_opacity;
    const float4* rgb;
    float* out_rgb;
    float* out_T;
    uint32_t* out_last;
    uint32_t* out_count;       // nullable: blended splats per pixel (for cfg.grad_limit)
    unsigned long long capacity;   // instance capacity (GS_DEBUG range checks)
    gs_device_status* status;
    uint32_t* contrib;         // per warp of a tile block: bit i set when the warp blended instance i (zeroed)
    uint32_t contrib_words;    // words per warp
    const uint32_t* order;     // [tiles] the tile of each block (k_tile_order)
};

struct RenderBwdArgs {
    int n;
    CamK cam;
    CfgK cfg;
    float bg[3];
    int batch;
    const uint32_t* ranges;
    const uint32_t* vals;
    const float4* xy;
    const float4* conic_opacity;
    const float4* rgb;
    const float* dL_drgb;
    const float* T_final;
    const uint32_t* last;
    const uint32_t* count;     // blended splats per pixel when cfg.grad_limit > 0, else null
    float* grad2d;             // [n, 12] accumulators, zeroed
    unsigned long long* blended;   // count of back-propagated (pixel, splat) pairs, zeroed
    unsigned long long capacity;   // instance capacity (GS_DEBUG range checks)
    gs_device_status* status;
    const uint32_t* contrib;   // the forward pass's contribution bits (see RenderFwdArgs)
    uint32_t contrib_words;
    const uint32_t* order;     // [tiles] the tile of each block (k_tile_order)
};

// Render order of a frame's tiles (k_tile_order): decreasing instance count.
struct TileOrderArgs {
    const uint32_t* ranges;    // [2 * tiles] the binning stage's tile ranges
    uint32_t* order;           // [tiles] out: tile ids, longest lists first, stable
    int tiles;
};

// Host-side launchers (defined next to their kernels).  Each returns the launch status.
// Persistent kernels size their grid as SM count x resident blocks per SM.
int persistent_grid(const void* kernel, int threads);
template <int MAXF> cudaError_t launch_preprocess(Multi<PreprocessArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_preprocess_backward(BwdPlan<MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_depth_hist(Multi<DepthHistArgs, MAXF>& m, cudaStream_t s);
template <typename KeyT, int MAXF>
cudaError_t launch_onesweep(const Multi<SortPassArgs<KeyT>, MAXF>& m, int max_chunks, cudaStream_t s);
template <int MAXF> cudaError_t launch_scan_tiles(const Multi<ScanArgs, MAXF>& m, bool key64, cudaStream_t s);
template <int MAXF> cudaError_t launch_ranges(const Multi<RangesArgs, MAXF>& m, bool key64, cudaStream_t s);
template <int MAXF> cudaError_t launch_emit(const Multi<EmitArgs, MAXF>& m, bool key64, cudaStream_t s);
template <int MAXF> cudaError_t launch_sort_prepare(const Multi<SortPrepareArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_col_count(const Multi<ColArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_tile_scan(const Multi<ColArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_col_scatter(const Multi<ColArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_render_forward(Multi<RenderFwdArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_render_backward(Multi<RenderBwdArgs, MAXF>& m, cudaStream_t s);
template <int MAXF> cudaError_t launch_tile_order(const Multi<TileOrderArgs, MAXF>& m, cudaStream_t s);
cudaError_t launch_clear(const Multi<ClearArgs, kMaxFrames>& m, cudaStream_t s);

}  // namespace gs
