/*
 * gs.h -- C ABI of the GB300 (sm_103a) differentiable tile rasterizer for 3D Gaussian
 * Splatting (Kerbl et al., "3D Gaussian Splatting for Real-Time Radiance Field
 * Rendering", SIGGRAPH 2023).
 *
 * The paper states the problem as Rasterize(w, h, M, S, C, A, V) (Algorithm 2): image size,
 * Gaussian means M, covariances S = (scales s, rotations q) (Sec. 4), colours C as
 * spherical-harmonic coefficients (Sec. 4, Sec. 7.1), opacities A and the view
 * configuration V.  This header splits Algorithm 2 into four stages:
 *
 *   gs_preprocess      CullGaussian + ScreenspaceGaussians   (Sec. 4, Sec. 6, App. C)
 *   gs_bin_sort        DuplicateWithKeys + SortByKeys + IdentifyTileRanges (Sec. 6, App. C)
 *   gs_render_forward  per-tile BlendInOrder, eq. (front-to-back) with the App. C rules
 *   gs_render_backward back-to-front traversal (Sec. 6) + chain rule of App. A
 *
 * Conventions for every entry point:
 *   - Pointers documented as "device" point to CUDA global memory on the current device.  The
 *     library never allocates or frees memory and keeps no state between calls.  Every call
 *     except gs_read_status is asynchronous on the given stream and issues only kernels and
 *     cudaMemsetAsync (no host synchronisation, no host copies), so a sequence of calls can be
 *     captured into a CUDA graph.
 *   - Floating-point arrays are fp32, contiguous, row-major.  Images are planar [3, H, W].
 *   - Inputs are activated values: scales s > 0 (exp already applied), opacities in (0, 1)
 *     (sigmoid already applied); quaternions (q_r, q_i, q_j, q_k) need not be unit length
 *     (they are normalised inside, Sec. 4).
 *   - Synchronous errors (bad arguments, launch failures) are returned.  Conditions found on
 *     the device (instance capacity exceeded, a bounded spin-wait that gave up, non-finite
 *     inputs) are recorded in the workspace status block and read with gs_read_status.
 */
#ifndef GS_GB300_H
#define GS_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,   /* a null pointer, a non-positive size, a workspace too small   */
    GS_ERR_CAPACITY = 2,      /* more (Gaussian, tile) instances than the workspace holds      */
    GS_ERR_TIMEOUT = 3,       /* a bounded device spin-wait gave up (results are invalid)      */
    GS_ERR_CUDA = 4,          /* a CUDA launch or memset failed                                */
    GS_ERR_NUMERIC = 5,       /* non-finite inputs were found and culled (results are valid)   */
    GS_ERR_INTERNAL = 6       /* a device-side consistency check failed: the per-tile instance
                                 counts did not add up to the instance count, or (in a GS_DEBUG
                                 build) an instance or range index was out of bounds while no
                                 capacity overflow or timeout had been reported; results are
                                 invalid, nothing was written out of bounds                   */
} gs_status;

/* Pinhole camera (the paper's view configuration V, Algorithm 2; viewing transformation W
 * of eq. volume-render).  x_cam = R x_world + t; camera x right, y down, z forward;
 * pixel (px, py) is sampled at (px + 0.5, py + 0.5). */
typedef struct gs_camera {
    int width, height;        /* image size in pixels                                     */
    float fx, fy, cx, cy;     /* focal lengths and principal point, pixels               */
    float R[9];               /* world -> camera rotation, row-major                      */
    float t[3];               /* world -> camera translation                              */
    float near_z;             /* near plane: Gaussians with z <= near_z are rejected      */
} gs_camera;

/* Sort schedule of gs_bin_sort; both give bit-identical instance order and tile ranges. */
enum {
    GS_SORT_TWO_PHASE = 0,    /* depth sort of the N Gaussians, then a stable tile sort of the instances:
                                 up to 255 tile columns the per-row tile runs are sorted by row
                                 and their instances placed by column, else byte passes over
                                 the tile ids */
    GS_SORT_KEY64 = 1         /* one LSD sort of the 64-bit (tile << 32 | depth) keys, as in App. C      */
};

/* Which tiles of a splat's 3-sigma rectangle get an instance (see gs_bin_sort). */
enum {
    GS_TILES_REACH = 0,       /* tiles holding a pixel centre the splat can reach with alpha >= alpha_min */
    GS_TILES_RECT = 1         /* every tile of the rectangle, as in Sec. 6                               */
};

/* Rasterizer constants.  gs_default_config() fills the paper's values. */
typedef struct gs_raster_config {
    int tile_w, tile_h;       /* tile size in pixels: 16 x 16 (Sec. 6); 8 x 8 and 16 x 8 also supported */
    int batch_depth;          /* Gaussians staged in shared memory per batch; <= tile_w * tile_h   */
    int sort_mode;            /* GS_SORT_TWO_PHASE or GS_SORT_KEY64                                */
    float alpha_min;          /* 1/255: skip blending updates with smaller alpha (App. C)          */
    float alpha_max;          /* 0.99: clamp alpha from above (App. C)                             */
    float T_min;              /* 1e-4: stop before the accumulated opacity exceeds 0.9999 (App. C) */
    float dilation;           /* 0.3 px^2 low-pass filter added to the diagonal of Sigma'          */
    float guard;              /* 1.3: reject |x/z| > guard * tan(fov_x/2) or |y/z| > guard * tan(fov_y/2) */
    float extent;             /* 3: screen radius = ceil(extent * sqrt(lambda_max(Sigma')))        */
    int tile_rule;            /* GS_TILES_REACH (default) or GS_TILES_RECT; same images either way */
    int grad_limit;           /* > 0: only the grad_limit front-most blended splats of each pixel
                                 receive gradients (the Limited-BW ablation of Sec. 7.3, N = 10 there);
                                 0: all of them (the paper's method).  The image is unchanged.     */
    int isotropic;            /* 1: one scale per Gaussian for all three axes (the isotropic ablation
                                 of Sec. 7.3): scales and their gradients are [n], quaternions are
                                 neither read nor differentiated (may be NULL); 0: anisotropic      */
    unsigned int spin_limit;  /* polls a thread block of the binning stage makes while waiting for
                                 a predecessor's published prefix before it gives up, sets the
                                 timeout flag (GS_ERR_TIMEOUT) and goes on without waiting;
                                 GS_DEFAULT_SPIN_LIMIT by default, 0 gives up at the first wait   */
} gs_raster_config;

#define GS_DEFAULT_SPIN_LIMIT (1u << 22)

/* Gaussian parameters (Sec. 4): device pointers, n rows each. */
typedef struct gs_gaussians {
    const float* means;       /* [n, 3] world-space means mu                                      */
    const float* scales;      /* [n, 3] s > 0 ([n] with cfg.isotropic)                            */
    const float* quats;       /* [n, 4] (q_r, q_i, q_j, q_k), 16-byte aligned (unused with
                                 cfg.isotropic)                                                   */
    const float* opacities;   /* [n]    o in (0, 1)                                               */
    const float* sh;          /* [n, sh_stride, 3] SH coefficients, bands 0..sh_degree used       */
    int n;                    /* number of Gaussians, >= 0                                        */
    int sh_degree;            /* 0..3                                                             */
    int sh_stride;            /* coefficients per Gaussian in the buffer, >= (sh_degree + 1)^2    */
} gs_gaussians;

/* Gradient outputs of gs_render_backward: device pointers shaped like gs_gaussians. */
typedef struct gs_gradients {
    float* means;             /* [n, 3]                                                         */
    float* scales;            /* [n, 3] ([n] with cfg.isotropic: dL/ds summed over the axes)     */
    float* quats;             /* [n, 4] (not written with cfg.isotropic, may be NULL)            */
    float* opacities;         /* [n]                                                            */
    float* sh;                /* [n, sh_stride, 3]; coefficients beyond the degree get 0         */
    float* mean2d;            /* [n, 2] dL/d(u, v) in pixels (view-space position gradient used
                                 by densification, Sec. 5.2); may be NULL                        */
} gs_gradients;

/* One frame: the Gaussian count, the camera, the constants and the caller-owned device
 * workspace that holds every intermediate of Algorithm 2 (screen-space Gaussians, instance
 * keys and values, tile ranges, sort state, gradient accumulators, status block).  The same
 * frame (same workspace contents) must be passed to all four stages of one render, and the
 * workspace must stay untouched between gs_render_forward and gs_render_backward. */
typedef struct gs_frame {
    int n;                    /* number of Gaussians                                           */
    gs_camera cam;
    gs_raster_config cfg;
    uint64_t capacity;        /* instance capacity: max (Gaussian, tile) pairs, <= 2^30 - 1      */
    void* ws;                 /* device workspace, 256-byte aligned                            */
    size_t ws_bytes;          /* >= gs_workspace_size(n, width, height, capacity, &cfg)          */
} gs_frame;

/* Offsets (bytes from the workspace start) of the named sub-buffers; for inspection and
 * tests.  Screen-space Gaussians (Algorithm 2 M', S'):
 *   xy            float4[n]  screen mean as a double-float (u_hi, v_hi, u_lo, v_lo), u = u_hi + u_lo
 *   depth         float[n]   camera-space z
 *   conic_opacity float4[n]  (l11, l21, l22, o): lower Cholesky factor L of the conic
 *                            Q = Sigma'^-1 = L L^T (power = -|L^T d|^2 / 2) and the opacity
 *   rgb           float4[n]  (r, g, b, bits of the channels clamped at 0)
 *   radius        int32[n]   screen radius in pixels, 0 = culled
 *   tau           float[n]   2 ln(o / alpha_min): a pixel at offset d is blended only if
 *                            |L^T d|^2 <= tau (used by gs_bin_sort's tile rule)
 * Instances: sorted Gaussian indices uint32[capacity] at vals_sorted; tile ranges
 * uint32[2 * tiles] ([start, end) into vals_sorted, [0, 0) for empty tiles); keys_sorted: the
 * sorted keys as uint64[capacity] (KEY64 mode) or the sorted tile ids as uint32[capacity]
 * (TWO_PHASE mode). */
typedef struct gs_layout {
    uint64_t xy, depth, conic_opacity, rgb, radius;
    uint64_t tau;             /* float[n] alpha level 2 ln(o / alpha_min) of every splat       */
    uint64_t vals_sorted, keys_sorted, ranges;
    uint64_t grad2d;          /* float[n, 12] per-Gaussian screen-space gradient accumulators,
                                 the mean and Sigma' terms in the whitened frame (p, q) = L^T d
                                 of the conic's Cholesky factor L (conic_opacity): P, Q =
                                 sum dL/dpower (p, q); K00, K01, K11 = (1/2) sum dL/dpower
                                 (p, q)(p, q)^T; then dL/do, dL/d(r, g, b), 3 unused.  dL/du, dL/dv
                                 = L (P, Q) and dL/dSigma' = L K L^T (full-matrix convention). */
    uint64_t status;          /* gs_device_status                                           */
    uint64_t total_bytes;
    int tiles_x, tiles_y;
    int key_passes;           /* passes of the tile sort: TWO_PHASE up to 255 tile columns,
                                 the row passes over the segment records + the column pass;
                                 otherwise the radix passes over the instance keys            */
    int depth_passes;         /* radix passes over the Gaussian depths (TWO_PHASE), else 0    */
    uint64_t tile_order;      /* uint32[tiles] render order written by gs_bin_sort: the tiles
                                 by decreasing list length (four classes per power of two),
                                 equal classes in tile order; block b of the render passes
                                 takes tile_order[b]                                          */
} gs_layout;

/* Device-side status block (in the workspace). */
typedef struct gs_device_status {
    uint32_t flags;           /* bit 0: capacity exceeded, bit 1: spin-wait timeout, bit 2: a
                                 consistency check failed (GS_ERR_INTERNAL)                    */
    uint32_t num_instances;   /* (Gaussian, tile) pairs (may exceed capacity, see flags)       */
    uint32_t num_visible;     /* Gaussians that survived culling                               */
    uint32_t num_nonfinite;   /* Gaussians culled because an input was NaN or Inf              */
    uint64_t blended_pairs;   /* (pixel, splat) pairs the last gs_render_backward(_tiles) call
                                 back-propagated through (alpha >= alpha_min, before the stop) */
    uint32_t num_segments;    /* tile-row runs of instances written by gs_bin_sort            */
    uint32_t reserved;
} gs_device_status;

/* Fill cfg with the paper's constants: 16x16 tiles, batch 128, alpha in [1/255, 0.99],
 * T_min 1e-4, dilation 0.3, guard 1.3, extent 3, GS_SORT_TWO_PHASE, GS_TILES_REACH, no gradient
 * limit, anisotropic. */
void gs_default_config(gs_raster_config* cfg);

/* Workspace bytes for a frame; 0 if the arguments are invalid. */
size_t gs_workspace_size(int n, int width, int height, uint64_t capacity, const gs_raster_config* cfg);

/* Sub-buffer offsets of the workspace (see gs_layout). */
gs_status gs_workspace_layout(int n, int width, int height, uint64_t capacity, const gs_raster_config* cfg,
                              gs_layout* out);

/* Algorithm 2, CullGaussian + ScreenspaceGaussians, one thread per Gaussian:
 * camera-space mean, near-plane / guard-band rejection (Sec. 6), Sigma = R S S^T R^T with
 * R from the normalised quaternion (Sec. 4, eq. quat), Sigma' = J W Sigma W^T J^T
 * (eq. volume-render) plus the 0.3 px^2 dilation, conic = Sigma'^-1, radius
 * ceil(3 sqrt(lambda_max)), screen mean, tile rectangle, SH colour max(0, sum_k c_k Y_k(d)).
 * Writes the screen-space Gaussians into the workspace and resets the status block.
 * Errors: GS_ERR_INVALID_ARG for a bad frame or Gaussian description, GS_ERR_CUDA. */
gs_status gs_preprocess(const gs_frame* frame, const gs_gaussians* g, cudaStream_t stream);

/* Algorithm 2, DuplicateWithKeys + SortByKeys + IdentifyTileRanges (App. C): one instance per
 * (visible Gaussian, tile it can reach) with key (tile id << 32) | fp32 bits of depth, ordered
 * as one stable sort of those keys emitted in (Gaussian index, row-major tile) order, and the
 * [start, end) range of every tile.  The tiles are those of the paper's 3-sigma rectangle
 * (Sec. 6) that hold at least one pixel centre where o G >= alpha_min could hold: per tile row,
 * the interval of columns where the ellipse |L^T d|^2 <= tau (widened by 2^-10 relative and
 * absolute, and by 0.01 px) meets the row's pixel centres, in IEEE fp32 round-to-nearest
 * arithmetic.  Every dropped pair would be skipped by the alpha test at every pixel of its
 * tile, so the images and gradients are those of the full rectangle.  The instance count stays on the device (status block);
 * if it exceeds frame->capacity, no instance is written past the capacity and the status
 * flag GS_ERR_CAPACITY is raised (the caller grows the workspace and re-runs).  Last, the
 * render order of the tiles (gs_layout.tile_order: longest lists first) is written for
 * gs_render_forward and gs_render_backward, which therefore need a gs_bin_sort of the frame
 * before them. 
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_bin_sort(const gs_frame* frame, cudaStream_t stream);

/* Algorithm 2, BlendInOrder, one thread block per tile: every pixel blends its tile's list
 * front to back, C = sum_i c_i a_i prod_{j<i} (1 - a_j), a = min(0.99, o G), skipping a < 1/255
 * and stopping before T (1 - a) < 1e-4 (App. C).  Outputs (device, caller-owned):
 *   out_rgb  float[3, H, W]   C + T_final * bg
 *   out_T    float[H, W]      final transmittance T_final
 *   out_last uint32[H, W]     1 + position (in the tile list) of the last blended Gaussian, 0 if none
 * bg is a host array of 3 floats.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_render_forward(const gs_frame* frame, const float bg[3], float* out_rgb, float* out_T,
                            uint32_t* out_last, cudaStream_t stream);

/* Backward pass (Sec. 6 and App. A): every tile is traversed back to front from its last
 * contributor; each pixel recovers T_i = T_{i+1} / (1 - a_i) from the stored T_final and
 * accumulates dL/d(mean2D, Sigma', opacity, colour) of every Gaussian it blended (reduced per
 * warp before global atomics); then, per Gaussian, the chain rule through Sigma',
 * Sigma = M M^T, M = R S, the quaternion normalisation, the projection Jacobian, the screen
 * mean and the SH colour gives the gradients of every input.  dL_drgb float[3, H, W], T and
 * last are the forward outputs.  accumulate != 0 adds into the gradient arrays (several views
 * of one scene); accumulate == 0 overwrites them.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_render_backward(const gs_frame* frame, const gs_gaussians* g, const float bg[3],
                             const float* dL_drgb, const float* T, const uint32_t* last,
                             const gs_gradients* grads, int accumulate, cudaStream_t stream);

/* The two halves of gs_render_backward, callable separately (gs_render_backward is exactly
 * gs_render_backward_tiles followed by gs_render_backward_gaussians):
 *   gs_render_backward_tiles      zeroes the workspace's per-Gaussian screen-space gradient
 *                                 accumulators, then runs the back-to-front tile traversal (Sec. 6)
 *                                 that fills them: dL/d(mean2D, Sigma', opacity, colour).
 *   gs_render_backward_gaussians  per Gaussian, the chain rule of App. A from those accumulators to
 *                                 the input gradients (see gs_render_backward for the arguments).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_render_backward_tiles(const gs_frame* frame, const float bg[3], const float* dL_drgb, const float* T,
                                   const uint32_t* last, cudaStream_t stream);
gs_status gs_render_backward_gaussians(const gs_frame* frame, const gs_gaussians* g, const gs_gradients* grads,
                                       int accumulate, cudaStream_t stream);

/* ---- Batches: several frames in one launch per stage --------------------------------------
 * A batch is an array of `views` frames (1 <= views <= GS_MAX_BATCH), each with its own
 * camera, image size, capacity and workspace, all with the same tile shape, batch depth, sort
 * mode and tile rule.  Each stage runs as one launch per kernel for the whole batch (the work
 * of all frames is split over one grid), so views of uneven size share the GPU instead of
 * running one after another.  Every frame's results are those of the single-frame call.
 *   gaussians[v]  the Gaussians frame v renders; views of one scene give equal descriptions.
 *   bg            host float[views][3].
 *   out_rgb, out_T, out_last, dL_drgb, T, last: host arrays of `views` device pointers, each
 *                 laid out as in the single-frame call for that frame's image size.
 *   grads[v]      gradient outputs of frame v.  Frames whose gaussians[] and grads[] are equal
 *                 form a group: the group's gradients are the sum over its frames, written once
 *                 (accumulate = 0) or added (accumulate = 1).  Frames of different groups must
 *                 not share any gradient buffer.
 * Errors: GS_ERR_INVALID_ARG (bad frame, mismatched configuration, views out of range,
 * overlapping gradient outputs), GS_ERR_CUDA.  Device conditions are in each frame's status. */
#define GS_MAX_BATCH 32
gs_status gs_batch_preprocess(const gs_frame* frames, const gs_gaussians* gaussians, int views, cudaStream_t stream);
gs_status gs_batch_bin_sort(const gs_frame* frames, int views, cudaStream_t stream);
gs_status gs_batch_render_forward(const gs_frame* frames, int views, const float* bg, float* const* out_rgb,
                                  float* const* out_T, uint32_t* const* out_last, cudaStream_t stream);
gs_status gs_batch_render_backward(const gs_frame* frames, const gs_gaussians* gaussians, int views,
                                   const float* bg, const float* const* dL_drgb, const float* const* T,
                                   const uint32_t* const* last, const gs_gradients* grads, int accumulate,
                                   cudaStream_t stream);

/* ---- Training step (Sec. 5.1, Algorithm 1): loss and parameter update ---------------------
 * L = (1 - lambda) L1 + lambda (1 - SSIM) of a rendered image against a target (the paper uses
 * lambda = 0.2), with its gradient with respect to the rendered image.  SSIM per channel with an
 * 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero padding, averaged over all
 * pixels and channels; L1 the mean absolute difference; d|x - y|/dx = sign(x - y) (0 at x = y).
 *   img, target  device float[3, H, W] planar
 *   ws           device workspace of gs_loss_workspace_size(width, height) bytes, 256-aligned
 *   out_loss     device float[3]: L, L1, mean SSIM
 *   dL_dimg      device float[3, H, W]
 * Asynchronous on `stream`.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
size_t gs_loss_workspace_size(int width, int height);
gs_status gs_loss_l1_dssim(const float* img, const float* target, int width, int height, float lambda, void* ws,
                           size_t ws_bytes, float* out_loss, float* dL_dimg, cudaStream_t stream);

/* Activation of a parameter tensor: the rasterizer sees act(raw) (Sec. 5.1: sigmoid for the
 * opacity, exp for the scales). */
enum { GS_ACT_NONE = 0, GS_ACT_EXP = 1, GS_ACT_SIGMOID = 2 };

/* One parameter tensor of an Adam step; `grad` is the gradient with respect to act(param). */
typedef struct gs_adam_group {
    float* param;             /* device float[n], raw values, updated in place                  */
    const float* grad;        /* device float[n]                                                */
    float* m;                 /* device float[n], first moment, updated in place (zero at start) */
    float* v;                 /* device float[n], second moment, updated in place               */
    float* activated;         /* device float[n] or NULL: receives act(updated param)           */
    uint64_t n;
    float lr;                 /* learning rate of this step (schedules are the caller's)        */
    int activation;           /* GS_ACT_*                                                       */
} gs_adam_group;

/* Adam (Kingma & Ba) with bias correction, step >= 1, over up to 8 groups in one launch:
 *   g = grad * act'(param); m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 *   param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_adam_step(const gs_adam_group* groups, int count, float beta1, float beta2, float eps, int step,
                       cudaStream_t stream);

/* ---- Adaptive density control (Sec. 5.2, the refinement step of Algorithm 1) ---------------
 * Between refinements the caller accumulates, per view, the magnitude of each Gaussian's
 * view-space positional gradient (gs_density_stats); a refinement (gs_densify) then removes
 * transparent or oversized Gaussians, clones small ones with a large mean gradient
 * (under-reconstruction) and splits large ones (over-reconstruction) into two children
 * sampled from the original Gaussian with their scale divided by phi (the paper: 1.6).
 * gs_opacity_reset lowers every opacity to a small value (the paper: every 3000 iterations).
 * Parameters are the raw tensors the optimiser updates: log scales (scale = exp) and logit
 * opacities (opacity = sigmoid). */

/* The five parameter tensors of a model (device float arrays, rows contiguous):
 *   means [n, 3], log_scales [n, 3], quats [n, 4] (q_r, q_i, q_j, q_k), logit_opacities [n],
 *   sh [n, sh_floats] (the SH coefficients of one Gaussian, any layout; sh_floats <= 192). */
typedef struct gs_param_arrays {
    float* means;
    float* log_scales;
    float* quats;
    float* logit_opacities;
    float* sh;
} gs_param_arrays;

typedef struct gs_density_config {
    float grad_threshold;     /* tau_pos: densify when the mean view-space gradient > this (0.0002) */
    float min_opacity;        /* epsilon_alpha: prune when opacity < this, in (0, 1)              */
    float split_scale;        /* tau_S, world units: split when the largest scale > this, else clone */
    float max_world_scale;    /* prune when the largest scale > this; <= 0 disables               */
    float max_screen_radius;  /* prune when the largest screen radius seen > this (px); <= 0 disables */
    float split_factor;       /* phi: split children have scale / phi (1.6)                       */
} gs_density_config;

/* One view's statistics (after gs_render_backward of `frame`): for every Gaussian that the
 * frame's preprocessing did not cull (screen radius > 0),
 *   grad_accum[i] += |(g_u W / 2, g_v H / 2)|   (the mean gradient in normalised device
 *                                                 coordinates, g = mean2d_grad[i] in pixels),
 *   grad_count[i] += 1,   max_radius[i] = max(max_radius[i], screen radius).
 *   mean2d_grad   device float[n, 2], the gradients' mean2d output of gs_render_backward
 *   grad_accum, grad_count   device float[n], updated in place
 *   max_radius    device float[n] or NULL, updated in place
 * Asynchronous.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_density_stats(const gs_frame* frame, const float* mean2d_grad, float* grad_accum, float* grad_count,
                           float* max_radius, cudaStream_t stream);

/* Scratch bytes gs_densify needs for n Gaussians (0 for n < 0). */
size_t gs_densify_scratch_size(int n);

/* One refinement.  Decision of Gaussian i, in fp32 (thresholds moved to the raw domains on
 * the host in double and rounded to fp32: logit(min_opacity), ln(split_scale),
 * ln(max_world_scale)), every comparison strict:
 *   prune  if sigmoid(logit_opacity) < min_opacity, or max scale > max_world_scale (when
 *          enabled), or max_radius[i] > max_screen_radius (when enabled);
 *   else densify if grad_count[i] > 0 and grad_accum[i] / grad_count[i] > grad_threshold:
 *          split if max scale > split_scale, else clone;
 *   else keep.
 * Outputs (rows in source order, each source's rows adjacent): keep -> the row with its Adam
 * moments; clone -> the row with its moments, then an exact copy with zero moments; split ->
 * two children with means mu + R(q / |q|) diag(exp(log_scales)) z_k (z_k = normals[i][k],
 * standard normal draws supplied by the caller; identity rotation for q = 0), log_scales
 * lowered by ln(split_factor), the other tensors copied, zero moments.  The output statistics
 * (when given) are zeroed.
 *   params, adam_m, adam_v   input tensors (read only) of n rows
 *   normals       device float[n, 2, 3] (rows of non-split Gaussians are not read)
 *   out_*         output tensors with room for out_capacity rows; they must not overlap the
 *                 inputs.  out_grad_accum, out_grad_count, out_max_radius may be NULL.
 *   out_scales    device float[out_capacity, 3] or NULL: exp of the output log_scales
 *   out_opacities device float[out_capacity] or NULL: sigmoid of the output logit_opacities
 *   result        device uint32[2]: [0] rows produced (may exceed out_capacity), [1] flags
 *                 (bit 0: out_capacity exceeded -- rows past it are not written; bit 1: a
 *                 bounded spin-wait gave up -- outputs invalid)
 *   scratch       device, 256-byte aligned, >= gs_densify_scratch_size(n) bytes
 * Asynchronous (cudaMemsetAsync + two kernels).  Errors: GS_ERR_INVALID_ARG (also for
 * n > 2^29 - 1 or sh_floats > 192), GS_ERR_CUDA. */
gs_status gs_densify(const gs_density_config* config, int n, int sh_floats, const gs_param_arrays* params,
                     const gs_param_arrays* adam_m, const gs_param_arrays* adam_v, const float* grad_accum,
                     const float* grad_count, const float* max_radius, const float* normals,
                     const gs_param_arrays* out_params, const gs_param_arrays* out_m, const gs_param_arrays* out_v,
                     float* out_grad_accum, float* out_grad_count, float* out_max_radius, float* out_scales,
                     float* out_opacities, int out_capacity, uint32_t* result, void* scratch,
                     size_t scratch_bytes, cudaStream_t stream);

/* Opacity reset: logit_opacities[i] = min(logit_opacities[i], fp32(logit(max_opacity))); when
 * given, the opacity moments adam_m, adam_v (device float[n]) are zeroed and opacities
 * (device float[n]) receives sigmoid of the new values.
 * Errors: GS_ERR_INVALID_ARG (max_opacity outside (0, 1)), GS_ERR_CUDA. */
gs_status gs_opacity_reset(float* logit_opacities, float* adam_m, float* adam_v, float* opacities, int n,
                           float max_opacity, cudaStream_t stream);

/* Depth ordering without workspace or allocation (no counterpart in the paper; it is the
 * first phase of the GS_SORT_TWO_PHASE binning schedule offered on its own).
 * Writes order[0..n): the indices i with radius[i] > 0 sorted by the fp32 bits of depth[i]
 * (ties by index), followed by the culled indices (radius[i] <= 0) in increasing order; the
 * same order gs_bin_sort uses internally.  status->num_visible receives the count of visible
 * Gaussians and status->flags bit 1 a spin-wait timeout (results then invalid); the other
 * fields are zero.  Asynchronous on `stream`.
 *   depth   device float[n]   camera-space depth of every Gaussian (positive for visible ones)
 *   radius  device int32[n]   screen radius, <= 0 = culled
 *   order   device uint32[n]  output, caller-owned
 *   status  device gs_device_status, caller-owned, overwritten
 * All scratch lives in a file-scope device array of the library sized for
 * n <= GS_STATIC_ORDER_MAX_N (about 4.3 MB per device), so the call allocates nothing: for
 * callers that cannot allocate where they need the ordering (cudaMalloc / cudaFree may
 * synchronise the device and stall other streams; a fixed memory budget leaves no room for a
 * workspace).  The scratch address is looked up once per device on the first call, which may
 * load the module on that device: make the first call on each device outside stream capture.
 * The address stays cached for the life of the process: after cudaDeviceReset (or anything else
 * that destroys the device's primary context and unloads the module) it is stale, so a process
 * that resets a device must not call this entry point on that device again.
 * The scratch is shared by every call on a device, so calls that overlap in time (two streams
 * or two host threads) race and must be ordered by the caller.
 * Errors: GS_ERR_INVALID_ARG for n < 0, n > GS_STATIC_ORDER_MAX_N or a null pointer,
 * GS_ERR_CUDA. */
#define GS_STATIC_ORDER_MAX_N 262144
gs_status gs_depth_order_static(int n, const float* depth, const int* radius, uint32_t* order,
                                gs_device_status* status, cudaStream_t stream);

/* gs_bin_sort with its launches timed (a measurement utility; the binning it performs is
 * gs_bin_sort's, App. C DuplicateWithKeys / SortByKeys / IdentifyTileRanges).  An event is
 * recorded on `stream` before the first launch and after each one; the call synchronises the
 * stream and writes, for up to `cap` launches in order, the milliseconds between consecutive
 * events to ms[i] and a static label of the launch ("depth radix pass", "segment pass", "row
 * radix pass", "column count", "tile scan", "column pass", ...) to names[i]; *count receives
 * how many were written.  Host arrays, caller-owned.  Creates and destroys its own events;
 * allocates no device memory.  Errors: GS_ERR_INVALID_ARG (also for null ms, names or count, or
 * cap <= 0), GS_ERR_CUDA. */
gs_status gs_bin_sort_timed(const gs_frame* frame, float* ms, const char** names, int cap, int* count,
                            cudaStream_t stream);

/* Copy the workspace status block to the host (synchronises the stream) and return the first
 * device-side error as a status: GS_ERR_INTERNAL, GS_ERR_TIMEOUT, GS_ERR_CAPACITY,
 * GS_ERR_NUMERIC or GS_OK. */
gs_status gs_read_status(const gs_frame* frame, gs_device_status* out, cudaStream_t stream);

/* Throughput microbenchmarks (no counterpart in the paper; measurement utilities).  The render
 * kernels' work per (pixel, splat) pair is FP32 fused multiply-adds and one 2^x (PTX
 * ex2.approx.ftz.f32, the instruction the render kernels use); these two kernels measure this
 * GPU's rate of each, the denominator of the render kernels' roofline.
 *   gs_peak_fma   `blocks` blocks of 1024 threads, each running independent chains of fmaf
 *   gs_peak_ex2   the same with ex2.approx.ftz.f32
 *   gs_peak_ops   operations one launch of either performs (FMA instructions per lane, i.e.
 *                 flops / 2, or 2^x evaluations), for (blocks, iters)
 * sink: a device float[blocks] that is never written in practice (it keeps the chains live).
 * Asynchronous on `stream`; time them with events.  Errors: GS_ERR_INVALID_ARG for blocks <= 0,
 * iters <= 0 or a null sink, GS_ERR_CUDA. */
gs_status gs_peak_fma(int blocks, int iters, float* sink, cudaStream_t stream);
gs_status gs_peak_ex2(int blocks, int iters, float* sink, cudaStream_t stream);
unsigned long long gs_peak_ops(int blocks, int iters);

/* Human-readable name of a status code (static string). */
const char* gs_status_string(gs_status s);

#ifdef __cplusplus
}
#endif

#endif /* GS_GB300_H */
