/*
 * libgs -- GB300 (sm_103a) differentiable tile rasterizer for 3D Gaussian splatting,
 * with the densification bookkeeping of the paper's training loop.
 *
 * Paper: "Decomposing Densification in Gaussian Splatting for Faster 3D Scene
 * Reconstruction" (arXiv 2507.20239). The rasterizer computes the paper's Eq. 1 /
 * EWA projection / Eq. 2 (Sec. "Preliminary"); densification follows the
 * split/clone rule (Sec. "Preliminary", last paragraph), global-to-local gating
 * (Sec. "Global-to-local framework") and adaptive opacity pruning (Sec. "Adaptive
 * Opacity Pruning").
 *
 * Conventions for every entry point:
 *  - Every pointer named *_dev or documented as "device" is CUDA device memory
 *    owned by the caller. The library never allocates, frees or synchronises:
 *    each call enqueues kernels on `stream` and returns. Calls on one stream may
 *    be captured into a CUDA graph.
 *  - Scratch memory is the caller's `ws` buffer of at least the size returned by
 *    the matching *_workspace_size function, 256-byte aligned.
 *  - Argument errors are detected on the host before anything is enqueued and
 *    returned as GS_ERR_INVALID_ARG. Launch failures return GS_ERR_CUDA.
 *    Conditions only the device can see (duplicate or output capacity exceeded)
 *    are OR-ed as GS_ERR_* bits into the caller's device word `d_error`, which
 *    the caller reads after the stream has been synchronised (outside any graph).
 *  - Floating point data are IEEE fp32, contiguous, row-major; all base pointers
 *    are 16-byte aligned. Records of view v and Gaussian g have index r = v*n + g.
 *  - No entry point traps or spins without a bound.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,
  GS_ERR_CAPACITY = 2,     /* a device-side count exceeded a caller capacity     */
  GS_ERR_CUDA = 3,         /* a CUDA launch or runtime call failed               */
  GS_ERR_TIMEOUT = 4,      /* a bounded device wait ran out (reserved)           */
  GS_ERR_UNSUPPORTED = 5   /* valid request this build does not implement        */
} gs_status_t;

typedef void *gs_stream_t; /* a cudaStream_t; NULL = the legacy default stream */

/* One pinhole view. World->camera rotation R (row-major) and translation t, OpenCV
 * axes (x right, y down, z forward); pixel (i, j) is sampled at (i + 0.5, j + 0.5).
 * The last five fields are layout, written by gs_frame_init. */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_plane;        /* records with camera-space z <= near_plane are culled */
  int32_t grid_x, grid_y;  /* tiles per row / column                              */
  int32_t tile_offset;     /* first global tile index of this view                */
  int64_t pixel_offset;    /* first pixel of this view in planar batch buffers    */
} gs_camera_t;

/* A batch of views rendered together. cams_dev is a device copy of the cameras
 * (after gs_frame_init). Tiles of all views form one global index space
 * [0, n_tiles); images are stored view after view, each planar [3][H][W] starting
 * at float offset 3 * pixel_offset. */
typedef struct {
  const gs_camera_t *cams_dev;
  int32_t n_views;
  int32_t tile_w, tile_h;  /* 16x16 (default), 8x8 or 16x32 (w x h); see gs_tile_supported */
  int32_t n_tiles;
  int64_t n_pixels;
  int32_t max_width, max_height;
  int32_t sort_fused_bits; /* gs_bin_sort: low tile-id bits sorted while emitting
                            * (1..8, at most the tile-id width); 0 = automatic.
                            * A tuning knob: the order produced is the same. */
} gs_frame_t;

/* Gaussian parameters, device SoA (Eq. 1: position, scale, rotation, opacity, SH):
 * means [n][3]; log_scales [n][3] (scale = exp); quats [n][4] as (w, x, y, z), any
 * norm > 0 (normalised inside); opacity_logits [n] (opacity = sigmoid);
 * sh [n][sh_stride][3] real SH coefficients, index k = l*l + l + m, Condon-Shortley
 * phase, colour = sum_k sh_k Y_k(dir) + 0.5 clamped at 0, dir = unit vector from
 * the camera centre to the mean. sh_degree in 0..3, sh_stride >= (sh_degree+1)^2. */
typedef struct {
  const float *means;
  const float *log_scales;
  const float *quats;
  const float *opacity_logits;
  const float *sh;
  int64_t n;
  int32_t sh_degree;
  int32_t sh_stride;
} gs_params_t;

/* Projected records (device, caller-allocated, n_records = n_views * n rows each).
 * mean2d [R][2] pixels; conic_opacity [R][4] = (A, beta, gamma, opacity): with the
 * dilated covariance Sigma'' = Sigma' + 0.3 I = (a b; b c), det = ac - b^2,
 * A = c/det, beta = -b/c, gamma = 1/c, so that d^T Sigma''^-1 d = A (dx + beta dy)^2
 * + gamma dy^2 (d = pixel mean - pixel centre) and the falloff is exp(-1/2 of it);
 * rgb [R][4] = (r, g, b, q_max), q_max = 2 ln(255 opacity), the bound on
 * d^T Sigma''^-1 d where alpha can reach 1/255; depth [R] camera-space z;
 * radius [R] = the ceiling of the larger half-extent of that ellipse (with the
 * binning's 0.2% margin), 0 = culled; rect [R][4] tile rectangle x0, y0, x1, y1
 * (exclusive) under its bounding box; clamped [R] bit c set when colour channel c
 * was clamped at 0. */
typedef struct {
  float *mean2d;
  float *conic_opacity;
  float *rgb;
  float *depth;
  int32_t *radius;
  uint16_t *rect;
  uint8_t *clamped;
  int64_t n_records;
} gs_proj_t;

/* Per-tile depth-sorted lists (device). vals [capacity]: record indices ordered by
 * (global tile, FP32 depth bits, record index); keys [capacity] optional (may be
 * NULL): tile << 32 | depth bits of the same entries; ranges [n_tiles][2]: start,
 * end of each tile in vals (start == end for an empty tile); d_count [1] (int64):
 * the number of entries M, written by gs_bin_sort. */
typedef struct {
  uint32_t *vals;
  uint64_t *keys;
  uint32_t *ranges;
  int64_t *d_count;
  int64_t capacity;
} gs_bins_t;

typedef struct {
  float bg[3];             /* background colour (default black)                   */
  int32_t store_stop;      /* write the per-pixel stop index in gs_raster_fwd     */
  int32_t stage_depth;     /* gs_raster_bwd: list entries staged per CTA step,
                            * 0 = one per thread, 1 = half as many. A tuning
                            * knob: gradients agree up to summation order. */
  uint32_t *d_queue;       /* gs_raster_fwd / gs_raster_fwd_ckpt: NULL = one CTA
                            * per tile; else a device word (overwritten) that a
                            * persistent grid's warps claim (tile, 8x8 block)
                            * units from. A tuning knob: images are identical. */
} gs_raster_cfg_t;

/* Gradients of the loss w.r.t. the projected records (device, [R] rows, same row
 * layout as gs_proj_t): d_mean2d [R][2], d_conic_opacity [R][4], d_rgb [R][4].
 * gs_raster_bwd OVERWRITES them (it clears them, then accumulates). */
typedef struct {
  float *d_mean2d;
  float *d_conic_opacity;
  float *d_rgb;
} gs_rec_grads_t;

/* Gradients w.r.t. the Gaussian parameters (device, same shapes as gs_params_t;
 * d_sh uses the params' sh_stride). gs_project_bwd OVERWRITES them. */
typedef struct {
  float *d_means;
  float *d_log_scales;
  float *d_quats;
  float *d_opacity_logits;
  float *d_sh;
} gs_param_grads_t;

/* ---------------------------------------------------------------------- host helpers */

const char *gs_status_str(gs_status_t s);
const char *gs_version(void);

/* Number of CUDA kernels this library has enqueued since it was loaded (a host-side
 * counter; graph replays of captured launches are not counted again). */
uint64_t gs_launch_count(void);

/* Nonzero when the tile shape tile_w x tile_h has compiled kernels. */
int32_t gs_tile_supported(int32_t tile_w, int32_t tile_h);

/* Fill the layout fields of cams_host[0..n_views) and the frame's counts (tile grid
 * per view, global tile and pixel offsets). Host memory only; cams_dev is left for
 * the caller to set after copying cams_host to the device. */
gs_status_t gs_frame_init(gs_camera_t *cams_host, int32_t n_views, int32_t tile_w,
                          int32_t tile_h, gs_frame_t *frame);

/* Bytes of scratch gs_bin_sort needs for n_records records and dup_capacity
 * duplicates on this frame (NULL frame: the most any frame needs); 0 for an
 * invalid size or sort_fused_bits. */
size_t gs_bin_sort_workspace_size(int64_t n_records, int64_t dup_capacity, const gs_frame_t *frame);

/* ---------------------------------------------------------------------- hot path */

/* EWA projection + SH colour of every (view, Gaussian) record -- Eq. 1, the paper's
 * Sigma' = J W Sigma W^T J^T, and the SH-evaluated colour c_i of Eq. 2.
 * Readings: near-plane cull; J at the mean with t_x/t_z, t_y/t_z clamped to
 * +-1.3 (W/2)/f; Sigma' + 0.3 I; cull det <= 0 and opacity < 1/255; the footprint
 * is the ellipse where alpha = min(0.99, opacity G) can reach 1/255, d^T Sigma''^-1 d
 * <= 2 ln(255 opacity) (x 1.002), and radius and rect come from its half-extents;
 * cull when the tile rectangle is empty. Culled records get radius 0 and an empty
 * rect; their other fields are zero. */
gs_status_t gs_project(const gs_params_t *params, const gs_frame_t *frame, gs_proj_t *out,
                       gs_stream_t stream);

/* Tile binning and depth sort ("tile-based", "depth-sorted"; Sec. "Preliminary").
 * Every visible record is duplicated into each tile of its rectangle whose box of
 * pixel centres its footprint ellipse (alpha >= 1/255, with a 0.2% margin) meets;
 * duplicates are ordered by (global tile, FP32 depth bits, record index) and the
 * per-tile ranges written. The capacity also holds, while the lists are built, one
 * entry per tile row of each visible record's rectangle (in practice fewer than M).
 * Device-side: if M or that row count exceeds bins->capacity, GS_ERR_CAPACITY is
 * OR-ed into *d_error, *bins->d_count receives the larger of the two (the capacity
 * needed) and vals holds no lists, every range being [0, 0). */
gs_status_t gs_bin_sort(const gs_proj_t *proj, const gs_frame_t *frame, gs_bins_t *bins,
                        void *ws, size_t ws_bytes, int32_t *d_error, gs_stream_t stream);

/* Front-to-back alpha compositing, Eq. 2, per pixel over its tile's list:
 * sigma = min(0.99, o exp(P)), entries with P > 0 or sigma < 1/255 skipped, the walk
 * stops before the entry that would make T < 1e-4; out = C + T bg.
 * image [3 * n_pixels] planar per view; T_final [n_pixels]; stop [n_pixels] (one
 * past the last contributing list position) written when cfg->store_stop and stop
 * is not NULL. */
gs_status_t gs_raster_fwd(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                          const gs_raster_cfg_t *cfg, float *image, float *T_final,
                          uint32_t *stop, gs_stream_t stream);

/* Work count of Eq. 2 (a measurement aid, not part of training): runs the forward's
 * per-pixel walk and writes, per pixel, counts[2p] = list entries examined up to and
 * including the one that triggers the transmittance cut-off (or the whole list) and
 * counts[2p+1] = entries composited. counts [n_pixels][2], 8-byte aligned. */
gs_status_t gs_raster_count(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                            uint32_t *counts, gs_stream_t stream);

/* L1 photometric loss (the L1 term of Eq. 3) per view, mean over 3*H*W:
 * d_image = sign(image - target) / (3 H W) (0 at equality); loss_dev [n_views]
 * receives each view's loss (overwritten). */
gs_status_t gs_l1_loss_grad(const gs_frame_t *frame, const float *image, const float *target,
                            float *d_image, float *loss_dev, gs_stream_t stream);

/* Gradient of Eq. 2 w.r.t. every record's mean2d, conic, opacity and colour, given
 * dL/d image. Re-walks each pixel's list front to back with the forward's exact
 * FP32 recurrence. stop (device, [n_pixels], may be NULL) is the forward's per-pixel
 * stop index (gs_raster_fwd with store_stop): each pixel then walks only up to it;
 * with NULL the stop position is recomputed from the transmittance cut-off. Uses
 * dL/dsigma_i = T_i <c_i, g> - (<out, g> - sum_{j<=i} <c_j, g> sigma_j T_j) / (1 - sigma_i),
 * out being the forward's image; zero through the 0.99 clamp. Per-pixel terms are
 * summed per Gaussian in registers, across the warp and the CTA, then added once
 * per (tile, record) into grads (see gs_rec_grads_t). */
gs_status_t gs_raster_bwd(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                          const gs_raster_cfg_t *cfg, const float *image, const float *d_image,
                          const uint32_t *stop, gs_rec_grads_t *grads, gs_stream_t stream);

/* Per-splat backward (the per-splat parallel back-propagation of the Taming-3DGS
 * lineage that the paper's base trainer uses; a measured alternative to
 * gs_raster_bwd, chosen by the autotuner). Same gradient as gs_raster_bwd (up to
 * summation order), parallel over list entries: each tile's list is cut into
 * buckets of 64 entries, two consecutive entries per lane, and the tile's pixels
 * flow through each bucket from a checkpoint the forward stored at its first
 * position.
 *
 * Checkpoints are stored per (bucket, 8 x 8 pixel block) that the forward actually
 * walks, in 1 KB slots (64 pixels x float4); a table of 4 bytes per possible
 * (bucket, block) pair locates them. The slot count is the caller's choice: a
 * buffer with a slot for every pair cannot overflow; a smaller one (sized from a
 * measured gs_raster_ckpt_usage with headroom, as the duplicate capacity is) holds
 * only the walked pairs, and a forward that needs more reports it through
 * gs_raster_ckpt_usage and leaves the excess pairs without checkpoints (the
 * backward then treats them as T = 1, so the gradients are wrong until the caller
 * grows the buffer and runs the step again).
 *
 * gs_raster_ckpt_size: bytes of a checkpoint buffer with n_slots slots for a frame
 * whose lists hold at most `capacity` entries (the gs_bins_t capacity); n_slots < 0
 * gives a slot for every possible (32-entry table row, block) pair, (ceil(capacity
 * / 32) + n_tiles) x tile_w tile_h / 64 (only every other row is used). 0 for an
 * invalid frame or capacity.
 *
 * gs_raster_fwd_ckpt: gs_raster_fwd that always writes stop [n_pixels] and also,
 * for every pixel still compositing at list position 64 b of its tile, the float4
 * (T, R, G, B) of the state before that position (transmittance and the colour
 * composited so far) into ckpt. ckpt: device, 16-byte aligned, ckpt_bytes at least
 * gs_raster_ckpt_size(frame, bins->capacity, 0); its slot count is what the bytes
 * beyond that hold. Layout is private to these calls.
 *
 * gs_raster_ckpt_usage: d_usage [2] (device int64) <- (slots the last
 * gs_raster_fwd_ckpt on this buffer needed, 1 if it ran out of slots else 0).
 *
 * gs_raster_bwd_splat: gradient of Eq. 2 from the image, stop and ckpt of the
 * gs_raster_fwd_ckpt call on the same bins; dL/dsigma as in gs_raster_bwd.
 * OVERWRITES grads (clears, then accumulates once per (tile, list entry)). */
size_t gs_raster_ckpt_size(const gs_frame_t *frame, int64_t capacity, int64_t n_slots);
gs_status_t gs_raster_ckpt_usage(const gs_frame_t *frame, int64_t capacity, const void *ckpt,
                                 size_t ckpt_bytes, int64_t *d_usage, gs_stream_t stream);
gs_status_t gs_raster_fwd_ckpt(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                               const gs_raster_cfg_t *cfg, float *image, float *T_final, uint32_t *stop,
                               void *ckpt, size_t ckpt_bytes, gs_stream_t stream);
gs_status_t gs_raster_bwd_splat(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                const float *image, const float *d_image, const uint32_t *stop,
                                const void *ckpt, size_t ckpt_bytes, gs_rec_grads_t *grads,
                                gs_stream_t stream);

/* Vector-Jacobian product of gs_project: record gradients -> parameter gradients,
 * summed over views (chain rule through the conic inverse, Sigma' = J W Sigma W^T J^T,
 * Sigma = R S S^T R^T, the quaternion normalisation, exp scales, the J clamp, the
 * pinhole mean, SH colour with its clamp and direction, and the opacity sigmoid).
 * If densify_accum / densify_count are not NULL the densification statistic of
 * gs_densify_accum is fused in. */
gs_status_t gs_project_bwd(const gs_params_t *params, const gs_frame_t *frame,
                           const gs_proj_t *proj, const gs_rec_grads_t *rec_grads,
                           gs_param_grads_t *out, float *densify_accum,
                           int32_t *densify_count, gs_stream_t stream);

/* ---------------------------------------------------------------------- densification */

typedef enum {
  GS_DENSIFY_ADAPTIVE = 0,   /* split if large, clone otherwise (the standard rule)      */
  GS_DENSIFY_SPLIT_ONLY = 1, /* global phase of global-to-local: clone disabled          */
  GS_DENSIFY_ALL_SPLIT = 2,  /* every selected Gaussian splits (split-only analysis)     */
  GS_DENSIFY_ALL_CLONE = 3   /* every selected Gaussian clones (clone-only analysis)     */
} gs_densify_mode_t;

typedef struct {
  int32_t mode;              /* gs_densify_mode_t                                         */
  float grad_threshold;      /* 2e-4: select when accum/count > this                      */
  float log_scale_threshold; /* split when max log-scale > this (FP32 of log(0.01 extent)) */
  int32_t prune_adaptive;    /* 0: fixed logit threshold; 1: adaptive order statistic     */
  float prune_logit;         /* fixed: prune when logit < prune_logit                     */
  float prune_upper_logit;   /* adaptive: FP32 logit(tau_u)                               */
  double prune_ratio;        /* adaptive: p, k = min(floor(N' p), N' - 1)                 */
  uint64_t seed;             /* Philox key for split children                             */
  uint32_t event;            /* densification event counter (Philox counter word 2)      */
} gs_densify_cfg_t;

/* View-space gradient statistic (Sec. "Preliminary": norm of the average position
 * gradient): for each view v in order and Gaussian g with radius > 0,
 * accum[g] += sqrt(gx^2 + gy^2), (gx, gy) = d_mean2d[v*n+g] * (W_v/2, H_v/2),
 * count[g] += 1 (FP32, one rounding per operation). */
gs_status_t gs_densify_accum(const float *d_mean2d, const int32_t *radius, const gs_frame_t *frame,
                             int64_t n, float *accum, int32_t *count, gs_stream_t stream);

size_t gs_densify_workspace_size(int64_t n);

/* Split/clone masks and the pruning threshold. split[g], clone[g] in {0,1};
 * *d_tau_logit receives the prune threshold in logit space (fixed, or
 * min(k-th smallest logit of the post-densification multiset, prune_upper_logit)
 * for adaptive pruning, Sec. "Adaptive Opacity Pruning"); *d_new_n receives the
 * Gaussian count after densification and pruning. */
gs_status_t gs_densify_select(const gs_densify_cfg_t *cfg, const float *log_scales,
                              const float *opacity_logits, const float *accum,
                              const int32_t *count, int64_t n, uint8_t *split, uint8_t *clone,
                              float *d_tau_logit, int64_t *d_new_n, void *ws, size_t ws_bytes,
                              gs_stream_t stream);

/* Allocation-free variant of gs_densify_select (the paper has no counterpart; this is
 * a library-integration entry point). For callers that cannot allocate device memory
 * for a workspace -- custom operators and plugins running inside another runtime's
 * execution callbacks, where allocating is forbidden or would bypass that runtime's
 * memory accounting, and fixed-budget deployments that must not grow their device
 * footprint at run time. Same arguments, results and stream semantics as
 * gs_densify_select, without ws / ws_bytes: the scratch (1,056 bytes: the selection
 * counters and a 256-bin histogram) lives in a file-scope device array of the
 * library that every GPU loading the library holds until the process exits.
 *  - n must not exceed GS_DENSIFY_SELECT_STATIC_MAX_N (the scratch's 32-bit
 *    histogram counts); larger n returns GS_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address on the current
 *    device (cudaGetSymbolAddress) and caches it; make that first call before any
 *    stream capture on the device.
 *  - The cached address is not valid across cudaDeviceReset: after a reset of a
 *    device in the same process the next call would use a stale device address.
 *    Do not reset a device between calls to this entry point.
 *  - Every call shares the one array and clears it on its stream before use; calls
 *    that overlap on the GPU (different streams, or concurrent threads) race on it.
 *  - Calls no cudaMalloc, cudaFree or allocating routine. */
#define GS_DENSIFY_SELECT_STATIC_MAX_N (1ll << 30)
gs_status_t gs_densify_select_static(const gs_densify_cfg_t *cfg, const float *log_scales,
                                     const float *opacity_logits, const float *accum,
                                     const int32_t *count, int64_t n, uint8_t *split, uint8_t *clone,
                                     float *d_tau_logit, int64_t *d_new_n, gs_stream_t stream);

/* One extra per-Gaussian float array carried through compaction (e.g. an optimiser
 * moment): survivors keep their row, new rows are zero. */
typedef struct {
  const float *src;
  float *dst;
  int32_t width;           /* floats per Gaussian */
} gs_extra_array_t;

/* Output parameter arrays of gs_densify_apply (device, capacity rows each). */
typedef struct {
  float *means;
  float *log_scales;
  float *quats;
  float *opacity_logits;
  float *sh;
} gs_params_out_t;

/* Per-Gaussian provenance carried through compaction (the split/clone analysis of
 * Sec. "Global-to-local framework"): origin = index of the Gaussian of the initial
 * set a row descends from, splits / clones = how many split / clone operations lie
 * on its lineage. Survivors keep their values; the copy a clone adds inherits its
 * parent's and adds 1 to clones; both children of a split inherit the parent's and
 * add 1 to splits. Inputs have n rows, outputs out_capacity rows (device int32). */
typedef struct {
  const int32_t *origin_in, *splits_in, *clones_in;
  int32_t *origin_out, *splits_out, *clones_out;
} gs_provenance_t;

/* Densify + prune + compaction. Output rows: survivors (kept, not split) in
 * original order, then clones in parent order, then split children in parent order
 * (child 0, child 1); a row is kept iff its (inherited) logit >= *d_tau_logit.
 * Child: log-scale - FP32(log 1.6), mean + R(q) (exp(s) * z), z ~ N(0, I) from
 * Philox4x32-10 (Salmon et al., SC'11) with counter (parent, 0, event, child) and key
 * (seed), Box-Muller on u = ((x >> 8) + 0.5) 2^-24. prov (NULL: none) carries the
 * provenance arrays (all six pointers set). If the new count exceeds out_capacity,
 * GS_ERR_CAPACITY is OR-ed into *d_error and nothing is written. */
gs_status_t gs_densify_apply(const gs_densify_cfg_t *cfg, const gs_params_t *in,
                             const uint8_t *split, const uint8_t *clone,
                             const float *d_tau_logit, gs_params_out_t *out,
                             const gs_extra_array_t *extra, int32_t n_extra,
                             const gs_provenance_t *prov,
                             int64_t out_capacity, int64_t *d_new_n, int32_t *d_error,
                             void *ws, size_t ws_bytes, gs_stream_t stream);

/* Debug builds (libgs_debug.so, compiled with -DGS_DEBUG): the hot path checks its
 * index accesses (record ids from the lists, the lists' ranges, checkpoint table
 * entries and slots, list positions) before making them; a failed check is recorded
 * and the access skipped. gs_debug_status returns the first failure since the last
 * call as (code << 48 | index), 0 if none, and clears it (synchronising the device).
 * Codes: 1 record id >= records, 2 tile range outside the list, 3 checkpoint table
 * index or slot out of range, 4 list position >= capacity. The release library
 * returns GS_ERR_UNSUPPORTED (and 0). */
gs_status_t gs_debug_status(uint64_t *word);

/* ------------------------------------------------------------ training step */
/* Eq. 3: L = (1 - lambda) ||I - I_hat||_1 + lambda D-SSIM(I, I_hat), per view: the L1
 * term as the mean over 3 H W values, D-SSIM = 1 - SSIM with SSIM averaged over the
 * 3 H W values, per channel with an 11 x 11 Gaussian window (sigma 1.5), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2. image, target, d_image: planar batch layout of
 * the frame (device); loss_dev [n_views] overwritten; d_image = dL/dimage
 * (overwritten). ws: 16-byte aligned, gs_photometric_workspace_size bytes. */
size_t gs_photometric_workspace_size(const gs_frame_t *frame);
gs_status_t gs_photometric_loss_grad(const gs_frame_t *frame, const float *image, const float *target,
                                     float lambda, float *d_image, float *loss_dev, void *ws,
                                     size_t ws_bytes, gs_stream_t stream);

/* Adam moments per parameter group (device, same shapes as the parameters), in
 * the order means, log_scales, quats, opacity_logits, sh. */
typedef struct {
  float *m[5];
  float *v[5];
} gs_adam_state_t;

typedef struct {
  float lr[5];             /* per group, same order as gs_adam_state_t */
  float eps;
  double beta1, beta2;     /* double: 1 - beta2^t is formed on the host, and beta2 in
                            * FP32 would move it by ~1e-5 relative at t = 3 */
  int32_t step;            /* 1 for the first step (bias correction) */
} gs_adam_cfg_t;

/* One Adam step in place: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr / (1 - b1^t) m / (sqrt(v) / sqrt(1 - b2^t) + eps), FP32. If radius is not
 * NULL ([n_views][n] record radii of the step's projection), rows of Gaussians no
 * view saw (radius 0 everywhere) are left untouched, moments included ("sparse"
 * Adam). params: the parameter arrays (updated); sh rows of 3 sh_stride floats. */
gs_status_t gs_adam_step(const gs_adam_cfg_t *cfg, gs_params_out_t *params, int64_t n, int32_t sh_stride,
                         const gs_param_grads_t *grads, gs_adam_state_t *state, const int32_t *radius,
                         int32_t n_views, gs_stream_t stream);

/* Opacity reset of the densification schedule: every opacity logit is lowered to
 * at most logit(max_opacity); the opacity moments m, v (may be NULL) are cleared. */
gs_status_t gs_opacity_reset(float *opacity_logits, float *m, float *v, int64_t n, float max_opacity,
                             gs_stream_t stream);

/* ------------------------------------------------- coarse-to-fine schedule energy */
/* Sec. "Energy-aware multi-resolution": the downscaling operator D_r (bilinear with
 * anti-aliasing) and the energy ||E(I)||_1 = sum over channels and frequencies of
 * the magnitude of the 2D DFT. The schedule built on them (E_r = ||E(D_r(I))||_1 r^2,
 * T_r = Round(E_r / E_1 T_densify)) is host arithmetic in the Python binding. */

/* Rows or columns after D_r: floor(n / r + 1/2), at least 1 (0 for bad input). */
int32_t gs_downscaled_size(int32_t n, int32_t r);

/* D_r of a planar image [C][H][W] (device, FP32) into out [C][Hr][Wr] (device,
 * Hr x Wr = gs_downscaled_size of H x W): separable triangle filter of half-width
 * s = W / Wr (rows: H / Hr); output column j samples the input at (j + 1/2) s - 1/2,
 * weights max(0, 1 - |k - c| / s) over the columns inside the image, normalised to
 * sum 1. r = 1 copies. */
gs_status_t gs_downscale(const float *image, int32_t C, int32_t H, int32_t W, int32_t r, float *out,
                         gs_stream_t stream);

/* Bytes of scratch gs_spectrum_l1 needs (0 if C < 1 or H, W outside 1..4096). */
size_t gs_spectrum_workspace_size(int32_t C, int32_t H, int32_t W);

/* ||E(I)||_1 of a planar image [C][H][W] (device, FP32), written to *d_sum (device,
 * one double, overwritten). Unnormalised forward DFT, FP32 products, FP64 sums of the
 * magnitudes. ws: 16-byte aligned, gs_spectrum_workspace_size bytes. */
gs_status_t gs_spectrum_l1(const float *image, int32_t C, int32_t H, int32_t W, double *d_sum, void *ws,
                           size_t ws_bytes, gs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
