/*
 * tgs.h -- C ABI of libtgs, a GB300 (sm_103a) differentiable Gaussian-splatting rasterizer
 * with the learned volume masks and SH-band masks of Trick-GS (arXiv 2501.14534).
 *
 * The library computes, for N Gaussians and V pinhole views:
 *   (a) preprocess: the straight-through volume mask M applied to opacity and scale
 *       (Sec. "Pruning with Volume Masking", mask equation), the EWA projection of each 3D
 *       Gaussian to the 2D Gaussian G'(x) = exp(-1/2 (x-mu')^T Sigma'^-1 (x-mu')) with
 *       Sigma' = J W Sigma W^T J^T + sI (Sec. "Preliminaries", Eq. 1; s = 0.3 from Sec.
 *       "Progressive training by scales of Gaussians"), the footprint radius and pixel rect,
 *       and the view-dependent colour from SH of degree <= 3 with per-band straight-through
 *       masks (Sec. "Spherical Harmonic (SH) Masking", Eq. sh-masks);
 *   (b) key emission of (tile id, depth bits) per touched tile, a stable radix sort and
 *       per-tile ranges;
 *   (c) front-to-back alpha blending C = sum_i c_i a_i prod_{j<i} (1 - a_j) (Eq. 2);
 *   (d) the backward of (c) and (a), including the gradients of the mask logits through the
 *       straight-through estimator, and the 2D-mean gradient-norm statistics used for
 *       densification and pruning (Sec. "Preliminaries": pruning and densification by
 *       gradient magnitudes).
 *
 * Conventions the paper inherits from 3DGS, fixed here:
 *   - camera: world->camera 4x4 row-major matrix, x right, y down, z forward; pixel (px, py)
 *     samples the Gaussian at integer coordinates in the frame mean2d = f t_xy / t_z + c - 1/2;
 *   - near plane: Gaussians with t_z <= near are culled; the Jacobian uses t_x/t_z clamped to
 *     +-1.3 * W / (2 fx) (y likewise) and is differentiated exactly, clamp included;
 *   - radius r = ceil(3 sqrt(lambda_max)) (TGS_SUPPORT_BOX3) or the exact alpha >= 1/255 radius
 *     (TGS_SUPPORT_ALPHA), lambda_max = mid + sqrt(max(0.1, mid^2 - det));
 *   - a Gaussian covers exactly the pixels of its inclusive pixel rect
 *     [ceil(mx - r), floor(mx + r)] x [ceil(my - r), floor(my + r)] clipped to the image, so
 *     the image does not depend on the tile size;
 *   - blending: a = min(0.99, o' G'(p)); fragments with a < 1/255 are skipped; a pixel stops
 *     before the fragment that would bring T below 1e-4; out = C + T_final * bg;
 *   - keys: a Gaussian emits a key for a tile of its rect only if some point of (tile x rect)
 *     has Q = (p - mean2d)^T conic (p - mean2d) <= tau (float32 test, fixed steps, in
 *     tgs_internal.cuh); since tau carries a 1e-3 margin, a dropped tile holds no pixel with
 *     a >= 1/255, so the image is the same as with every tile of the rect;
 *   - colour: c = max(0, 1/2 + sum_l M^l sum_m Y_lm(d) f_lm), d = unit(mean - campos);
 *   - mask thresholds: M = 1 iff logit > float32(log(eps / (1 - eps))).
 *
 * Data layout (all float32 unless stated, device memory, C-contiguous):
 *   Gaussians (structure of arrays): means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z;
 *   normalised inside), opacity_logits [N], sh_dc [N,3], sh_rest [N,15,3] (bands 1..3,
 *   coefficient-major, channel-minor), sh_degree uint8 [N] (optional), mask_logits [N]
 *   (optional), sh_mask_logits [N,3] (optional).
 *   Images: [3,H,W] planar RGB. T_final [H,W]. last [H,W] int32: 1-based position, within
 *   the pixel's tile list, of its last contributing Gaussian (0: none).
 *   Splat record (one per (view, Gaussian), 16 x 32 bit, index v * N + g):
 *     [0..1] mean2d, [2..4] conic a, b, c of Sigma'^-1 = [[a, b], [b, c]], [5] opacity o',
 *     [6..8] rgb, [9] uint32 x_lo | x_hi << 16, [10] uint32 y_lo | y_hi << 16, [11] depth t_z,
 *     [12] cull threshold tau = 2 ln(255 o' / (1 - 1e-3)), [13] b / c, [14] b / a, [15] zero.
 *   Splat gradient record (12 floats, same index): dL/d mean2d [0..1], conic a, b, c [2..4]
 *     (with respect to the scalar b of power = -1/2 (a dx^2 + c dy^2) - b dx dy), opacity [5],
 *     rgb [6..8]; [9..11] unused.
 *
 * Ownership: the caller allocates every input and output pointer passed in (device memory
 * unless stated). A tgs_ctx owns a device scratch arena (sort buffers, splat records, key
 * lists) that it grows on demand outside stream capture and frees in tgs_destroy. Nothing is
 * freed across the ABI. Calls are asynchronous on the given stream except where stated.
 * The calls on one context share its arena: they must not overlap on the GPU (issue them on
 * one stream, or give each stream or host thread a context of its own).
 *
 * Errors: every call returns a tgs_status; no C++ exception crosses the ABI. Errors found on
 * the device (key capacity overflow, key counts that fail the emission's consistency check)
 * are recorded in a device status word and returned by tgs_poll_status (which synchronises
 * the stream). No kernel waits on another block or launch, so no call can hang on the device;
 * the work of every kernel is bounded by its launch sizes and the key capacity.
 */
#ifndef TGS_H
#define TGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tgs_status;
#define TGS_OK 0
#define TGS_ERR_INVALID_ARG 1   /* a pointer, size or setting is out of range */
#define TGS_ERR_CUDA 2          /* a CUDA runtime call failed */
#define TGS_ERR_CAPACITY 3      /* more (Gaussian, tile) keys than the key capacity */
#define TGS_ERR_TIMEOUT 4       /* reserved: no kernel of the library waits on another, so no call
                                   returns it */
#define TGS_ERR_OOM 5           /* device memory for the scratch arena could not be had */
#define TGS_ERR_NOT_SUPPORTED 6 /* e.g. a tile size or launch shape that is not compiled */
#define TGS_ERR_SCRATCH_LIMIT 7 /* input larger than the fixed scratch of tgs_bin_noalloc */
#define TGS_ERR_INCONSISTENT 8  /* a device-side check of scratch data failed: the per-record key
                                   counts of a block did not add up to the keys the count pass
                                   scanned for it; that block emitted no keys and the step's
                                   results are invalid (returned by tgs_poll_status) */

#define TGS_SUPPORT_BOX3 0      /* 3-sigma square box (3DGS) */
#define TGS_SUPPORT_ALPHA 1     /* smallest box outside which a < 1/255 */

#define TGS_MAX_VIEWS 64        /* views per call */

/* flags */
#define TGS_ACCUMULATE 1u       /* add parameter gradients into the outputs instead of overwriting */
#define TGS_NO_SH_REST_GRAD 2u  /* skip dL/d sh_rest (SH rest bands updated every 16 steps) */
#define TGS_USE_GRAPH 4u        /* batched step: replay a captured CUDA graph when arguments repeat */
#define TGS_UNFUSED 8u          /* batched step: separate forward, loss and backward kernels (A/B) */
#define TGS_LOSS_DSSIM 16u      /* batched step: loss (1 - lambda) L1 + lambda D-SSIM (Eq. loss3dgs),
                                   lambda = tgs_config.ssim_lambda; implies separate kernels */
#define TGS_MASK_LOSS 32u       /* add the mask losses lambda_m L_m + lambda_sh L_sh of Eq. loss3dgs
                                   (see tgs_mask_loss) to the gradients of the mask logits, folded
                                   into the preprocess backward (once per call, not per view), and,
                                   in the batched step, to the loss */

typedef struct tgs_ctx tgs_ctx;
typedef void *tgs_stream; /* a cudaStream_t; NULL is the legacy default stream */

typedef struct {
    int32_t tile;          /* tile edge in pixels: 8, 16 or 32 */
    int32_t ppt;           /* pixels per thread in the blend kernels: 1, 2 or 4 */
    int32_t support;       /* TGS_SUPPORT_BOX3 or TGS_SUPPORT_ALPHA */
    float low_pass;        /* s of Sigma' + sI (default 0.3) */
    float eps_mask;        /* volume-mask threshold eps_m (default 0.05) */
    float eps_sh;          /* SH-band-mask threshold eps_sh (default 0.1) */
    float near_plane;      /* default 0.2 */
    float bg[3];           /* background colour (default 0) */
    int64_t key_capacity;  /* (Gaussian, tile) keys the batched path may hold; 0 = sized by tgs_plan */
    int64_t spin_limit;    /* reserved (no kernel waits on another); ignored, default 0 */
    float ssim_lambda;     /* lambda_SSIM of Eq. loss3dgs for TGS_LOSS_DSSIM, in [0, 1] (default 0.2) */
    float lambda_mask;     /* lambda_m of Eq. loss3dgs for TGS_MASK_LOSS, >= 0 (default 0.05) */
    float lambda_sh_mask;  /* lambda_sh of Eq. loss3dgs for TGS_MASK_LOSS, >= 0 (default 0.05) */
    int32_t batch;         /* Gaussians staged per shared-memory batch of the fused blend, as a
                              multiple of its threads: 1 or 2 (0 = 1); tuned by tgs_autotune */
} tgs_config;

#define TGS_PARAM_F32 0         /* parameter arrays hold float32 */
#define TGS_PARAM_F16 1         /* parameter arrays hold IEEE half (FP16 storage; render path only) */

typedef struct {
    int64_t n;                   /* number of Gaussians */
    int32_t sh_degree_max;       /* 0..3; rest bands above it are not read */
    int32_t param_dtype;         /* TGS_PARAM_F32 (0) or TGS_PARAM_F16: every float array below
                                    then holds halves of the same shape; accepted by
                                    tgs_preprocess, tgs_forward and tgs_count_hits, the other
                                    calls return TGS_ERR_NOT_SUPPORTED */
    const float *means;          /* [n,3] */
    const float *log_scales;     /* [n,3] */
    const float *quats;          /* [n,4] */
    const float *opacity_logits; /* [n] */
    const float *sh_dc;          /* [n,3] */
    const float *sh_rest;        /* [n,15,3]; may be NULL when sh_degree_max == 0 */
    const uint8_t *sh_degree;    /* [n] or NULL */
    const float *mask_logits;    /* [n] or NULL: no volume mask */
    const float *sh_mask_logits; /* [n,3] or NULL: no band masks */
} tgs_gaussians;

typedef struct {
    float viewmat[16];  /* world -> camera, row-major */
    float campos[3];    /* camera centre in world space */
    float fx, fy, cx, cy;
    int32_t width, height;
    float low_pass;     /* per-view s; <= 0 selects tgs_config.low_pass */
} tgs_camera;           /* host memory */

typedef struct {
    float *image;        /* [3,H,W] */
    float *T_final;      /* [H,W] or NULL */
    int32_t *last;       /* [H,W] or NULL */
    int32_t *n_examined; /* [H,W] or NULL: list entries each pixel looked at */
    int32_t *radii;      /* [n] or NULL */
    int32_t *n_contrib;  /* [H,W] or NULL: fragments blended into the pixel */
    int32_t *n_eval;     /* [H,W] or NULL: fragments whose rect holds the pixel, evaluated
                            before the pixel stopped (the blend's algorithmic work) */
} tgs_view_out;

typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *sh_dc, *sh_rest, *mask_logits,
        *sh_mask_logits; /* same shapes as the inputs; NULL = not wanted */
} tgs_grads;

typedef struct {
    float *grad_norm_accum; /* [n] += |dL/d mean2d|_2 (pixels) per view where visible, or NULL */
    int32_t *vis_count;     /* [n] += 1 per view where visible, or NULL */
    int32_t *max_radius;    /* [n] = max(max_radius, radius), or NULL */
    uint32_t *hit_count;    /* [n] += pixels whose forward blend blends the Gaussian, or NULL: the
                               ray hits of the significance score (Eq. significance-score);
                               counted by the batched step when not NULL */
} tgs_stats;

/* --- context ------------------------------------------------------------------------ */

/* Fills *cfg with the defaults named in tgs_config. */
void tgs_default_config(tgs_config *cfg);
/* Creates a context on the current CUDA device. cfg may be NULL (defaults). */
tgs_status tgs_create(tgs_ctx **out, const tgs_config *cfg);
void tgs_destroy(tgs_ctx *ctx);
tgs_status tgs_get_config(const tgs_ctx *ctx, tgs_config *cfg);
/* Replaces the settings (tile, ppt, thresholds ...). Invalidates captured graphs. */
tgs_status tgs_set_config(tgs_ctx *ctx, const tgs_config *cfg);
const char *tgs_status_string(tgs_status s);
/* Synchronises the stream, returns and clears the device status word. */
tgs_status tgs_poll_status(tgs_ctx *ctx, tgs_stream stream);

/* --- the plain single-view path (3DGS-like: one host read-back of the key count) ---- */

/* Renders each view in turn (preprocess, keys, sort, blend). The binning of the last view
   rendered stays in the context so that an immediately following tgs_backward of that view
   reuses it; other views are re-binned in tgs_backward (per-view checkpointing).
   Synchronises the stream once per view to size the key buffers. */
tgs_status tgs_forward(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                       const tgs_view_out *outs, uint32_t flags, tgs_stream stream);
/* Backward of tgs_forward given dL/d image per view (device [3,H,W] each) and each view's
   saved T_final and last (outs[v].T_final, outs[v].last). Writes (or with TGS_ACCUMULATE
   adds) parameter gradients summed over the V views, and adds statistics. */
tgs_status tgs_backward(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams,
                        int32_t V, const tgs_view_out *outs, const float *const *dL_dimages,
                        const tgs_grads *grads, const tgs_stats *stats, uint32_t flags,
                        tgs_stream stream);
/* L1 loss of one image: *loss += scale * sum |img - target|, grad = scale * sign(img -
   target) (sign(0) = 0). count = 3 H W. loss_accum is a device float. */
tgs_status tgs_l1_loss(const float *image, const float *target, int64_t count, float scale,
                       float *loss_accum, float *grad, tgs_stream stream);
/* L1 + D-SSIM loss of Eq. loss3dgs (its mask terms excluded) over V views of any sizes:
   *loss_accum += mean over views of ((1 - lambda) mean_3HW |x - y| + lambda (1 - SSIM(x, y))),
   grads[v] = dL/d images[v] (overwritten). images, targets, grads: host arrays of V device
   pointers to [3,H,W] planar images, the sizes taken from cams[v].width, height (the rest of
   the camera is not read). SSIM per channel as 3DGS trains it (Wang et al.): local means,
   variances and covariance under an 11 x 11 Gaussian window of sigma 1.5 normalised to sum 1,
   the image taken as 0 outside its border, C1 = 0.01^2, C2 = 0.03^2, averaged over the 3HW
   outputs; the window sums run as two 1D passes (Sec. "Accelerated training"). loss_accum may
   be NULL. The context provides scratch (3 floats per element; grown outside stream capture,
   else TGS_ERR_CAPACITY). lambda in [0, 1], else TGS_ERR_INVALID_ARG. Asynchronous. */
tgs_status tgs_l1_dssim_loss(tgs_ctx *ctx, const tgs_camera *cams, int32_t V, const float *const *images,
                             const float *const *targets, float lambda, float *loss_accum,
                             float *const *grads, tgs_stream stream);

/* Mask losses of Eq. loss3dgs: adds lambda_m L_m + lambda_sh L_sh (tgs_config.lambda_mask,
   lambda_sh_mask) to *loss_accum (device float, or NULL) and their gradients to
   grads->mask_logits and grads->sh_mask_logits (device, always added to; NULL fields and absent
   logit arrays are skipped). The paper fixes the weights (0.05 each) and that each SH band's
   masking loss is weighted by its number of coefficients (Sec. "Spherical Harmonic (SH)
   Masking"), and leaves the definitions to the cited works; this library takes
     L_m  = (1/N) sum_n sigmoid(m_n),
     L_sh = (1/N) sum_n sum_{l=1..3} (2l + 1) / 15 * sigmoid(m_n^l),
   over every Gaussian and band, visible or not. The batched step, tgs_backward and
   tgs_preprocess_backward do the same when given TGS_MASK_LOSS. Asynchronous. */
tgs_status tgs_mask_loss(tgs_ctx *ctx, const tgs_gaussians *g, float *loss_accum, const tgs_grads *grads,
                         tgs_stream stream);

/* --- the batched path ---------------------------------------------------------------- */

/* Sizes the key capacity for these views: runs preprocess and the key count once, waits,
   and sets capacity = ceil(headroom * K). */
tgs_status tgs_plan(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                    double headroom, int64_t *keys_out);
/* One training step over V views of any sizes: preprocess of all views, one key sort, a
   persistent fused forward + L1 loss + backward over (view, tile) work items heaviest first
   (TGS_UNFUSED: one forward launch, V loss launches and one backward launch instead), and
   the preprocess backward. loss_out (device float) = mean over views of mean |C - t|; with
   TGS_LOSS_DSSIM the loss of tgs_l1_dssim_loss at lambda = tgs_config.ssim_lambda, whose
   gradient is not pixel-local, so forward, loss and backward run as separate launches.
   images (optional, host array of V device pointers) receives the rendered views.
   Never synchronises; with TGS_USE_GRAPH the whole step is captured once into a CUDA graph
   and replayed while g, cams, targets, images, grads, stats and loss_out are unchanged.
   A key-capacity overflow sets TGS_ERR_CAPACITY in the device status word. */
tgs_status tgs_train_step_batched(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams,
                                  int32_t V, const float *const *targets, float *const *images,
                                  const tgs_grads *grads, const tgs_stats *stats,
                                  float *loss_out, uint32_t flags, tgs_stream stream);
/* The batched step for a caller whose parameters and target images live in host memory (a
   data loader on the CPU, an application without device buffers of its own): one call copies
   every parameter array of g_host (host pointers, same layouts as tgs_gaussians, float32) and
   the V target images (host [3,H,W] each) into device buffers the context owns, runs
   tgs_train_step_batched on them, and copies the loss into *loss_host (host float, may be
   NULL). grads and stats are device memory, as for tgs_train_step_batched.
   The copies go on an upload stream of the context, one cudaMemcpyAsync per array, into one
   of three buffer sets used in turn, so that the next calls' copies overlap this call's step
   (up to two steps ahead); the step waits for its copies, and the copies into a set wait for
   the step that last read it. Host buffers should be pinned (cudaHostAlloc / cudaHostRegister) for the copies to be
   asynchronous, and must not change until the copies have run (e.g. until the next call
   returns, or a stream synchronisation). With TGS_USE_GRAPH each buffer set keeps its own
   captured graph. Not capturable (TGS_ERR_NOT_SUPPORTED inside stream capture); the first
   calls, and any call with larger inputs than before, allocate (and synchronise). */
tgs_status tgs_train_step_batched_host(tgs_ctx *ctx, const tgs_gaussians *g_host, const tgs_camera *cams,
                                       int32_t V, const float *const *targets_host, const tgs_grads *grads,
                                       const tgs_stats *stats, float *loss_host, uint32_t flags,
                                       tgs_stream stream);
/* Forward-only render of V views of any sizes through the batched machinery (Eq. 2; the FPS
   protocol of the paper's experiments renders trained scenes this way, one view after another):
   preprocess of all V views, one binning at the context's planned key capacity, one forward blend
   launch over every (view, tile). outs[v].image ([3,H,W], required), T_final, last, n_examined,
   n_contrib and n_eval (each optional) are device buffers written as by tgs_forward; radii are
   not written (leave NULL).
   Accepts FP16 parameters. Never synchronises while the key capacity is planned (tgs_plan; if it
   is 0 the call plans first, one synchronisation), so it may run inside stream capture; with
   TGS_USE_GRAPH the work is captured into a CUDA graph once and replayed while g, cams, V, outs
   and the config repeat. A key-capacity overflow sets TGS_ERR_CAPACITY in the status word. */
tgs_status tgs_render_batched(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                              const tgs_view_out *outs, uint32_t flags, tgs_stream stream);
/* Times the batched step for tile in {8, 16, 32} x ppt in {1, 2, 4} x batch in {1, 2} (the
   supported combinations; 2 warm-up and 3 timed steps each) and keeps the fastest in the
   context's config, with a key capacity planned for it. cache_path (may be NULL) is a JSON file
   {"n<N>_V<V>_<W>x<H>...": {"tile": T, "ppt": P, "batch": B}, ...}: an entry for these Gaussian
   count and view sizes is adopted without timing; otherwise the result is added and the file
   rewritten. Synchronises the stream. Images do not depend on the choice (a Gaussian covers
   the pixels of its rect, whatever the tile). */
tgs_status tgs_autotune(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                        const float *const *targets, const char *cache_path,
                        tgs_stream stream);

/* --- the individual steps (caller-owned buffers) --------------------------------------- */

/* (a) Writes splat records [V*n,16] and radii [V*n] (0 = culled). */
tgs_status tgs_preprocess(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams,
                          int32_t V, float *splats, int32_t *radii, tgs_stream stream);
/* (b) From splat records and radii: sorted Gaussian record indices (v*n + g) in tile order,
   the sorted 64-bit keys ((global tile << 32) | float32 bits of depth, or NULL) and per-tile
   [start, end) ranges [tiles,2] (uint32). Global tile ids count the views' tiles in order,
   row-major within a view. Synchronises once to read the key count K into *K_out; returns
   TGS_ERR_CAPACITY without sorting when K > capacity. */
tgs_status tgs_bin(tgs_ctx *ctx, const float *splats, const int32_t *radii, int64_t n,
                   const tgs_camera *cams, int32_t V, uint32_t *sorted_ids, uint64_t *sorted_keys,
                   uint32_t *ranges, int64_t capacity, int64_t *K_out, tgs_stream stream);
/* (c) Forward blend of V views from the binned lists. */
tgs_status tgs_blend_forward(tgs_ctx *ctx, const float *splats, const uint32_t *sorted_ids,
                             const uint32_t *ranges, const tgs_camera *cams, int32_t V,
                             const tgs_view_out *outs, tgs_stream stream);
/* (d) Backward blend: adds into splat gradient records [V*n,12] (zero them first). */
tgs_status tgs_blend_backward(tgs_ctx *ctx, const float *splats, const uint32_t *sorted_ids,
                              const uint32_t *ranges, const tgs_camera *cams, int32_t V,
                              const tgs_view_out *outs, const float *const *dL_dimages,
                              float *splat_grads, tgs_stream stream);
/* (e) Backward preprocess: parameter gradients (overwritten, or added with TGS_ACCUMULATE)
   summed over the V views, and statistics (always added). */
tgs_status tgs_preprocess_backward(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams,
                                   int32_t V, const float *splat_grads, const int32_t *radii,
                                   const tgs_grads *grads, const tgs_stats *stats,
                                   uint32_t flags, tgs_stream stream);

/* --- binning without any device allocation ------------------------------------------ */

/* Limits of tgs_bin_noalloc: (view, Gaussian) records (n * V) and (Gaussian, tile) keys. */
#define TGS_NOALLOC_MAX_RECORDS 131072
#define TGS_NOALLOC_MAX_KEYS 524288

/* The same binning as tgs_bin -- same outputs, bit for bit -- for callers that cannot call
   cudaMalloc: a host application that hands all device memory to its own allocator or
   memory pool, a real-time loop that must not pay for an allocation, or code under a fixed
   device-memory budget. The paper has no counterpart; this is a deployment variant.
   It needs no tgs_ctx and allocates nothing. Its scratch is one fixed array of about 13.4 MB
   of device memory that is part of the library image, so every GPU that loads libtgs holds
   it until the process exits. The caller still allocates every output: sorted_ids
   [capacity], sorted_keys [capacity] (or NULL) and ranges [tiles,2]; splats are [n*V,16]
   records as tgs_preprocess writes them. tile is 8, 16 or 32.
   Limits: n * V <= TGS_NOALLOC_MAX_RECORDS, else TGS_ERR_SCRATCH_LIMIT without launching
   anything; K <= TGS_NOALLOC_MAX_KEYS, else TGS_ERR_SCRATCH_LIMIT after counting the keys
   (*K_out is set); K > capacity gives TGS_ERR_CAPACITY (*K_out is set).
   The first call on a device looks up the array's device address (cudaGetSymbolAddress,
   once per device, under a lock) and caches it; make that first call before any stream
   capture. Like tgs_bin it synchronises the stream once to read K.
   All calls share the one array, which keeps the previous call's contents (the call clears
   what must start at zero). Calls that overlap on the GPU -- on two streams, or from two
   host threads -- race on it and give wrong results: serialise them. */
tgs_status tgs_bin_noalloc(const float *splats, const int32_t *radii, int64_t n,
                           const tgs_camera *cams, int32_t V, int32_t tile, uint32_t *sorted_ids,
                           uint64_t *sorted_keys, uint32_t *ranges, int64_t capacity,
                           int64_t *K_out, tgs_stream stream);

/* --- significance pruning (Eq. significance-score) ---------------------------------- */

/* Ray hits of the significance score: renders the V views (forward only, nothing else
   written) and adds to hit_count [n] (device, uint32) the number of pixels of each view
   whose blend (Eq. 2) blends the Gaussian -- alpha >= 1/255 and before the pixel's stop.
   Same decisions as tgs_forward. All V views are preprocessed, binned and blended together
   (scratch for n * V records and all their keys); synchronises the stream once to read the key
   count. Errors: TGS_ERR_INVALID_ARG for a null pointer or V <= 0. */
tgs_status tgs_count_hits(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                          uint32_t *hit_count, tgs_stream stream);
/* Significance score of each Gaussian, scores [n] (device float):
   GS_j = hits_j * alpha_j * gamma_j, with hits_j = hit_count[j] summed over the training
   views, alpha_j = M_j sigmoid(o_j) the opacity the blend uses and gamma_j = min(V_j / V_q, 1)
   the volume V_j = s_x s_y s_z (masked scales M exp(l)) relative to V_q, the volume at rank
   floor(quantile * (n - 1)) of all n volumes in ascending order (gamma = 1 where V_q = 0).
   quantile in [0, 1] (the paper normalises at the 90 % point: 0.9). Uses the context's mask threshold.
   Asynchronous; TGS_ERR_INVALID_ARG for a null pointer or a quantile outside [0, 1]. */
tgs_status tgs_significance(tgs_ctx *ctx, const tgs_gaussians *g, const uint32_t *hit_count,
                            double quantile, float *scores, tgs_stream stream);
/* The significance-pruning schedule (Sec. "Implementation details": pruning applied a fixed
   number of times, 60 % of the Gaussians the first time, the rate decayed by a constant factor
   each time): fractions[r] = first * decay^r for r < rounds (host array of rounds doubles).
   The paper's values are rounds = 6, first = 0.6, decay = 0.7. Host-only, no device work.
   TGS_ERR_INVALID_ARG for rounds < 0, first or decay outside [0, 1], or a null fractions. */
tgs_status tgs_prune_schedule(int32_t rounds, double first, double decay, double *fractions);
/* The Gaussians a pruning round removes: prune [n] (device bytes) = 1 for the
   floor(fraction * n) lowest scores (equal scores: lower index first), 0 for the others.
   scores [n] device float, non-negative. fraction in [0, 1]. Asynchronous. */
tgs_status tgs_prune_select(tgs_ctx *ctx, const float *scores, int64_t n, double fraction,
                            uint8_t *prune, tgs_stream stream);

/* --- FP16 storage -------------------------------------------------------------------------- */

/* Half-precision copies of the parameter arrays (device, same shapes as tgs_gaussians). */
typedef struct {
    uint16_t *means, *log_scales, *quats, *opacity_logits, *sh_dc, *sh_rest, *mask_logits,
        *sh_mask_logits; /* NULL = not wanted */
} tgs_half_params;

/* The paper's post-processing (Sec. "Experiments", setup): every Gaussian parameter stored
   with 16-bit precision after training. Writes each float32 array of g (param_dtype
   TGS_PARAM_F32) rounded to the nearest IEEE half, ties to even, values beyond the half range
   to +-inf; sh_degree stays uint8. Render from it with param_dtype = TGS_PARAM_F16: the
   preprocess widens each half to float32 exactly, so the images equal those of the float32
   path on the rounded values, bit for bit. Asynchronous. */
tgs_status tgs_params_to_half(const tgs_gaussians *g, const tgs_half_params *out, tgs_stream stream);

/* --- compaction ---------------------------------------------------------------------------- */

#define TGS_COMPACT_MASKED 1u   /* also remove the Gaussians whose volume mask M is 0 */

/* Removes Gaussians from the parameter arrays, keeping the others in their order: those with
   remove[j] != 0 (remove: device bytes [n], e.g. from tgs_prune_select, or NULL) and, with
   TGS_COMPACT_MASKED and g->mask_logits given, those whose volume mask is 0 by the same
   float32 threshold test as the preprocess (Sec. "Pruning with Volume Masking": masked
   Gaussians are removed at densification steps and every 500 iterations afterwards).
   out: caller-allocated arrays with room for n Gaussians, in the layouts of tgs_gaussians
   under the field names of tgs_grads; a NULL field (or a NULL input array) is not copied.
   sh_degree_out [n] uint8 or NULL. kept_index [n] (device uint32, or NULL) receives, for each
   new index, the old one -- the gather map for per-Gaussian optimiser state and statistics.
   The outputs must not overlap the inputs. *n_kept (host) = number kept; the call
   synchronises the stream once to read it. TGS_ERR_INVALID_ARG for a null ctx, g, out or
   n_kept or an invalid g. */
tgs_status tgs_compact(tgs_ctx *ctx, const tgs_gaussians *g, const uint8_t *remove, uint32_t flags,
                       const tgs_grads *out, uint8_t *sh_degree_out, uint32_t *kept_index,
                       int64_t *n_kept, tgs_stream stream);

/* --- densification --------------------------------------------------------------------- */

/* Densification by clone and split, driven by the statistics the preprocess backward
   accumulates (Sec. "Preliminaries": Gaussians are densified by their gradient magnitudes; Sec.
   "Implementation details": the paper densifies as 3DGS does, every 100 iterations until 15K
   and again from 20K to 20.5K). The paper states no rule of its own; this library takes 3DGS's:
     avg = grad_norm_accum / vis_count (float32 division; vis_count 0 is never chosen),
     chosen = avg >= grad_threshold (pixel units of the accumulated |dL/d mean2d|),
     large = max_k log_scale_k > float32(log(scale_threshold)) (3DGS: 0.01 x scene extent),
     clone = chosen and not large: an identical copy is added,
     split = chosen and large: replaced by 2 children with means mu + R(q/|q|)(exp(l) * z_c),
             z_c = normals[i, c] (device float [n,2,3], the caller's standard normal draws; only
             the rows of split Gaussians are read), log-scales l - log(1.6), every other
             parameter copied.
   New order: the Gaussians not split (in order), the clones (in order), the first children of
   the split Gaussians (in order), their second children.
   out: caller-allocated arrays with room for `capacity` Gaussians, in the layouts of
   tgs_gaussians under the field names of tgs_grads (NULL fields, or absent inputs, are not
   written); sh_degree_out [capacity] uint8 or NULL; src_index [capacity] device uint32 or NULL
   receives the old index of each new row (children and clones: their source). The outputs must
   not overlap the inputs. *n_out (host) = n + n_clone + n_split; n_clone and n_split (host) may
   be NULL. Synchronises the stream once to read the counts; returns TGS_ERR_CAPACITY (counts
   set, nothing written) when *n_out > capacity. TGS_ERR_INVALID_ARG for null arguments, a
   non-positive scale_threshold or float16 parameters. */
tgs_status tgs_densify(tgs_ctx *ctx, const tgs_gaussians *g, const tgs_stats *stats, const float *normals,
                       float grad_threshold, float scale_threshold, const tgs_grads *out, uint8_t *sh_degree_out,
                       uint32_t *src_index, int64_t capacity, int64_t *n_out, int64_t *n_clone, int64_t *n_split,
                       tgs_stream stream);

/* --- measurement ------------------------------------------------------------------------ */

/* With profiling on, the batched step records a CUDA event between its stages (also inside
   a captured graph). tgs_stage_times synchronises on the last event and writes the duration
   in milliseconds of each stage of the most recent step; *n_out = number of stages. */
#define TGS_MAX_STAGES 8
tgs_status tgs_set_profiling(tgs_ctx *ctx, int32_t on);
tgs_status tgs_stage_times(tgs_ctx *ctx, float *ms, int32_t max, int32_t *n_out);
const char *tgs_stage_name(tgs_ctx *ctx, int32_t i);
/* Kernels the most recent batched step launched (for a graph replay: the kernel nodes of the
   graph). */
int64_t tgs_kernels_per_step(const tgs_ctx *ctx);
/* Device bytes the context's scratch arena holds now (every buffer it has allocated). */
size_t tgs_arena_bytes(const tgs_ctx *ctx);

/* Arithmetic peaks of the current GPU, measured by microbenchmark kernels (each thread runs 8
   independent chains of one instruction over a grid of SMs x 2048 threads; about 20 ms in
   all): the denominators of the roofline of the blend kernels, which are bound by FP32
   instruction issue and the special-function unit (SFU) rather than by memory.
   Synchronises the stream. Allocates a small buffer (freed before returning). */
typedef struct {
    double fp32_fma_per_s;   /* scalar fma.rn.f32 per second over all lanes (FP32 issue rate) */
    double fp32x2_fma_per_s; /* FP32 FMAs per second issued as packed fma.rn.f32x2 pairs */
    double ex2_per_s;        /* ex2.approx.ftz.f32 per second (SFU) */
    double rcp_per_s;        /* rcp.approx.ftz.f32 per second (SFU) */
    int32_t sms;             /* streaming multiprocessors */
    double ms;               /* device time of the timed launches */
} tgs_peaks;
tgs_status tgs_measure_peaks(tgs_peaks *out, tgs_stream stream);

/* Number of tiles of a view at the context's tile size, and bytes of scratch the batched
   path needs for n Gaussians and these views at the current key capacity. */
int64_t tgs_num_tiles(const tgs_ctx *ctx, const tgs_camera *cams, int32_t V);
size_t tgs_workspace_bytes(const tgs_ctx *ctx, int64_t n, const tgs_camera *cams, int32_t V);

#ifdef __cplusplus
}
#endif
#endif /* TGS_H */
