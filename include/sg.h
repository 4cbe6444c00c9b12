/*
 * sg.h -- C ABI of the GB300 (sm_103a) multi-level-pyramid Gaussian splatting library.
 *
 * The library implements the data-parallel hot path of RGBDS-SLAM's mapping step
 * (Sec. III-B..D): project 3D Gaussians into every (view, pyramid level), build per-tile
 * depth-sorted instance lists, composite RGB / depth / semantic images front to back,
 * evaluate the tightly coupled reconstruction loss per level, and run the hand-written
 * adjoint back to every Gaussian parameter.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All pointers in the structs below are DEVICE pointers owned by the caller.  The
 *    library never allocates or frees device memory; scratch space is passed in as a
 *    workspace sized by the matching *_workspace_size() call.
 *  - float tensors are FP32, contiguous, row-major; arrays read with 16-byte vector loads
 *    (quat, sem, geo, images of a view) must be 16-byte aligned (checked).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream)
 *    and capturable into a CUDA graph: no call synchronises or copies to the host.
 *  - Host-checkable problems return an error code before anything is launched.  Problems
 *    found on the device (instance capacity exceeded, non-finite values) set bits of the
 *    caller's device status word (SG_STATUS_*), which the caller reads after the stream
 *    work completes; the kernels themselves always exit normally.
 *  - sg_last_error() returns a thread-local message for the last failing call.
 *
 * Images are planar and packed per view-level: view-level v (see sg_view) with W x H
 * pixels starting at pixel offset p0 stores channel c of an image with K channels at
 * base + K*p0 + c*W*H + y*W + x.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sg_stream_t; /* same type as cudaStream_t */

typedef enum {
    SG_OK = 0,
    SG_ERR_INVALID_ARG = 1, /* null/misaligned pointer, bad size, unsupported C, ...     */
    SG_ERR_CAPACITY = 2,    /* a caller buffer or workspace is too small                */
    SG_ERR_TIMEOUT = 3,     /* a bounded device wait gave up                            */
    SG_ERR_NUMERIC = 4,     /* non-finite values detected                               */
    SG_ERR_CUDA = 5         /* a CUDA launch or runtime call failed                     */
} sg_status;

/* Bits of the caller's device status word (uint32). */
#define SG_STATUS_CAPACITY 1u /* more tile instances than sg_tile_lists.capacity  */
#define SG_STATUS_NUMERIC 2u  /* non-finite value met (checks on: sg_config /
                                 sg_loss_config check_numeric, sg_adam_multi status) */
#define SG_STATUS_TIMEOUT 4u  /* a bounded wait inside a tensor-core kernel gave up */

#define SG_MAX_VIEWS 64

/* Pinhole camera of pyramid level 0 (Eq. 2: K and T_cw).  Pixel (x, y) is evaluated at
 * the point (x, y): pixel centres sit at integer coordinates. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t W, H;
    float R_cw[9]; /* world -> camera rotation, row-major */
    float t_cw[3]; /* world -> camera translation         */
} sg_camera;

/* One (view, pyramid level) render target.  Built on the host by sg_make_views and copied
 * by the caller into a device array (the `views` argument of the calls below). */
typedef struct {
    float fx, fy, cx, cy; /* intrinsics of this level (Eq. 4-6 pyramid, see sg_make_views) */
    float R[9], t[3];     /* world -> camera                                             */
    int32_t W, H;         /* level image size                                            */
    int32_t tiles_x, tiles_y;
    int32_t tile_offset;  /* first global tile id of this view-level                     */
    int32_t pixel_offset; /* first pixel of this view-level in packed image buffers      */
    int32_t level;        /* pyramid level (0 = full resolution)                         */
    int32_t camera;       /* index of the source camera                                  */
} sg_view;

/* Gaussian parameters (Sec. III-B: position, shape, colour, semantic feature, opacity);
 * shape is anisotropic: log-scale (3) + unit quaternion (w, x, y, z). */
typedef struct {
    const float *mean;          /* N x 3                                  */
    const float *log_scale;     /* N x 3                                  */
    const float *quat;          /* N x 4 (w, x, y, z), 16-byte aligned    */
    const float *opacity_logit; /* N; opacity = sigmoid(logit)            */
    const float *rgb;           /* N x 3                                  */
    const float *sem;           /* N x C semantic feature, 16-byte aligned */
    int32_t N, C;               /* C % 4 == 0, C in {4, 8, 16, 32, 40}    */
    /* View-dependent colour (Sec. III-B, spherical-harmonic colour): with sh_degree D in
     * 1..3, the colour of Gaussian i seen from a view whose camera centre is
     * c = -R^T t is rgb_i + sum_k sh[i][k][:] Y_k(d), k = 1 .. (D+1)^2 - 1, where
     * d = (mean_i - c) / |mean_i - c| and Y_k are the real spherical harmonics of degree
     * 1..D in the usual graphics order (m = -l..l within a degree, Condon-Shortley signs;
     * Y_1 = -sqrt(3/4pi) y, sqrt(3/4pi) z, -sqrt(3/4pi) x).  The constant term is rgb
     * itself (no offset, no clamp).  The semantic feature takes the same view dependence
     * when sem_sh is given: sem_i + sum_k sem_sh[i][k][:] Y_k(d).  With sh_degree > 0 at
     * least one of sh and sem_sh is non-NULL; a NULL one leaves that feature view-
     * independent.  sh_degree 0: both are unused (may be NULL).                     */
    const float *sh;            /* N x ((D+1)^2 - 1) x 3                  */
    int32_t sh_degree;          /* D in 0..3                              */
    const float *sem_sh;        /* N x ((D+1)^2 - 1) x C, 16-byte aligned */
} sg_gaussians;

/* Gradients with respect to every Gaussian parameter; same layouts as sg_gaussians.
 * The backward call ADDS into these (the caller zeroes them).  sh and sh_degree as in
 * sg_gaussians (the degree must match). */
typedef struct {
    float *mean, *log_scale, *quat, *opacity_logit, *rgb, *sem;
    int32_t N, C;
    float *sh;
    int32_t sh_degree;
    float *sem_sh; /* 16-byte aligned, as is sem when sem_sh is given */
} sg_gaussian_grads;

/* Rendering constants (3D Gaussian splatting conventions, Sec. III-C) and launch shape. */
typedef struct {
    float alpha_max; /* 0.99:   alpha = min(alpha_max, o * exp(-sigma))              */
    float alpha_min; /* 1/255:  a Gaussian with alpha < alpha_min is skipped           */
    float T_min;     /* 1e-4:   stop before a Gaussian that would make T < T_min       */
    float z_near;    /* 0.2:    Gaussians with camera z <= z_near are culled           */
    float dilation;  /* 0.3:    added to the 2D covariance diagonal (pixels^2)         */
    float fov_clamp; /* 1.3:    Jacobian evaluated at t_x/t_z clamped to fov_clamp*W/2fx */
    float bg[3];     /* background RGB (depth and semantic background are 0)          */
    int32_t tile_w, tile_h; /* screen tile: 8x8, 16x8, 16x16 or 32x8                  */
    int32_t batch;          /* Gaussians staged per shared-memory batch: 16..512, step 16 */
    int32_t persistent;     /* 1: persistent grid with an atomic work queue           */
    int32_t pixels_per_thread;     /* forward: 1, 2 or 4 pixels per thread (rows 4 apart);
                                      tile_h % (4 * it) == 0, tile pixels >= 32 * it       */
    int32_t pixels_per_thread_bwd; /* the same for the backward kernel                    */
    int32_t batch_bwd;      /* batch of the backward kernel; 0: the same as `batch`    */
    int32_t isotropic;      /* 0: EWA projection of the anisotropic Gaussian (log_scale,
                               quat); 1: Eq. 2 as printed: an isotropic Gaussian of radius
                               r = exp(log_scale[0]) projects to a circle of radius f r / d
                               (fx along x, fy along y), Sigma2D = diag((fx r/d)^2,
                               (fy r/d)^2) + dilation; quat and log_scale[1..2] are unused
                               and get zero gradient                                    */
    int32_t check_numeric;  /* 1: sg_project_gaussians sets SG_STATUS_NUMERIC in its status
                               word when a Gaussian parameter it reads (mean, log-scale,
                               quaternion, opacity logit, rgb, semantic feature, SH
                               coefficients) is NaN or infinite; 0: no check (the default)  */
    int32_t half_tile_fwd;  /* with half masks in the lists, 8x8 tiles and one pixel per
                               thread: 1 = the forward compositing also runs one warp per
                               half tile, each taking only its half's entries with no block
                               barrier and stopping when its own pixels saturate (faster on
                               long lists); 0 = the tile's warps share staged batches.  The
                               output is the same either way.                            */
} sg_config;

/* Projected records of all (view-level, Gaussian) pairs: record r = v*N + g. */
typedef struct {
    float *geo;     /* R x 8 (16-B aligned): u_frac, v_frac, depth, opacity, m00, m10, m11,
                       (u_int | v_int << 16) as int16 bits; the 2D mean is
                       (u_int + u_frac, v_int + v_frac) and
                       1/2 d^T Sigma2D^{-1} d = (m00 dx)^2 + (m10 dx + m11 dy)^2            */
    uint32_t *rect; /* R x 2: tile rectangle [tx0,tx1) x [ty0,ty1) as (tx0|ty0<<16, tx1|ty1<<16);
                       an empty rectangle means the record is culled                    */
    float *ext;     /* R x 2: half extents (pixels) of the region where alpha can reach
                       alpha_min, with margin (8-B aligned)                             */
    float *rgb;     /* R x 3: colour of each record seen from its view-level, written by
                       the projection when the Gaussians carry sh and read by the
                       compositing kernels in place of the Gaussian's rgb (may be NULL
                       otherwise); entries of culled records are left unwritten       */
    float *sem;     /* R x C (16-B aligned): the same for the semantic feature when the
                       Gaussians carry sem_sh                                           */
} sg_projected;

/* Per-tile depth-sorted instance lists (the set N of Eq. 7-9, restricted to a tile). */
typedef struct {
    int32_t capacity; /* K_cap: instances the arrays below can hold                      */
    uint32_t *tile;   /* K_cap: global tile id of each instance, ascending               */
    uint32_t *record; /* K_cap: record id v*N+g; within a tile by (depth, record id)
                         (with half_masks, plus the mask in bits 30-31)                  */
    int32_t *ranges;  /* n_tiles x 2: [start, end) of each tile's instances              */
    int32_t *count;   /* device scalar: K = instances emitted (may exceed capacity)      */
    int32_t *order;   /* n_tiles or NULL: every tile id once, by descending instance count
                         in power-of-two half-octave buckets (ascending id within a
                         bucket); the compositing kernels take tiles in this order, so the
                         longest lists start first and the short ones fill the tail.  NULL:
                         tiles in id order.                                             */
    int32_t half_masks; /* nonzero: each listed record also carries, in bits 30-31, which
                         halves of its tile its footprint may reach (bit 30: pixel rows
                         [0, tile_h / 2), bit 31: the rest), by the culling rule applied to
                         each half: a conservative superset (a half left out holds no pixel
                         with alpha >= alpha_min); a tile then keeps a record if either
                         half's rule keeps it (otherwise the rule runs once on the whole
                         tile row), and N * n_views must be below 2^30.  The compositing
                         kernels take the record id from bits 0-29; the adjoint of 8 x 8
                         tiles at one pixel per thread runs one warp per half tile, each
                         staging only its half's entries (faster on long lists; the masks
                         make the lists slower to build).  0: plain record ids.          */
} sg_tile_lists;

/* Rendered images (all view-levels packed, planar). */
typedef struct {
    float *rgb;   /* 3 planes per view-level */
    float *depth; /* 1 plane                 */
    float *sem;   /* C planes                */
} sg_images;

/* Per-pixel state saved by the forward pass for the backward pass (no per-Gaussian
 * intermediates are stored). */
typedef struct {
    float *T_final;     /* transmittance after the last contributor                      */
    int32_t *last;      /* list entries examined up to and including the last contributor */
    int32_t *n_contrib; /* number of contributing Gaussians                              */
} sg_saved;

/* Ground-truth pyramid of every view-level, same packing as sg_images. */
typedef struct {
    const float *rgb;     /* 3 planes                                  */
    const float *depth;   /* 1 plane; <= 0 marks missing depth          */
    const int32_t *label; /* 1 plane; < 0 = ignore (sem_mode 0)         */
    const float *sem;     /* C planes of semantic colour (sem_mode 1)    */
} sg_targets;

/* Eq. 10-13 weights and the semantic term. */
typedef struct {
    float lambda_r;        /* 0.2: weight of D-SSIM in the RGB term (Eq. 10)             */
    float lambda_s;        /* 0.2: weight of D-SSIM in the semantic term (Eq. 12)        */
    float w_depth, w_sem;  /* 1, 1: weights of the depth and semantic terms (Eq. 13)     */
    int32_t sem_mode;      /* 0: cross-entropy of softmax(decoder * S) vs label;
                              1: (1-lambda_s) L1 + lambda_s (1 - SSIM) vs semantic colour */
    int32_t n_classes;     /* K (sem_mode 0)                                              */
    const float *decoder;  /* K x C linear decoder, or NULL for identity (K == C)         */
    float *decoder_grad;   /* K x C gradient (added), or NULL                             */
    int32_t check_numeric; /* 1: set SG_STATUS_NUMERIC when a view-level's loss terms come
                              out NaN or infinite (a non-finite rendered or target value
                              reached the loss); 0: no check (the default)                 */
} sg_loss_config;

/* ---------------------------------------------------------------------------------- */
/* Host helpers                                                                         */
/* ---------------------------------------------------------------------------------- */

const char *sg_last_error(void);
const char *sg_version(void);

/* Reads a device status word after the work queued on `stream` before this call has
 * completed (it synchronises the stream: call it outside graph capture), writes its bits to
 * *bits (may be NULL) and maps them to a status: SG_ERR_CAPACITY if SG_STATUS_CAPACITY is
 * set, else SG_ERR_TIMEOUT for SG_STATUS_TIMEOUT, else SG_ERR_NUMERIC for SG_STATUS_NUMERIC,
 * else SG_OK; the message (sg_last_error) names every bit that is set.  The word is left as
 * it is (the caller clears it). */
sg_status sg_read_status(const uint32_t *status, sg_stream_t stream, uint32_t *bits);
/* Number of kernels this library has launched (or recorded into a graph) since it was
 * loaded; a diagnostic used by the benchmark to report its launch count. */
uint64_t sg_kernel_launch_count(void);
void sg_default_config(sg_config *cfg);
void sg_default_loss_config(sg_loss_config *cfg);

/* Eq. 4-6 / Sec. IV-A (3 levels): expand n_cams level-0 cameras into n_cams*levels
 * view-levels (camera-major, level-minor).  Level l+1 halves the size (floor) and maps
 * pixel centres consistently: f' = f/2, c' = (c - 0.5)/2.  Writes out[n_cams*levels];
 * returns total pixels and tiles.  SG_ERR_INVALID_ARG when a level would be empty or
 * n_cams*levels > SG_MAX_VIEWS. */
sg_status sg_make_views(const sg_camera *cams, int32_t n_cams, int32_t levels, int32_t tile_w,
                        int32_t tile_h, sg_view *out, int64_t *total_pixels,
                        int32_t *total_tiles);

/* ---------------------------------------------------------------------------------- */
/* Forward path                                                                         */
/* ---------------------------------------------------------------------------------- */

/* Eq. 2-3 generalised by the EWA covariance projection: for every view-level and every
 * Gaussian writes the 2D mean, depth, opacity, conic and the tile rectangle covering every
 * pixel where alpha can reach alpha_min; with spherical-harmonic features also the
 * view-dependent colour (semantic feature) of every visible record into out->rgb (out->sem),
 * required when g->sh (g->sem_sh) is given.  views: device array of
 * n_views sg_view.  status: device status word, required when cfg->check_numeric is set
 * (see sg_config), else may be NULL. */
sg_status sg_project_gaussians(const sg_gaussians *g, const sg_view *views, int32_t n_views,
                               const sg_config *cfg, sg_projected *out, uint32_t *status,
                               sg_stream_t stream);

/* Scratch bytes sg_build_tile_lists needs for n_records = n_views*N records and the
 * lists' capacity. */
size_t sg_tile_lists_workspace_size(int64_t n_records, int32_t capacity);

/* Sec. III-C "sorted 2D gaussian primitives": instances (tile, record) of every non-culled
 * record, ordered by global tile id, then float32 depth bits, then record id (a stable,
 * deterministic radix sort), plus each tile's [start, end) and (with lists->half_masks)
 * each instance's half mask.  n_tiles: total tiles of the views (sg_make_views); with half
 * masks N * n_views must be below 2^30.  If more than capacity instances arise, the surplus
 * is dropped, *count holds the required number and SG_STATUS_CAPACITY is set in *status. */
sg_status sg_build_tile_lists(const sg_projected *proj, int32_t N, int32_t n_views,
                              const sg_view *views, int32_t n_tiles, const sg_config *cfg,
                              sg_tile_lists *lists, void *workspace, size_t workspace_bytes,
                              uint32_t *status, sg_stream_t stream);

/* Eq. 7-9 for every view-level in one launch: per tile, front-to-back compositing of RGB,
 * depth and C semantic channels.  work_counter: 2 int32 of device scratch for the persistent
 * work queue, zero before the first call; every call leaves them zero (the last CTA resets
 * them), so one pair can serve all calls on a stream. */
sg_status sg_render_pyramid(const sg_gaussians *g, const sg_projected *proj,
                            const sg_tile_lists *lists, const sg_view *views, int32_t n_views,
                            int32_t n_tiles, const sg_config *cfg, sg_images *out,
                            sg_saved *saved, int32_t *work_counter, sg_stream_t stream);

/* Scratch bytes sg_pyramid_loss needs for the view-levels in views_host (host table), C
 * semantic channels and n_classes decoder outputs (covers the decoder gradient's
 * per-block partials). */
size_t sg_loss_workspace_size(const sg_view *views_host, int32_t n_views, int32_t C,
                              int32_t n_classes);

/* Eq. 10-13 at every view-level: writes terms[4*v + {0,1,2,3}] = L_r, L_d, L_s, total of
 * view-level v (device floats) and the gradient of sum_v total_v with respect to the
 * rendered images into dL (same packing as sg_images).  views_host: host copy of the
 * view table (sizes are needed to size the launch).  SSIM uses an 11x11 Gaussian window
 * (sigma 1.5) with zero padding.  workspace: sg_loss_workspace_size() bytes, 16-byte
 * aligned.  status: device status word, required when lcfg->check_numeric is set, else may
 * be NULL. */
sg_status sg_pyramid_loss(const sg_images *rendered, const sg_targets *gt, const sg_view *views,
                          const sg_view *views_host, int32_t n_views, int32_t C,
                          const sg_loss_config *lcfg, float *terms, sg_images *dL,
                          void *workspace, size_t workspace_bytes, uint32_t *status,
                          sg_stream_t stream);

/* Same as sg_pyramid_loss, for callers that cannot allocate device memory: a host
 * framework that owns the device memory pool and passes this library only its input and
 * output buffers, or a latency-critical thread that must not call cudaMalloc because it
 * can block on or synchronise with other work on the device.  The paper has no
 * counterpart; this is a deployment variant of the loss call.
 * Instead of a caller workspace it uses a scratch array of SG_LOSS_NOALLOC_SCRATCH_BYTES
 * (16 MiB) built into the library; every GPU that loads the library holds that array
 * until the process exits.  Images whose scratch need exceeds it (roughly P/16 bytes for
 * P pixels, plus P*K*C/64 bytes when a decoder gradient is requested) are rejected with
 * SG_ERR_CAPACITY and a message (after the same argument checks as sg_pyramid_loss).  The
 * first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that first call before
 * any stream capture, and do not use this call across a device reset (cudaDeviceReset or a
 * re-created primary context may move the array and leave the kept address stale).  All
 * calls share the array and leave their contents in it: the call clears what it needs, but
 * calls whose GPU work overlaps race on it.  No allocation or free happens inside the call. */
#define SG_LOSS_NOALLOC_SCRATCH_BYTES (16u << 20)
sg_status sg_pyramid_loss_noalloc(const sg_images *rendered, const sg_targets *gt,
                                  const sg_view *views, const sg_view *views_host, int32_t n_views,
                                  int32_t C, const sg_loss_config *lcfg, float *terms,
                                  sg_images *dL, uint32_t *status, sg_stream_t stream);

/* ---------------------------------------------------------------------------------- */
/* Backward path                                                                        */
/* ---------------------------------------------------------------------------------- */

/* Scratch bytes sg_render_pyramid_backward needs: 12 + sem_channels floats per record, in
 * three blocks: R x 8 2D gradients, R x 4 view-dependent colour gradients, R x sem_channels
 * view-dependent semantic gradients.  sem_channels = C when the Gaussians carry sem_sh,
 * else 0.  Zero the workspace once after allocating it; every backward leaves it zero (see
 * sg_render_pyramid_backward_raster below). */
size_t sg_backward_workspace_size(int64_t n_records, int32_t sem_channels);

/* Adjoint of sg_render_pyramid followed by the adjoint of sg_project_gaussians (Sec. III-D
 * backpropagation): back-to-front per tile from each pixel's saved `last`, warp-level
 * reductions before the atomics, then the chain rule through the EWA projection.  ADDS
 * dL/d{mean, log_scale, quat, opacity_logit, rgb, sem} into grads. */
sg_status sg_render_pyramid_backward(const sg_gaussians *g, const sg_projected *proj,
                                     const sg_tile_lists *lists, const sg_view *views,
                                     int32_t n_views, int32_t n_tiles, const sg_config *cfg,
                                     const sg_saved *saved, const sg_images *dL,
                                     sg_gaussian_grads *grads, void *workspace,
                                     size_t workspace_bytes, int32_t *work_counter,
                                     sg_stream_t stream);

/* The two halves of sg_render_pyramid_backward, for callers that time or schedule them
 * apart (same arguments, same workspace):
 *   sg_render_pyramid_backward_raster: the compositing adjoint.  ADDS dL/d(2D mean, conic,
 *     opacity, depth) per record into the workspace's first block; dL/drgb and dL/dsem go
 *     into grads, except that with sh (sem_sh) the gradient of the record's colour
 *     (semantic feature) goes into the workspace's colour (semantic) block instead.
 *   sg_project_gaussians_backward: the chain rule through the EWA projection from those
 *     per-record gradients; ADDS dL/d{mean, log_scale, quat, opacity_logit} into grads (with
 *     SH also dL/d{sh, rgb} and/or dL/d{sem_sh, sem} and the view direction's share of
 *     dL/dmean) and zeroes the per-record slots it consumed.
 * The workspace must be all zero when the compositing adjoint starts: zero it once after
 * allocating it; each projection adjoint then leaves it zero again (only records visible in
 * some view-level are ever written, and those are the ones it consumes).  Calling both in
 * this order on one stream equals sg_render_pyramid_backward. */
sg_status sg_render_pyramid_backward_raster(const sg_gaussians *g, const sg_projected *proj,
                                            const sg_tile_lists *lists, const sg_view *views,
                                            int32_t n_views, int32_t n_tiles, const sg_config *cfg,
                                            const sg_saved *saved, const sg_images *dL,
                                            sg_gaussian_grads *grads, void *workspace,
                                            size_t workspace_bytes, int32_t *work_counter,
                                            sg_stream_t stream);
sg_status sg_project_gaussians_backward(const sg_gaussians *g, const sg_projected *proj,
                                        const sg_view *views, int32_t n_views, const sg_config *cfg,
                                        void *workspace, size_t workspace_bytes,
                                        sg_gaussian_grads *grads, sg_stream_t stream);

/* ---------------------------------------------------------------------------------- */
/* Support: pyramid construction and the optimizer                                      */
/* ---------------------------------------------------------------------------------- */

/* Eq. 4-6 "PyramidImageExtraction": fills levels 1..L-1 of every camera in `tgt` (packed
 * like the views) from level 0: 2x2 box mean for RGB, mean of the valid (> 0) depths,
 * majority label of the valid (>= 0) labels with ties to the lowest id.  n_sem_ch planes of
 * semantic colour (may be 0) are box-averaged like RGB. */
sg_status sg_build_pyramid(float *rgb, float *depth, int32_t *label, float *sem, int32_t n_sem_ch,
                           const sg_view *views_host, int32_t n_views, sg_stream_t stream);

/* One parameter tensor for sg_adam_multi. */
typedef struct {
    float *param, *grad, *m, *v;
    int64_t n;
    float lr;
} sg_adam_group;
#define SG_ADAM_MAX_GROUPS 8

/* Adam over up to SG_ADAM_MAX_GROUPS tensors in one launch (same update as sg_adam_step,
 * per-group learning rate); with zero_grad != 0 every gradient is set to 0 after use.
 * status: NULL, or a device status word in which SG_STATUS_NUMERIC is set when a gradient
 * it reads is NaN or infinite (the update itself is applied as usual). */
sg_status sg_adam_multi(const sg_adam_group *groups, int32_t n_groups, float beta1, float beta2,
                        float eps, int32_t step, int32_t zero_grad, uint32_t *status,
                        sg_stream_t stream);

/* Adam (the paper leaves the optimizer unspecified): for i < n
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr * mhat / (sqrt(vhat) + eps). */
sg_status sg_adam_step(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int32_t step, sg_stream_t stream);

/* ---------------------------------------------------------------------------------- */
/* Learned initializer (not in the paper; its only counterpart is Sec. III-A's insertion  */
/* of new Gaussians from a keyframe): a 3-layer BF16 MLP with FP32 accumulation on the    */
/* tcgen05 tensor cores, 2048 (2009 used) -> 128 -> ReLU -> 128 -> ReLU -> 32 (20 used).   */
/* ---------------------------------------------------------------------------------- */

#define SG_MLP_IN 2048
#define SG_MLP_HIDDEN 128
#define SG_MLP_OUT 32

/* bf16 operands are passed as uint16_t bit patterns. */
typedef struct {
    const uint16_t *W1, *W2, *W3; /* bf16 [128][2048], [128][128], [32][128]  ([out][in])      */
    const uint16_t *W2t, *W3t;    /* bf16 W2^T [128][128]; W3^T zero-padded to [128][64]      */
    const float *b1, *b2, *b3;    /* [128], [128], [32]                                        */
} sg_mlp;

typedef struct {
    uint16_t *H1, *H1t, *H2, *H2t; /* bf16 [B][128] and transposed [128][B]                  */
    float *Y;                      /* fp32 [B][32]                                            */
    uint16_t *dY, *dYt;            /* bf16 [B][64] (columns >= 32 written as 0), [32][B]      */
    uint16_t *dH2, *dH2t, *dH1t;   /* bf16 [B][128], [128][B], [128][B]                       */
} sg_mlp_acts;

typedef struct {
    float *W1, *W2, *W3, *b1, *b2, *b3; /* fp32, same shapes as the weights; ADDED into      */
} sg_mlp_grads;

/* D[M][N] (+)= A[M][K] B[N][K]^T on the tensor cores (A, B bf16 with K contiguous, rows
 * 16-byte aligned, K % 64 == 0; D fp32 row-major with leading dimension ldd).  accumulate:
 * 0 stores D, 1 atomically adds (the K range is then split over CTAs).  Timeouts of the
 * kernel's bounded waits set SG_STATUS_TIMEOUT in *status (may be NULL). */
sg_status sg_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int32_t M,
                       int32_t N, int32_t K, float *D, int64_t ldd, int32_t accumulate,
                       uint32_t *status, sg_stream_t stream);

/* Self-test of the failure detection of the tensor-core kernels (no counterpart in the
 * paper).  Launches sg_gemm_bf16's kernel (store mode) whose CTAs first wait on an mbarrier
 * that nothing arrives on, bounded by `polls` polls (1..2^20).  Each CTA must give up, set
 * SG_STATUS_TIMEOUT in *status, skip its output (D is left untouched), release its tensor
 * memory and return, so the context stays usable.  Arguments as for sg_gemm_bf16. */
sg_status sg_gemm_bf16_timeout_probe(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                                     int32_t M, int32_t N, int32_t K, float *D, int64_t ldd,
                                     uint32_t polls, uint32_t *status, sg_stream_t stream);

/* fp32 master weights ([out][in]) -> the bf16 operand copies of sg_mlp.  W3t's padding
 * columns 32..63 are not written: the caller zeroes W3t once. */
sg_status sg_mlp_pack_weights(const float *W1, const float *W2, const float *W3, uint16_t *W1b,
                              uint16_t *W2b, uint16_t *W3b, uint16_t *W2t, uint16_t *W3t,
                              sg_stream_t stream);

/* Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for B rows of X (bf16 [B][2048], B % 128 == 0).
 * Writes acts->H1/H1t/H2/H2t (bf16, needed by the backward; H1t/H2t may be NULL for
 * inference) and acts->Y (fp32). */
sg_status sg_mlp_forward(const sg_mlp *net, const uint16_t *X, int32_t B, sg_mlp_acts *acts,
                         uint32_t *status, sg_stream_t stream);

/* Gradient of L = sum_o out_weight[o] * mean_b (Y[b][o] - target[b][o])^2 after
 * sg_mlp_forward on the same batch.  Xt: bf16 [2048][B] (the transposed input).  ADDS the
 * weight and bias gradients into grads and L into *loss (device float). */
sg_status sg_mlp_backward(const sg_mlp *net, const uint16_t *Xt, const float *target,
                          const float *out_weight, int32_t B, sg_mlp_acts *acts,
                          sg_mlp_grads *grads, float *loss, uint32_t *status, sg_stream_t stream);

/* Sec. III-A (the mapping thread converts keyframe data into Gaussian primitives): for B
 * pixels (x, y) of a level-0 frame (planar rgb 3 x H x W, depth H x W, label H x W or NULL)
 * with valid depth, writes B new Gaussians into out (device arrays with room for B; out->C
 * is the semantic width): mean = back-projection, rgb = pixel colour, log-scale = ln(D/fx)
 * on every axis, identity rotation, opacity logit 0, semantic feature =
 * kappa * sem_code[label] (sem_code: n_classes x C, or NULL for zeros).  pixels: int32 (x, y)
 * pairs. */
sg_status sg_init_gaussians(const float *rgb, const float *depth, const int32_t *label,
                            const sg_camera *cam, const int32_t *pixels, int32_t B,
                            const float *sem_code, int32_t n_classes, float kappa,
                            sg_gaussian_grads *out, sg_stream_t stream);

/* Input features of the learned initializer: the 7 x 7 patch around each pixel, 41
 * channels per patch pixel (rgb 3, depth 1, one-hot label 32, unit camera ray 3, depth
 * valid 1, 1/fx 1) = 2009 features, zero-padded to SG_MLP_IN; pixels outside the image
 * give zeros; rows b >= B of the B_pad (multiple of 128) output rows are zero.  X: bf16
 * [B_pad][2048] and/or Xt: bf16 [2048][B_pad] (either may be NULL). */
sg_status sg_extract_patches(const float *rgb, const float *depth, const int32_t *label,
                             const sg_camera *cam, const int32_t *pixels, int32_t B, int32_t B_pad,
                             uint16_t *X, uint16_t *Xt, sg_stream_t stream);

/* Overwrites log-scale (3), opacity logit (1) and semantic feature (C) of B Gaussians in
 * out with the MLP output Y ([B][32], standardised): value = Y * y_std + y_mean. */
sg_status sg_apply_mlp_init(const float *Y, int32_t B, const float *y_mean, const float *y_std,
                            sg_gaussian_grads *out, sg_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
