// api.cu -- the extern "C" boundary: argument checks, workspace carving, launches.
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <cstring>

#include "raster.cuh"

namespace sg {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

sg_status check_launch(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    return SG_OK;
}

// defined in the kernel files
sg_status launch_project_fwd(const sg_gaussians *, const sg_view *, int, const sg_config *,
                             sg_projected *, uint32_t *, cudaStream_t);
sg_status launch_project_bwd(const sg_gaussians *, const sg_view *, int, const sg_config *,
                             const sg_projected *, float *, sg_gaussian_grads *, cudaStream_t);
size_t tile_lists_workspace_size(int64_t R, int32_t cap);
sg_status launch_build_tile_lists(const sg_projected *, int, int, const sg_view *, int, int, int,
                                  sg_tile_lists *, void *, size_t, uint32_t *, cudaStream_t);
size_t loss_workspace_size(const sg_view *vh, int n_views, int C, int n_classes);
sg_status launch_loss(const sg_images *, const sg_targets *, const sg_view *, const sg_view *, int,
                      int, const sg_loss_config *, float *, sg_images *, void *, size_t, uint32_t *,
                      cudaStream_t);
sg_status launch_pyramid(float *, float *, int *, float *, int, const sg_view *, int, cudaStream_t);
sg_status launch_adam(float *, const float *, float *, float *, int64_t, float, float, float, float, int,
                      cudaStream_t);
sg_status launch_adam_multi(const sg_adam_group *, int, float, float, float, int, int, uint32_t *,
                            cudaStream_t);

}  // namespace sg


using namespace sg;

#define SG_REQUIRE(cond, ...)                   \
    do {                                        \
        if (!(cond)) {                          \
            set_error(__VA_ARGS__);             \
            return SG_ERR_INVALID_ARG;          \
        }                                       \
    } while (0)

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static sg_status check_gaussians(const sg_gaussians *g) {
    SG_REQUIRE(g, "gaussians is NULL");
    SG_REQUIRE(g->N >= 0, "N = %d < 0", g->N);
    SG_REQUIRE(raster_supports(g->C), "unsupported semantic width C=%d (supported: 4, 8, 16, 32, 40)", g->C);
    SG_REQUIRE(g->sh_degree >= 0 && g->sh_degree <= 3, "sh_degree = %d not in 0..3", g->sh_degree);
    if (g->N == 0) return SG_OK;
    SG_REQUIRE(g->mean && g->log_scale && g->quat && g->opacity_logit && g->rgb && g->sem,
               "a Gaussian parameter pointer is NULL");
    SG_REQUIRE(aligned16(g->quat) && aligned16(g->sem), "quat and sem must be 16-byte aligned");
    SG_REQUIRE(g->sh_degree == 0 || g->sh || g->sem_sh, "sh_degree = %d needs sh and/or sem_sh",
               g->sh_degree);
    SG_REQUIRE(!g->sem_sh || aligned16(g->sem_sh), "sem_sh must be 16-byte aligned");
    return SG_OK;
}

static bool sh_colour(const sg_gaussians *g) { return g->sh_degree > 0 && g->sh; }
static bool sh_semantic(const sg_gaussians *g) { return g->sh_degree > 0 && g->sem_sh; }

// With spherical-harmonic features the compositing kernels read the per-record colour and
// semantic feature the projection wrote.
static sg_status check_record_colour(const sg_gaussians *g, const sg_projected *proj) {
    SG_REQUIRE(!sh_colour(g) || proj->rgb, "sh colour needs projected->rgb");
    SG_REQUIRE(!sh_semantic(g) || (proj->sem && aligned16(proj->sem)),
               "sem_sh needs a 16-byte aligned projected->sem");
    return SG_OK;
}

static sg_status check_cfg(const sg_config *c) {
    SG_REQUIRE(c, "config is NULL");
    const int t = c->tile_w * c->tile_h;
    SG_REQUIRE((c->tile_w == 8 && c->tile_h == 8) || (c->tile_w == 16 && c->tile_h == 16) ||
                   (c->tile_w == 32 && c->tile_h == 8) || (c->tile_w == 16 && c->tile_h == 8),
               "tile %dx%d not supported (8x8, 16x8, 16x16, 32x8)", c->tile_w, c->tile_h);
    SG_REQUIRE(t <= kMaxTileThreads, "tile too large");
    SG_REQUIRE(c->batch >= 16 && c->batch <= 512 && (c->batch % 16) == 0, "batch %d not in [16, 512] step 16",
               c->batch);
    SG_REQUIRE(c->batch_bwd == 0 || (c->batch_bwd >= 16 && c->batch_bwd <= 512 && (c->batch_bwd % 16) == 0),
               "batch_bwd %d not 0 or in [16, 512] step 16", c->batch_bwd);
    SG_REQUIRE(c->isotropic == 0 || c->isotropic == 1, "isotropic must be 0 or 1");
    SG_REQUIRE(c->check_numeric == 0 || c->check_numeric == 1, "check_numeric must be 0 or 1");
    SG_REQUIRE(c->half_tile_fwd == 0 || c->half_tile_fwd == 1, "half_tile_fwd must be 0 or 1");
    SG_REQUIRE(c->alpha_min > 0.f && c->alpha_max <= 1.f && c->alpha_min < c->alpha_max,
               "need 0 < alpha_min < alpha_max <= 1");
    SG_REQUIRE(c->T_min >= 0.f && c->z_near > 0.f && c->dilation >= 0.f && c->fov_clamp > 0.f,
               "bad T_min / z_near / dilation / fov_clamp");
    for (int ppt : {c->pixels_per_thread, c->pixels_per_thread_bwd}) {
        SG_REQUIRE(ppt == 1 || ppt == 2 || ppt == 4, "pixels per thread must be 1, 2 or 4");
        SG_REQUIRE(c->tile_h % (4 * ppt) == 0 && t / ppt >= 32,
                   "tile %dx%d cannot give %d pixels per thread", c->tile_w, c->tile_h, ppt);
    }
    return SG_OK;
}

static sg_status check_views(const sg_view *views, int n_views) {
    SG_REQUIRE(views, "views is NULL");
    SG_REQUIRE(n_views >= 1 && n_views <= SG_MAX_VIEWS, "n_views = %d not in [1, %d]", n_views, SG_MAX_VIEWS);
    return SG_OK;
}

#define SG_TRY(expr)                  \
    do {                              \
        const sg_status _s = (expr);  \
        if (_s != SG_OK) return _s;   \
    } while (0)

namespace sg {
// Every host-checkable condition of sg_pyramid_loss except the workspace (shared with the
// entry point that brings its own scratch).
sg_status check_loss_args(const sg_images *rendered, const sg_targets *gt, const sg_view *views,
                          const sg_view *views_host, int32_t n_views, int32_t C, const sg_loss_config *lcfg,
                          float *terms, sg_images *dL, uint32_t *status) {
    SG_TRY(check_views(views, n_views));
    SG_REQUIRE(views_host, "views_host is NULL");
    SG_REQUIRE(rendered && gt && lcfg && terms && dL, "NULL argument");
    SG_REQUIRE(C >= 1, "C = %d < 1", C);
    SG_REQUIRE(rendered->rgb && rendered->depth && rendered->sem && gt->rgb && gt->depth,
               "image buffers are NULL");
    SG_REQUIRE(dL->rgb && dL->depth && dL->sem, "gradient buffers are NULL");
    SG_REQUIRE(lcfg->sem_mode == 0 || lcfg->sem_mode == 1, "sem_mode must be 0 or 1");
    if (lcfg->sem_mode == 0) {
        SG_REQUIRE(gt->label, "cross-entropy mode needs labels");
        SG_REQUIRE(lcfg->n_classes >= 1, "n_classes must be >= 1");
        SG_REQUIRE(lcfg->decoder || lcfg->n_classes == C, "without a decoder n_classes must equal C");
    } else {
        SG_REQUIRE(gt->sem, "semantic-colour mode needs gt->sem");
    }
    for (int v = 0; v < n_views; ++v)
        SG_REQUIRE(views_host[v].W >= 1 && views_host[v].H >= 1, "view %d is empty", v);
    SG_REQUIRE(lcfg->check_numeric == 0 || lcfg->check_numeric == 1, "check_numeric must be 0 or 1");
    SG_REQUIRE(!lcfg->check_numeric || status, "check_numeric needs a status word");
    return SG_OK;
}
}  // namespace sg

extern "C" {

const char *sg_last_error(void) { return g_err; }

const char *sg_version(void) { return "pyramid-splat-gb300 0.1 (sm_103a)"; }

uint64_t sg_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void sg_default_config(sg_config *c) {
    if (!c) return;
    c->alpha_max = 0.99f;
    c->alpha_min = 1.f / 255.f;
    c->T_min = 1e-4f;
    c->z_near = 0.2f;
    c->dilation = 0.3f;
    c->fov_clamp = 1.3f;
    c->bg[0] = c->bg[1] = c->bg[2] = 0.f;
    c->tile_w = 16;
    c->tile_h = 16;
    c->batch = 256;
    c->persistent = 1;
    c->pixels_per_thread = 1;
    c->pixels_per_thread_bwd = 2;
    c->batch_bwd = 0;
    c->isotropic = 0;
    c->check_numeric = 0;
    c->half_tile_fwd = 0;
}

void sg_default_loss_config(sg_loss_config *c) {
    if (!c) return;
    c->lambda_r = 0.2f;
    c->lambda_s = 0.2f;
    c->w_depth = 1.f;
    c->w_sem = 1.f;
    c->sem_mode = 0;
    c->n_classes = 0;
    c->decoder = nullptr;
    c->decoder_grad = nullptr;
    c->check_numeric = 0;
}

sg_status sg_read_status(const uint32_t *status, sg_stream_t stream, uint32_t *bits) {
    SG_REQUIRE(status, "status is NULL");
    uint32_t b = 0;
    cudaError_t e = cudaMemcpyAsync(&b, status, sizeof(b), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("read_status: %s", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    if (bits) *bits = b;
    set_error("status word 0x%x:%s%s%s", b, (b & SG_STATUS_CAPACITY) ? " capacity exceeded;" : "",
              (b & SG_STATUS_TIMEOUT) ? " a bounded device wait gave up;" : "",
              (b & SG_STATUS_NUMERIC) ? " non-finite value met;" : "");
    if (b & SG_STATUS_CAPACITY) return SG_ERR_CAPACITY;
    if (b & SG_STATUS_TIMEOUT) return SG_ERR_TIMEOUT;
    if (b & SG_STATUS_NUMERIC) return SG_ERR_NUMERIC;
    return SG_OK;
}

sg_status sg_make_views(const sg_camera *cams, int32_t n_cams, int32_t levels, int32_t tile_w,
                        int32_t tile_h, sg_view *out, int64_t *total_pixels, int32_t *total_tiles) {
    SG_REQUIRE(cams && out, "cams/out is NULL");
    SG_REQUIRE(n_cams >= 1 && levels >= 1, "n_cams and levels must be >= 1");
    SG_REQUIRE((int64_t)n_cams * levels <= SG_MAX_VIEWS, "n_cams*levels = %d > %d", n_cams * levels,
               SG_MAX_VIEWS);
    SG_REQUIRE(tile_w > 0 && tile_h > 0, "bad tile size");
    int64_t pix = 0;
    int64_t tiles = 0;
    int v = 0;
    for (int c = 0; c < n_cams; ++c) {
        float fx = cams[c].fx, fy = cams[c].fy, cx = cams[c].cx, cy = cams[c].cy;
        int W = cams[c].W, H = cams[c].H;
        for (int l = 0; l < levels; ++l, ++v) {
            if (l > 0) {
                fx *= 0.5f;
                fy *= 0.5f;
                cx = (cx - 0.5f) * 0.5f;
                cy = (cy - 0.5f) * 0.5f;
                W /= 2;
                H /= 2;
            }
            SG_REQUIRE(W >= 1 && H >= 1, "camera %d level %d has an empty image", c, l);
            SG_REQUIRE(W <= 16 * 65535 && H <= 8 * 65535, "image too large");
            sg_view &o = out[v];
            o.fx = fx; o.fy = fy; o.cx = cx; o.cy = cy;
            memcpy(o.R, cams[c].R_cw, sizeof(o.R));
            memcpy(o.t, cams[c].t_cw, sizeof(o.t));
            o.W = W; o.H = H;
            o.tiles_x = (W + tile_w - 1) / tile_w;
            o.tiles_y = (H + tile_h - 1) / tile_h;
            o.tile_offset = (int32_t)tiles;
            o.pixel_offset = (int32_t)pix;
            o.level = l;
            o.camera = c;
            tiles += (int64_t)o.tiles_x * o.tiles_y;
            pix += (int64_t)W * H;
            SG_REQUIRE(pix < (1ll << 31) && tiles < (1ll << 31), "too many pixels/tiles");
        }
    }
    if (total_pixels) *total_pixels = pix;
    if (total_tiles) *total_tiles = (int32_t)tiles;
    return SG_OK;
}

sg_status sg_project_gaussians(const sg_gaussians *g, const sg_view *views, int32_t n_views,
                               const sg_config *cfg, sg_projected *out, uint32_t *status,
                               sg_stream_t stream) {
    SG_TRY(check_gaussians(g));
    SG_TRY(check_cfg(cfg));
    SG_TRY(check_views(views, n_views));
    SG_REQUIRE(out && out->geo && out->rect && out->ext, "projected buffers are NULL");
    SG_REQUIRE(aligned16(out->geo), "geo must be 16-byte aligned");
    SG_TRY(check_record_colour(g, out));
    SG_REQUIRE((int64_t)g->N * n_views < (1ll << 32), "too many records");
    SG_REQUIRE(!cfg->check_numeric || status, "check_numeric needs a status word");
    return launch_project_fwd(g, views, n_views, cfg, out, cfg->check_numeric ? status : nullptr,
                              (cudaStream_t)stream);
}

size_t sg_tile_lists_workspace_size(int64_t n_records, int32_t capacity) {
    return tile_lists_workspace_size(n_records, capacity);
}

sg_status sg_build_tile_lists(const sg_projected *proj, int32_t N, int32_t n_views,
                              const sg_view *views, int32_t n_tiles, const sg_config *cfg,
                              sg_tile_lists *lists, void *workspace, size_t workspace_bytes,
                              uint32_t *status, sg_stream_t stream) {
    SG_REQUIRE(proj && proj->geo && proj->rect && proj->ext, "projected buffers are NULL");
    SG_TRY(check_cfg(cfg));
    SG_TRY(check_views(views, n_views));
    SG_REQUIRE(N >= 0 && n_tiles >= 1, "bad N / n_tiles");
    SG_REQUIRE(!lists || !lists->half_masks || (int64_t)N * n_views < (int64_t)1 << 30,
               "N * n_views = %lld records: with half masks at most 2^30 - 1", (long long)N * n_views);
    SG_REQUIRE(lists && lists->tile && lists->record && lists->ranges && lists->count, "tile-list buffers are NULL");
    SG_REQUIRE(lists->capacity >= 1, "capacity must be >= 1");
    SG_REQUIRE(workspace && status, "workspace/status is NULL");
    SG_REQUIRE(aligned16(workspace), "workspace must be 16-byte aligned");
    return launch_build_tile_lists(proj, N, n_views, views, n_tiles, cfg->tile_w, cfg->tile_h, lists, workspace,
                                   workspace_bytes,
                                   status, (cudaStream_t)stream);
}

sg_status sg_render_pyramid(const sg_gaussians *g, const sg_projected *proj,
                            const sg_tile_lists *lists, const sg_view *views, int32_t n_views,
                            int32_t n_tiles, const sg_config *cfg, sg_images *out, sg_saved *saved,
                            int32_t *work_counter, sg_stream_t stream) {
    SG_TRY(check_gaussians(g));
    SG_TRY(check_cfg(cfg));
    SG_TRY(check_views(views, n_views));
    SG_REQUIRE(proj && lists && out && saved, "NULL argument");
    SG_REQUIRE(out->rgb && out->depth && out->sem && saved->T_final && saved->last && saved->n_contrib,
               "output buffers are NULL");
    SG_REQUIRE(!cfg->persistent || work_counter, "persistent launch needs work_counter");
    SG_TRY(check_record_colour(g, proj));
    RasterArgs a{};
    fill_raster_args(a, g, proj, lists, views, n_views, n_tiles, cfg, work_counter);
    a.img_rgb = out->rgb;
    a.img_depth = out->depth;
    a.img_sem = out->sem;
    a.T_final = saved->T_final;
    a.last = saved->last;
    a.n_contrib = saved->n_contrib;
    a.ppt = cfg->pixels_per_thread;
    return launch_raster(a, g->C, false, (cudaStream_t)stream);
}

size_t sg_loss_workspace_size(const sg_view *views_host, int32_t n_views, int32_t C,
                              int32_t n_classes) {
    if (!views_host || n_views < 1 || n_views > SG_MAX_VIEWS) return 0;
    return loss_workspace_size(views_host, n_views, C, n_classes);
}

sg_status sg_pyramid_loss(const sg_images *rendered, const sg_targets *gt, const sg_view *views,
                          const sg_view *views_host, int32_t n_views, int32_t C,
                          const sg_loss_config *lcfg, float *terms, sg_images *dL, void *workspace,
                          size_t workspace_bytes, uint32_t *status, sg_stream_t stream) {
    SG_TRY(check_loss_args(rendered, gt, views, views_host, n_views, C, lcfg, terms, dL, status));
    SG_REQUIRE(workspace, "workspace is NULL");
    SG_REQUIRE(aligned16(workspace), "workspace must be 16-byte aligned");
    return launch_loss(rendered, gt, views, views_host, n_views, C, lcfg, terms, dL, workspace,
                       workspace_bytes, lcfg->check_numeric ? status : nullptr, (cudaStream_t)stream);
}

size_t sg_backward_workspace_size(int64_t n_records, int32_t sem_channels) {
    if (n_records < 0 || sem_channels < 0) return 0;
    return (size_t)n_records * (12 + (size_t)sem_channels) * sizeof(float);
}

static sg_status check_backward(const sg_gaussians *g, const sg_view *views, int32_t n_views, const sg_config *cfg,
                                const void *workspace, size_t workspace_bytes, const sg_gaussian_grads *grads) {
    SG_TRY(check_gaussians(g));
    SG_TRY(check_cfg(cfg));
    SG_TRY(check_views(views, n_views));
    SG_REQUIRE(grads && workspace, "NULL argument");
    SG_REQUIRE(g->N == 0 || (grads->mean && grads->log_scale && grads->quat && grads->opacity_logit &&
                             grads->rgb && grads->sem),
               "gradient buffers are NULL");
    SG_REQUIRE(grads->N == g->N && grads->C == g->C, "grads shape differs from gaussians");
    SG_REQUIRE(grads->sh_degree == g->sh_degree, "grads sh_degree %d differs from gaussians' %d",
               grads->sh_degree, g->sh_degree);
    SG_REQUIRE(g->N == 0 || !sh_colour(g) || grads->sh, "grads->sh is NULL");
    SG_REQUIRE(g->N == 0 || !sh_semantic(g) || (grads->sem_sh && aligned16(grads->sem_sh) && aligned16(grads->sem)),
               "grads->sem_sh is NULL, or it or grads->sem is not 16-byte aligned");
    SG_REQUIRE(aligned16(workspace), "workspace must be 16-byte aligned");
    const size_t need = sg_backward_workspace_size((int64_t)g->N * n_views, sh_semantic(g) ? g->C : 0);
    if (workspace_bytes < need) {
        set_error("render_pyramid_backward: workspace %zu bytes < %zu needed", workspace_bytes, need);
        return SG_ERR_CAPACITY;
    }
    return SG_OK;
}

sg_status sg_render_pyramid_backward_raster(const sg_gaussians *g, const sg_projected *proj,
                                            const sg_tile_lists *lists, const sg_view *views,
                                            int32_t n_views, int32_t n_tiles, const sg_config *cfg,
                                            const sg_saved *saved, const sg_images *dL,
                                            sg_gaussian_grads *grads, void *workspace,
                                            size_t workspace_bytes, int32_t *work_counter,
                                            sg_stream_t stream) {
    SG_TRY(check_backward(g, views, n_views, cfg, workspace, workspace_bytes, grads));
    SG_REQUIRE(proj && lists && saved && dL, "NULL argument");
    SG_REQUIRE(!cfg->persistent || work_counter, "persistent launch needs work_counter");
    SG_TRY(check_record_colour(g, proj));
    cudaStream_t st = (cudaStream_t)stream;
    float *g2d = (float *)workspace;  // zero on entry (see sg.h)
    RasterArgs a{};
    fill_raster_args(a, g, proj, lists, views, n_views, n_tiles, cfg, work_counter);
    a.T_final = saved->T_final;
    a.last = saved->last;
    a.n_contrib = saved->n_contrib;
    a.dL_rgb = dL->rgb;
    a.dL_depth = dL->depth;
    a.dL_sem = dL->sem;
    a.g2d = g2d;
    const size_t R = (size_t)g->N * n_views;
    if (sh_colour(g)) {
        // per-record colour gradients in the workspace's colour block (4 floats per record)
        a.g_col = g2d + 8 * R;
        a.col_stride = 4;
    } else {
        a.g_col = grads->rgb;
        a.col_stride = 3;
    }
    // with sem_sh, per-record semantic gradients in the workspace's semantic block
    a.g_sem = sh_semantic(g) ? g2d + 12 * R : grads->sem;
    a.sem_v2 = ((uintptr_t)a.g_sem % 8) == 0 && (g->C % 2) == 0;
    a.ppt = cfg->pixels_per_thread_bwd;
    if (cfg->batch_bwd) a.batch = cfg->batch_bwd;
    return launch_raster(a, g->C, true, st);
}

sg_status sg_project_gaussians_backward(const sg_gaussians *g, const sg_projected *proj,
                                        const sg_view *views, int32_t n_views, const sg_config *cfg,
                                        void *workspace, size_t workspace_bytes,
                                        sg_gaussian_grads *grads, sg_stream_t stream) {
    SG_TRY(check_backward(g, views, n_views, cfg, workspace, workspace_bytes, grads));
    SG_REQUIRE(proj, "NULL argument");
    return launch_project_bwd(g, views, n_views, cfg, proj, (float *)workspace, grads,
                              (cudaStream_t)stream);
}

sg_status sg_render_pyramid_backward(const sg_gaussians *g, const sg_projected *proj,
                                     const sg_tile_lists *lists, const sg_view *views,
                                     int32_t n_views, int32_t n_tiles, const sg_config *cfg,
                                     const sg_saved *saved, const sg_images *dL,
                                     sg_gaussian_grads *grads, void *workspace,
                                     size_t workspace_bytes, int32_t *work_counter,
                                     sg_stream_t stream) {
    SG_TRY(sg_render_pyramid_backward_raster(g, proj, lists, views, n_views, n_tiles, cfg, saved, dL, grads,
                                             workspace, workspace_bytes, work_counter, stream));
    return sg_project_gaussians_backward(g, proj, views, n_views, cfg, workspace, workspace_bytes, grads, stream);
}

sg_status sg_build_pyramid(float *rgb, float *depth, int32_t *label, float *sem, int32_t n_sem_ch,
                           const sg_view *views_host, int32_t n_views, sg_stream_t stream) {
    SG_REQUIRE(rgb && depth && views_host, "NULL argument");
    SG_REQUIRE(n_views >= 1 && n_views <= SG_MAX_VIEWS, "bad n_views");
    SG_REQUIRE(n_sem_ch == 0 || sem, "sem is NULL");
    return launch_pyramid(rgb, depth, label, sem, n_sem_ch, views_host, n_views, (cudaStream_t)stream);
}

sg_status sg_adam_step(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int32_t step, sg_stream_t stream) {
    SG_REQUIRE(n >= 0, "n < 0");
    if (n == 0) return SG_OK;
    SG_REQUIRE(param && grad && m && v, "NULL argument");
    SG_REQUIRE(step >= 1, "step must be >= 1");
    return launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
}

sg_status sg_adam_multi(const sg_adam_group *groups, int32_t n_groups, float beta1, float beta2, float eps,
                        int32_t step, int32_t zero_grad, uint32_t *status, sg_stream_t stream) {
    SG_REQUIRE(groups && n_groups >= 1 && n_groups <= SG_ADAM_MAX_GROUPS, "n_groups must be in [1, %d]",
               SG_ADAM_MAX_GROUPS);
    SG_REQUIRE(step >= 1, "step must be >= 1");
    for (int k = 0; k < n_groups; ++k) {
        SG_REQUIRE(groups[k].n >= 0, "group %d: n < 0", k);
        SG_REQUIRE(groups[k].n == 0 || (groups[k].param && groups[k].grad && groups[k].m && groups[k].v),
                   "group %d: NULL pointer", k);
    }
    return launch_adam_multi(groups, n_groups, beta1, beta2, eps, step, zero_grad, status, (cudaStream_t)stream);
}

}  // extern "C"
