/*
 * sg_oracle.c -- plain, slow FP64 CPU oracle of the multi-level-pyramid Gaussian
 * splatting rasterizer (RGBDS-SLAM, Sec. III-B..D).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file; only the tests, the package entry's smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or constant table with the CUDA path.
 *
 * What it computes (all in double precision):
 *   oc_project          Eq. 2-3, generalised to anisotropic Gaussians by the EWA
 *                       covariance projection that Sec. III-C defers to (3D Gaussian
 *                       splatting); reduces to Eq. 2 for isotropic Gaussians on the axis.
 *                       With cfg isotropic = 1 it is Eq. 2 itself: an isotropic Gaussian of
 *                       radius r = exp(log_scale[0]) projects to a circle of radius
 *                       f r / d (fx along x, fy along y), i.e. Sigma2D = diag((fx r/d)^2,
 *                       (fy r/d)^2) + dilation; quaternion and log_scale[1..2] are unused.
 *   oc_render           Eq. 7-9: per-pixel brute force over all Gaussians, sorted by
 *                       depth (the camera-space depth t_z rounded to float32, then ascending
 *                       Gaussian id), front-to-back compositing of RGB, depth and C semantic
 *                       channels.
 *   oc_render_backward  hand-derived adjoint of oc_render followed by the adjoint of
 *                       oc_project (Sec. III-D "perform backpropagation"), giving
 *                       dL/d{mean, log_scale, quat, opacity_logit, rgb, sem}.
 *   oc_ssim             mean SSIM (Wang et al. 2004, the SSIM cited in Sec. IV-A) with an
 *                       11x11 Gaussian window (sigma 1.5), zero-padded "same" windows, and
 *                       its gradient with respect to the first image (Eq. 10, 12).
 *
 * Compositing rules (the 3D Gaussian splatting conventions Sec. III-C refers to):
 *   alpha = min(alpha_max, o * exp(-sigma)),  sigma = 1/2 d^T conic d,  d = p - mu2D;
 *   a Gaussian with sigma < 0 or alpha < alpha_min is skipped; if T*(1-alpha) < T_min
 *   compositing stops before that Gaussian is added.  Pixel (x, y) is evaluated at the
 *   point (x, y).  The depth channel value d_i is the camera-space z of the mean (Eq. 8).
 *   Derivatives at the clamp and skip branches are those of the branch taken (zero).
 *
 * Camera packing (18 doubles): fx fy cx cy W H R_cw[9, row-major] t_cw[3].
 * Config packing (10 doubles): alpha_max alpha_min T_min z_near dilation bg_r bg_g bg_b
 *                              fov_clamp isotropic.
 * Image/pixel-list outputs are planar: channel ch of list entry k is at [ch*n_pix + k].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_PROJ_STRIDE 24

/* Projection record layout (OC_PROJ_STRIDE doubles per Gaussian). */
enum {
    P_VALID = 0, P_U, P_V, P_DEPTH, P_OPAC,
    P_CA, P_CB, P_CC,           /* conic = Sigma2D^{-1} = [[a, b], [b, c]] */
    P_S00, P_S01, P_S11,        /* Sigma2D (dilation included) */
    P_TX, P_TY, P_TZ,           /* camera-space mean */
    P_CLX, P_CLY,               /* Jacobian clamp active in x / y (0 or 1) */
    P_EXTX, P_EXTY,             /* half extents outside which alpha < alpha_min */
    P_LIMX, P_LIMY,             /* clamp limits of t_x/t_z and t_y/t_z */
    P_DKEY,                     /* depth ordering key: t_z rounded to float32 */
    P_DAMB,                     /* 1: t_z lies within DEPTH_KEY_BAND of a float32 rounding
                                   midpoint, so the key is not decided (see depth_key) */
    P_GEXTX, P_GEXTY            /* half extents outside which alpha < alpha_min / 2 (the
                                   candidates gathered per pixel, for the ambiguity flags) */
};

/* Per-pixel ambiguity flags (reported, never used to change a result). */
enum { F_SKIP = 1, F_STOP = 2, F_DEPTH = 4, F_CLAMP = 8 };

typedef struct {
    double fx, fy, cx, cy;
    int W, H;
    double R[9], t[3];
} cam_t;

typedef struct {
    double alpha_max, alpha_min, T_min, z_near, dilation, bg[3], fov_clamp;
    int isotropic;
} cfg_t;

static cam_t unpack_cam(const double *c) {
    cam_t k;
    k.fx = c[0]; k.fy = c[1]; k.cx = c[2]; k.cy = c[3];
    k.W = (int)c[4]; k.H = (int)c[5];
    for (int i = 0; i < 9; ++i) k.R[i] = c[6 + i];
    for (int i = 0; i < 3; ++i) k.t[i] = c[15 + i];
    return k;
}

static cfg_t unpack_cfg(const double *c) {
    cfg_t g;
    g.alpha_max = c[0]; g.alpha_min = c[1]; g.T_min = c[2]; g.z_near = c[3];
    g.dilation = c[4]; g.bg[0] = c[5]; g.bg[1] = c[6]; g.bg[2] = c[7]; g.fov_clamp = c[8];
    g.isotropic = c[9] != 0.0;
    return g;
}

/* Rotation matrix (row-major) of the unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* M = R(q/|q|) diag(exp(s)); Sigma = M M^T (the anisotropic covariance). */
static void scale_rot(const double *log_scale, const double *quat, double qhat[4], double R[9],
                      double M[9], double Sig[9]) {
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    for (int i = 0; i < 4; ++i) qhat[i] = quat[i] / qn;
    quat_to_rot(qhat, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * exp(log_scale[j]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += M[3 * i + k] * M[3 * j + k];
            Sig[3 * i + j] = s;
        }
}

/* J (2x3) of the perspective map at the clamped mean, and T = J W. */
static void jacobian(const cam_t *cam, const double t[3], double limx, double limy,
                     double J[6], int *clx, int *cly, double T[6]) {
    double rx = t[0] / t[2], ry = t[1] / t[2];
    *clx = 0; *cly = 0;
    if (rx > limx) { rx = limx; *clx = 1; } else if (rx < -limx) { rx = -limx; *clx = 1; }
    if (ry > limy) { ry = limy; *cly = 1; } else if (ry < -limy) { ry = -limy; *cly = 1; }
    double xt = rx * t[2], yt = ry * t[2], z2 = t[2] * t[2];
    J[0] = cam->fx / t[2]; J[1] = 0; J[2] = -cam->fx * xt / z2;
    J[3] = 0; J[4] = cam->fy / t[2]; J[5] = -cam->fy * yt / z2;
    const double *W = cam->R;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = J[3 * i] * W[j] + J[3 * i + 1] * W[3 + j] + J[3 * i + 2] * W[6 + j];
}

/* The sorted set N of Eq. 7-9 is ordered by depth: the key is the camera-space depth t_z
 * (computed here in double precision) rounded to the nearest float32, ties broken by
 * Gaussian id.  Any evaluation of t_z = R20 x + R21 y + R22 z + t_z0 whose error stays
 * below DEPTH_KEY_BAND times the magnitude of its terms rounds to the same key, unless t_z
 * itself lies within that distance of a midpoint between two float32 values; such a key
 * is not decided by the definition and is flagged (*ambiguous = 1). */
#define DEPTH_KEY_BAND 0x1p-40
static float depth_key(const double *mean, const cam_t *cam, double tz, int *ambiguous) {
    const float key = (float)tz;
    const double lo = 0.5 * ((double)key + (double)nextafterf(key, -INFINITY));
    const double hi = 0.5 * ((double)key + (double)nextafterf(key, INFINITY));
    const double mag = fabs(cam->R[6] * mean[0]) + fabs(cam->R[7] * mean[1]) +
                       fabs(cam->R[8] * mean[2]) + fabs(cam->t[2]);
    const double band = DEPTH_KEY_BAND * mag;
    *ambiguous = fabs(tz - lo) <= band || fabs(tz - hi) <= band;
    return key;
}

/* Projection of one Gaussian (Eq. 2-3 via EWA).  Writes OC_PROJ_STRIDE values. */
static void project_one(const double *mean, const double *log_scale, const double *quat,
                        double opacity_logit, const cam_t *cam, const cfg_t *cfg, double *out) {
    memset(out, 0, sizeof(double) * OC_PROJ_STRIDE);
    const double *W = cam->R;
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = W[3 * i] * mean[0] + W[3 * i + 1] * mean[1] + W[3 * i + 2] * mean[2] + cam->t[i];
    out[P_TX] = t[0]; out[P_TY] = t[1]; out[P_TZ] = t[2];
    int damb;
    out[P_DKEY] = (double)depth_key(mean, cam, t[2], &damb);
    out[P_DAMB] = damb;
    if (!(t[2] > cfg->z_near)) return;                    /* at or behind the near plane */
    double o = 1.0 / (1.0 + exp(-opacity_logit));
    out[P_OPAC] = o;
    out[P_DEPTH] = t[2];
    out[P_U] = cam->fx * t[0] / t[2] + cam->cx;
    out[P_V] = cam->fy * t[1] / t[2] + cam->cy;
    double limx = cfg->fov_clamp * 0.5 * cam->W / cam->fx;
    double limy = cfg->fov_clamp * 0.5 * cam->H / cam->fy;
    out[P_LIMX] = limx; out[P_LIMY] = limy;
    double S[4];                                          /* projected covariance */
    if (cfg->isotropic) {                                 /* Eq. 2: radius f r / d */
        double r = exp(log_scale[0]);
        double rx = cam->fx * r / t[2], ry = cam->fy * r / t[2];
        S[0] = rx * rx; S[1] = S[2] = 0.0; S[3] = ry * ry;
    } else {                                              /* EWA: T Sig T^T */
        double J[6], T[6], qh[4], R[9], M[9], Sig[9];
        int clx, cly;
        jacobian(cam, t, limx, limy, J, &clx, &cly, T);
        out[P_CLX] = clx; out[P_CLY] = cly;
        scale_rot(log_scale, quat, qh, R, M, Sig);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double s = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) s += T[3 * i + k] * Sig[3 * k + l] * T[3 * j + l];
                S[2 * i + j] = s;
            }
    }
    double s00 = S[0] + cfg->dilation, s01 = 0.5 * (S[1] + S[2]), s11 = S[3] + cfg->dilation;
    out[P_S00] = s00; out[P_S01] = s01; out[P_S11] = s11;
    double det = s00 * s11 - s01 * s01;
    if (!(det > 0)) return;
    out[P_CA] = s11 / det; out[P_CB] = -s01 / det; out[P_CC] = s00 / det;
    if (o < cfg->alpha_min) return;                       /* alpha <= o < alpha_min everywhere */
    /* min over d_y of 1/2 d^T Sigma^{-1} d is d_x^2 / (2 s00): outside |d_x| > extx the
     * exponent exceeds ln(o/alpha_min), hence alpha < alpha_min (exact bound). */
    double thr = log(o / cfg->alpha_min);
    out[P_EXTX] = sqrt(2.0 * thr * s00) * (1.0 + 1e-9) + 1e-9;
    out[P_EXTY] = sqrt(2.0 * thr * s11) * (1.0 + 1e-9) + 1e-9;
    double thr2 = log(2.0 * o / cfg->alpha_min);
    out[P_GEXTX] = sqrt(2.0 * thr2 * s00) * (1.0 + 1e-9) + 1e-9;
    out[P_GEXTY] = sqrt(2.0 * thr2 * s11) * (1.0 + 1e-9) + 1e-9;
    out[P_VALID] = 1.0;
}

int oc_proj_stride(void) { return OC_PROJ_STRIDE; }

void oc_project(int N, const double *mean, const double *log_scale, const double *quat,
                const double *opacity_logit, const double *camp, const double *cfgp,
                double *out) {
    cam_t cam = unpack_cam(camp);
    cfg_t cfg = unpack_cfg(cfgp);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i)
        project_one(mean + 3 * i, log_scale + 3 * i, quat + 4 * i, opacity_logit[i], &cam, &cfg,
                    out + (size_t)OC_PROJ_STRIDE * i);
}

/* ------------------------------------------------------------------------------------ */
/* Per-pixel candidate list and compositing (Eq. 7-9)                                    */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    float dkey;        /* depth rounded to float32: the ordering key */
    int id;            /* Gaussian id: tie-break */
    int damb;          /* the key is undecided (P_DAMB) */
    int order_amb;     /* an undecided key next to a key within one float32 step: the
                          order of this candidate is not fixed by the definition */
    double raw;        /* o * exp(-sigma) before the clamp */
    double alpha;      /* min(alpha_max, raw) */
    double G;          /* exp(-sigma) */
    double dx, dy;     /* p - mu2D */
} cand_t;

static int cand_cmp(const void *pa, const void *pb) {
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->dkey < b->dkey) return -1;
    if (a->dkey > b->dkey) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

static int32_t f32_bits(float f) { int32_t i; memcpy(&i, &f, 4); return i; }

/* Gather the candidates of pixel (x, y) whose alpha reaches alpha_min, sorted. */
static int gather(double x, double y, int N, const double *proj, const cfg_t *cfg, cand_t *buf) {
    int n = 0;
    for (int i = 0; i < N; ++i) {
        const double *p = proj + (size_t)OC_PROJ_STRIDE * i;
        if (p[P_VALID] == 0.0) continue;
        double dx = x - p[P_U], dy = y - p[P_V];
        if (fabs(dx) > p[P_GEXTX] || fabs(dy) > p[P_GEXTY]) continue; /* alpha < alpha_min / 2 */
        double sigma = 0.5 * (p[P_CA] * dx * dx + p[P_CC] * dy * dy) + p[P_CB] * dx * dy;
        if (sigma < 0) continue;
        double G = exp(-sigma);
        double raw = p[P_OPAC] * G;
        double alpha = raw < cfg->alpha_max ? raw : cfg->alpha_max;
        /* keep the near-threshold ones too: the flags below need them */
        if (alpha < cfg->alpha_min * 0.5) continue;
        cand_t c;
        c.dkey = (float)p[P_DKEY]; c.id = i; c.raw = raw; c.alpha = alpha; c.G = G;
        c.dx = dx; c.dy = dy; c.damb = p[P_DAMB] != 0.0; c.order_amb = 0;
        buf[n++] = c;
    }
    qsort(buf, (size_t)n, sizeof(cand_t), cand_cmp);
    /* an undecided key can move by one float32 step: it may then pass a neighbour whose
       key is equal or one step away (keys are sorted, so the neighbours suffice) */
    for (int k = 0; k < n; ++k) {
        if (!buf[k].damb) continue;
        const int32_t b = f32_bits(buf[k].dkey);
        if (k > 0 && abs(b - f32_bits(buf[k - 1].dkey)) <= 1) buf[k].order_amb = buf[k - 1].order_amb = 1;
        if (k + 1 < n && abs(b - f32_bits(buf[k + 1].dkey)) <= 1) buf[k].order_amb = buf[k + 1].order_amb = 1;
    }
    return n;
}

/* Composites the sorted list.  Writes the contributing positions to contrib[] (indices
 * into buf) with their transmittance before them in Tb[]; returns their count.
 *
 * Ambiguity flags, for an evaluation whose alpha carries a relative error up to `tol` and
 * whose transmittance a relative error up to `tol_T`: a decision is flagged when the exact
 * value lies within that error of its threshold -- raw alpha within tol of alpha_min (skip,
 * F_SKIP) or of alpha_max (clamp, F_CLAMP), the transmittance T' = T (1 - alpha) within tol_T
 * of T_min (stop, F_STOP) -- or when a contributor's depth order is undecided (F_DEPTH). */
static int composite(const cand_t *buf, int n, const cfg_t *cfg, double tol, double tol_T, int *contrib,
                     double *Tb, double *T_out, int *flags) {
    double T = 1.0;
    int m = 0, fl = 0;
    for (int k = 0; k < n; ++k) {
        const cand_t *c = buf + k;
        if (fabs(c->raw - cfg->alpha_min) <= tol * cfg->alpha_min) fl |= F_SKIP;
        if (c->alpha < cfg->alpha_min) continue;
        if (fabs(c->raw - cfg->alpha_max) <= tol * cfg->alpha_max) fl |= F_CLAMP;
        if (c->order_amb) fl |= F_DEPTH;
        double Tn = T * (1.0 - c->alpha);
        if (fabs(Tn - cfg->T_min) <= tol_T * cfg->T_min) fl |= F_STOP;
        if (Tn < cfg->T_min) break;
        contrib[m] = k; Tb[m] = T; ++m;
        T = Tn;
    }
    *T_out = T;
    *flags = fl;
    return m;
}

/*
 * Render the listed pixels (or, with pix == NULL, every pixel of the W x H image in
 * row-major order).  rgb: N x 3, sem: N x C.  Outputs planar over the pixel list.
 */
void oc_render(int N, int C, const double *proj, const double *rgb, const double *sem,
               const double *camp, const double *cfgp, int n_pix, const int *pix, double tol, double tol_T,
               double *out_rgb, double *out_depth, double *out_sem, double *out_T,
               int *out_ncontrib, int *out_flags) {
    cam_t cam = unpack_cam(camp);
    cfg_t cfg = unpack_cfg(cfgp);
    if (!pix) n_pix = cam.W * cam.H;
#pragma omp parallel
    {
        cand_t *buf = (cand_t *)malloc(sizeof(cand_t) * (size_t)(N > 0 ? N : 1));
        int *contrib = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
        double *Tb = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double *acc = (double *)malloc(sizeof(double) * (size_t)(4 + C));
#pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < n_pix; ++k) {
            int px = pix ? pix[2 * k] : k % cam.W;
            int py = pix ? pix[2 * k + 1] : k / cam.W;
            int n = gather((double)px, (double)py, N, proj, &cfg, buf);
            double T;
            int fl;
            int m = composite(buf, n, &cfg, tol, tol_T, contrib, Tb, &T, &fl);
            for (int ch = 0; ch < 4 + C; ++ch) acc[ch] = 0.0;
            for (int j = 0; j < m; ++j) {
                const cand_t *c = buf + contrib[j];
                double w = c->alpha * Tb[j];
                for (int ch = 0; ch < 3; ++ch) acc[ch] += w * rgb[3 * (size_t)c->id + ch];
                acc[3] += w * proj[(size_t)OC_PROJ_STRIDE * c->id + P_DEPTH];
                for (int ch = 0; ch < C; ++ch) acc[4 + ch] += w * sem[(size_t)C * c->id + ch];
            }
            for (int ch = 0; ch < 3; ++ch) out_rgb[(size_t)ch * n_pix + k] = acc[ch] + T * cfg.bg[ch];
            out_depth[k] = acc[3];
            for (int ch = 0; ch < C; ++ch) out_sem[(size_t)ch * n_pix + k] = acc[4 + ch];
            out_T[k] = T;
            out_ncontrib[k] = m;
            out_flags[k] = fl;
        }
        free(buf); free(contrib); free(Tb); free(acc);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Adjoint of the projection (chain rule through Eq. 2-3 / EWA)                          */
/* ------------------------------------------------------------------------------------ */

/* g2: dL/d{u, v, conic a, conic b, conic c, opacity, depth} of one Gaussian. */
static void project_backward_one(const double *mean, const double *log_scale, const double *quat,
                                 const double *p, const cam_t *cam, int isotropic, const double *g2,
                                 double *g_mean, double *g_ls, double *g_q, double *g_ol) {
    (void)mean;
    double gu = g2[0], gv = g2[1], ga = g2[2], gb = g2[3], gc = g2[4], go = g2[5], gd = g2[6];
    double a = p[P_CA], b = p[P_CB], c = p[P_CC];
    /* conic = Sigma2D^{-1}:  dQ = -Q dS Q  (dS symmetric, S01 is one parameter) */
    double gS00 = -(a * a * ga + a * b * gb + b * b * gc);
    double gS01 = -(2 * a * b * ga + (a * c + b * b) * gb + 2 * b * c * gc);
    double gS11 = -(b * b * ga + b * c * gb + c * c * gc);
    if (isotropic) {
        /* S00 = (fx r/tz)^2 + b, S11 = (fy r/tz)^2 + b, r = e^{s0}, S01 = 0 (constant) */
        const double *W = cam->R;
        double t[3] = {p[P_TX], p[P_TY], p[P_TZ]};
        double fx = cam->fx, fy = cam->fy, tz = t[2], tz2 = tz * tz, tz3 = tz2 * tz;
        double r = exp(log_scale[0]);
        double gr = gS00 * 2.0 * fx * fx * r / tz2 + gS11 * 2.0 * fy * fy * r / tz2;
        g_ls[0] += gr * r;
        double gt[3] = {gu * fx / tz, gv * fy / tz,
                        -gu * fx * t[0] / tz2 - gv * fy * t[1] / tz2 + gd
                            - gS00 * 2.0 * fx * fx * r * r / tz3 - gS11 * 2.0 * fy * fy * r * r / tz3};
        for (int j = 0; j < 3; ++j) g_mean[j] += W[j] * gt[0] + W[3 + j] * gt[1] + W[6 + j] * gt[2];
        double o = p[P_OPAC];
        *g_ol += go * o * (1.0 - o);
        (void)quat; (void)g_q;
        return;
    }
    double G[4] = {gS00, 0.5 * gS01, 0.5 * gS01, gS11};   /* full-entry symmetric gradient */
    double t[3] = {p[P_TX], p[P_TY], p[P_TZ]};
    double J[6], T[6], qh[4], R[9], M[9], Sig[9];
    int clx, cly;
    jacobian(cam, t, p[P_LIMX], p[P_LIMY], J, &clx, &cly, T);
    scale_rot(log_scale, quat, qh, R, M, Sig);
    /* S = T Sig T^T:  dL/dSig = T^T G T,  dL/dT = 2 G T Sig */
    double gSig[9], gT[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) s += T[3 * k + i] * G[2 * k + l] * T[3 * l + j];
            gSig[3 * i + j] = s;
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 3; ++l) s += G[2 * i + k] * T[3 * k + l] * Sig[3 * l + j];
            gT[3 * i + j] = 2.0 * s;
        }
    /* T = J W:  dL/dJ = dL/dT W^T */
    const double *W = cam->R;
    double gJ[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            gJ[3 * i + j] = gT[3 * i] * W[3 * j] + gT[3 * i + 1] * W[3 * j + 1] + gT[3 * i + 2] * W[3 * j + 2];
    double fx = cam->fx, fy = cam->fy, tz = t[2], tz2 = tz * tz, tz3 = tz2 * tz;
    double gt[3] = {0, 0, 0};
    gt[2] += gJ[0] * (-fx / tz2) + gJ[4] * (-fy / tz2);
    if (!clx) {                              /* J02 = -fx tx / tz^2 */
        gt[0] += gJ[2] * (-fx / tz2);
        gt[2] += gJ[2] * (2.0 * fx * t[0] / tz3);
    } else {                                 /* J02 = -fx (+-limx) / tz */
        gt[2] += gJ[2] * (-J[2] / tz);
    }
    if (!cly) {
        gt[1] += gJ[5] * (-fy / tz2);
        gt[2] += gJ[5] * (2.0 * fy * t[1] / tz3);
    } else {
        gt[2] += gJ[5] * (-J[5] / tz);
    }
    /* mean2D and depth */
    gt[0] += gu * fx / tz;
    gt[1] += gv * fy / tz;
    gt[2] += -gu * fx * t[0] / tz2 - gv * fy * t[1] / tz2 + gd;
    /* t = W mu + t_cw */
    for (int j = 0; j < 3; ++j) g_mean[j] += W[j] * gt[0] + W[3 + j] * gt[1] + W[6 + j] * gt[2];
    /* Sig = M M^T,  M = R diag(e^s):  dL/dM = 2 gSig M */
    double gM[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += gSig[3 * i + k] * M[3 * k + j];
            gM[3 * i + j] = 2.0 * s;
        }
    double gR[9];
    for (int j = 0; j < 3; ++j) {
        double e = exp(log_scale[j]), s = 0;
        for (int i = 0; i < 3; ++i) {
            gR[3 * i + j] = gM[3 * i + j] * e;
            s += gM[3 * i + j] * R[3 * i + j] * e;
        }
        g_ls[j] += s;
    }
    /* R(qhat) */
    double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
    double gw = 2 * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    double gx = 2 * (y * gR[1] + z * gR[2] + y * gR[3] - 2 * x * gR[4] - w * gR[5] + z * gR[6] +
                     w * gR[7] - 2 * x * gR[8]);
    double gy = 2 * (-2 * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] +
                     z * gR[7] - 2 * y * gR[8]);
    double gz = 2 * (-2 * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2 * z * gR[4] + y * gR[5] +
                     x * gR[6] + y * gR[7]);
    double gqh[4] = {gw, gx, gy, gz};
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double dot = qh[0] * gqh[0] + qh[1] * gqh[1] + qh[2] * gqh[2] + qh[3] * gqh[3];
    for (int i = 0; i < 4; ++i) g_q[i] += (gqh[i] - qh[i] * dot) / qn;
    /* o = sigmoid(l) */
    double o = p[P_OPAC];
    *g_ol += go * o * (1.0 - o);
}

/*
 * Adjoint of oc_render over the listed pixels (or all pixels when pix == NULL), followed
 * by the projection adjoint.  Upstream gradients g_rgb (3 x n_pix), g_depth (n_pix),
 * g_sem (C x n_pix), planar over the pixel list.  Parameter gradients are ADDED to
 * gm (N x 3), gls (N x 3), gq (N x 4), gol (N), grgb (N x 3), gsem (N x C).  If g2d is
 * not NULL it receives (adds) the per-Gaussian 2D gradients (N x 8: u v a b c o depth 0).
 */
void oc_render_backward(int N, int C, const double *mean, const double *log_scale,
                        const double *quat, const double *proj, const double *rgb,
                        const double *sem, const double *camp, const double *cfgp, int n_pix,
                        const int *pix, const double *g_rgb, const double *g_depth,
                        const double *g_sem, double *gm, double *gls, double *gq, double *gol,
                        double *grgb, double *gsem, double *g2d) {
    cam_t cam = unpack_cam(camp);
    cfg_t cfg = unpack_cfg(cfgp);
    if (!pix) n_pix = cam.W * cam.H;
    double *g2 = (double *)calloc((size_t)(N > 0 ? N : 1) * 8, sizeof(double));
#pragma omp parallel
    {
        cand_t *buf = (cand_t *)malloc(sizeof(cand_t) * (size_t)(N > 0 ? N : 1));
        int *contrib = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
        double *Tb = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double *A = (double *)malloc(sizeof(double) * (size_t)(4 + C));
        double *g = (double *)malloc(sizeof(double) * (size_t)(4 + C));
        double *f = (double *)malloc(sizeof(double) * (size_t)(4 + C));
#pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < n_pix; ++k) {
            int px = pix ? pix[2 * k] : k % cam.W;
            int py = pix ? pix[2 * k + 1] : k / cam.W;
            for (int ch = 0; ch < 3; ++ch) g[ch] = g_rgb[(size_t)ch * n_pix + k];
            g[3] = g_depth[k];
            for (int ch = 0; ch < C; ++ch) g[4 + ch] = g_sem[(size_t)ch * n_pix + k];
            int nz = 0;
            for (int ch = 0; ch < 4 + C; ++ch) nz |= (g[ch] != 0.0);
            if (!nz) continue;
            int n = gather((double)px, (double)py, N, proj, &cfg, buf);
            double Tfin;
            int fl;
            int m = composite(buf, n, &cfg, 0.0, 0.0, contrib, Tb, &Tfin, &fl);
            /* suffix accumulator A = (sum_{k>i} w_k f_k + T_final bg) / T_{i+1} */
            for (int ch = 0; ch < 4 + C; ++ch) A[ch] = ch < 3 ? cfg.bg[ch] : 0.0;
            for (int j = m - 1; j >= 0; --j) {
                const cand_t *c = buf + contrib[j];
                const double *p = proj + (size_t)OC_PROJ_STRIDE * c->id;
                for (int ch = 0; ch < 3; ++ch) f[ch] = rgb[3 * (size_t)c->id + ch];
                f[3] = p[P_DEPTH];
                for (int ch = 0; ch < C; ++ch) f[4 + ch] = sem[(size_t)C * c->id + ch];
                double Ti = Tb[j], al = c->alpha, w = al * Ti;
                double dalpha = 0.0;
                for (int ch = 0; ch < 4 + C; ++ch) dalpha += g[ch] * (f[ch] - A[ch]);
                dalpha *= Ti;
                for (int ch = 0; ch < 4 + C; ++ch) A[ch] = al * f[ch] + (1.0 - al) * A[ch];
                /* feature gradients */
                for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
                    grgb[3 * (size_t)c->id + ch] += w * g[ch];
                }
#pragma omp atomic
                g2[8 * (size_t)c->id + 6] += w * g[3];
                for (int ch = 0; ch < C; ++ch) {
#pragma omp atomic
                    gsem[(size_t)C * c->id + ch] += w * g[4 + ch];
                }
                if (c->raw >= cfg.alpha_max) continue;   /* clamped: d alpha / d(o, sigma) = 0 */
                double go = dalpha * c->G;
                double gsig = -dalpha * p[P_OPAC] * c->G;
                double dx = c->dx, dy = c->dy;
                double ca = p[P_CA], cb = p[P_CB], cc = p[P_CC];
                double vals[6] = {
                    gsig * -(ca * dx + cb * dy),     /* d sigma / d u = -(a dx + b dy) */
                    gsig * -(cb * dx + cc * dy),
                    gsig * 0.5 * dx * dx,
                    gsig * dx * dy,
                    gsig * 0.5 * dy * dy,
                    go};
                for (int q = 0; q < 6; ++q) {
#pragma omp atomic
                    g2[8 * (size_t)c->id + q] += vals[q];
                }
            }
        }
        free(buf); free(contrib); free(Tb); free(A); free(g); free(f);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        const double *p = proj + (size_t)OC_PROJ_STRIDE * i;
        if (p[P_VALID] == 0.0) continue;
        project_backward_one(mean + 3 * i, log_scale + 3 * i, quat + 4 * i, p, &cam, cfg.isotropic,
                             g2 + 8 * (size_t)i, gm + 3 * i, gls + 3 * i, gq + 4 * i, gol + i);
    }
    if (g2d)
        for (size_t i = 0; i < (size_t)N * 8; ++i) g2d[i] += g2[i];
    free(g2);
}

/* ------------------------------------------------------------------------------------ */
/* SSIM (Wang et al. 2004): 11x11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2     */
/* ------------------------------------------------------------------------------------ */

/* Mean SSIM over nch planes of H x W; if grad != NULL, it receives d(mean SSIM)/dx. */
double oc_ssim(int H, int W, int nch, const double *x, const double *y, double *grad) {
    double g1[11], s = 0;
    for (int i = 0; i < 11; ++i) { g1[i] = exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += g1[i]; }
    for (int i = 0; i < 11; ++i) g1[i] /= s;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    size_t P = (size_t)H * W;
    double total = 0.0;
    double *Pm = (double *)malloc(sizeof(double) * P), *Qm = (double *)malloc(sizeof(double) * P),
           *Rm = (double *)malloc(sizeof(double) * P);
    double norm = 1.0 / ((double)nch * (double)P);
    for (int ch = 0; ch < nch; ++ch) {
        const double *X = x + ch * P, *Y = y + ch * P;
        double sum = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sum)
        for (int r = 0; r < H; ++r)
            for (int q = 0; q < W; ++q) {
                double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
                for (int i = -5; i <= 5; ++i) {
                    int rr = r + i;
                    if (rr < 0 || rr >= H) continue;
                    for (int j = -5; j <= 5; ++j) {
                        int cc = q + j;
                        if (cc < 0 || cc >= W) continue;
                        double w = g1[i + 5] * g1[j + 5];
                        double xv = X[(size_t)rr * W + cc], yv = Y[(size_t)rr * W + cc];
                        mx += w * xv; my += w * yv;
                        exx += w * xv * xv; eyy += w * yv * yv; exy += w * xv * yv;
                    }
                }
                double sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                double A1 = 2 * mx * my + C1, A2 = 2 * sxy + C2;
                double B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
                double ss = (A1 * A2) / (B1 * B2);
                sum += ss;
                if (grad) {
                    double ds_dmx = 2 * my * A2 / (B1 * B2) - ss * 2 * mx / B1;
                    double ds_dsxx = -ss / B2;
                    double ds_dsxy = 2 * A1 / (B1 * B2);
                    size_t o = (size_t)r * W + q;
                    /* s as a function of (mx, my, Exx, Eyy, Exy) */
                    Pm[o] = norm * (ds_dmx - 2 * mx * ds_dsxx - my * ds_dsxy);
                    Qm[o] = norm * ds_dsxx;
                    Rm[o] = norm * ds_dsxy;
                }
            }
        total += sum;
        if (grad) {
            double *Gd = grad + ch * P;
#pragma omp parallel for schedule(static)
            for (int r = 0; r < H; ++r)
                for (int q = 0; q < W; ++q) {
                    double a = 0, bq = 0, cr = 0;
                    for (int i = -5; i <= 5; ++i) {
                        int rr = r + i;
                        if (rr < 0 || rr >= H) continue;
                        for (int j = -5; j <= 5; ++j) {
                            int cc = q + j;
                            if (cc < 0 || cc >= W) continue;
                            double w = g1[i + 5] * g1[j + 5];
                            size_t o = (size_t)rr * W + cc;
                            a += w * Pm[o]; bq += w * Qm[o]; cr += w * Rm[o];
                        }
                    }
                    size_t o = (size_t)r * W + q;
                    Gd[o] = a + 2.0 * X[o] * bq + Y[o] * cr;
                }
        }
    }
    free(Pm); free(Qm); free(Rm);
    return total * norm;
}

int oc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
