// project.cu -- EWA projection of 3D Gaussians into every (view, pyramid level) and its
// adjoint (Eq. 2-3 generalised to anisotropic Gaussians; Sec. III-D backpropagation).
//
// One thread per Gaussian loops over the view-levels.  Forward: the Gaussian's parameters
// (44 B) are read once and its 3D covariance is formed once, then one 32-byte record, one
// 8-byte tile rectangle and the 8-byte extents are written per view-level.  Backward: the
// view-levels where it is visible are gathered first (all rectangle loads in flight at once),
// then the chain rule runs on each with the next one's 2D gradients already loading.  The
// view table sits in shared memory.
//
// View-dependent colour and semantic feature (spherical harmonics of degree D = 1..3) is a
// template parameter: the forward evaluates each visible record's colour (and, with sem_sh,
// its semantic feature) from the camera-to-mean direction, and the adjoint chains the
// per-record gradients to the SH coefficients, rgb / sem and the mean; D = 0 compiles to the
// plain kernels.
#include "sg_common.cuh"

namespace sg {

struct ProjConsts {
    float z_near, dilation, fov_clamp, alpha_min;
    int tile_w, tile_h;
    int isotropic;     // Eq. 2 projection instead of EWA
    uint32_t *status;  // non-NULL: flag non-finite parameters (SG_STATUS_NUMERIC)
};


// Rotation (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

struct GaussianFrame {
    float q[4];    // normalised quaternion
    float qn;      // |q| before normalisation
    float R[9];    // rotation
    float S[3];    // exp(log_scale)
    float Sig[6];  // 3D covariance: xx xy xz yy yz zz
};

__device__ __forceinline__ void gaussian_frame(const float *log_scale, float4 q4, int g,
                                               GaussianFrame &f) {
    f.qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float r = 1.f / f.qn;
    f.q[0] = q4.x * r; f.q[1] = q4.y * r; f.q[2] = q4.z * r; f.q[3] = q4.w * r;
    quat_rot(f.q[0], f.q[1], f.q[2], f.q[3], f.R);
    f.S[0] = expf(log_scale[3 * g + 0]);
    f.S[1] = expf(log_scale[3 * g + 1]);
    f.S[2] = expf(log_scale[3 * g + 2]);
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = f.R[3 * i + j] * f.S[j];
    f.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    f.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    f.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    f.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    f.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    f.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

__device__ __forceinline__ float sym3(const float *S, int i, int j) {
    // index into xx xy xz yy yz zz
    const int a = i < j ? i : j, b = i < j ? j : i;
    const int idx = a == 0 ? b : (a == 1 ? 2 + b : 5);
    return S[idx];
}

// Camera-space mean, Jacobian rows of T = J W and the clamp flags of one view-level.
struct ViewGeom {
    float t[3];
    DF tz;  // camera z in double-float (its rounded head is t[2])
    float T0[3], T1[3];
    float J00, J02, J11, J12;
    bool clx, cly;
};

// The pose part: camera-space mean (the view's R, t only, so shared by every pyramid level
// of a keyframe).
struct PoseGeom {
    float t0, t1;
    DF tz;  // camera z in double-float (its rounded head is the float32 z)
};
__device__ __forceinline__ void pose_geom(const sg_view &vw, const float mu[3], PoseGeom &p) {
    p.t0 = vw.R[0] * mu[0] + vw.R[1] * mu[1] + vw.R[2] * mu[2] + vw.t[0];
    p.t1 = vw.R[3] * mu[0] + vw.R[4] * mu[1] + vw.R[5] * mu[2] + vw.t[1];
    // camera z is also the depth ordering key of the tile lists (the order of the set N of
    // Eq. 7-9): t_z rounded to the nearest float32.  It is summed in double-float (exact
    // products, error near 2^-46 of the terms), whose rounded head is the nearest float32 of
    // the exact depth unless that lies within the sum's error of a rounding midpoint.
    DF z = two_prod(vw.R[6], mu[0]);
    z = df_add(z, two_prod(vw.R[7], mu[1]));
    z = df_add(z, two_prod(vw.R[8], mu[2]));
    p.tz = df_add_f(z, vw.t[2]);
}

// The level part.  (limx, limy) = the Jacobian clamp fov_clamp W / (2 fx), fov_clamp H / (2 fy)
// of the view.
__device__ __forceinline__ void level_geom(const sg_view &vw, const PoseGeom &p, float2 lim, ViewGeom &q) {
    q.t[0] = p.t0;
    q.t[1] = p.t1;
    q.tz = p.tz;
    q.t[2] = q.tz.hi;
    const float itz = 1.f / q.t[2];
    const float limx = lim.x, limy = lim.y;
    float rx = q.t[0] * itz, ry = q.t[1] * itz;
    q.clx = rx > limx || rx < -limx;
    q.cly = ry > limy || ry < -limy;
    rx = fminf(limx, fmaxf(-limx, rx));
    ry = fminf(limy, fmaxf(-limy, ry));
    q.J00 = vw.fx * itz;
    q.J11 = vw.fy * itz;
    q.J02 = -q.J00 * rx;  // = -fx * x~ / tz^2 with x~ = rx * tz
    q.J12 = -q.J11 * ry;
    for (int j = 0; j < 3; ++j) {
        q.T0[j] = q.J00 * vw.R[j] + q.J02 * vw.R[6 + j];
        q.T1[j] = q.J11 * vw.R[3 + j] + q.J12 * vw.R[6 + j];
    }
}

// Sigma2D = A A^T + dil I with A = T M (M = R diag(S)); det by Cauchy-Binet,
// det(A A^T) = |a0 x a1|^2, so it is a sum of non-negative terms.
__device__ __forceinline__ void cov2d(const ViewGeom &q, const GaussianFrame &f, float dil,
                                      float &s00, float &s01, float &s11, float &det) {
    float a0[3], a1[3];
    for (int j = 0; j < 3; ++j) {
        a0[j] = (q.T0[0] * f.R[j] + q.T0[1] * f.R[3 + j] + q.T0[2] * f.R[6 + j]) * f.S[j];
        a1[j] = (q.T1[0] * f.R[j] + q.T1[1] * f.R[3 + j] + q.T1[2] * f.R[6 + j]) * f.S[j];
    }
    const float n0 = a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2];
    const float n1 = a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2];
    s00 = n0 + dil;
    s11 = n1 + dil;
    s01 = a0[0] * a1[0] + a0[1] * a1[1] + a0[2] * a1[2];
    const float c0 = diff_of_products(a0[1], a1[2], a0[2], a1[1]);
    const float c1 = diff_of_products(a0[2], a1[0], a0[0], a1[2]);
    const float c2 = diff_of_products(a0[0], a1[1], a0[1], a1[0]);
    det = (c0 * c0 + c1 * c1 + c2 * c2) + dil * (n0 + n1) + dil * dil;
}

// Eq. 2 as printed: radius r = exp(log_scale[0]) projects to f r / t_z along each axis.
__device__ __forceinline__ void cov2d_eq2(const sg_view &vw, float tz, const GaussianFrame &f, float dil,
                                          float &s00, float &s01, float &s11, float &det) {
    const float rx = vw.fx * f.S[0] / tz, ry = vw.fy * f.S[0] / tz;
    s00 = rx * rx + dil;
    s11 = ry * ry + dil;
    s01 = 0.f;
    det = s00 * s11;
}

// Real spherical harmonics of degree 1..D at the unit direction (x, y, z), in the graphics
// order (m = -l..l within each degree, Condon-Shortley signs).  Constants from their closed
// forms: c1 = sqrt(3/4pi); a2 = sqrt(15/pi)/2, b2 = sqrt(5/pi)/4, c2 = sqrt(15/pi)/4;
// e3 = sqrt(35/2pi)/4, f3 = sqrt(105/pi)/2, h3 = sqrt(21/2pi)/4, k3 = sqrt(7/pi)/4,
// m3 = sqrt(105/pi)/4.
namespace shc {
constexpr float c1 = 0.48860251190291992f;
constexpr float a2 = 1.09254843059207907f, b2 = 0.31539156525252005f, c2 = 0.54627421529603959f;
constexpr float e3 = 0.59004358992664352f, f3 = 2.89061144264055405f, h3 = 0.45704579946446573f;
constexpr float k3 = 0.37317633259011540f, m3 = 1.44530572132027702f;
}  // namespace shc

template <int D>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float *Y) {
    Y[0] = -shc::c1 * y;
    Y[1] = shc::c1 * z;
    Y[2] = -shc::c1 * x;
    if constexpr (D >= 2) {
        Y[3] = shc::a2 * x * y;
        Y[4] = -shc::a2 * y * z;
        Y[5] = shc::b2 * (2.f * z * z - x * x - y * y);
        Y[6] = -shc::a2 * x * z;
        Y[7] = shc::c2 * (x * x - y * y);
    }
    if constexpr (D >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[8] = -shc::e3 * y * (3.f * xx - yy);
        Y[9] = shc::f3 * x * y * z;
        Y[10] = -shc::h3 * y * (4.f * zz - xx - yy);
        Y[11] = shc::k3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
        Y[12] = -shc::h3 * x * (4.f * zz - xx - yy);
        Y[13] = shc::m3 * z * (xx - yy);
        Y[14] = -shc::e3 * x * (xx - 3.f * yy);
    }
}

// sum_k w_k grad Y_k at (x, y, z), the gradient of each basis polynomial (before restriction
// to the sphere).
template <int D>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float *w, float gd[3]) {
    gd[0] = -shc::c1 * w[2];
    gd[1] = -shc::c1 * w[0];
    gd[2] = shc::c1 * w[1];
    if constexpr (D >= 2) {
        gd[0] += shc::a2 * (y * w[3] - z * w[6]) - 2.f * shc::b2 * x * w[5] + 2.f * shc::c2 * x * w[7];
        gd[1] += shc::a2 * (x * w[3] - z * w[4]) - 2.f * shc::b2 * y * w[5] - 2.f * shc::c2 * y * w[7];
        gd[2] += -shc::a2 * (y * w[4] + x * w[6]) + 4.f * shc::b2 * z * w[5];
    }
    if constexpr (D >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gd[0] += -6.f * shc::e3 * x * y * w[8] + shc::f3 * y * z * w[9] + 2.f * shc::h3 * x * y * w[10] -
                 6.f * shc::k3 * x * z * w[11] - shc::h3 * (4.f * zz - 3.f * xx - yy) * w[12] +
                 2.f * shc::m3 * x * z * w[13] - 3.f * shc::e3 * (xx - yy) * w[14];
        gd[1] += -3.f * shc::e3 * (xx - yy) * w[8] + shc::f3 * x * z * w[9] -
                 shc::h3 * (4.f * zz - xx - 3.f * yy) * w[10] - 6.f * shc::k3 * y * z * w[11] +
                 2.f * shc::h3 * x * y * w[12] - 2.f * shc::m3 * y * z * w[13] + 6.f * shc::e3 * x * y * w[14];
        gd[2] += shc::f3 * x * y * w[9] - 8.f * shc::h3 * y * z * w[10] +
                 shc::k3 * (6.f * zz - 3.f * xx - 3.f * yy) * w[11] - 8.f * shc::h3 * x * z * w[12] +
                 shc::m3 * (xx - yy) * w[13];
    }
}

// Jacobian clamp limits of every view-level (thread tid of nthr in the block).
__device__ __forceinline__ void view_limits(const sg_view *s_views, int n_views, float fov_clamp, float2 *s_lim,
                                            int tid, int nthr) {
    for (int i = tid; i < n_views; i += nthr)
        s_lim[i] = make_float2(fov_clamp * 0.5f * (float)s_views[i].W / s_views[i].fx,
                               fov_clamp * 0.5f * (float)s_views[i].H / s_views[i].fy);
}

// s_same[v]: view-level v has the bit-identical pose (R, t) of view-level v - 1 (the next
// pyramid level of the same keyframe).
__device__ __forceinline__ void view_same_pose(const sg_view *s_views, int n_views, bool *s_same, int tid, int nthr) {
    for (int i = tid; i < n_views; i += nthr) {
        bool same = i > 0;
        for (int k = 0; k < 9 && same; ++k) same = __float_as_uint(s_views[i].R[k]) == __float_as_uint(s_views[i - 1].R[k]);
        for (int k = 0; k < 3 && same; ++k) same = __float_as_uint(s_views[i].t[k]) == __float_as_uint(s_views[i - 1].t[k]);
        s_same[i] = same;
    }
}

// Camera centre c = -R^T t of every view-level, next to the view table in shared memory
// (thread tid of nthr in the block).
__device__ __forceinline__ void view_centres(const sg_view *s_views, int n_views, float3 *s_centre,
                                             int tid, int nthr) {
    for (int i = tid; i < n_views; i += nthr) {
        const float *R = s_views[i].R, *t = s_views[i].t;
        s_centre[i] = make_float3(-(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]),
                                  -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]),
                                  -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]));
    }
}

template <int D>
__global__ void __launch_bounds__(256) __maxnreg__((D == 0 ? 64 : D <= 2 ? 128 : 255)) project_fwd_kernel(
    const float *__restrict__ mean, const float *__restrict__ log_scale,
    const float4 *__restrict__ quat, const float *__restrict__ ologit, int N,
    const sg_view *__restrict__ views, int n_views, ProjConsts pc, float4 *__restrict__ geo,
    uint2 *__restrict__ rect, float2 *__restrict__ ext, const float *__restrict__ rgb,
    const float *__restrict__ sh, float *__restrict__ rec_rgb, int C, const float *__restrict__ sem,
    const float *__restrict__ sem_sh, float *__restrict__ rec_sem) {
    constexpr int K = (D + 1) * (D + 1) - 1;
    pdl_begin();
    __shared__ sg_view s_views[SG_MAX_VIEWS];
    __shared__ float3 s_centre[SG_MAX_VIEWS];
    __shared__ float2 s_lim[SG_MAX_VIEWS];
    __shared__ bool s_same[SG_MAX_VIEWS];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < n_views; i += nthr) s_views[i] = views[i];
    __syncthreads();
    view_limits(s_views, n_views, pc.fov_clamp, s_lim, tid, nthr);
    view_same_pose(s_views, n_views, s_same, tid, nthr);
    if constexpr (D > 0) view_centres(s_views, n_views, s_centre, tid, nthr);
    __syncthreads();
    // threadIdx.x picks the Gaussian, threadIdx.y a contiguous run of view-levels, so that the
    // levels of one keyframe share the camera-space mean and its double-float ratios
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const float mu[3] = {mean[3 * g], mean[3 * g + 1], mean[3 * g + 2]};
    GaussianFrame f;
    gaussian_frame(log_scale, quat[g], g, f);
    const float o = 1.f / (1.f + expf(-ologit[g]));
    // alpha >= alpha_min needs sigma <= ln(o / alpha_min) (+ 1e-3 margin, see below)
    const float thr = logf(o / pc.alpha_min) + 1e-3f;
    float shv[3 * K + 1], c0[3];
    if (D > 0 && sh) {
        for (int i = 0; i < 3 * K; ++i) shv[i] = sh[(size_t)3 * K * g + i];
        for (int c = 0; c < 3; ++c) c0[c] = rgb[3 * g + c];
    }
    if (pc.status && threadIdx.y == 0) {
        // every parameter of the Gaussian the path reads
        const float4 q = quat[g];
        bool bad = !isfinite(q.x) || !isfinite(q.y) || !isfinite(q.z) || !isfinite(q.w) || !isfinite(ologit[g]);
        for (int i = 0; i < 3; ++i)
            bad |= !isfinite(mu[i]) || !isfinite(log_scale[3 * g + i]) || !isfinite(rgb[3 * g + i]);
        for (int c = 0; c < C; ++c) bad |= !isfinite(sem[(size_t)C * g + c]);
        if (D > 0 && sh)
            for (int i = 0; i < 3 * K; ++i) bad |= !isfinite(shv[i]);
        if (D > 0 && sem_sh)
            for (int i = 0; i < K * C; ++i) bad |= !isfinite(sem_sh[(size_t)K * C * g + i]);
        flag_status(bad, pc.status, SG_STATUS_NUMERIC);
    }
    const int per = (n_views + (int)blockDim.y - 1) / (int)blockDim.y;
    const int v_begin = (int)threadIdx.y * per, v_end = min(n_views, v_begin + per);
    PoseGeom pose;
    DF xz, yz;              // t_x / t_z and t_y / t_z of the pose, in double-float
    bool have_ratios = false;
    for (int v = v_begin; v < v_end; ++v) {
        const sg_view &vw = s_views[v];
        const size_t r = (size_t)v * N + g;
        if (v == v_begin || !s_same[v]) {
            pose_geom(vw, mu, pose);
            have_ratios = false;
        }
        ViewGeom q;
        level_geom(vw, pose, s_lim[v], q);
        float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
        uint2 rc = make_uint2(0u, 0u);
        float2 e2 = make_float2(0.f, 0.f);
        const float tz = q.t[2];
        if (tz > pc.z_near && o >= pc.alpha_min) {
            // the 2D mean in double-float: t = R mu + t_cw and (fx t_x / t_z + cx, ...)
            // carry ~1e-4 px of float32 error at 1200 px otherwise
            if (!have_ratios) {
                DF tdf[2];
                for (int i = 0; i < 2; ++i) {
                    DF acc = two_prod(vw.R[3 * i], mu[0]);
                    acc = df_add(acc, two_prod(vw.R[3 * i + 1], mu[1]));
                    acc = df_add(acc, two_prod(vw.R[3 * i + 2], mu[2]));
                    tdf[i] = df_add_f(acc, vw.t[i]);
                }
                xz = df_div(tdf[0], q.tz);
                yz = df_div(tdf[1], q.tz);
                have_ratios = true;
            }
            const DF udf = df_add_f(df_mul_f(xz, vw.fx), vw.cx);
            const DF vdf = df_add_f(df_mul_f(yz, vw.fy), vw.cy);
            const float u = udf.hi, vv = vdf.hi;
            float s00, s01, s11, det;
            if (pc.isotropic)
                cov2d_eq2(vw, tz, f, pc.dilation, s00, s01, s11, det);
            else
                cov2d(q, f, pc.dilation, s00, s01, s11, det);
            if (det > 0.f && s00 > 0.f) {
                // alpha >= alpha_min needs sigma <= ln(o/alpha_min); the smallest sigma at a
                // horizontal offset dx is dx^2/(2 s00): half extents (with float32 slack)
                // (thr + 1e-3: at the boundary alpha is at least 0.1% below alpha_min, far
                // beyond float32 rounding, so no pixel outside can pass the alpha test)
                const float ex = sqrtf(2.f * thr * s00) * 1.002f + 0.01f;
                const float ey = sqrtf(2.f * thr * s11) * 1.002f + 0.01f;
                const float xmin = fmaxf(ceilf(u - ex), 0.f);
                const float xmax = fminf(floorf(u + ex), (float)(vw.W - 1));
                const float ymin = fmaxf(ceilf(vv - ey), 0.f);
                const float ymax = fminf(floorf(vv + ey), (float)(vw.H - 1));
                if (xmin <= xmax && ymin <= ymax && fabsf(u) < 32000.f && fabsf(vv) < 32000.f) {
                    const int tx0 = (int)xmin / pc.tile_w, tx1 = (int)xmax / pc.tile_w + 1;
                    const int ty0 = (int)ymin / pc.tile_h, ty1 = (int)ymax / pc.tile_h + 1;
                    rc = make_uint2(pack16(tx0, ty0), pack16(tx1, ty1));
                    // 2D mean = integer part + float fraction, so that the compositing kernels
                    // can form tile-relative offsets without losing bits
                    const float ui = rintf(u), vi = rintf(vv);
                    const float uf = __fadd_rn(__fsub_rn(udf.hi, ui), udf.lo);
                    const float vf = __fadd_rn(__fsub_rn(vdf.hi, vi), vdf.lo);
                    g0 = make_float4(uf, vf, tz, o);
                    // conditional form of 1/2 d^T Sigma2D^{-1} d (see eval_alpha)
                    const float m00 = rsqrtf(2.f * s00);
                    const float m11 = sqrtf(s00 / (2.f * det));
                    const float m10 = -s01 / sqrtf(2.f * s00 * det);
                    const uint32_t packed = ((uint32_t)(int)ui & 0xffffu) | (((uint32_t)(int)vi & 0xffffu) << 16);
                    g1 = make_float4(m00, m10, m11, __uint_as_float(packed));
                    e2 = make_float2(ex, ey);
                    if constexpr (D > 0) {
                        // colour = rgb + sum_k sh_k Y_k(d), d = (mu - c) / |mu - c|; the same
                        // for the semantic feature with sem_sh
                        const float3 cc = s_centre[v];
                        const float dx = mu[0] - cc.x, dy = mu[1] - cc.y, dz = mu[2] - cc.z;
                        const float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
                        float Y[K];
                        sh_eval<D>(dx * rn, dy * rn, dz * rn, Y);
                        if (sh) {
                            for (int c = 0; c < 3; ++c) {
                                float col = c0[c];
#pragma unroll
                                for (int k = 0; k < K; ++k) col = fmaf(Y[k], shv[3 * k + c], col);
                                rec_rgb[3 * r + c] = col;
                            }
                        }
                        if (sem_sh) {
                            const int C4 = C / 4;
                            const float4 *s0 = reinterpret_cast<const float4 *>(sem + (size_t)C * g);
                            const float4 *ss = reinterpret_cast<const float4 *>(sem_sh + (size_t)K * C * g);
                            float4 *so = reinterpret_cast<float4 *>(rec_sem + (size_t)C * r);
                            for (int c4 = 0; c4 < C4; ++c4) {
                                float4 acc = s0[c4];
#pragma unroll
                                for (int k = 0; k < K; ++k) {
                                    const float4 t = ss[k * C4 + c4];
                                    acc.x = fmaf(Y[k], t.x, acc.x);
                                    acc.y = fmaf(Y[k], t.y, acc.y);
                                    acc.z = fmaf(Y[k], t.z, acc.z);
                                    acc.w = fmaf(Y[k], t.w, acc.w);
                                }
                                so[c4] = acc;
                            }
                        }
                    }
                }
            }
        }
        geo[2 * r] = g0;
        geo[2 * r + 1] = g1;
        rect[r] = rc;
        ext[r] = e2;
    }
}

// Adjoint.  g2d: per record (u, v, conic a, conic b, conic c, opacity, depth, 0); with SH,
// gcol: per record dL/d(colour) (r, g, b, 0) and gsem_rec: per record dL/d(semantic feature).
template <int D>
__global__ void __launch_bounds__(256) project_bwd_kernel(
    const float *__restrict__ mean, const float *__restrict__ log_scale,
    const float4 *__restrict__ quat, const float *__restrict__ ologit, int N,
    const sg_view *__restrict__ views, int n_views, ProjConsts pc,
    const uint2 *__restrict__ rect, float4 *__restrict__ g2d, float *__restrict__ g_mean, float *__restrict__ g_ls,
    float *__restrict__ g_quat, float *__restrict__ g_ologit, const float *__restrict__ sh,
    float4 *__restrict__ gcol, float *__restrict__ g_rgb, float *__restrict__ g_sh, int C,
    const float *__restrict__ sem_sh, float4 *__restrict__ gsem_rec, float *__restrict__ g_sem,
    float *__restrict__ g_sem_sh) {
    constexpr int K = (D + 1) * (D + 1) - 1;
    pdl_begin();
    __shared__ sg_view s_views[SG_MAX_VIEWS];
    __shared__ float3 s_centre[SG_MAX_VIEWS];
    __shared__ float2 s_lim[SG_MAX_VIEWS];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    for (int i = tid; i < n_views; i += nthr) s_views[i] = views[i];
    __syncthreads();
    view_limits(s_views, n_views, pc.fov_clamp, s_lim, tid, nthr);
    if constexpr (D > 0) view_centres(s_views, n_views, s_centre, tid, nthr);
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const float mu[3] = {mean[3 * g], mean[3 * g + 1], mean[3 * g + 2]};
    GaussianFrame f;
    gaussian_frame(log_scale, quat[g], g, f);
    const float o = 1.f / (1.f + expf(-ologit[g]));
    float gmu[3] = {0.f, 0.f, 0.f};
    float gSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // full-entry gradient, symmetric
    float go_total = 0.f;
    float gls0 = 0.f;  // Eq. 2 mode: dL/dlog_scale[0]
    float shv[3 * K + 1], gsh[3 * K + 1], grgb[3] = {0.f, 0.f, 0.f};
    if (D > 0 && sh) {
        for (int i = 0; i < 3 * K; ++i) {
            shv[i] = sh[(size_t)3 * K * g + i];
            gsh[i] = 0.f;
        }
    }
    // Visible view-levels first, 32 at a time, with all tile-rectangle loads in flight
    // together; then the visible ones, each one's 2D gradients loaded one view ahead.
    for (int v0 = 0; v0 < n_views; v0 += 32) {
    uint32_t vis = 0;
    const int nv = min(32, n_views - v0);
#pragma unroll 8
    for (int i = 0; i < nv; ++i) {
        const uint2 rc = rect[(size_t)(v0 + i) * N + g];
        vis |= (rc.x != rc.y ? 1u : 0u) << i;  // an empty rectangle means culled
    }
    float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na, nc = na;
    if (vis) {
        const size_t r = (size_t)(v0 + __ffs(vis) - 1) * N + g;
        na = g2d[2 * r];
        nb = g2d[2 * r + 1];
        if (D > 0 && sh) nc = gcol[r];
    }
    while (vis) {
        const int v = v0 + __ffs(vis) - 1;
        vis &= vis - 1;
        const float4 a = na, b = nb, cg = nc;
        {
            // consumed: zero the record's slots, so the workspace is all zero for the next
            // compositing adjoint (only visible records are ever written)
            const size_t r = (size_t)v * N + g;
            g2d[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
            g2d[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (D > 0 && sh) gcol[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (vis) {
            const size_t rn = (size_t)(v0 + __ffs(vis) - 1) * N + g;
            na = g2d[2 * rn];
            nb = g2d[2 * rn + 1];
            if (D > 0 && sh) nc = gcol[rn];
        }
        const float gu = a.x, gv = a.y, ga = a.z, gb = a.w, gc = b.x, go = b.y, gd = b.z;
        const sg_view &vw = s_views[v];
        if constexpr (D > 0) {
            // feature f = f0 + sum_k coef_k Y_k(d) (colour: rgb, sh; semantic: sem, sem_sh):
            // dL/dcoef_k += Y_k dL/df, dL/df0 += dL/df,
            // dL/dmu += (I - d d^T) / |mu - c| sum_k (coef_k . dL/df) grad Y_k(d)
            const float gcv[3] = {cg.x, cg.y, cg.z};
            const float3 cc = s_centre[v];
            const float dx = mu[0] - cc.x, dy = mu[1] - cc.y, dz = mu[2] - cc.z;
            const float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
            const float x = dx * rn, y = dy * rn, z = dz * rn;
            float Y[K], w[K];
            sh_eval<D>(x, y, z, Y);
#pragma unroll
            for (int k = 0; k < K; ++k) w[k] = 0.f;
            if (sh) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        gsh[3 * k + c] = fmaf(Y[k], gcv[c], gsh[3 * k + c]);
                        w[k] = fmaf(shv[3 * k + c], gcv[c], w[k]);
                    }
                }
                for (int c = 0; c < 3; ++c) grgb[c] += gcv[c];
            }
            if (sem_sh) {
                // this thread owns Gaussian g's rows of g_sem and g_sem_sh: plain read-modify-
                // write per view; the record's semantic slots are zeroed once read
                const int C4 = C / 4;
                const size_t r = (size_t)v * N + g;
                float4 *gs = reinterpret_cast<float4 *>(g_sem + (size_t)C * g);
                float4 *gss = reinterpret_cast<float4 *>(g_sem_sh + (size_t)K * C * g);
                const float4 *ss = reinterpret_cast<const float4 *>(sem_sh + (size_t)K * C * g);
                for (int c4 = 0; c4 < C4; ++c4) {
                    const float4 t = gsem_rec[r * C4 + c4];
                    gsem_rec[r * C4 + c4] = make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 a0 = gs[c4];
                    a0.x += t.x; a0.y += t.y; a0.z += t.z; a0.w += t.w;
                    gs[c4] = a0;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float4 u = gss[k * C4 + c4];
                        u.x = fmaf(Y[k], t.x, u.x);
                        u.y = fmaf(Y[k], t.y, u.y);
                        u.z = fmaf(Y[k], t.z, u.z);
                        u.w = fmaf(Y[k], t.w, u.w);
                        gss[k * C4 + c4] = u;
                        const float4 sv = ss[k * C4 + c4];
                        w[k] += sv.x * t.x + sv.y * t.y + sv.z * t.z + sv.w * t.w;
                    }
                }
            }
            float gdir[3];
            sh_grad<D>(x, y, z, w, gdir);
            const float radial = gdir[0] * x + gdir[1] * y + gdir[2] * z;
            gmu[0] += (gdir[0] - radial * x) * rn;
            gmu[1] += (gdir[1] - radial * y) * rn;
            gmu[2] += (gdir[2] - radial * z) * rn;
        }
        PoseGeom pose;
        pose_geom(vw, mu, pose);
        ViewGeom q;
        level_geom(vw, pose, s_lim[v], q);
        // conic = Sigma2D^{-1} of this view-level, recomputed in float32
        float ca, cb, cc;
        {
            float s00, s01, s11, det;
            if (pc.isotropic)
                cov2d_eq2(vw, q.t[2], f, pc.dilation, s00, s01, s11, det);
            else
                cov2d(q, f, pc.dilation, s00, s01, s11, det);
            const float id = 1.f / det;
            ca = s11 * id;
            cb = -s01 * id;
            cc = s00 * id;
        }
        const float tz = q.t[2], tz2 = tz * tz;
        // conic = Sigma2D^{-1}: dQ = -Q dS Q
        const float gS00 = -(ca * ca * ga + ca * cb * gb + cb * cb * gc);
        const float gS01 = -(2.f * ca * cb * ga + (ca * cc + cb * cb) * gb + 2.f * cb * cc * gc);
        const float gS11 = -(cb * cb * ga + cb * cc * gb + cc * cc * gc);
        if (pc.isotropic) {
            // Eq. 2: S00 = (fx r/tz)^2 + b, S11 = (fy r/tz)^2 + b with r = e^{s0}; S01 = 0
            const float r = f.S[0];
            const float q2 = (gS00 * vw.fx * vw.fx + gS11 * vw.fy * vw.fy) * 2.f * r * r / tz2;
            gls0 += q2;  // dL/ds0 = dL/dr * r
            const float gt0 = gu * vw.fx / tz, gt1 = gv * vw.fy / tz;
            const float gt2 = -gu * vw.fx * q.t[0] / tz2 - gv * vw.fy * q.t[1] / tz2 + gd - q2 / tz;
            const float *W = vw.R;
            for (int j = 0; j < 3; ++j) gmu[j] += W[j] * gt0 + W[3 + j] * gt1 + W[6 + j] * gt2;
            go_total += go;
            continue;
        }
        const float G00 = gS00, G01 = 0.5f * gS01, G11 = gS11;
        // Sigma2D = T Sig T^T: dSig += T^T G T; dT = 2 G T Sig
        const float *T0 = q.T0, *T1 = q.T1;
        {
            int k = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = i; j < 3; ++j, ++k)
                    gSig[k] += T0[i] * G00 * T0[j] + T0[i] * G01 * T1[j] + T1[i] * G01 * T0[j] +
                               T1[i] * G11 * T1[j];
        }
        float TS0[3], TS1[3];  // T Sig
        for (int j = 0; j < 3; ++j) {
            TS0[j] = T0[0] * sym3(f.Sig, 0, j) + T0[1] * sym3(f.Sig, 1, j) + T0[2] * sym3(f.Sig, 2, j);
            TS1[j] = T1[0] * sym3(f.Sig, 0, j) + T1[1] * sym3(f.Sig, 1, j) + T1[2] * sym3(f.Sig, 2, j);
        }
        float gT0[3], gT1[3];
        for (int j = 0; j < 3; ++j) {
            gT0[j] = 2.f * (G00 * TS0[j] + G01 * TS1[j]);
            gT1[j] = 2.f * (G01 * TS0[j] + G11 * TS1[j]);
        }
        // T0 = J00 W0 + J02 W2, T1 = J11 W1 + J12 W2 (W rows)
        const float *W = vw.R;
        const float gJ00 = gT0[0] * W[0] + gT0[1] * W[1] + gT0[2] * W[2];
        const float gJ02 = gT0[0] * W[6] + gT0[1] * W[7] + gT0[2] * W[8];
        const float gJ11 = gT1[0] * W[3] + gT1[1] * W[4] + gT1[2] * W[5];
        const float gJ12 = gT1[0] * W[6] + gT1[1] * W[7] + gT1[2] * W[8];
        // (J00 = fx / tz, J11 = fy / tz: the divisions by tz are products with them)
        const float itz = 1.f / tz;
        float gt0 = 0.f, gt1 = 0.f, gt2 = 0.f;
        gt2 += -(gJ00 * q.J00 + gJ11 * q.J11) * itz;
        if (!q.clx) {
            gt0 += gJ02 * (-q.J00 * itz);
            gt2 += gJ02 * (2.f * q.J00 * q.t[0] * itz * itz);
        } else {
            gt2 += gJ02 * (-q.J02 * itz);
        }
        if (!q.cly) {
            gt1 += gJ12 * (-q.J11 * itz);
            gt2 += gJ12 * (2.f * q.J11 * q.t[1] * itz * itz);
        } else {
            gt2 += gJ12 * (-q.J12 * itz);
        }
        gt0 += gu * q.J00;
        gt1 += gv * q.J11;
        gt2 += -(gu * q.J00 * q.t[0] + gv * q.J11 * q.t[1]) * itz + gd;
        for (int j = 0; j < 3; ++j) gmu[j] += W[j] * gt0 + W[3 + j] * gt1 + W[6 + j] * gt2;
        go_total += go;
    }
    }
    // Sig = M M^T with M = R diag(S): dM = 2 gSig M
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = f.R[3 * i + j] * f.S[j];
    float gR[9], gls[3] = {0.f, 0.f, 0.f};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const float gM = 2.f * (sym3(gSig, i, 0) * M[j] + sym3(gSig, i, 1) * M[3 + j] +
                                    sym3(gSig, i, 2) * M[6 + j]);
            gR[3 * i + j] = gM * f.S[j];
            gls[j] += gM * f.R[3 * i + j] * f.S[j];
        }
    const float w = f.q[0], x = f.q[1], y = f.q[2], z = f.q[3];
    float gq[4];
    gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] +
                   w * gR[7] - 2.f * x * gR[8]);
    gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] +
                   z * gR[7] - 2.f * y * gR[8]);
    gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] +
                   y * gR[5] + x * gR[6] + y * gR[7]);
    const float dot = f.q[0] * gq[0] + f.q[1] * gq[1] + f.q[2] * gq[2] + f.q[3] * gq[3];
    const float rq = 1.f / f.qn;
    for (int i = 0; i < 4; ++i) g_quat[4 * g + i] += (gq[i] - f.q[i] * dot) * rq;
    gls[0] += gls0;
    for (int j = 0; j < 3; ++j) {
        g_mean[3 * g + j] += gmu[j];
        g_ls[3 * g + j] += gls[j];
    }
    g_ologit[g] += go_total * o * (1.f - o);
    if (D > 0 && sh) {
        for (int c = 0; c < 3; ++c) g_rgb[3 * g + c] += grgb[c];
        for (int i = 0; i < 3 * K; ++i) g_sh[(size_t)3 * K * g + i] += gsh[i];
    }
}

sg_status launch_project_fwd(const sg_gaussians *g, const sg_view *views, int n_views,
                             const sg_config *cfg, sg_projected *out, uint32_t *status, cudaStream_t st) {
    ProjConsts pc{cfg->z_near, cfg->dilation, cfg->fov_clamp, cfg->alpha_min, cfg->tile_w,
                  cfg->tile_h, cfg->isotropic, status};
    // a block of bx Gaussians x vy view-levels (each thread loops over every vy-th view-level):
    // with many view-levels, eight short threads per Gaussian instead of one long loop (the
    // Gaussian's frame is then formed eight times); with few, one thread per Gaussian
    const int vy = n_views >= 8 ? 8 : 1;
    const int bx = 256 / vy;
    const int blocks = (g->N + bx - 1) / bx;
    if (blocks > 0) {
        auto kern = g->sh_degree == 3 ? project_fwd_kernel<3>
                  : g->sh_degree == 2 ? project_fwd_kernel<2>
                  : g->sh_degree == 1 ? project_fwd_kernel<1> : project_fwd_kernel<0>;
        launch_pdl(kern, blocks, dim3(bx, vy), 0, st,
            g->mean, g->log_scale, reinterpret_cast<const float4 *>(g->quat), g->opacity_logit,
            g->N, views, n_views, pc, reinterpret_cast<float4 *>(out->geo),
            reinterpret_cast<uint2 *>(out->rect), reinterpret_cast<float2 *>(out->ext), g->rgb,
            g->sh_degree > 0 ? g->sh : nullptr, out->rgb, g->C, g->sem,
            g->sh_degree > 0 ? g->sem_sh : nullptr, out->sem);
        count_launches(1);
    }
    return check_launch("project_fwd");
}

sg_status launch_project_bwd(const sg_gaussians *g, const sg_view *views, int n_views,
                             const sg_config *cfg, const sg_projected *proj, float *g2d,
                             sg_gaussian_grads *gr, cudaStream_t st) {
    ProjConsts pc{cfg->z_near, cfg->dilation, cfg->fov_clamp, cfg->alpha_min, cfg->tile_w,
                  cfg->tile_h, cfg->isotropic, nullptr};
    const int threads = 256;
    const int blocks = (g->N + threads - 1) / threads;
    if (blocks > 0) {
        auto kern = g->sh_degree == 3 ? project_bwd_kernel<3>
                  : g->sh_degree == 2 ? project_bwd_kernel<2>
                  : g->sh_degree == 1 ? project_bwd_kernel<1> : project_bwd_kernel<0>;
        // workspace blocks: R x 8 2D gradients, R x 4 colour gradients, R x C semantic ones
        const size_t R = (size_t)g->N * n_views;
        float4 *gcol = reinterpret_cast<float4 *>(g2d + 8 * R);
        float4 *gsem = reinterpret_cast<float4 *>(g2d + 12 * R);
        launch_pdl(kern, blocks, threads, 0, st,
            g->mean, g->log_scale, reinterpret_cast<const float4 *>(g->quat), g->opacity_logit,
            g->N, views, n_views, pc, reinterpret_cast<const uint2 *>(proj->rect),
            reinterpret_cast<float4 *>(g2d),
            gr->mean, gr->log_scale, gr->quat, gr->opacity_logit, g->sh_degree > 0 ? g->sh : nullptr, gcol,
            gr->rgb, gr->sh, g->C, g->sh_degree > 0 ? g->sem_sh : nullptr, gsem, gr->sem, gr->sem_sh);
        count_launches(1);
    }
    return check_launch("project_bwd");
}

}  // namespace sg
