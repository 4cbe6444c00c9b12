// init.cu -- insertion of new Gaussians from a keyframe (Sec. III-A: the mapping thread
// converts keyframe data into Gaussian primitives with position, colour, semantics, depth
// and opacity) and the patch features of the learned initializer.
//
// Heuristic initializer, per inserted pixel (x, y) with valid depth D at level 0:
//   mean = back-projection of (x, y, D); rgb = pixel colour; log-scale = ln(D / fx) on all
//   three axes (a one-pixel footprint, Eq. 2's r2D = f r / d = 1); quaternion = identity;
//   opacity logit = 0 (opacity 0.5); semantic feature = kappa * code[label] (or 0).
// Patch features, per inserted pixel: the 7x7 neighbourhood, 41 channels per pixel:
//   rgb (3), depth in metres (1), one-hot label (32), unit ray direction in the camera frame
//   (3), depth-valid flag (1), 1/fx (1) -- 49 * 41 = 2009 features, zero-padded to 2048.
//   Pixels outside the image contribute zeros.
#include <cuda_bf16.h>

#include "sg_common.cuh"

namespace sg {

constexpr int kPatch = 7, kPatchCh = 41, kPatchFeat = kPatch * kPatch * kPatchCh;  // 2009
static_assert(kPatchFeat <= SG_MLP_IN, "patch features exceed the MLP input");

struct Frame {
    const float *rgb, *depth;
    const int *label;
    int W, H;
    float fx, fy, cx, cy;
};

__device__ __forceinline__ float patch_feature(const Frame &fr, int x0, int y0, int f) {
    if (f >= kPatchFeat) return 0.f;
    const int pix = f / kPatchCh, ch = f % kPatchCh;
    const int x = x0 + pix % kPatch - kPatch / 2, y = y0 + pix / kPatch - kPatch / 2;
    if (x < 0 || y < 0 || x >= fr.W || y >= fr.H) return 0.f;
    const size_t p = (size_t)y * fr.W + x, HW = (size_t)fr.W * fr.H;
    if (ch < 3) return fr.rgb[ch * HW + p];
    const float d = fr.depth[p];
    if (ch == 3) return d > 0.f ? d : 0.f;
    if (ch < 36) return fr.label && fr.label[p] == ch - 4 ? 1.f : 0.f;
    if (ch < 39) {
        const float rx = (x - fr.cx) / fr.fx, ry = (y - fr.cy) / fr.fy;
        const float inv = rsqrtf(rx * rx + ry * ry + 1.f);
        return ch == 36 ? rx * inv : (ch == 37 ? ry * inv : inv);
    }
    if (ch == 39) return d > 0.f ? 1.f : 0.f;
    return 1.f / fr.fx;
}

// X [B_pad][2048] row-major (coalesced over features)
__global__ void patch_rows_kernel(Frame fr, const int2 *__restrict__ pix, int B, int B_pad,
                                  __nv_bfloat16 *__restrict__ X) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B_pad * SG_MLP_IN) return;
    const int b = (int)(i / SG_MLP_IN), f = (int)(i % SG_MLP_IN);
    float v = 0.f;
    if (b < B) {
        const int2 q = pix[b];
        v = patch_feature(fr, q.x, q.y, f);
    }
    X[i] = __float2bfloat16_rn(v);
}

// Xt [2048][B_pad] (coalesced over rows of the batch)
__global__ void patch_cols_kernel(Frame fr, const int2 *__restrict__ pix, int B, int B_pad,
                                  __nv_bfloat16 *__restrict__ Xt) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B_pad * SG_MLP_IN) return;
    const int f = (int)(i / B_pad), b = (int)(i % B_pad);
    float v = 0.f;
    if (b < B) {
        const int2 q = pix[b];
        v = patch_feature(fr, q.x, q.y, f);
    }
    Xt[i] = __float2bfloat16_rn(v);
}

struct InitOut {
    float *mean, *log_scale, *quat, *opacity_logit, *rgb, *sem;
};

__global__ void heuristic_init_kernel(Frame fr, sg_camera cam, const int2 *__restrict__ pix, int B, int C,
                                      const float *__restrict__ code, int n_classes, float kappa, InitOut o) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int2 q = pix[b];
    const size_t p = (size_t)q.y * fr.W + q.x, HW = (size_t)fr.W * fr.H;
    float D = fr.depth[p];
    if (!(D > 0.f)) D = 1.f;  // callers insert valid-depth pixels; keep the state finite
    // camera-frame point, then world = R_cw^T (t - t_cw)
    const float xc = (q.x - cam.cx) / cam.fx * D, yc = (q.y - cam.cy) / cam.fy * D, zc = D;
    const float dx = xc - cam.t_cw[0], dy = yc - cam.t_cw[1], dz = zc - cam.t_cw[2];
    const float *R = cam.R_cw;
    o.mean[3 * b + 0] = R[0] * dx + R[3] * dy + R[6] * dz;
    o.mean[3 * b + 1] = R[1] * dx + R[4] * dy + R[7] * dz;
    o.mean[3 * b + 2] = R[2] * dx + R[5] * dy + R[8] * dz;
    const float ls = logf(D / cam.fx);
    o.log_scale[3 * b + 0] = ls;
    o.log_scale[3 * b + 1] = ls;
    o.log_scale[3 * b + 2] = ls;
    o.quat[4 * b + 0] = 1.f;
    o.quat[4 * b + 1] = 0.f;
    o.quat[4 * b + 2] = 0.f;
    o.quat[4 * b + 3] = 0.f;
    o.opacity_logit[b] = 0.f;
    for (int c = 0; c < 3; ++c) o.rgb[3 * b + c] = fr.rgb[c * HW + p];
    const int lab = fr.label ? fr.label[p] : -1;
    for (int c = 0; c < C; ++c)
        o.sem[(size_t)C * b + c] = (code && lab >= 0 && lab < n_classes) ? kappa * code[(size_t)lab * C + c] : 0.f;
}

// MLP output (standardised) -> log-scale (3), opacity logit (1), semantic feature (C)
__global__ void apply_mlp_kernel(const float *__restrict__ Y, int B, int C, const float *__restrict__ mu,
                                 const float *__restrict__ sd, float *__restrict__ log_scale,
                                 float *__restrict__ opacity_logit, float *__restrict__ sem) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *y = Y + (size_t)b * SG_MLP_OUT;
    for (int k = 0; k < 3; ++k) log_scale[3 * b + k] = y[k] * sd[k] + mu[k];
    opacity_logit[b] = y[3] * sd[3] + mu[3];
    for (int c = 0; c < C && 4 + c < SG_MLP_OUT; ++c) sem[(size_t)C * b + c] = y[4 + c] * sd[4 + c] + mu[4 + c];
}

}  // namespace sg

using namespace sg;

extern "C" {

sg_status sg_extract_patches(const float *rgb, const float *depth, const int32_t *label, const sg_camera *cam,
                             const int32_t *pixels, int32_t B, int32_t B_pad, uint16_t *X, uint16_t *Xt,
                             sg_stream_t stream) {
    if (!rgb || !depth || !cam || !pixels || (!X && !Xt) || B < 0 || B_pad < B || B_pad % 128 != 0) {
        set_error("extract_patches: bad argument (B=%d, B_pad=%d must be a multiple of 128 >= B)", B, B_pad);
        return SG_ERR_INVALID_ARG;
    }
    Frame fr{rgb, depth, label, cam->W, cam->H, cam->fx, cam->fy, cam->cx, cam->cy};
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)B_pad * SG_MLP_IN;
    const int blocks = (int)((n + 255) / 256);
    if (blocks > 0) {
        if (X) {
            patch_rows_kernel<<<blocks, 256, 0, st>>>(fr, (const int2 *)pixels, B, B_pad, (__nv_bfloat16 *)X);
            count_launches(1);
        }
        if (Xt) {
            patch_cols_kernel<<<blocks, 256, 0, st>>>(fr, (const int2 *)pixels, B, B_pad, (__nv_bfloat16 *)Xt);
            count_launches(1);
        }
    }
    return check_launch("extract_patches");
}

sg_status sg_init_gaussians(const float *rgb, const float *depth, const int32_t *label, const sg_camera *cam,
                            const int32_t *pixels, int32_t B, const float *sem_code, int32_t n_classes,
                            float kappa, sg_gaussian_grads *out, sg_stream_t stream) {
    if (!rgb || !depth || !cam || !pixels || !out || B < 0 || !out->mean || !out->log_scale || !out->quat ||
        !out->opacity_logit || !out->rgb || !out->sem) {
        set_error("init_gaussians: NULL argument");
        return SG_ERR_INVALID_ARG;
    }
    if (B == 0) return SG_OK;
    Frame fr{rgb, depth, label, cam->W, cam->H, cam->fx, cam->fy, cam->cx, cam->cy};
    InitOut o{out->mean, out->log_scale, out->quat, out->opacity_logit, out->rgb, out->sem};
    heuristic_init_kernel<<<(B + 127) / 128, 128, 0, (cudaStream_t)stream>>>(fr, *cam, (const int2 *)pixels, B,
                                                                             out->C, sem_code, n_classes, kappa, o);
    count_launches(1);
    return check_launch("init_gaussians");
}

sg_status sg_apply_mlp_init(const float *Y, int32_t B, const float *y_mean, const float *y_std,
                            sg_gaussian_grads *out, sg_stream_t stream) {
    if (!Y || !y_mean || !y_std || !out || !out->log_scale || !out->opacity_logit || !out->sem || B < 0) {
        set_error("apply_mlp_init: NULL argument");
        return SG_ERR_INVALID_ARG;
    }
    if (B == 0) return SG_OK;
    apply_mlp_kernel<<<(B + 127) / 128, 128, 0, (cudaStream_t)stream>>>(Y, B, out->C, y_mean, y_std, out->log_scale,
                                                                        out->opacity_logit, out->sem);
    count_launches(1);
    return check_launch("apply_mlp_init");
}

}  // extern "C"
