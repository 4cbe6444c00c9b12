// loss.cu -- Eq. 10-13 per pyramid level, the Eq. 4-6 image pyramid, and Adam.
//
// RGB term (Eq. 10) and, in semantic-colour mode, the semantic term (Eq. 12):
//   (1 - lambda) mean|I - I_gt| + lambda (1 - SSIM(I, I_gt)),
// SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero padding.
// One CTA owns a 32x32 output tile of one view-level and one group of planes.  It stages
// the planes with a 10-pixel halo, forms the five window moments (separable, horizontal
// then vertical) on the tile plus a 5-pixel halo, turns them into the three per-pixel
// partials of SSIM (w.r.t. the window mean, E[x^2] and E[xy]), and convolves those once
// more to get dL/dI for the tile -- one read of I and I_gt and one write of dL/dI per
// pixel, no intermediate maps in HBM.
// Depth term (Eq. 11): mean |D - D_gt| over pixels with D_gt > 0.
// Semantic term, cross-entropy mode: mean CE(softmax(decoder * S), label) over label >= 0.
// Sums are per-CTA partials reduced in a fixed order (deterministic).
#include <cstdio>

#include "sg_common.cuh"

namespace sg {

constexpr int kLTW = 32, kLTH = 32;           // loss tile (outputs)
constexpr int kXW = kLTW + 20, kXH = kLTH + 20;  // staged planes (10-px halo)
constexpr int kMW = kLTW + 10, kMH = kLTH + 10;  // moment / partial maps (5-px halo)
constexpr int kXP = kXW + 1, kMP = kMW + 1;      // padded row pitches (odd: no bank conflicts)
constexpr int kLossThreads = 256;

struct LossViews {
    int n;
    int tile_off[SG_MAX_VIEWS + 1];  // loss tiles (32x32) per view, prefix
    int pix_blk_off[SG_MAX_VIEWS + 1];  // 256-pixel blocks per view, prefix
};

__device__ __forceinline__ void gauss_window(float *w) {
    float s = 0.f;
    for (int i = 0; i < 11; ++i) {
        w[i] = expf(-(float)((i - 5) * (i - 5)) / (2.f * 1.5f * 1.5f));
        s += w[i];
    }
    for (int i = 0; i < 11; ++i) w[i] /= s;
}

__device__ __forceinline__ int find_prefix(const int *off, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float block_sum(float v, float *s_red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SG_FULL_MASK, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLossThreads / 32; ++w) t += s_red[w];
    return t;  // valid in thread 0
}

struct SsimArgs {
    const float *x, *y;  // planar images (rendered, target), nch planes per view
    float *grad;         // dL/dx
    int nch;
    float l1_coef_num;   // (1 - lambda) * weight  (divided by n = nch*W*H per view)
    float ssim_coef_num; // lambda * weight
    const sg_view *views;
    LossViews lv;
    float *partials;     // per CTA: (sum |x - y|, sum ssim)
    // valid-pixel counts (counts[2v]: target depth > 0, counts[2v+1]: label >= 0) gathered
    // on the side, or null
    const float *gt_depth;
    const int *label;
    int *counts;
};

// Sliding-window separable passes: each thread produces a run of consecutive outputs of one
// row (horizontal) or column (vertical) from a register window of input values.
__global__ void __launch_bounds__(kLossThreads, 3) ssim_l1_kernel(SsimArgs a) {
    pdl_begin();
    extern __shared__ __align__(16) float sm[];
    float *X = sm;                   // kXH x kXP
    float *Y = X + kXH * kXP;        // kXH x kXP
    float *Hm = Y + kXH * kXP;       // 5 x kXH x kMP (later: 3 x kMH x kMP)
    float *Mp = X;                   // 3 x kMH x kMP: reuses the staged planes once the
                                     // horizontal pass has consumed them
    static_assert(3 * kMH * kMP <= 2 * kXH * kXP, "partials must fit the staged planes");
    __shared__ int s_cnt[2];
    __shared__ float w[11];
    __shared__ float s_red[kLossThreads / 32];
    if (threadIdx.x == 0) gauss_window(w);
    const int item = blockIdx.x;
    const int v = find_prefix(a.lv.tile_off, a.lv.n, item);
    const sg_view &vw = a.views[v];
    const int W = vw.W, H = vw.H;
    const int tiles_x = (W + kLTW - 1) / kLTW;
    const int local = item - a.lv.tile_off[v];
    const int bx = local % tiles_x, by = local / tiles_x;
    const int ox = bx * kLTW - 10, oy = by * kLTH - 10;
    const size_t HW = (size_t)W * H;
    const float n = (float)a.nch * (float)HW;
    const float l1c = a.l1_coef_num / n, sc = -a.ssim_coef_num / n;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float l1_sum = 0.f, ssim_sum = 0.f;
    int n_depth = 0, n_label = 0;
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    float wr[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) wr[i] = w[i];
    for (int ch = 0; ch < a.nch; ++ch) {
        const float *xs = a.x + (size_t)a.nch * vw.pixel_offset + ch * HW;
        const float *ys = a.y + (size_t)a.nch * vw.pixel_offset + ch * HW;
        // stage x, y with a 10-pixel halo (zero outside the image)
        for (int i = threadIdx.x; i < kXH * kXW; i += kLossThreads) {
            const int r = i / kXW, c = i - r * kXW;
            const int gy = oy + r, gx = ox + c;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            X[r * kXP + c] = in ? xs[(size_t)gy * W + gx] : 0.f;
            Y[r * kXP + c] = in ? ys[(size_t)gy * W + gx] : 0.f;
        }
        __syncthreads();
        // Run lengths are chosen so that every phase's work items fill whole rounds of the
        // block's 256 threads (728, 252, 504 and 256 items).
        // horizontal window sums of x, y, x^2, y^2, xy: rows kXH, outputs kMW in runs of 3
        {
            constexpr int RUN = 3, SEGS = kMW / RUN;  // 42 = 14 * 3
            for (int it = threadIdx.x; it < SEGS * kXH; it += kLossThreads) {
                const int seg = it / kXH, r = it - seg * kXH;
                const int c0 = seg * RUN;
                float xv[RUN + 10], yv[RUN + 10];
#pragma unroll
                for (int i = 0; i < RUN + 10; ++i) {
                    xv[i] = X[r * kXP + c0 + i];
                    yv[i] = Y[r * kXP + c0 + i];
                }
#pragma unroll
                for (int o = 0; o < RUN; ++o) {
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
                    for (int j = 0; j < 11; ++j) {
                        const float x = xv[o + j], y = yv[o + j];
                        s0 = fmaf(wr[j], x, s0);
                        s1 = fmaf(wr[j], y, s1);
                        s2 = fmaf(wr[j], x * x, s2);
                        s3 = fmaf(wr[j], y * y, s3);
                        s4 = fmaf(wr[j], x * y, s4);
                    }
                    const int idx = r * kMP + c0 + o;
                    Hm[0 * kXH * kMP + idx] = s0;
                    Hm[1 * kXH * kMP + idx] = s1;
                    Hm[2 * kXH * kMP + idx] = s2;
                    Hm[3 * kXH * kMP + idx] = s3;
                    Hm[4 * kXH * kMP + idx] = s4;
                }
            }
        }
        __syncthreads();
        // vertical window sums -> SSIM and its partials (zero outside the image): columns
        // kMW, output rows kMH in runs of 7
        {
            constexpr int RUN = 7, SEGS = kMH / RUN;  // 42 = 6 * 7
            for (int it = threadIdx.x; it < SEGS * kMW; it += kLossThreads) {
                const int seg = it / kMW, c = it - seg * kMW;
                const int r0 = seg * RUN;
                float m[5][RUN];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    float col[RUN + 10];
#pragma unroll
                    for (int i = 0; i < RUN + 10; ++i) col[i] = Hm[k * kXH * kMP + (r0 + i) * kMP + c];
#pragma unroll
                    for (int o = 0; o < RUN; ++o) {
                        float acc = 0.f;
#pragma unroll
                        for (int j = 0; j < 11; ++j) acc = fmaf(wr[j], col[o + j], acc);
                        m[k][o] = acc;
                    }
                }
#pragma unroll
                for (int o = 0; o < RUN; ++o) {
                    const int r = r0 + o;
                    const int gy = by * kLTH - 5 + r, gx = bx * kLTW - 5 + c;
                    float P = 0.f, Q = 0.f, R = 0.f;
                    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                        const float mx = m[0][o], my = m[1][o];
                        const float sxx = m[2][o] - mx * mx, syy = m[3][o] - my * my, sxy = m[4][o] - mx * my;
                        const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
                        const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
                        const float inv = 1.f / (B1 * B2);
                        const float s = A1 * A2 * inv;
                        if (r >= 5 && r < kLTH + 5 && c >= 5 && c < kLTW + 5) ssim_sum += s;
                        const float d_mx = 2.f * my * A2 * inv - s * 2.f * mx / B1;
                        const float d_sxx = -s / B2;
                        const float d_sxy = 2.f * A1 * inv;
                        P = sc * (d_mx - 2.f * mx * d_sxx - my * d_sxy);
                        Q = sc * d_sxx;
                        R = sc * d_sxy;
                    }
                    Mp[0 * kMH * kMP + r * kMP + c] = P;
                    Mp[1 * kMH * kMP + r * kMP + c] = Q;
                    Mp[2 * kMH * kMP + r * kMP + c] = R;
                }
            }
        }
        __syncthreads();
        float *Hp = Hm;  // 3 x kMH x kMP, reuses the moment buffer
        // horizontal sums of the partials: (partial, row, run of 8 outputs) per item
        {
            constexpr int RUN = 8, SEGS = kLTW / RUN;
            for (int it = threadIdx.x; it < 3 * SEGS * kMH; it += kLossThreads) {
                const int k = it / (SEGS * kMH), rem = it - k * (SEGS * kMH);
                const int seg = rem / kMH, r = rem - seg * kMH;
                const int c0 = seg * RUN;
                {
                    float row[RUN + 10];
#pragma unroll
                    for (int i = 0; i < RUN + 10; ++i) row[i] = Mp[k * kMH * kMP + r * kMP + c0 + i];
#pragma unroll
                    for (int o = 0; o < RUN; ++o) {
                        float acc = 0.f;
#pragma unroll
                        for (int j = 0; j < 11; ++j) acc = fmaf(wr[j], row[o + j], acc);
                        Hp[k * kMH * kMP + r * kMP + c0 + o] = acc;
                    }
                }
            }
        }
        __syncthreads();
        // vertical sums of the partials -> dL/dx on the tile: columns kLTW, rows in runs of 4
        float *gs = a.grad + (size_t)a.nch * vw.pixel_offset + ch * HW;
        {
            constexpr int RUN = 4, SEGS = kLTH / RUN;
            for (int it = threadIdx.x; it < SEGS * kLTW; it += kLossThreads) {
                const int seg = it / kLTW, c = it - seg * kLTW;
                const int r0 = seg * RUN;
                float cv[3][RUN];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float col[RUN + 10];
#pragma unroll
                    for (int i = 0; i < RUN + 10; ++i) col[i] = Hp[k * kMH * kMP + (r0 + i) * kMP + c];
#pragma unroll
                    for (int o = 0; o < RUN; ++o) {
                        float acc = 0.f;
#pragma unroll
                        for (int j = 0; j < 11; ++j) acc = fmaf(wr[j], col[o + j], acc);
                        cv[k][o] = acc;
                    }
                }
#pragma unroll
                for (int o = 0; o < RUN; ++o) {
                    const int r = r0 + o;
                    const int gy = by * kLTH + r, gx = bx * kLTW + c;
                    if (gx >= W || gy >= H) continue;
                    const size_t gp = (size_t)gy * W + gx;
                    const float xv = xs[gp], yv = ys[gp];  // the staged planes now hold partials
                    if (ch == 0 && a.counts) {
                        n_depth += a.gt_depth[(size_t)vw.pixel_offset + gp] > 0.f;
                        if (a.label) n_label += a.label[(size_t)vw.pixel_offset + gp] >= 0;
                    }
                    const float d = xv - yv;
                    l1_sum += fabsf(d);
                    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                    gs[(size_t)gy * W + gx] = l1c * sg + cv[0][o] + 2.f * xv * cv[1][o] + yv * cv[2][o];
                }
            }
        }
        __syncthreads();
    }
    if (a.counts) {
        n_depth = __reduce_add_sync(SG_FULL_MASK, n_depth);
        n_label = __reduce_add_sync(SG_FULL_MASK, n_label);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_cnt[0], n_depth);
            atomicAdd(&s_cnt[1], n_label);
        }
    }
    const float t1 = block_sum(l1_sum, s_red);  // (its barriers also order the counts above)
    const float t2 = block_sum(ssim_sum, s_red);
    if (threadIdx.x == 0) {
        a.partials[2 * item] = t1;
        a.partials[2 * item + 1] = t2;
        // integer atomics: the totals do not depend on the order
        if (a.counts && s_cnt[0]) atomicAdd(a.counts + 2 * v, s_cnt[0]);
        if (a.counts && s_cnt[1]) atomicAdd(a.counts + 2 * v + 1, s_cnt[1]);
    }
}

// ---------------------------------------------------------------------------------------
// depth L1, cross-entropy
// ---------------------------------------------------------------------------------------


struct PixelArgs {
    const float *depth, *gt_depth, *sem;
    const int *label;
    float *g_depth, *g_sem;
    const float *decoder;   // K x C or null
    float *decoder_grad;    // K x C or null
    int C, K, ce;           // ce: cross-entropy mode
    float w_depth, w_sem;
    const int *counts;
    const sg_view *views;
    LossViews lv;
    float *partials;        // per pixel block, kPixSlots slots of (sum |D - D_gt| over valid, sum CE over valid)
    float *dec_partials;    // per CTA: K x C share of the decoder gradient
};

// Loss-sum slots per 256-pixel block: one per warp (the SIMT kernel fills slot 0 with its
// block sum and zeroes the others).
constexpr int kPixSlots = kLossThreads / 32;

// Two-level, fixed-order reduction of the per-CTA decoder-gradient shares:
// level 1: chunk c of kDecChunks sums CTAs [c n / kDecChunks, (c+1) n / kDecChunks);
// level 2: decoder_grad[o] += sum over chunks.
constexpr int kDecChunks = 128;
__global__ void decoder_reduce1_kernel(const float *__restrict__ part, int n_blocks, int KC,
                                       float *__restrict__ chunk_sums) {
    pdl_begin();
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (o >= KC) return;
    const int b0 = (int)((long long)c * n_blocks / kDecChunks), b1 = (int)((long long)(c + 1) * n_blocks / kDecChunks);
    float s = 0.f;
    for (int b = b0; b < b1; ++b) s += part[(size_t)b * KC + o];
    chunk_sums[(size_t)c * KC + o] = s;
}
__global__ void decoder_reduce2_kernel(const float *__restrict__ chunk_sums, int KC, float *__restrict__ out) {
    pdl_begin();
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= KC) return;
    float s = 0.f;
    for (int c = 0; c < kDecChunks; ++c) s += chunk_sums[(size_t)c * KC + o];
    out[o] += s;
}

// Row pitches of the per-thread stashes of dz (K floats) and S (C floats).  Rows stay
// 16-byte aligned, and the 8 rows written by a quarter-warp's 16-byte stores start in 8
// different 4-bank groups, so neither the stores nor the 16-byte reads of the decoder
// gradient loop have bank conflicts.
template <int K> __host__ __device__ constexpr int stash_pitch() { return K + 4; }

template <int C, int K>
__global__ void __launch_bounds__(kLossThreads) loss_pixel_kernel(PixelArgs a) {
    pdl_begin();
    static_assert(C % 4 == 0 && K % 4 == 0, "float4 stashes");
    constexpr int KP = stash_pitch<K>(), CP = stash_pitch<C>();
    __shared__ __align__(16) float s_dec[K * C];
    __shared__ float s_red[kLossThreads / 32];
    // only used when the decoder gradient is requested
    extern __shared__ __align__(16) float s_dyn[];
    float *s_dz = s_dyn;                          // kLossThreads x KP
    float *s_S = s_dyn + kLossThreads * KP;       // kLossThreads x CP
    float *s_dec_acc = s_S + kLossThreads * CP;   // K x C
    const bool has_dec = a.decoder != nullptr;
    for (int i = threadIdx.x; i < K * C; i += kLossThreads) s_dec[i] = has_dec ? a.decoder[i] : (i / C == i % C ? 1.f : 0.f);
    if (a.decoder_grad)
        for (int o = threadIdx.x; o < K * C; o += kLossThreads) s_dec_acc[o] = 0.f;
    const int blk = blockIdx.x;
    const int v = find_prefix(a.lv.pix_blk_off, a.lv.n, blk);
    const sg_view &vw = a.views[v];
    const int HW = vw.W * vw.H;
    const int p = (blk - a.lv.pix_blk_off[v]) * kLossThreads + threadIdx.x;
    const bool in = p < HW;
    const size_t p0 = (size_t)vw.pixel_offset;
    const int nd = a.counts[2 * v], nl = a.counts[2 * v + 1];
    __syncthreads();
    float l1d = 0.f, ce = 0.f;
    if (in) {
        const float gd = a.gt_depth[p0 + p];
        float gdep = 0.f;
        if (gd > 0.f) {
            const float d = a.depth[p0 + p] - gd;
            l1d = fabsf(d);
            gdep = a.w_depth * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) / (float)nd;
        }
        a.g_depth[p0 + p] = gdep;
    }
    if (a.ce) {
        float S[C], z[K];
        const int lab = in ? a.label[p0 + p] : -1;
#pragma unroll
        for (int c = 0; c < C; ++c) S[c] = in ? a.sem[(size_t)C * p0 + (size_t)c * HW + p] : 0.f;
        if (has_dec) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c) s = fmaf(s_dec[k * C + c], S[c], s);
                z[k] = s;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) z[k] = S[k < C ? k : 0];
        }
        float zmax = -INFINITY;
#pragma unroll
        for (int k = 0; k < K; ++k) zmax = fmaxf(zmax, z[k]);
        // z <- exp(z - max); softmax = z / sum
        float se = 0.f, zl = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k == lab) zl = z[k] - zmax;
            z[k] = expf(z[k] - zmax);
            se += z[k];
        }
        const float lse_rel = logf(se);   // log-sum-exp minus zmax
        const bool valid = in && lab >= 0;
        if (valid) ce = lse_rel - zl;
        const float sc = valid ? a.w_sem / (float)nl : 0.f;
        const float inv = 1.f / se;
        float dS[C];
#pragma unroll
        for (int c = 0; c < C; ++c) dS[c] = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float dz = sc * (z[k] * inv - (k == lab ? 1.f : 0.f));
            z[k] = dz;
            if (has_dec) {
#pragma unroll
                for (int c = 0; c < C; ++c) dS[c] = fmaf(s_dec[k * C + c], dz, dS[c]);
            } else if (k < C) {
                dS[k] = dz;
            }
        }
        if (in)
#pragma unroll
            for (int c = 0; c < C; ++c) a.g_sem[(size_t)C * p0 + (size_t)c * HW + p] = dS[c];
        if (a.decoder_grad) {
            float4 *dz4 = reinterpret_cast<float4 *>(s_dz + threadIdx.x * KP);
            float4 *S4 = reinterpret_cast<float4 *>(s_S + threadIdx.x * CP);
#pragma unroll
            for (int k = 0; k < K; k += 4) dz4[k / 4] = make_float4(z[k], z[k + 1], z[k + 2], z[k + 3]);
#pragma unroll
            for (int c = 0; c < C; c += 4) S4[c / 4] = make_float4(S[c], S[c + 1], S[c + 2], S[c + 3]);
            __syncwarp();
            // this warp's 32 pixels: each lane accumulates 4 x 4 blocks of dz_p S_p^T in registers
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            constexpr int KB = K / 4, CB = C / 4;
            for (int blk4 = lane; blk4 < KB * CB; blk4 += 32) {
                const int k0 = (blk4 / CB) * 4, c0 = (blk4 % CB) * 4;
                float acc[4][4] = {};
#pragma unroll 4
                for (int t = warp * 32; t < warp * 32 + 32; ++t) {
                    const float4 dz = *reinterpret_cast<const float4 *>(s_dz + t * KP + k0);
                    const float4 sv = *reinterpret_cast<const float4 *>(s_S + t * CP + c0);
                    const float dzv[4] = {dz.x, dz.y, dz.z, dz.w}, svv[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(dzv[i], svv[jj], acc[i][jj]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) atomicAdd(s_dec_acc + (k0 + i) * C + c0 + jj, acc[i][jj]);
            }
            __syncthreads();
            // this block's share of dL/ddecoder, reduced later in block order
            for (int o = threadIdx.x; o < K * C; o += kLossThreads)
                a.dec_partials[(size_t)blk * K * C + o] = s_dec_acc[o];
        }
    }
    const float t1 = block_sum(l1d, s_red);
    const float t2 = block_sum(ce, s_red);
    if (threadIdx.x < kPixSlots) {
        a.partials[2 * (kPixSlots * blk + threadIdx.x)] = threadIdx.x == 0 ? t1 : 0.f;
        a.partials[2 * (kPixSlots * blk + threadIdx.x) + 1] = threadIdx.x == 0 ? t2 : 0.f;
    }
}

// Cross-entropy through a linear decoder on the tensor cores.  One warp owns 32 consecutive
// pixels; with S (32 x C) their semantic features and W (K x C) the decoder:
//   Z = S W^T (logits), softmax and CE per pixel row on the accumulator fragments (a row's
//   K logits sit in the 4 lanes of a quad), dZ = scale (softmax - onehot) in place,
//   dS = dZ W with dZ taken from registers as the A operand (the k index of each 8-class
//   step is permuted so that A column tig / tig + 4 is class 2 tig / 2 tig + 1, and the B
//   rows follow the same permutation), and dW = dZ^T S with dZ transposed through shared
//   memory.  All three run as 3xTF32 MMAs (FP32-level accuracy).  Shared-memory operands
//   are read with ldmatrix (a 32-bit 8 x 4 tile is an 8 x 8 tile of 16-bit halves, and
//   ldmatrix hands thread t the word at row t / 4, column t % 4: exactly the (gid, tig)
//   element of an m16n8k8 TF32 fragment), and each decoder fragment serves both 16-pixel
//   tiles.
//
// Persistent: the warps of a resident grid walk the 32-pixel units of the image set, so the
// decoder is split into shared memory once per CTA and each warp keeps its share of dL/dW in
// registers across all of its units; no block barrier inside the loop.  Each warp stages its
// units in shared memory with asynchronous copies: the next unit's features, labels and
// depths are requested as soon as the current unit's last read of them (the dW contraction)
// is done, so they arrive while dS is computed and stored.  Each unit's two loss
// sums go to its own partial slot (kPixSlots per 256-pixel block); the CTA writes one K x C
// row of decoder-gradient partials at the end, its warps summed in a fixed order.
template <int C, int K>
struct CeLayout {
    static constexpr int CP = C + 4;   // W rows (class-major): 16-byte rows, conflict-free ldmatrix
    static constexpr int KT = K + 4;   // W^T rows (feature-major, classes permuted)
    static constexpr int PP = 32 + 4;  // dZ^T rows (class-major over the warp's 32 pixels)
    static constexpr int SP = 32 + 8;  // staged S rows (feature-major): conflict-free A fragments
    static constexpr int W_FLOATS = 2 * K * CP + 2 * C * KT;
    static constexpr int WARP_FLOATS = K * PP > K * C ? K * PP : K * C;
    // per warp: the unit's S (C x SP), labels, depth and GT depth (32 each)
    static constexpr int STAGE_FLOATS = C * SP + 3 * 32;
};

template <int C, int K>
__host__ __device__ constexpr int ce_mma_smem_floats() {
    return CeLayout<C, K>::W_FLOATS + (kLossThreads / 32) * (CeLayout<C, K>::WARP_FLOATS + CeLayout<C, K>::STAGE_FLOATS);
}

// 4-byte asynchronous copy global -> shared (zero-filled when !valid; src must still be a
// mapped address), and its group fences.
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_groups() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void ldsm_x2(const float *p, uint32_t &r0, uint32_t &r1) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a) : "memory");
}
__device__ __forceinline__ void ldsm_x4(const float *p, uint32_t (&r)[4]) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a) : "memory");
}

// Two CTAs per SM (up to 128 registers): with the per-warp stage, three CTAs at 80 registers
// spilled the warp's fragments and measured slower (loss 0.975 against 0.954 ms on the batched
// workload), and four at 64 slower still.
template <int C, int K>
__global__ void __launch_bounds__(kLossThreads, 2) ce_decoder_mma_kernel(PixelArgs a) {
    pdl_begin();
    static_assert(C % 8 == 0 && K % 16 == 0, "MMA tiles");
    using L = CeLayout<C, K>;
    constexpr int CP = L::CP, KT = L::KT, PP = L::PP, SP = L::SP;
    constexpr int NK = K / 8, NC = C / 8;
    extern __shared__ __align__(16) float s_dyn[];
    float *s_whi = s_dyn, *s_wlo = s_whi + K * CP;     // W [class][feature]
    float *s_thi = s_wlo + K * CP, *s_tlo = s_thi + C * KT;  // W^T [feature][permuted class]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
    float *s_dz = s_dyn + L::W_FLOATS + warp * L::WARP_FLOATS;  // dZ^T [class][pixel]
    for (int i = threadIdx.x; i < K * C; i += kLossThreads) {
        uint32_t h, l;
        split_tf32(a.decoder[i], h, l);
        const int k = i / C, c = i % C;
        s_whi[k * CP + c] = __uint_as_float(h);
        s_wlo[k * CP + c] = __uint_as_float(l);
        // class k = 8 q + 2 j + e sits at column 8 q + j + 4 e of W^T
        const int kc = (k & ~7) + ((k & 7) >> 1) + 4 * (k & 1);
        s_thi[c * KT + kc] = __uint_as_float(h);
        s_tlo[c * KT + kc] = __uint_as_float(l);
    }
    __syncthreads();
    const bool dec_grad = a.decoder_grad != nullptr;
    // ldmatrix row addresses: lanes 0-7 give rows 0-7 of the first 8 x 4 tile, lanes 8-15 of
    // the second (4 columns further), lanes 16-31 (x4 only) the same 8 rows further down
    const int lr = lane & 7, lc = (lane >> 3) & 1, lh = lane >> 4;
    // this warp's share of dW = dZ^T S over all of its pixels (M = classes, N = features)
    float dw[K / 16][NC][4];
#pragma unroll
    for (int mt = 0; mt < K / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < NC; ++nt) dw[mt][nt][0] = dw[mt][nt][1] = dw[mt][nt][2] = dw[mt][nt][3] = 0.f;
    // work unit u = 32 pixels: slot u % kPixSlots of 256-pixel block u / kPixSlots; the warps
    // of the grid take units u = w, w + n_warps, ... (w the warp's grid-wide index)
    const int n_units = kPixSlots * a.lv.pix_blk_off[a.lv.n];
    const int n_warps = (int)gridDim.x * kPixSlots;
    float *s_st = s_dyn + L::W_FLOATS + (kLossThreads / 32) * L::WARP_FLOATS + warp * L::STAGE_FLOATS;
    int *s_lab = reinterpret_cast<int *>(s_st + C * SP);
    float *s_dep = s_st + C * SP + 32, *s_gd = s_dep + 32;
    // unit u: view v, its pixel count and offset, the unit's first pixel pw
    struct Unit {
        int v, HW, pw;
        size_t p0;
    };
    auto unit_of = [&](int u) {
        Unit x;
        const int blk = u / kPixSlots, slot = u % kPixSlots;
        x.v = find_prefix(a.lv.pix_blk_off, a.lv.n, blk);
        const sg_view &vw = a.views[x.v];
        x.HW = vw.W * vw.H;
        x.pw = (blk - a.lv.pix_blk_off[x.v]) * kLossThreads + slot * 32;
        x.p0 = (size_t)vw.pixel_offset;
        return x;
    };
    // lane l requests pixel pw + l of every feature plane, its label and both depths
    auto prefetch = [&](const Unit &x) {
        const int p = x.pw + lane;
        const bool ok = p < x.HW;
        const size_t q = x.p0 + (ok ? p : 0);
        const float *src = a.sem + (size_t)C * x.p0 + (ok ? p : 0);
#pragma unroll
        for (int f = 0; f < C; ++f) cp_async4(s_st + f * SP + lane, src + (size_t)f * x.HW, ok);
        cp_async4(s_lab + lane, a.label + q, ok);
        cp_async4(s_dep + lane, a.depth + q, ok);
        cp_async4(s_gd + lane, a.gt_depth + q, ok);
        cp_async_commit_group();
    };
    int u = (int)blockIdx.x * kPixSlots + warp;
    if (u < n_units) prefetch(unit_of(u));
    for (; u < n_units; u += n_warps) {
        const Unit x = unit_of(u);
        const int v = x.v, HW = x.HW, pw = x.pw;
        const size_t p0 = x.p0;
        const int nd = a.counts[2 * v], nl = a.counts[2 * v + 1];
        cp_async_wait_all_groups();
        __syncwarp();
        float l1d = 0.f, ce = 0.f;
        {
            const int p = pw + lane;
            if (p < HW) {
                const float gd = s_gd[lane];
                float gdep = 0.f;
                if (gd > 0.f) {
                    const float d = s_dep[lane] - gd;
                    l1d = fabsf(d);
                    gdep = a.w_depth * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) / (float)nd;
                }
                a.g_depth[p0 + p] = gdep;
            }
        }
        // staged S (pixels past the view's end read as zero)
        auto S = [&](int px, int f) -> float { return s_st[f * SP + px]; };
        // ---- Z = S W^T: M = pixels (2 x 16), N = classes, K = features ----
        // all of the warp's feature loads are issued before the first MMA (memory-level parallelism)
        float sa[NC][2][4];
#pragma unroll
        for (int ks = 0; ks < NC; ++ks)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = 16 * mt + gid, f0 = 8 * ks + tig;
                sa[ks][mt][0] = S(r0, f0);
                sa[ks][mt][1] = S(r0 + 8, f0);
                sa[ks][mt][2] = S(r0, f0 + 4);
                sa[ks][mt][3] = S(r0 + 8, f0 + 4);
            }
        int labs[2][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = pw + 16 * mt + gid + 8 * h;
                labs[mt][h] = p < HW ? s_lab[16 * mt + gid + 8 * h] : -1;
            }
        float z[2][NK][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NK; ++nt) z[mt][nt][0] = z[mt][nt][1] = z[mt][nt][2] = z[mt][nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < NC; ++ks) {
            uint32_t ah[2][4], al[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int i = 0; i < 4; ++i) split_tf32(sa[ks][mt][i], ah[mt][i], al[mt][i]);
#pragma unroll
            for (int nt = 0; nt < NK; ++nt) {
                // B (8 x 8): b0 (tig, gid) = W[8 nt + gid][8 ks + tig], b1 four features further
                const int w0 = (8 * nt + lr) * CP + 8 * ks + 4 * lc;
                uint32_t bh0, bh1, bl0, bl1;
                ldsm_x2(s_whi + w0, bh0, bh1);
                ldsm_x2(s_wlo + w0, bl0, bl1);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) mma_tf32x3(z[mt][nt], ah[mt], al[mt], bh0, bh1, bl0, bl1);
            }
        }
        // ---- softmax, CE and dZ per pixel row (row 16 mt + gid + 8 h; classes 8 nt + 2 tig + c) ----
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int lab = labs[mt][h];
                float m = -INFINITY;
#pragma unroll
                for (int nt = 0; nt < NK; ++nt) m = fmaxf(m, fmaxf(z[mt][nt][2 * h], z[mt][nt][2 * h + 1]));
                m = fmaxf(m, __shfl_xor_sync(SG_FULL_MASK, m, 1));
                m = fmaxf(m, __shfl_xor_sync(SG_FULL_MASK, m, 2));
                float se = 0.f, zl = 0.f;
                bool has_lab = false;
#pragma unroll
                for (int nt = 0; nt < NK; ++nt)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int cls = 8 * nt + 2 * tig + c;
                        if (cls == lab) {
                            zl = z[mt][nt][2 * h + c] - m;
                            has_lab = true;
                        }
                        const float e = __expf(z[mt][nt][2 * h + c] - m);
                        z[mt][nt][2 * h + c] = e;
                        se += e;
                    }
                se += __shfl_xor_sync(SG_FULL_MASK, se, 1);
                se += __shfl_xor_sync(SG_FULL_MASK, se, 2);
                const bool valid = lab >= 0;
                if (valid && has_lab) ce += logf(se) - zl;
                const float sc = valid ? a.w_sem / (float)nl : 0.f;
                const float inv = 1.f / se;
#pragma unroll
                for (int nt = 0; nt < NK; ++nt)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int cls = 8 * nt + 2 * tig + c;
                        z[mt][nt][2 * h + c] = sc * (z[mt][nt][2 * h + c] * inv - (cls == lab ? 1.f : 0.f));
                    }
            }
        }
        // the two loss sums of this unit
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l1d += __shfl_xor_sync(SG_FULL_MASK, l1d, o);
            ce += __shfl_xor_sync(SG_FULL_MASK, ce, o);
        }
        if (lane == 0) {
            a.partials[2 * u] = l1d;
            a.partials[2 * u + 1] = ce;
        }
        // ---- dW += dZ^T S: M = classes, N = features, K = pixels ----
        if (dec_grad) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NK; ++nt)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        s_dz[(8 * nt + 2 * tig + (i & 1)) * PP + 16 * mt + gid + 8 * (i >> 1)] = z[mt][nt][i];
            __syncwarp();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t bh[NC][2], bl[NC][2];
#pragma unroll
                for (int nt = 0; nt < NC; ++nt) {
                    split_tf32(S(8 * ks + tig, 8 * nt + gid), bh[nt][0], bl[nt][0]);
                    split_tf32(S(8 * ks + tig + 4, 8 * nt + gid), bh[nt][1], bl[nt][1]);
                }
#pragma unroll
                for (int mt = 0; mt < K / 16; ++mt) {
                    // A (16 x 8): rows = classes 16 mt .., columns = pixels 8 ks ..
                    uint32_t ar[4], ah[4], al[4];
                    ldsm_x4(s_dz + (16 * mt + lr + 8 * lc) * PP + 8 * ks + 4 * lh, ar);
#pragma unroll
                    for (int i = 0; i < 4; ++i) split_tf32(__uint_as_float(ar[i]), ah[i], al[i]);
#pragma unroll
                    for (int nt = 0; nt < NC; ++nt)
                        mma_tf32x3(dw[mt][nt], ah, al, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
                }
            }
            __syncwarp();  // the stash is rewritten by the next unit
        }
        // the stage's last read is done: request the next unit (it arrives during dS)
        __syncwarp();
        if (u + n_warps < n_units) prefetch(unit_of(u + n_warps));
        // ---- dS = dZ W: M = pixels, N = features, K = classes (permuted within each 8-class step) ----
        {
            float ds[2][NC][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NC; ++nt) ds[mt][nt][0] = ds[mt][nt][1] = ds[mt][nt][2] = ds[mt][nt][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < NK; ++ks) {
                uint32_t ah[2][4], al[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    // A column tig = class 8 ks + 2 tig (d0 / d2), column tig + 4 = class 8 ks + 2 tig + 1 (d1 / d3)
                    split_tf32(z[mt][ks][0], ah[mt][0], al[mt][0]);
                    split_tf32(z[mt][ks][2], ah[mt][1], al[mt][1]);
                    split_tf32(z[mt][ks][1], ah[mt][2], al[mt][2]);
                    split_tf32(z[mt][ks][3], ah[mt][3], al[mt][3]);
                }
#pragma unroll
                for (int nt = 0; nt < NC; ++nt) {
                    // B (8 x 8): b0 (tig, gid) = W[8 ks + 2 tig][8 nt + gid], b1 = W[8 ks + 2 tig + 1][..]:
                    // rows 8 nt + gid, columns 8 ks + tig (+ 4) of the permuted W^T
                    const int t0 = (8 * nt + lr) * KT + 8 * ks + 4 * lc;
                    uint32_t bh0, bh1, bl0, bl1;
                    ldsm_x2(s_thi + t0, bh0, bh1);
                    ldsm_x2(s_tlo + t0, bl0, bl1);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) mma_tf32x3(ds[mt][nt], ah[mt], al[mt], bh0, bh1, bl0, bl1);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NC; ++nt)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int p = pw + 16 * mt + gid + 8 * (i >> 1);
                        const int f = 8 * nt + 2 * tig + (i & 1);
                        if (p < HW) a.g_sem[(size_t)C * p0 + (size_t)f * HW + p] = ds[mt][nt][i];
                    }
        }
    }
    if (!dec_grad) return;
    // this CTA's share of dL/dW: every warp's fragments into its own stash, then summed over
    // the warps in order (deterministic), one K x C row per CTA
#pragma unroll
    for (int mt = 0; mt < K / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < NC; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                s_dz[(16 * mt + gid + 8 * (i >> 1)) * C + 8 * nt + 2 * tig + (i & 1)] = dw[mt][nt][i];
    __syncthreads();
    const float *s_all = s_dyn + L::W_FLOATS;
    for (int o = threadIdx.x; o < K * C; o += kLossThreads) {
        float s = 0.f;
        for (int w = 0; w < kLossThreads / 32; ++w) s += s_all[w * L::WARP_FLOATS + o];
        a.dec_partials[(size_t)blockIdx.x * K * C + o] = s;
    }
}

// Resident grid of the persistent decoder kernel (at most one CTA per pixel block); returns
// the number of CTAs, i.e. of decoder-gradient partial rows.
template <int C, int K>
static int launch_ce_mma(PixelArgs &pa, int blocks, cudaStream_t st) {
    const size_t smem = sizeof(float) * ce_mma_smem_floats<C, K>();
    static int resident = 0;
    if (!resident) {
        cudaFuncSetAttribute(ce_decoder_mma_kernel<C, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ce_decoder_mma_kernel<C, K>, kLossThreads, smem);
        resident = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    const int grid = blocks < resident ? blocks : resident;
    launch_pdl(ce_decoder_mma_kernel<C, K>, grid, kLossThreads, smem, st, pa);
    return grid;
}

struct FinalArgs {
    const float *ssim_rgb, *ssim_sem, *pix;  // partial arrays
    const int *counts;
    const sg_view *views;
    LossViews lv;
    int C, sem_mode;
    float lambda_r, lambda_s, w_depth, w_sem;
    float *terms;
    uint32_t *status;  // non-NULL: flag non-finite loss terms (SG_STATUS_NUMERIC)
};

// Sum of v over the block in double, in a fixed order (warp butterflies, then the warps in
// order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v, double *s_w) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SG_FULL_MASK, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLossThreads / 32; ++w) t += s_w[w];
    return t;
}

__global__ void loss_finalize_kernel(FinalArgs a) {
    pdl_begin();
    const int v = blockIdx.x;
    const sg_view &vw = a.views[v];
    const double HW = (double)vw.W * vw.H;
    __shared__ double s_w[kLossThreads / 32];
    double acc[4] = {0, 0, 0, 0};
    for (int i = a.lv.tile_off[v] + threadIdx.x; i < a.lv.tile_off[v + 1]; i += kLossThreads) {
        acc[0] += a.ssim_rgb[2 * i];
        acc[1] += a.ssim_rgb[2 * i + 1];
        if (a.ssim_sem) {
            acc[2] += a.ssim_sem[2 * i];
            acc[3] += a.ssim_sem[2 * i + 1];
        }
    }
    // the per-unit (depth L1, CE) sums: two units per 16-byte load, four loads in flight per
    // thread, summed in a fixed order (a latency-bound chain of dependent adds otherwise)
    double b[2] = {0, 0};
    {
        const float4 *p4 = reinterpret_cast<const float4 *>(a.pix);
        const int s1 = kPixSlots * a.lv.pix_blk_off[v + 1] / 2;
        double c[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        int i = kPixSlots * a.lv.pix_blk_off[v] / 2 + threadIdx.x;
        for (; i + 3 * kLossThreads < s1; i += 4 * kLossThreads) {
            float4 q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = p4[i + k * kLossThreads];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                c[k][0] += (double)q[k].x + (double)q[k].z;
                c[k][1] += (double)q[k].y + (double)q[k].w;
            }
        }
        for (; i < s1; i += kLossThreads) {
            const float4 q = p4[i];
            c[0][0] += (double)q.x + (double)q.z;
            c[0][1] += (double)q.y + (double)q.w;
        }
        b[0] = (c[0][0] + c[1][0]) + (c[2][0] + c[3][0]);
        b[1] = (c[0][1] + c[1][1]) + (c[2][1] + c[3][1]);
    }
    double r[4];
    for (int k = 0; k < 4; ++k) r[k] = block_sum_d(acc[k], s_w);
    const double l1d_sum = block_sum_d(b[0], s_w);
    const double ce_sum = block_sum_d(b[1], s_w);
    if (threadIdx.x == 0) {
        const double l1d = l1d_sum, ce = ce_sum;
        const int nd = a.counts[2 * v], nl = a.counts[2 * v + 1];
        const double n_rgb = 3.0 * HW;
        const double L_r = (1.0 - a.lambda_r) * r[0] / n_rgb + a.lambda_r * (1.0 - r[1] / n_rgb);
        const double L_d = nd > 0 ? a.w_depth * l1d / nd : 0.0;
        double L_s;
        if (a.sem_mode == 0) {
            L_s = nl > 0 ? a.w_sem * ce / nl : 0.0;
        } else {
            const double n_s = (double)a.C * HW;
            L_s = a.w_sem * ((1.0 - a.lambda_s) * r[2] / n_s + a.lambda_s * (1.0 - r[3] / n_s));
        }
        a.terms[4 * v + 0] = (float)L_r;
        a.terms[4 * v + 1] = (float)L_d;
        a.terms[4 * v + 2] = (float)L_s;
        a.terms[4 * v + 3] = (float)(L_r + L_d + L_s);
        if (a.status && !isfinite(L_r + L_d + L_s)) atomicOr(a.status, SG_STATUS_NUMERIC);
    }
}

// ---------------------------------------------------------------------------------------

static size_t ssim_smem() { return sizeof(float) * (2 * kXH * kXP + 5 * kXH * kMP); }

static void make_loss_views(const sg_view *vh, int n_views, LossViews &lv) {
    lv.n = n_views;
    lv.tile_off[0] = 0;
    lv.pix_blk_off[0] = 0;
    for (int v = 0; v < n_views; ++v) {
        const int tx = (vh[v].W + kLTW - 1) / kLTW, ty = (vh[v].H + kLTH - 1) / kLTH;
        lv.tile_off[v + 1] = lv.tile_off[v] + tx * ty;
        lv.pix_blk_off[v + 1] = lv.pix_blk_off[v] + (vh[v].W * vh[v].H + kLossThreads - 1) / kLossThreads;
    }
}

static size_t loss_ws_bytes(int n_views, int n_tiles, int n_blocks, int KC) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(sizeof(int) * 2 * n_views) + 2 * al(sizeof(float) * 2 * n_tiles) +
           al(sizeof(float) * 2 * kPixSlots * n_blocks) + al(sizeof(float) * (size_t)n_blocks * KC) +
           al(sizeof(float) * (size_t)kDecChunks * KC);
}

// Decoder-gradient floats the loss keeps per pixel block: K x C partials in cross-entropy
// mode when a decoder gradient is requested, none otherwise (paper mode has no decoder).
int loss_decoder_partials(const sg_loss_config *lc, int C) {
    return (lc->sem_mode == 0 && lc->decoder_grad) ? lc->n_classes * C : 0;
}

// Exact scratch bytes when KC decoder-gradient floats per block are needed (0 = none).
size_t loss_workspace_size_kc(const sg_view *vh, int n_views, int KC) {
    LossViews lv;
    make_loss_views(vh, n_views, lv);
    return loss_ws_bytes(n_views, lv.tile_off[n_views], lv.pix_blk_off[n_views], KC);
}

size_t loss_workspace_size(const sg_view *vh, int n_views, int C, int n_classes) {
    LossViews lv;
    make_loss_views(vh, n_views, lv);
    const int K = n_classes > C ? n_classes : C;
    return loss_ws_bytes(n_views, lv.tile_off[n_views], lv.pix_blk_off[n_views], K * C);
}

template <int C, int K>
static void launch_pixel_t(PixelArgs &pa, int blocks, cudaStream_t st) {
    const size_t full = sizeof(float) * (kLossThreads * (stash_pitch<K>() + stash_pitch<C>()) + K * C);
    const size_t dyn = pa.decoder_grad ? full : 0;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(loss_pixel_kernel<C, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)full);
        attr = true;
    }
    launch_pdl(loss_pixel_kernel<C, K>, blocks, kLossThreads, dyn, st, pa);
}

// Launches the per-pixel loss kernel; returns the number of decoder-gradient partial rows it
// writes (its CTAs), or 0 for an unsupported (C, K).
static int launch_pixel(PixelArgs &pa, int blocks, cudaStream_t st) {
    const int C = pa.C, K = pa.K;
    if (pa.ce && pa.decoder) {
#define SG_CE(c, k) if (C == c && K == k) return launch_ce_mma<c, k>(pa, blocks, st);
        SG_CE(16, 16) SG_CE(16, 32) SG_CE(32, 32)
#undef SG_CE
    }
#define SG_PIX(c, k) if (C == c && K == k) { launch_pixel_t<c, k>(pa, blocks, st); return blocks; }
    SG_PIX(4, 4) SG_PIX(8, 8) SG_PIX(16, 16) SG_PIX(16, 32) SG_PIX(32, 32) SG_PIX(40, 40)
#undef SG_PIX
    return 0;
}

sg_status launch_loss(const sg_images *r, const sg_targets *gt, const sg_view *views,
                      const sg_view *vh, int n_views, int C, const sg_loss_config *lc,
                      float *terms, sg_images *dL, void *ws, size_t ws_bytes, uint32_t *status,
                      cudaStream_t st) {
    LossViews lv;
    make_loss_views(vh, n_views, lv);
    const int n_tiles = lv.tile_off[n_views], n_blocks = lv.pix_blk_off[n_views];
    char *base = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = base + off; off += (bytes + 255) & ~(size_t)255; return p; };
    int *counts = (int *)take(sizeof(int) * 2 * n_views);
    float *p_rgb = (float *)take(sizeof(float) * 2 * n_tiles);
    float *p_sem = (float *)take(sizeof(float) * 2 * n_tiles);
    float *p_pix = (float *)take(sizeof(float) * 2 * kPixSlots * n_blocks);
    const int ce = lc->sem_mode == 0;
    const int K = ce ? lc->n_classes : C;
    const int KC = loss_decoder_partials(lc, C);
    float *p_dec = (float *)take(sizeof(float) * (size_t)n_blocks * KC);
    float *p_dec2 = (float *)take(sizeof(float) * (size_t)kDecChunks * KC);
    if (loss_ws_bytes(n_views, n_tiles, n_blocks, KC) > ws_bytes) {
        set_error("pyramid_loss: workspace %zu bytes < %zu needed", ws_bytes,
                  loss_ws_bytes(n_views, n_tiles, n_blocks, KC));
        return SG_ERR_CAPACITY;
    }
    cudaMemsetAsync(counts, 0, sizeof(int) * 2 * n_views, st);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(ssim_l1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssim_smem());
        attr = true;
    }
    SsimArgs sa{r->rgb, gt->rgb, dL->rgb, 3, 1.f - lc->lambda_r, lc->lambda_r, views, lv, p_rgb,
                gt->depth, ce ? gt->label : nullptr, counts};
    launch_pdl(ssim_l1_kernel, n_tiles, kLossThreads, ssim_smem(), st, sa);
    if (!ce) {
        SsimArgs ss{r->sem, gt->sem, dL->sem, C, lc->w_sem * (1.f - lc->lambda_s), lc->w_sem * lc->lambda_s,
                    views, lv, p_sem, nullptr, nullptr, nullptr};
        launch_pdl(ssim_l1_kernel, n_tiles, kLossThreads, ssim_smem(), st, ss);
    }
    PixelArgs pa{r->depth, gt->depth, r->sem, gt->label, dL->depth, dL->sem, lc->decoder,
                 KC ? lc->decoder_grad : nullptr, C, K, ce, lc->w_depth, lc->w_sem, counts, views, lv, p_pix, p_dec};
    const int dec_rows = launch_pixel(pa, n_blocks, st);
    if (!dec_rows) {
        set_error("pyramid_loss: unsupported (C=%d, classes=%d)", C, K);
        return SG_ERR_INVALID_ARG;
    }
    if (ce && lc->decoder_grad) {
        launch_pdl(decoder_reduce1_kernel, dim3((KC + 127) / 128, kDecChunks), 128, 0, st, p_dec, dec_rows, KC, p_dec2);
        launch_pdl(decoder_reduce2_kernel, (KC + 127) / 128, 128, 0, st, p_dec2, KC, lc->decoder_grad);
        count_launches(2);
    }
    FinalArgs fa{p_rgb, ce ? nullptr : p_sem, p_pix, counts, views, lv, C, lc->sem_mode,
                 lc->lambda_r, lc->lambda_s, lc->w_depth, lc->w_sem, terms, status};
    launch_pdl(loss_finalize_kernel, n_views, kLossThreads, 0, st, fa);
    count_launches(ce ? 3 : 4);
    return check_launch("pyramid_loss");
}

// ---------------------------------------------------------------------------------------
// Eq. 4-6 pyramid: level l+1 from level l of the same camera
// ---------------------------------------------------------------------------------------

__global__ void pyramid_down_kernel(float *rgb, float *depth, int *label, float *sem, int n_sem,
                                    sg_view src, sg_view dst) {
    pdl_begin();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= dst.W || y >= dst.H) return;
    const size_t sHW = (size_t)src.W * src.H, dHW = (size_t)dst.W * dst.H;
    const size_t s00 = (size_t)(2 * y) * src.W + 2 * x;
    const size_t idx[4] = {s00, s00 + 1, s00 + src.W, s00 + src.W + 1};
    const size_t o = (size_t)y * dst.W + x;
    for (int c = 0; c < 3; ++c) {
        const float *s = rgb + 3 * (size_t)src.pixel_offset + c * sHW;
        rgb[3 * (size_t)dst.pixel_offset + c * dHW + o] = 0.25f * ((s[idx[0]] + s[idx[1]]) + (s[idx[2]] + s[idx[3]]));
    }
    for (int c = 0; c < n_sem; ++c) {
        const float *s = sem + (size_t)n_sem * src.pixel_offset + c * sHW;
        sem[(size_t)n_sem * dst.pixel_offset + c * dHW + o] = 0.25f * ((s[idx[0]] + s[idx[1]]) + (s[idx[2]] + s[idx[3]]));
    }
    float ds = 0.f;
    int dn = 0;
    for (int k = 0; k < 4; ++k) {
        const float d = depth[src.pixel_offset + idx[k]];
        if (d > 0.f) { ds += d; ++dn; }
    }
    depth[dst.pixel_offset + o] = dn ? ds / (float)dn : 0.f;
    if (label) {
        int l[4];
        for (int k = 0; k < 4; ++k) l[k] = label[src.pixel_offset + idx[k]];
        int best = -1, bc = 0;
        for (int k = 0; k < 4; ++k) {
            if (l[k] < 0) continue;
            int c = 0;
            for (int j = 0; j < 4; ++j) c += l[j] == l[k];
            if (c > bc || (c == bc && l[k] < best)) { best = l[k]; bc = c; }
        }
        label[dst.pixel_offset + o] = best;
    }
}

sg_status launch_pyramid(float *rgb, float *depth, int *label, float *sem, int n_sem,
                         const sg_view *vh, int n_views, cudaStream_t st) {
    int max_level = 0;
    for (int v = 0; v < n_views; ++v) max_level = vh[v].level > max_level ? vh[v].level : max_level;
    for (int l = 1; l <= max_level; ++l)
        for (int v = 0; v < n_views; ++v) {
            if (vh[v].level != l) continue;
            int s = -1;
            for (int u = 0; u < n_views; ++u)
                if (vh[u].camera == vh[v].camera && vh[u].level == l - 1) s = u;
            if (s < 0) {
                set_error("build_pyramid: view %d (camera %d, level %d) has no parent level", v, vh[v].camera, l);
                return SG_ERR_INVALID_ARG;
            }
            const dim3 blk(32, 8), grd((vh[v].W + 31) / 32, (vh[v].H + 7) / 8);
            launch_pdl(pyramid_down_kernel, grd, blk, 0, st, rgb, depth, label, sem, n_sem, vh[s], vh[v]);
            count_launches(1);
        }
    return check_launch("build_pyramid");
}

// ---------------------------------------------------------------------------------------
// Adam
// ---------------------------------------------------------------------------------------

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2) {
    pdl_begin();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// All parameter groups in one launch; the gradient is zeroed after it is read, ready for
// the next iteration's accumulation.
struct AdamGroups {
    sg_adam_group g[SG_ADAM_MAX_GROUPS];
    int64_t start[SG_ADAM_MAX_GROUPS + 1];  // prefix of element counts
    int n;
    uint32_t *status;  // non-NULL: flag non-finite gradients (SG_STATUS_NUMERIC)
};

__global__ void adam_multi_kernel(AdamGroups G, float b1, float b2, float eps, float bc1, float bc2,
                                  int zero_grad) {
    pdl_begin();
    const int64_t total = G.start[G.n];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < G.n && i >= G.start[k + 1]) ++k;
        const sg_adam_group &q = G.g[k];
        const int64_t j = i - G.start[k];
        const float gi = q.grad[j];
        if (G.status) flag_status(!isfinite(gi), G.status, SG_STATUS_NUMERIC);
        const float mi = b1 * q.m[j] + (1.f - b1) * gi;
        const float vi = b2 * q.v[j] + (1.f - b2) * gi * gi;
        q.m[j] = mi;
        q.v[j] = vi;
        q.param[j] -= q.lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        if (zero_grad) q.grad[j] = 0.f;
    }
}

// The same update, four elements per thread with 16-byte loads and stores: start[] counts
// quads (every group holds a multiple of 4 elements, all arrays 16-byte aligned).
// ibc1, ibc2: reciprocals of the bias corrections.  sqrt and the division use the fast
// hardware approximations (a few ulp; the update is a step size, not a value the path
// returns); sqrt(0) is taken as 0 so that a parameter with no gradient history stays put.
__device__ __forceinline__ float adam_one(float &m, float &v, float p, float g, float lr, float b1, float b2,
                                          float eps, float ibc1, float ibc2) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    const float vh = v * ibc2;
    const float s = vh > 0.f ? vh * rsqrtf(vh) : 0.f;
    return p - lr * __fdividef(m * ibc1, s + eps);
}

__global__ void adam_multi4_kernel(AdamGroups G, float b1, float b2, float eps, float ibc1, float ibc2,
                                   int zero_grad) {
    pdl_begin();
    const int64_t total = G.start[G.n];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < G.n && i >= G.start[k + 1]) ++k;
        const sg_adam_group &q = G.g[k];
        const int64_t j = i - G.start[k];
        float4 *gp = reinterpret_cast<float4 *>(q.grad) + j;
        float4 *mp = reinterpret_cast<float4 *>(q.m) + j;
        float4 *vp = reinterpret_cast<float4 *>(q.v) + j;
        float4 *pp = reinterpret_cast<float4 *>(q.param) + j;
        const float4 g = *gp;
        if (G.status)
            flag_status(!isfinite(g.x) || !isfinite(g.y) || !isfinite(g.z) || !isfinite(g.w), G.status,
                        SG_STATUS_NUMERIC);
        float4 m = *mp, v = *vp, p = *pp;
        p.x = adam_one(m.x, v.x, p.x, g.x, q.lr, b1, b2, eps, ibc1, ibc2);
        p.y = adam_one(m.y, v.y, p.y, g.y, q.lr, b1, b2, eps, ibc1, ibc2);
        p.z = adam_one(m.z, v.z, p.z, g.z, q.lr, b1, b2, eps, ibc1, ibc2);
        p.w = adam_one(m.w, v.w, p.w, g.w, q.lr, b1, b2, eps, ibc1, ibc2);
        *mp = m;
        *vp = v;
        *pp = p;
        if (zero_grad) *gp = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

sg_status launch_adam_multi(const sg_adam_group *groups, int n, float b1, float b2, float eps, int step,
                            int zero_grad, uint32_t *status, cudaStream_t st) {
    AdamGroups G{};
    G.n = n;
    G.status = status;
    G.start[0] = 0;
    for (int k = 0; k < n; ++k) {
        G.g[k] = groups[k];
        G.start[k + 1] = G.start[k] + groups[k].n;
    }
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bool quads = true;
    for (int k = 0; k < n; ++k) {
        const sg_adam_group &q = groups[k];
        quads = quads && q.n % 4 == 0 && ((uintptr_t)q.param | (uintptr_t)q.grad | (uintptr_t)q.m |
                                          (uintptr_t)q.v) % 16 == 0;
    }
    if (quads)
        for (int k = 0; k <= n; ++k) G.start[k] /= 4;
    int64_t blocks = (G.start[n] + 255) / 256;
    if (blocks > 8 * (int64_t)sms) blocks = 8 * (int64_t)sms;
    if (blocks > 0) {
        if (quads)
            launch_pdl(adam_multi4_kernel, (int)blocks, 256, 0, st, G, b1, b2, eps, 1.f / bc1, 1.f / bc2, zero_grad);
        else
            launch_pdl(adam_multi_kernel, (int)blocks, 256, 0, st, G, b1, b2, eps, bc1, bc2, zero_grad);
        count_launches(1);
    }
    return check_launch("adam_multi");
}

sg_status launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t st) {
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8 * (int64_t)sms) blocks = 8 * (int64_t)sms;
    if (blocks > 0) {
        launch_pdl(adam_kernel, (int)blocks, 256, 0, st, p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
        count_launches(1);
    }
    return check_launch("adam");
}

}  // namespace sg
