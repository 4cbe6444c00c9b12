// raster_impl.cuh -- tile compositing of RGB, depth and C semantic channels (Eq. 7-9) and its
// adjoint (Sec. III-D backpropagation), templated on the semantic width C and on the
// number of pixels each thread owns (PPT = 1, 2 or 4).
//
// One CTA owns one screen tile of one view-level.  Every view-level of every keyframe is
// addressed through one global tile id, so a single launch renders the whole pyramid of
// all keyframes; with `persistent` set, a grid of resident CTAs pulls tile ids from an
// atomic work counter.  Each warp owns an 8 x (4 PPT) pixel sub-tile: lane l has the PPT
// pixels (l mod 8, l div 8 + 4k), k < PPT.  A whole warp skips a Gaussian whose footprint
// misses its sub-tile (one uniform test), and with PPT > 1 every per-Gaussian cost
// (shared-memory loads, the per-chunk contractions of the backward) is shared by PPT pixels.
//
// Forward: the tile's depth-sorted list is walked in batches the CTA stages into shared
// memory; each pixel composites front to back and stops when T would fall below T_min;
// the CTA leaves the tile when all pixels are done.  Saved per pixel: T_final, last (list
// entries examined up to and including the last contributor), contributor count.
//
// Backward: back to front from the tile's largest `last`.  Each pixel rebuilds T by
// dividing by (1 - alpha) and tracks only the scalar a = g . A of the background-weighted
// suffix colour A.  Per chunk of 16 list entries every lane writes, for each entry, its
// weight w = alpha T and s = dL/dsigma into two chunk buffers; the three sums over the
// warp's pixels -- g . f, the 4 + C feature gradients dF = W^T G (colour, depth, semantics)
// and the six pixel moments of s, which give the 2D-mean, conic and opacity gradients --
// then run on the tensor cores (mma.m16n8k8, TF32 split into hi + lo parts for FP32-level
// accuracy); no shuffles in the per-entry loop.
#pragma once

#include "raster.cuh"

namespace sg {

// Stages entries [b0, b0 + cnt) of a tile's list.  Per entry:
//   s_geo0 = (ui - px0, vi - py0, uf, vf): integer part of the 2D mean relative to the tile
//            origin (exact in float) and its float fraction,
//   s_geo1 = (m00, m10, m11, opacity),
//   s_geo2 = (u, v, ex, ey): approximate tile-relative mean and the projection's conservative
//            half extents of the alpha >= alpha_min region (warp-level skip test only),
// the 4 + C features, and (backward) the Gaussian index.
template <int NF>
__device__ __forceinline__ void load_batch(const RasterArgs &a, int C, int list_start, int b0, int cnt,
                                           int px0, int py0, uint32_t rec_base, float4 *s_geo0,
                                           float4 *s_geo1, float4 *s_geo2, float *s_feat, uint32_t *s_rec,
                                           int nthreads) {
    for (int j = threadIdx.x; j < cnt; j += nthreads) {
        const uint32_t rec = a.record[list_start + b0 + j] & a.rec_mask;
        const float4 g0 = a.geo[2 * (size_t)rec];
        const float4 g1 = a.geo[2 * (size_t)rec + 1];
        const uint32_t packed = __float_as_uint(g1.w);
        const float uI = (float)((int)(short)(packed & 0xffffu) - px0);
        const float vI = (float)((int)(short)(packed >> 16) - py0);
        const float2 ex = a.ext[rec];
        s_geo0[j] = make_float4(uI, vI, g0.x, g0.y);
        s_geo1[j] = make_float4(g1.x, g1.y, g1.z, g0.w);
        s_geo2[j] = make_float4(uI + g0.x, vI + g0.y, ex.x, ex.y);
        const uint32_t gi = rec - rec_base;  // every record of a tile belongs to its view-level
        const size_t ci = a.col_rec ? rec : gi;
        float *f = s_feat + (size_t)j * NF;
        f[0] = a.rgb[3 * ci];
        f[1] = a.rgb[3 * ci + 1];
        f[2] = a.rgb[3 * ci + 2];
        f[3] = g0.z;  // depth (camera z of the mean, Eq. 8)
        const float4 *s4 = reinterpret_cast<const float4 *>(a.sem + (size_t)(a.sem_rec ? rec : gi) * C);
        float4 *f4 = reinterpret_cast<float4 *>(f + 4);
#pragma unroll
        for (int k = 0; k < (NF - 4) / 4; ++k) f4[k] = s4[k];
        if (s_rec) s_rec[j] = rec;
    }
}
// The same rows for one warp and at most 32 entries whose records are known (rec_of(j) is
// row j's record): lanes 0-15 stage the geometry of rows lane, lane + 16, lanes 16-31 their
// features.  s_geo2 and s_rec may be null (not staged).
template <int NF, class RecOf>
__device__ __forceinline__ void stage_rows_warp(const RasterArgs &a, int C, RecOf rec_of, int cnt, int px0,
                                                int py0, uint32_t rec_base, float4 *s_geo0, float4 *s_geo1,
                                                float4 *s_geo2, float *s_feat, uint32_t *s_rec) {
    const int lane = threadIdx.x & 31;
    for (int j = lane & 15; j < cnt; j += 16) {
        const uint32_t rec = rec_of(j);
        float *f = s_feat + (size_t)j * NF;
        if (lane < 16) {
            const float4 g0 = a.geo[2 * (size_t)rec];
            const float4 g1 = a.geo[2 * (size_t)rec + 1];
            const uint32_t packed = __float_as_uint(g1.w);
            const float uI = (float)((int)(short)(packed & 0xffffu) - px0);
            const float vI = (float)((int)(short)(packed >> 16) - py0);
            s_geo0[j] = make_float4(uI, vI, g0.x, g0.y);
            s_geo1[j] = make_float4(g1.x, g1.y, g1.z, g0.w);
            if (s_geo2) {
                const float2 ex = a.ext[rec];
                s_geo2[j] = make_float4(uI + g0.x, vI + g0.y, ex.x, ex.y);
            }
            if (s_rec) s_rec[j] = rec;
            f[3] = g0.z;  // depth (camera z of the mean, Eq. 8)
        } else {
            const uint32_t gi = rec - rec_base;
            const size_t ci = a.col_rec ? rec : gi;
            f[0] = a.rgb[3 * ci];
            f[1] = a.rgb[3 * ci + 1];
            f[2] = a.rgb[3 * ci + 2];
            const float4 *s4 = reinterpret_cast<const float4 *>(a.sem + (size_t)(a.sem_rec ? rec : gi) * C);
            float4 *f4 = reinterpret_cast<float4 *>(f + 4);
#pragma unroll
            for (int k = 0; k < (NF - 4) / 4; ++k) f4[k] = s4[k];
        }
    }
}

// Persistent work queue: work_counter[0] hands out slots, work_counter[1] counts the CTAs
// that have drawn their terminating slot; the last of them zeroes both, so the queue is
// ready for the next launch without a memset.
__device__ __forceinline__ int next_item(const RasterArgs &a, int n_items, int &s_item) {
    if (!a.persistent) return blockIdx.x;
    if (threadIdx.x == 0) {
        const int slot = atomicAdd(a.work_counter, 1);
        if (slot >= n_items && atomicAdd(a.work_counter + 1, 1) == (int)gridDim.x - 1) {
            a.work_counter[0] = 0;
            a.work_counter[1] = 0;
        }
        s_item = slot;
    }
    __syncthreads();
    return s_item;
}

template <int PPT>
struct WarpTile {
    int lx, ly;      // first pixel of the thread, relative to the tile origin (others: ly + 4k)
    float cxw, cyw;  // centre of the warp's 8 x (4 PPT) sub-tile
    __device__ WarpTile(int tile_w) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int warps_x = tile_w >> 3;
        const int wx = (warp % warps_x) * 8, wy = (warp / warps_x) * (4 * PPT);
        lx = wx + (lane & 7);
        ly = wy + (lane >> 3);
        cxw = wx + 3.5f;
        cyw = wy + 2.f * PPT - 0.5f;
    }
    // true if no pixel of the warp's sub-tile can reach alpha_min (g2 = u, v, ex, ey)
    __device__ __forceinline__ bool misses(const float4 &g2) const {
        return fabsf(g2.x - cxw) > g2.z + 3.5f || fabsf(g2.y - cyw) > g2.w + (2.f * PPT - 0.5f);
    }
    // The same, exactly for the ellipse: besides the box test, true if the minimum of
    // sigma = (m00 dx)^2 + (m10 dx + m11 dy)^2 over the rectangle spanned by the sub-tile's
    // pixel centres exceeds ln(o / alpha_min), so alpha < alpha_min at every pixel of the warp
    // (g1 = m00, m10, m11, o).  Conservative: the continuous rectangle contains every pixel
    // centre, and the 1e-3 margin on sigma covers rounding and the fast exponential.
    __device__ __forceinline__ bool misses(const float4 &g2, const float4 &g1, float ln_alpha_min) const {
        if (misses(g2)) return true;
        const float hx = 3.5f, hy = 2.f * PPT - 0.5f;
        // pixel offsets from the mean: dx in [x0, x1], dy in [y0, y1]
        const float x0 = cxw - g2.x - hx, x1 = cxw - g2.x + hx;
        const float y0 = cyw - g2.y - hy, y1 = cyw - g2.y + hy;
        if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return false;  // the mean is inside
        // sigma = A dx^2 + 2 B dx dy + Cq dy^2, a convex quadratic: with the mean outside, its
        // minimum over the rectangle lies on an edge, where it is a clamped 1D minimum
        const float A = g1.x * g1.x + g1.y * g1.y, B = g1.y * g1.z, Cq = g1.z * g1.z;
        const float iA = 1.f / A, iC = 1.f / Cq;
        auto on_x = [&](float dx) {
            const float dy = fminf(y1, fmaxf(y0, -B * dx * iC));
            return fmaf(A * dx, dx, fmaf(2.f * B * dx, dy, Cq * dy * dy));
        };
        auto on_y = [&](float dy) {
            const float dx = fminf(x1, fmaxf(x0, -B * dy * iA));
            return fmaf(A * dx, dx, fmaf(2.f * B * dx, dy, Cq * dy * dy));
        };
        const float smin = fminf(fminf(on_x(x0), on_x(x1)), fminf(on_y(y0), on_y(y1)));
        const float tau = __logf(g1.w) - ln_alpha_min;  // alpha >= alpha_min needs sigma <= tau
        return smin > tau * 1.0001f + 1e-3f;
    }
};

struct TileInfo {
    int v, px0, py0;
    const sg_view *vw;
};

__device__ __forceinline__ TileInfo tile_info(const RasterArgs &a, int item) {
    TileInfo t;
    t.v = find_view(a.views, a.n_views, item);
    t.vw = &a.views[t.v];
    const int local = item - t.vw->tile_offset;
    t.px0 = (local % t.vw->tiles_x) * a.tile_w;
    t.py0 = (local / t.vw->tiles_x) * a.tile_h;
    return t;
}

// Half mode of the forward (8 x 8 tiles, one pixel per thread, lists with half masks): a
// CTA is one warp that owns one half (8 x 4 pixels) of a tile; it walks the tile's list front
// to back, queues (position, record) of the entries whose mask holds its half, and stages and
// composites them 32 at a time with no block barrier, stopping as soon as its own 32 pixels
// are saturated.  The per-pixel sequence of contributing entries, and so the output, is the
// same as with shared batches.
constexpr int kFwdHalfChunk = 32;
constexpr int kFwdHalfQueue = kFwdHalfChunk + 32;  // < kFwdHalfChunk pending + one 32-entry scan

template <int C, int PPT, bool HALF = false>
__global__ void __launch_bounds__(kMaxTileThreads) raster_fwd_kernel(RasterArgs a) {
    pdl_begin();
    constexpr int NF = 4 + C;
    constexpr bool hm = HALF;
    static_assert(!HALF || PPT == 1, "half mode runs one pixel per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int batch = hm ? kFwdHalfChunk : a.batch;
    float4 *s_geo0 = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_geo1 = s_geo0 + batch;
    float4 *s_geo2 = hm ? nullptr : s_geo1 + batch;
    float *s_feat = reinterpret_cast<float *>(s_geo1 + (hm ? batch : 2 * batch));
    int *s_q = reinterpret_cast<int *>(s_feat + (size_t)batch * NF);  // half mode: the queue
    uint32_t *s_qr = reinterpret_cast<uint32_t *>(s_q + kFwdHalfQueue);
    const int nthreads = hm ? 32 : a.tile_w * a.tile_h / PPT;
    const int lane = threadIdx.x & 31;
    const WarpTile<PPT> wt(a.tile_w);
    const float fx = (float)wt.lx;
    const float ln_amin = __logf(a.alpha_min);
    const int n_items = hm ? 2 * a.n_tiles : a.n_tiles;
    for (int iter = 0;; ++iter) {
        if (!a.persistent && iter > 0) break;
        const int slot = next_item(a, n_items, s_item);
        if (slot >= n_items) break;
        const int tslot = hm ? slot >> 1 : slot, hf = hm ? slot & 1 : 0;
        const int item = a.order ? a.order[tslot] : tslot;  // tile id
        TileInfo ti = tile_info(a, item);
        ti.py0 += hf * (a.tile_h / 2);  // half mode: this warp's half
        const sg_view &vw = *ti.vw;
        const int px = ti.px0 + wt.lx;
        const int2 range = a.ranges[item];
        const int n = range.y - range.x;
        const uint32_t rec_base = (uint32_t)ti.v * (uint32_t)a.N;
        float acc[PPT][NF];
        float T[PPT];
        int last[PPT], nc[PPT];
        bool done[PPT];
        int n_done = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int py = ti.py0 + wt.ly + 4 * k;
#pragma unroll
            for (int c = 0; c < NF; ++c) acc[k][c] = 0.f;
            T[k] = 1.f;
            last[k] = 0;
            nc[k] = 0;
            done[k] = !(px < vw.W && py < vw.H);
            n_done += done[k];
        }
        // staged row j, list position pos: alpha at the thread's pixels, front to back
        auto entry = [&](const int j, const int pos) {
            const float4 g0 = s_geo0[j];
            const float4 g1 = s_geo1[j];
            float w[PPT];
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                w[k] = 0.f;
                if (done[k]) continue;
                AlphaEval e;
                if (!eval_alpha(fx - g0.x, (float)(wt.ly + 4 * k) - g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w,
                                a.alpha_max, a.alpha_min, e))
                    continue;
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, e.alpha));
                if (Tn < a.T_min) {
                    done[k] = true;
                    ++n_done;
                    continue;
                }
                w[k] = e.alpha * T[k];
                T[k] = Tn;
                last[k] = pos + 1;
                ++nc[k];
                any = true;
            }
            if (!any) return;
            const float4 *f4 = reinterpret_cast<const float4 *>(s_feat + (size_t)j * NF);
#pragma unroll
            for (int q = 0; q < NF / 4; ++q) {
                const float4 f = f4[q];
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    acc[k][4 * q + 0] = fmaf(w[k], f.x, acc[k][4 * q + 0]);
                    acc[k][4 * q + 1] = fmaf(w[k], f.y, acc[k][4 * q + 1]);
                    acc[k][4 * q + 2] = fmaf(w[k], f.z, acc[k][4 * q + 2]);
                    acc[k][4 * q + 3] = fmaf(w[k], f.w, acc[k][4 * q + 3]);
                }
            }
        };
        if (!hm) {
            for (int b0 = 0; b0 < n; b0 += batch) {
                if (__syncthreads_count(n_done == PPT) == nthreads) break;
                const int cnt = min(batch, n - b0);
                load_batch<NF>(a, C, range.x, b0, cnt, ti.px0, ti.py0, rec_base, s_geo0, s_geo1, s_geo2, s_feat,
                               nullptr, nthreads);
                __syncthreads();
                if (__all_sync(SG_FULL_MASK, n_done == PPT)) continue;
                // 32 entries at a time: lane l tests entry j0 + l against the warp's sub-tile, and
                // the warp walks the entries that can reach it, front to back
                for (int j0 = 0; j0 < cnt; j0 += 32) {
                    if (__all_sync(SG_FULL_MASK, n_done == PPT)) break;
                    const int jl = j0 + lane;
                    uint32_t cm = __ballot_sync(SG_FULL_MASK, jl < cnt && !wt.misses(s_geo2[jl], s_geo1[jl], ln_amin));
                    while (cm) {
                        const int j = j0 + __ffs(cm) - 1;
                        cm &= cm - 1;
                        entry(j, b0 + j);
                    }
                }
            }
        } else {
            // list positions whose half mask holds this half, ascending: (s_q, s_qr)[0 .. qn)
            // is the queue of (position, record), top the next position scanned
            const uint32_t lt = (1u << lane) - 1u;
            int top = 0, qn = 0;
            while (!__all_sync(SG_FULL_MASK, n_done == PPT)) {
                while (qn < kFwdHalfChunk && top < n) {
                    const int pos = top + lane;
                    uint32_t rec = 0u;
                    bool sel = false;
                    if (pos < n) {
                        const uint32_t word = a.record[range.x + pos];  // record | half mask << 30
                        rec = word & 0x3fffffffu;
                        sel = (word >> (30 + hf)) & 1u;
                    }
                    const uint32_t bal = __ballot_sync(SG_FULL_MASK, sel);
                    if (sel) {
                        s_q[qn + __popc(bal & lt)] = pos;
                        s_qr[qn + __popc(bal & lt)] = rec;
                    }
                    qn += __popc(bal);
                    top += 32;
                    __syncwarp();
                }
                if (qn == 0) break;
                const int c = min(kFwdHalfChunk, qn);
                stage_rows_warp<NF>(a, C, [&](int j) { return s_qr[j]; }, c, ti.px0, ti.py0, rec_base, s_geo0, s_geo1,
                                    nullptr, s_feat, nullptr);
                __syncwarp();
                for (int j = 0; j < c; ++j) {
                    if (__all_sync(SG_FULL_MASK, n_done == PPT)) break;
                    entry(j, s_q[j]);
                }
                __syncwarp();
                // drop the staged entries from the queue
                const int rest = qn - c;  // (< 32)
                const int keep = lane < rest ? s_q[c + lane] : 0;
                const uint32_t keep_rec = lane < rest ? s_qr[c + lane] : 0u;
                __syncwarp();
                if (lane < rest) {
                    s_q[lane] = keep;
                    s_qr[lane] = keep_rec;
                }
                qn = rest;
                __syncwarp();
            }
        }
        const size_t HW = (size_t)vw.W * vw.H;
        const size_t p0 = (size_t)vw.pixel_offset;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int py = ti.py0 + wt.ly + 4 * k;
            if (!(px < vw.W && py < vw.H)) continue;
            const size_t p = (size_t)py * vw.W + px;
            a.img_rgb[3 * p0 + p] = acc[k][0] + T[k] * a.bg0;
            a.img_rgb[3 * p0 + HW + p] = acc[k][1] + T[k] * a.bg1;
            a.img_rgb[3 * p0 + 2 * HW + p] = acc[k][2] + T[k] * a.bg2;
            a.img_depth[p0 + p] = acc[k][3];
#pragma unroll
            for (int c = 0; c < C; ++c) a.img_sem[(size_t)C * p0 + c * HW + p] = acc[k][4 + c];
            a.T_final[p0 + p] = T[k];
            a.last[p0 + p] = last[k];
            a.n_contrib[p0 + p] = nc[k];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Backward helpers
// ---------------------------------------------------------------------------------------

// The backward works on chunks of 16 consecutive list entries.  Three of its sums are
// contractions over the warp's pixels and run on the tensor cores (mma.m16n8k8, TF32
// operands split as x = hi + lo, hi = x with its 13 low mantissa bits cleared, lo = x - hi
// exactly; hi*hi + hi*lo + lo*hi keeps about 22 mantissa bits of every product, i.e.
// FP32-level accuracy):
//   gf[p][r] = sum_f g[p][f] F[r][f]          (pixel gradient . Gaussian features)
//   dF[r][f] = sum_p w[p][r] g[p][f]          (colour / depth / semantic gradients)
//   M[r][m]  = sum_p s[p][r] P_m(X_p, Y_p)    (moments of s = dL/dsigma)
// with w = alpha T and P = (1, X, Y, X^2, XY, Y^2) the pixel offsets from the warp centre.
// The 2D-mean, conic and opacity gradients are linear in the moments (see moment_grads).
constexpr int kChunk = 16;
constexpr int kHalfQueue = kChunk + 32;  // half mode: list positions pending (< 16 + one 32-entry scan)

template <int NPX>
__host__ __device__ constexpr int chunk_pitch() { return NPX + 4; }  // 4 mod 32: conflict-free fragments

template <int NF>
__host__ __device__ constexpr int padded_features() { return (NF + 7) / 8 * 8; }

// Row pitch of the per-warp copy of dL/dimage: the least odd multiple of 4 that holds the NF
// features (conflict-free fragment loads).  Features NF .. padded_features - 1 of the last
// 8-feature tile are not stored: their fragment loads are predicated to zero.
template <int NF>
__host__ __device__ constexpr int g_pitch() { return (NF / 4) % 2 == 1 ? NF : NF + 4; }

// shared memory of one warp: G (NPX x g_pitch) and two chunk buffers (16 x chunk_pitch)
template <int C, int PPT>
__host__ __device__ constexpr int bwd_warp_floats() {
    return 32 * PPT * g_pitch<4 + C>() + 2 * kChunk * chunk_pitch<32 * PPT>();
}

// A fragment (16 x 8, row-major, pitch ld) at column k0: a0 (gid, tig), a1 (gid + 8, tig),
// a2 (gid, tig + 4), a3 (gid + 8, tig + 4); rows outside `keep` read as zero, and so do
// columns k0 + 4 .. k0 + 7 unless `upper` (the part of the last feature tile that is not
// stored).
__device__ __forceinline__ void load_a_split(const float *m, int ld, int k0, int gid, int tig, bool keep0,
                                             bool keep1, uint32_t (&ah)[4], uint32_t (&al)[4],
                                             bool upper = true) {
    const float *p = m + gid * ld + k0 + tig;
    const float v[4] = {keep0 ? p[0] : 0.f, keep1 ? p[8 * ld] : 0.f, keep0 && upper ? p[4] : 0.f,
                        keep1 && upper ? p[8 * ld + 4] : 0.f};
#pragma unroll
    for (int i = 0; i < 4; ++i) split_tf32(v[i], ah[i], al[i]);
}

// Gradients of the 2D mean (u, v), the conic (a, b, c) and the opacity from the moments
// M = (sum s, sum s X, sum s Y, sum s X^2, sum s XY, sum s Y^2) of s = dL/dsigma over the
// pixels (X, Y offsets from the warp centre; U, V the mean's offset from it, so that
// dx = X - U, dy = Y - V).  With sigma = p1^2 + p2^2, p1 = m00 dx, p2 = m10 dx + m11 dy:
//   dL/du = -2 ((m00^2 + m10^2) S_x + m10 m11 S_y),  dL/dv = -2 (m10 m11 S_x + m11^2 S_y),
//   dL/d(a, b, c) = (S_xx / 2, S_xy, S_yy / 2),       dL/do = -S_1 / o,
// S_x = sum s dx, S_xx = sum s dx^2, ...; the last because s = -dL/dalpha alpha and
// dalpha/do = alpha / o wherever s is non-zero (alpha not clamped).  `part` (0..2) picks
// the pair this lane writes.
__device__ __forceinline__ void moment_grads(const float (&M)[6], float U, float V, const float4 &g1, int part,
                                             float &r0, float &r1) {
    const float M0 = M[0], Mx = M[1], My = M[2], Mxx = M[3], Mxy = M[4], Myy = M[5];
    if (part == 0) {
        const float Sx = fmaf(-U, M0, Mx), Sy = fmaf(-V, M0, My);
        const float m00 = g1.x, m10 = g1.y, m11 = g1.z;
        r0 = -2.f * ((m00 * m00 + m10 * m10) * Sx + m10 * m11 * Sy);
        r1 = -2.f * (m10 * m11 * Sx + m11 * m11 * Sy);
    } else if (part == 1) {
        r0 = 0.5f * (Mxx - 2.f * U * Mx + U * U * M0);
        r1 = Mxy - V * Mx - U * My + U * V * M0;
    } else {
        r0 = 0.5f * (Myy - 2.f * V * My + V * V * M0);
        r1 = -M0 / g1.w;
    }
}

// One pixel per thread and C = 4 or 16: at most 72 registers, so that occupancy is set by
// shared memory rather than registers (the adjoint is latency-bound and gains from warps):
// 13 CTAs of an 8 x 8 tile fit both (13 x 64 threads x 72 registers); 64 registers spilled
// nothing but measured 1 % slower, 80 cost a CTA.  The other widths keep the compiler's
// choice (with C >= 32 the staged entries hold occupancy lower than registers anyway).
template <int C, int PPT>
__host__ __device__ constexpr int bwd_max_regs() { return PPT == 1 && (C == 4 || C == 16) ? 72 : 255; }

template <int C, int PPT, bool HALF = false>
__global__ void __maxnreg__((bwd_max_regs<C, PPT>())) raster_bwd_kernel(RasterArgs a) {
    pdl_begin();
    constexpr int NF = 4 + C;                     // rgb(3) depth | sem(C)
    constexpr int NFP = padded_features<NF>();    // features padded to 8
    constexpr int NT = NFP / 8;                   // 8-feature tiles
    constexpr int NPX = 32 * PPT;                 // pixels of one warp (pixel q = 32 k + lane)
    constexpr int KS = NPX / 8;                   // 8-pixel steps
    constexpr int MT = NPX / 16;                  // 16-pixel tiles
    constexpr int WQ = chunk_pitch<NPX>();
    constexpr int GP = g_pitch<NF>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_max_last;
    // Half mode (8 x 8 tiles, one pixel per thread, half masks given): a CTA is one warp that
    // works on one half (8 x 4 pixels) of a tile at a time; it walks the tile's list back to
    // front, keeps the entries whose half mask holds its half in a queue, and stages and
    // processes them 16 at a time, so its chunks hold only its own entries; no block barrier.
    // Otherwise the CTA's warps share each batch of the list, staged between two block
    // barriers.
    constexpr bool hm = HALF;
    static_assert(!HALF || PPT == 1, "half mode runs one pixel per thread");
    const int batch = hm ? kChunk : a.batch;
    float4 *s_geo0 = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_geo1 = s_geo0 + batch;
    // (half mode stages no (u, v, ex, ey) rows: its entries passed the half's culling rule,
    // which rejects what the warp's ellipse test would)
    float4 *s_geo2 = hm ? nullptr : s_geo1 + batch;
    float *s_feat = reinterpret_cast<float *>(s_geo1 + (hm ? batch : 2 * batch));
    uint32_t *s_rec = reinterpret_cast<uint32_t *>(s_feat + (size_t)batch * NF);
    // half mode: the list position of each staged row, and the queue of pending entries
    // (list position, record)
    int *s_pos = reinterpret_cast<int *>(s_rec + batch);
    int *s_q = s_pos + (hm ? kChunk : 0);
    uint32_t *s_qr = reinterpret_cast<uint32_t *>(s_q + (hm ? kHalfQueue : 0));
    const int nthreads = hm ? 32 : a.tile_w * a.tile_h / PPT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *s_G = reinterpret_cast<float *>(s_qr + (hm ? kHalfQueue : 0)) + (size_t)warp * bwd_warp_floats<C, PPT>();
    float *s_gw = s_G + NPX * GP;     // per chunk row: gf, then overwritten with w = alpha T
    float *s_sg = s_gw + kChunk * WQ; // per chunk row: s = dL/dsigma
    const int gid = lane >> 2, tig = lane & 3;
    const WarpTile<PPT> wt(a.tile_w);
    const float fx = (float)wt.lx;
    const float ln_amin = __logf(a.alpha_min);
    // moment polynomials at the B-fragment pixels: pixel 8 ks + tig (+ 4) has X = tig - 3.5
    // (tig + 0.5), Y = (ks % 4) + 4 (ks / 4) - (2 PPT - 0.5); P_gid = P0 + Y (P1 + Y P2)
    // (all values small multiples of 1/4: exact in TF32, so B needs no split)
    const float X0 = tig - 3.5f, X1 = tig + 0.5f;
    const float P0a = gid == 0 ? 1.f : gid == 1 ? X0 : gid == 3 ? X0 * X0 : 0.f;
    const float P0b = gid == 0 ? 1.f : gid == 1 ? X1 : gid == 3 ? X1 * X1 : 0.f;
    const float P1a = gid == 2 ? 1.f : gid == 4 ? X0 : 0.f;
    const float P1b = gid == 2 ? 1.f : gid == 4 ? X1 : 0.f;
    const float P2 = gid == 5 ? 1.f : 0.f;
    // half mode: a work item is one half tile, or (half_pairs) a whole tile whose halves the
    // warp takes in turn, so that the second half's staging loads can hit L1
    const bool pairs = hm && a.half_pairs;
    const int n_items = hm && !pairs ? 2 * a.n_tiles : a.n_tiles;
    for (int iter = 0;; ++iter) {
        if (!a.persistent && iter > 0) break;
        const int slot = next_item(a, n_items, s_item);
        if (slot >= n_items) break;
        const int tslot = hm && !pairs ? slot >> 1 : slot;
        const int item = a.order ? a.order[tslot] : tslot;  // tile id
        const int hf0 = hm && !pairs ? slot & 1 : 0, hf1 = pairs ? 2 : hf0 + 1;
        for (int hf = hf0; hf < hf1; ++hf) {
        TileInfo ti = tile_info(a, item);
        ti.py0 += hf * (a.tile_h / 2);  // half mode: this warp's half
        const sg_view &vw = *ti.vw;
        const int px = ti.px0 + wt.lx;
        const int2 range = a.ranges[item];
        const size_t HW = (size_t)vw.W * vw.H;
        const size_t p0 = (size_t)vw.pixel_offset;
        const uint32_t rec_base = (uint32_t)ti.v * (uint32_t)a.N;
        float T[PPT], acc_a[PPT];
        int my_last[PPT];
        int thread_last = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int py = ti.py0 + wt.ly + 4 * k;
            const bool inside = px < vw.W && py < vw.H;
            const size_t p = (size_t)py * vw.W + px;
            float g[NFP];
#pragma unroll
            for (int f = 0; f < NFP; ++f) g[f] = 0.f;
            T[k] = 1.f;
            my_last[k] = 0;
            if (inside) {
                g[0] = a.dL_rgb[3 * p0 + p];
                g[1] = a.dL_rgb[3 * p0 + HW + p];
                g[2] = a.dL_rgb[3 * p0 + 2 * HW + p];
                g[3] = a.dL_depth[p0 + p];
#pragma unroll
                for (int c = 0; c < C; ++c) g[4 + c] = a.dL_sem[(size_t)C * p0 + c * HW + p];
                T[k] = a.T_final[p0 + p];
                my_last[k] = a.last[p0 + p];
            }
            acc_a[k] = g[0] * a.bg0 + g[1] * a.bg1 + g[2] * a.bg2;
            thread_last = max(thread_last, my_last[k]);
            float4 *row = reinterpret_cast<float4 *>(s_G + (32 * k + lane) * GP);
#pragma unroll
            for (int f = 0; f < NF; f += 4) row[f / 4] = make_float4(g[f], g[f + 1], g[f + 2], g[f + 3]);
        }
        const int warp_last = __reduce_max_sync(SG_FULL_MASK, thread_last);
        // One chunk of staged rows [jc0, jc0 + 16) (rows past jmax are left out), back to
        // front; pos_of(j) is the list position of row j.
        auto chunk = [&](const int jc0, const int jmax, auto pos_of) {
                // entries of the chunk whose footprint reaches the warp (lane r tests entry jc0 + r)
                bool cand = false;
                if (lane < kChunk)
                    cand = jc0 + lane < jmax && (hm || !wt.misses(s_geo2[jc0 + lane], s_geo1[jc0 + lane], ln_amin));
                uint32_t cmask = __ballot_sync(SG_FULL_MASK, cand);
                if (!cmask) return;
                // ---- gf = G F^T for the chunk (M = pixels, N = entries, K = features) ----
                if constexpr (MT <= 2) {
                    // features outside, pixel tiles inside: every F fragment is split once
                    float d[MT][2][4];
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.f;
#pragma unroll
                    for (int kk = 0; kk < NT; ++kk) {
                        const int f0 = 8 * kk + tig;
                        uint32_t bh[2][2], bl[2][2];
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt) {
                            const float *fr = s_feat + (size_t)(jc0 + 8 * nt + gid) * NF;
                            split_tf32(f0 < NF ? fr[f0] : 0.f, bh[nt][0], bl[nt][0]);
                            split_tf32(f0 + 4 < NF ? fr[f0 + 4] : 0.f, bh[nt][1], bl[nt][1]);
                        }
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt) {
                            uint32_t ah[4], al[4];
                            load_a_split(s_G + 16 * mt * GP, GP, 8 * kk, gid, tig, true, true, ah, al,
                                         8 * kk + 4 < NF);
#pragma unroll
                            for (int nt = 0; nt < 2; ++nt)
                                mma_tf32x3(d[mt][nt], ah, al, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
                        }
                    }
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                s_gw[(8 * nt + 2 * tig + (i & 1)) * WQ + 16 * mt + gid + 8 * (i >> 1)] = d[mt][nt][i];
                } else
#pragma unroll 1
                for (int mt = 0; mt < MT; ++mt) {
                    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
                    for (int kk = 0; kk < NT; ++kk) {
                        // B (8 x 8): b0 (tig, gid), b1 (tig + 4, gid) = F[entry][feature]
                        const int f0 = 8 * kk + tig;
                        uint32_t ah[4], al[4];
                        load_a_split(s_G + 16 * mt * GP, GP, 8 * kk, gid, tig, true, true, ah, al,
                                     8 * kk + 4 < NF);
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt) {
                            const float *fr = s_feat + (size_t)(jc0 + 8 * nt + gid) * NF;
                            uint32_t bh0, bl0, bh1, bl1;
                            split_tf32(f0 < NF ? fr[f0] : 0.f, bh0, bl0);
                            split_tf32(f0 + 4 < NF ? fr[f0 + 4] : 0.f, bh1, bl1);
                            mma_tf32x3(d[nt], ah, al, bh0, bh1, bl0, bl1);
                        }
                    }
                    // D (16 x 8): d0 (gid, 2 tig), d1 (gid, 2 tig + 1), d2 (gid + 8, 2 tig), d3 (gid + 8, 2 tig + 1)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            s_gw[(8 * nt + 2 * tig + (i & 1)) * WQ + 16 * mt + gid + 8 * (i >> 1)] = d[nt][i];
                }
                __syncwarp();
                // ---- back to front over the candidates: T, dL/dalpha, w and s per pixel ----
                uint32_t mask = 0;
                while (cmask) {
                    const int r = 31 - __clz(cmask);
                    cmask &= ~(1u << r);
                    const int j = jc0 + r;
                    const float4 g0 = s_geo0[j];
                    const float4 g1 = s_geo1[j];
                    const int pos = pos_of(j);
                    AlphaEval e[PPT];
                    bool hit[PPT];
                    bool any = false;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        hit[k] = pos < my_last[k] &&
                                 eval_alpha(fx - g0.x, (float)(wt.ly + 4 * k) - g0.y, g0.z, g0.w, g1.x, g1.y, g1.z,
                                            g1.w, a.alpha_max, a.alpha_min, e[k]);
                        any |= hit[k];
                    }
                    if (!__any_sync(SG_FULL_MASK, any)) continue;
                    mask |= 1u << r;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        float *gw = s_gw + r * WQ + 32 * k + lane;
                        float w = 0.f, sg = 0.f;
                        if (hit[k]) {
                            const float gf = *gw;
                            // transmittance before this Gaussian (only gradients depend on it)
                            T[k] = __fdividef(T[k], __fsub_rn(1.f, e[k].alpha));
                            const float dalpha = T[k] * (gf - acc_a[k]);
                            acc_a[k] = e[k].alpha * gf + (1.f - e[k].alpha) * acc_a[k];
                            w = e[k].alpha * T[k];
                            if (e[k].raw < a.alpha_max) sg = -dalpha * e[k].raw;
                        }
                        *gw = w;
                        s_sg[r * WQ + 32 * k + lane] = sg;
                    }
                }
                if (!mask) return;  // (warp-uniform)
                __syncwarp();
                // ---- dF = W G (M = entries, N = features, K = pixels), moments M = S P ----
                const bool keep0 = (mask >> gid) & 1u, keep1 = (mask >> (gid + 8)) & 1u;
                float df[NT][4], mom[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) df[nt][0] = df[nt][1] = df[nt][2] = df[nt][3] = 0.f;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    uint32_t ah[4], al[4];
                    load_a_split(s_gw, WQ, 8 * ks, gid, tig, keep0, keep1, ah, al);
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        // B (8 x 8): b0 (tig, gid), b1 (tig + 4, gid) = G[pixel][feature]
                        const float *gp = s_G + (8 * ks + tig) * GP + 8 * nt + gid;
                        const bool stored = 8 * nt + 8 <= NF || 8 * nt + gid < NF;
                        uint32_t bh0, bl0, bh1, bl1;
                        split_tf32(stored ? gp[0] : 0.f, bh0, bl0);
                        split_tf32(stored ? gp[4 * GP] : 0.f, bh1, bl1);
                        mma_tf32x3(df[nt], ah, al, bh0, bh1, bl0, bl1);
                    }
                    load_a_split(s_sg, WQ, 8 * ks, gid, tig, keep0, keep1, ah, al);
                    const float Y = (float)((ks & 3) + 4 * (ks >> 2)) - (2.f * PPT - 0.5f);
                    const uint32_t pb0 = __float_as_uint(fmaf(Y, fmaf(Y, P2, P1a), P0a));
                    const uint32_t pb1 = __float_as_uint(fmaf(Y, fmaf(Y, P2, P1b), P0b));
                    mma_tf32(mom, al, pb0, pb1);
                    mma_tf32(mom, ah, pb0, pb1);
                }
                // feature gradients: D rows gid, gid + 8 (entries), columns 2 tig, 2 tig + 1 (features)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    if (!(hr ? keep1 : keep0)) continue;
                    const uint32_t rec = s_rec[jc0 + gid + 8 * hr];
                    const uint32_t gi = rec - rec_base;
                    const size_t si = (size_t)C * (a.sem_rec ? rec : gi);
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        // features 2 tig, 2 tig + 1 of this n-tile: both semantic (C even) ->
                        // one 8-byte vector reduction when the buffer allows it
                        const int f0 = 8 * nt + 2 * tig;
                        if (a.sem_v2 && f0 >= 4 && f0 + 1 < NF) {
                            red_add_v2(a.g_sem + si + (f0 - 4), df[nt][2 * hr], df[nt][2 * hr + 1]);
                            continue;
                        }
#pragma unroll
                        for (int c2 = 0; c2 < 2; ++c2) {
                            const int f = f0 + c2;
                            const float val = df[nt][2 * hr + c2];
                            if (f >= NF) continue;
                            if (f < 3)
                                atomicAdd(a.g_col + (size_t)a.col_stride * (a.col_rec ? rec : gi) + f, val);
                            else if (f == 3)
                                atomicAdd(a.g2d + 8 * (size_t)rec + 6, val);
                            else
                                atomicAdd(a.g_sem + si + (f - 4), val);
                        }
                    }
                }
                // geometric gradients: lane tig of a quad holds moments (2 tig, 2 tig + 1) of its rows
                float Mr[2][6];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const int src = (lane & ~3) | t;
                    Mr[0][2 * t] = __shfl_sync(SG_FULL_MASK, mom[0], src);
                    Mr[0][2 * t + 1] = __shfl_sync(SG_FULL_MASK, mom[1], src);
                    Mr[1][2 * t] = __shfl_sync(SG_FULL_MASK, mom[2], src);
                    Mr[1][2 * t + 1] = __shfl_sync(SG_FULL_MASK, mom[3], src);
                }
                if (tig < 3) {
#pragma unroll
                    for (int hr = 0; hr < 2; ++hr) {
                        if (!(hr ? keep1 : keep0)) continue;
                        const int j = jc0 + gid + 8 * hr;
                        const float4 g0 = s_geo0[j];
                        const float4 g1 = s_geo1[j];
                        const float U = (g0.x - wt.cxw) + g0.z, V = (g0.y - wt.cyw) + g0.w;
                        float r0, r1;
                        moment_grads(Mr[hr], U, V, g1, tig, r0, r1);
                        float *dst = a.g2d + 8 * (size_t)s_rec[j] + 2 * tig;
                        atomicAdd(dst, r0);
                        atomicAdd(dst + 1, r1);
                    }
                }
                __syncwarp();  // the chunk buffers are rewritten next
        };
        if (!hm) {
            if (threadIdx.x == 0) s_max_last = 0;
            __syncthreads();
            if (lane == 0 && warp_last > 0) atomicMax(&s_max_last, warp_last);
            __syncthreads();
            const int max_last = s_max_last;
            const int n_batches = (max_last + batch - 1) / batch;
            for (int b = n_batches - 1; b >= 0; --b) {
                const int b0 = b * batch;
                const int cnt = min(batch, max_last - b0);
                __syncthreads();
                load_batch<NF>(a, C, range.x, b0, cnt, ti.px0, ti.py0, rec_base, s_geo0, s_geo1, s_geo2, s_feat,
                               s_rec, nthreads);
                __syncthreads();
                const int jmax = min(cnt, warp_last - b0);  // warp-uniform
                for (int jc0 = jmax > 0 ? (jmax - 1) & ~(kChunk - 1) : -kChunk; jc0 >= 0; jc0 -= kChunk)
                    chunk(jc0, jmax, [b0](int j) { return b0 + j; });
            }
            __syncthreads();
        } else {
            // list positions < warp_last whose half mask holds this half, in descending order:
            // (s_q, s_qr)[0 .. qn) is the queue of (position, record), top the next position
            // scanned (exclusive)
            const uint32_t lt = (1u << lane) - 1u;
            int top = warp_last, qn = 0;
            for (;;) {
                while (qn < kChunk && top > 0) {
                    const int pos = top - 1 - lane;
                    uint32_t rec = 0u;
                    bool sel = false;
                    if (pos >= 0) {
                        const uint32_t word = a.record[range.x + pos];  // record | half mask << 30
                        rec = word & 0x3fffffffu;
                        sel = (word >> (30 + hf)) & 1u;
                    }
                    const uint32_t bal = __ballot_sync(SG_FULL_MASK, sel);
                    if (sel) {
                        s_q[qn + __popc(bal & lt)] = pos;
                        s_qr[qn + __popc(bal & lt)] = rec;
                    }
                    qn += __popc(bal);
                    top = max(top - 32, 0);
                    __syncwarp();
                }
                if (qn == 0) break;
                const int c = min(kChunk, qn);
                // rows 0 .. c-1 in ascending list position: row r is queue entry c - 1 - r
                stage_rows_warp<NF>(a, C, [&](int j) { return s_qr[c - 1 - j]; }, c, ti.px0, ti.py0, rec_base, s_geo0,
                                    s_geo1, s_geo2, s_feat, s_rec);
                if (lane < c) s_pos[lane] = s_q[c - 1 - lane];
                const int rest = qn - c;  // (< 32)
                const int keep = lane < rest ? s_q[c + lane] : 0;
                const uint32_t keep_rec = lane < rest ? s_qr[c + lane] : 0u;
                __syncwarp();
                if (lane < rest) {
                    s_q[lane] = keep;
                    s_qr[lane] = keep_rec;
                }
                qn = rest;
                __syncwarp();
                chunk(0, c, [s_pos](int j) { return s_pos[j]; });
            }
            __syncwarp();
        }
        }
    }
}

// ---------------------------------------------------------------------------------------

template <int C>
inline size_t fwd_smem(int batch) {
    return (size_t)batch * (3 * 16 + 4 * (4 + C));
}
template <int C, int PPT>
inline size_t bwd_smem(int batch, int threads) {
    return fwd_smem<C>(batch) + (size_t)batch * 4 + sizeof(float) * (threads / 32) * bwd_warp_floats<C, PPT>();
}
// half mode: one 16-entry chunk staged without its (u, v, ex, ey) rows (+ its list positions),
// the (position, record) queue, one warp
template <int C>
inline size_t bwd_half_smem() {
    return fwd_smem<C>(kChunk) - (size_t)kChunk * 16 + (size_t)kChunk * 4 * 2 + (size_t)kHalfQueue * 4 * 2 +
           sizeof(float) * bwd_warp_floats<C, 1>();
}

// forward half mode: one 32-entry chunk staged without its (u, v, ex, ey) rows, and the
// (position, record) queue
template <int C>
inline size_t fwd_half_smem() {
    return (size_t)kFwdHalfChunk * (2 * 16 + 4 * (4 + C)) + (size_t)kFwdHalfQueue * 4 * 2;
}

inline int resident_grid(const void *fn, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

template <int C, int PPT>
sg_status launch_raster_cp(RasterArgs &a, bool backward, cudaStream_t st) {
    // with half masks, the adjoint of 8 x 8 tiles at one pixel per thread runs one warp per
    // half tile, and so does the forward when the config asks for it
    const bool half = a.half && PPT == 1 && a.tile_w == 8 && a.tile_h == 8 && (backward || a.half_fwd);
    const int threads = half ? 32 : a.tile_w * a.tile_h / PPT;
    const size_t smem = backward ? (half ? bwd_half_smem<C>() : bwd_smem<C, PPT>(a.batch, threads))
                                 : (half ? fwd_half_smem<C>() : fwd_smem<C>(a.batch));
    const void *fn = backward ? (half ? (const void *)raster_bwd_kernel<C, PPT, PPT == 1>
                                      : (const void *)raster_bwd_kernel<C, PPT>)
                              : (half ? (const void *)raster_fwd_kernel<C, PPT, PPT == 1>
                                      : (const void *)raster_fwd_kernel<C, PPT>);
    // opt in to the dynamic size whenever it grows: at 48 KB and just below, the kernel's
    // static shared variables alone take the total past the default limit
    static size_t configured[4] = {0, 0, 0, 0};
    const int which = 2 * (int)backward + (int)half;
    if (configured[which] < smem) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return check_launch("raster smem attribute");
        configured[which] = smem;
    }
    // the half-tile adjoint takes whole tiles as work items when there are at least 16 tiles
    // per resident CTA (measured: batched workload, 29 per CTA, -1.4 %); with fewer, twice as
    // long items leave the persistent grid's tail unbalanced
    const int resident = a.persistent ? resident_grid(fn, threads, smem) : 0;
    a.half_pairs = backward && half && a.persistent && (int64_t)a.n_tiles >= 16 * (int64_t)resident;
    const int n_items = half && !a.half_pairs ? 2 * a.n_tiles : a.n_tiles;
    int grid = n_items;
    if (a.persistent) {
        grid = resident;
        if (grid > n_items) grid = n_items;
    }
    if (grid <= 0) return SG_OK;
    if (backward && half)
        launch_pdl(raster_bwd_kernel<C, PPT, PPT == 1>, grid, threads, smem, st, a);
    else if (backward)
        launch_pdl(raster_bwd_kernel<C, PPT>, grid, threads, smem, st, a);
    else if (half)
        launch_pdl(raster_fwd_kernel<C, PPT, PPT == 1>, grid, threads, smem, st, a);
    else
        launch_pdl(raster_fwd_kernel<C, PPT>, grid, threads, smem, st, a);
    count_launches(1);
    return check_launch(backward ? "raster_bwd" : "raster_fwd");
}

template <int C>
sg_status launch_raster_c(RasterArgs &a, bool backward, cudaStream_t st) {
    switch (a.ppt) {
        case 1: return launch_raster_cp<C, 1>(a, backward, st);
        case 2: return launch_raster_cp<C, 2>(a, backward, st);
        default: return launch_raster_cp<C, 4>(a, backward, st);
    }
}

}  // namespace sg
