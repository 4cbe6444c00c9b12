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
// (shared-memory loads, the warp reduction of the backward) is shared by PPT pixels.
//
// Forward: the tile's depth-sorted list is walked in batches the CTA stages into shared
// memory; each pixel composites front to back and stops when T would fall below T_min;
// the CTA leaves the tile when all pixels are done.  Saved per pixel: T_final, last (list
// entries examined up to and including the last contributor), contributor count.
//
// Backward: back to front from the tile's largest `last`.  Each pixel rebuilds T by
// dividing by (1 - alpha) and tracks only the scalar a = g . A of the background-weighted
// suffix colour A.  A thread sums its pixels' 10 + C partial gradients of a Gaussian; the
// warp then adds its 32 lanes with a lane-transposed butterfly (NV - 1 shuffles for NV
// values) and issues one warp-wide set of atomics.
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
        const uint32_t rec = a.record[list_start + b0 + j];
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
        float *f = s_feat + (size_t)j * NF;
        f[0] = a.rgb[3 * (size_t)gi];
        f[1] = a.rgb[3 * (size_t)gi + 1];
        f[2] = a.rgb[3 * (size_t)gi + 2];
        f[3] = g0.z;  // depth (camera z of the mean, Eq. 8)
        const float4 *s4 = reinterpret_cast<const float4 *>(a.sem + (size_t)gi * C);
        float4 *f4 = reinterpret_cast<float4 *>(f + 4);
#pragma unroll
        for (int k = 0; k < (NF - 4) / 4; ++k) f4[k] = s4[k];
        if (s_rec) s_rec[j] = rec;
    }
}

__device__ __forceinline__ int next_item(const RasterArgs &a, int &s_item) {
    if (!a.persistent) return blockIdx.x;
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
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

template <int C, int PPT>
__global__ void __launch_bounds__(kMaxTileThreads) raster_fwd_kernel(RasterArgs a) {
    constexpr int NF = 4 + C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int batch = a.batch;
    float4 *s_geo0 = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_geo1 = s_geo0 + batch;
    float4 *s_geo2 = s_geo1 + batch;
    float *s_feat = reinterpret_cast<float *>(s_geo2 + batch);
    const int nthreads = a.tile_w * a.tile_h / PPT;
    const WarpTile<PPT> wt(a.tile_w);
    const float fx = (float)wt.lx;
    for (int iter = 0;; ++iter) {
        if (!a.persistent && iter > 0) break;
        const int item = next_item(a, s_item);
        if (item >= a.n_tiles) break;
        const TileInfo ti = tile_info(a, item);
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
        for (int b0 = 0; b0 < n; b0 += batch) {
            if (__syncthreads_count(n_done == PPT) == nthreads) break;
            const int cnt = min(batch, n - b0);
            load_batch<NF>(a, C, range.x, b0, cnt, ti.px0, ti.py0, rec_base, s_geo0, s_geo1, s_geo2, s_feat,
                           nullptr, nthreads);
            __syncthreads();
            if (__all_sync(SG_FULL_MASK, n_done == PPT)) continue;
            for (int j = 0; j < cnt; ++j) {
                if (wt.misses(s_geo2[j])) continue;  // warp-uniform
                const float4 g0 = s_geo0[j];
                const float4 g1 = s_geo1[j];
                float w[PPT];
                bool any = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    w[k] = 0.f;
                    if (done[k]) continue;
                    AlphaEval e;
                    if (!eval_alpha(fx - g0.x, (float)(wt.ly + 4 * k) - g0.y, g0.z, g0.w, g1.x, g1.y, g1.z,
                                    g1.w, a.alpha_max, a.alpha_min, e))
                        continue;
                    const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, e.alpha));
                    if (Tn < a.T_min) {
                        done[k] = true;
                        ++n_done;
                        continue;
                    }
                    w[k] = e.alpha * T[k];
                    T[k] = Tn;
                    last[k] = b0 + j + 1;
                    ++nc[k];
                    any = true;
                }
                if (!any) continue;
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

template <int X>
struct NextPow2 {
    static constexpr int v = X <= 32 ? 32 : (X <= 64 ? 64 : (X <= 128 ? 128 : 256));
};

template <int C, int PPT>
__global__ void __launch_bounds__(kMaxTileThreads) raster_bwd_kernel(RasterArgs a) {
    constexpr int NF = 4 + C;
    constexpr int NRAW = 10 + C;  // u v ca cb cc o depth | rgb(3) | sem(C)
    constexpr int NV = NextPow2<NRAW>::v;
    constexpr int PER = NV / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_max_last;
    const int batch = a.batch;
    float4 *s_geo0 = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_geo1 = s_geo0 + batch;
    float4 *s_geo2 = s_geo1 + batch;
    float *s_feat = reinterpret_cast<float *>(s_geo2 + batch);
    uint32_t *s_rec = reinterpret_cast<uint32_t *>(s_feat + (size_t)batch * NF);
    const int nthreads = a.tile_w * a.tile_h / PPT;
    const int lane = threadIdx.x & 31;
    const WarpTile<PPT> wt(a.tile_w);
    const float fx = (float)wt.lx;
    for (int iter = 0;; ++iter) {
        if (!a.persistent && iter > 0) break;
        const int item = next_item(a, s_item);
        if (item >= a.n_tiles) break;
        const TileInfo ti = tile_info(a, item);
        const sg_view &vw = *ti.vw;
        const int px = ti.px0 + wt.lx;
        const int2 range = a.ranges[item];
        const size_t HW = (size_t)vw.W * vw.H;
        const size_t p0 = (size_t)vw.pixel_offset;
        const uint32_t rec_base = (uint32_t)ti.v * (uint32_t)a.N;
        float g[PPT][NF];
        float T[PPT], acc_a[PPT];
        int my_last[PPT];
        int thread_last = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int py = ti.py0 + wt.ly + 4 * k;
            const bool inside = px < vw.W && py < vw.H;
            const size_t p = (size_t)py * vw.W + px;
            if (inside) {
                g[k][0] = a.dL_rgb[3 * p0 + p];
                g[k][1] = a.dL_rgb[3 * p0 + HW + p];
                g[k][2] = a.dL_rgb[3 * p0 + 2 * HW + p];
                g[k][3] = a.dL_depth[p0 + p];
#pragma unroll
                for (int c = 0; c < C; ++c) g[k][4 + c] = a.dL_sem[(size_t)C * p0 + c * HW + p];
                T[k] = a.T_final[p0 + p];
                my_last[k] = a.last[p0 + p];
                acc_a[k] = g[k][0] * a.bg0 + g[k][1] * a.bg1 + g[k][2] * a.bg2;
            } else {
#pragma unroll
                for (int c = 0; c < NF; ++c) g[k][c] = 0.f;
                T[k] = 1.f;
                my_last[k] = 0;
                acc_a[k] = 0.f;
            }
            thread_last = max(thread_last, my_last[k]);
        }
        const int warp_last = __reduce_max_sync(SG_FULL_MASK, thread_last);
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
            for (int j = jmax - 1; j >= 0; --j) {
                if (wt.misses(s_geo2[j])) continue;  // warp-uniform
                const float4 g0 = s_geo0[j];
                const float4 g1 = s_geo1[j];
                const int pos = b0 + j;
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
                float vals[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) vals[q] = 0.f;
                if (any) {
                    const float4 *f4 = reinterpret_cast<const float4 *>(s_feat + (size_t)j * NF);
                    float gf[PPT];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) gf[k] = 0.f;
#pragma unroll
                    for (int q = 0; q < NF / 4; ++q) {
                        const float4 f = f4[q];
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            gf[k] = fmaf(g[k][4 * q + 0], f.x, gf[k]);
                            gf[k] = fmaf(g[k][4 * q + 1], f.y, gf[k]);
                            gf[k] = fmaf(g[k][4 * q + 2], f.z, gf[k]);
                            gf[k] = fmaf(g[k][4 * q + 3], f.w, gf[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (!hit[k]) continue;
                        // transmittance before this Gaussian (only gradients depend on it)
                        T[k] = __fdividef(T[k], __fsub_rn(1.f, e[k].alpha));
                        const float dalpha = T[k] * (gf[k] - acc_a[k]);
                        acc_a[k] = e[k].alpha * gf[k] + (1.f - e[k].alpha) * acc_a[k];
                        const float w = e[k].alpha * T[k];
                        vals[6] = fmaf(w, g[k][3], vals[6]);
                        vals[7] = fmaf(w, g[k][0], vals[7]);
                        vals[8] = fmaf(w, g[k][1], vals[8]);
                        vals[9] = fmaf(w, g[k][2], vals[9]);
#pragma unroll
                        for (int c = 0; c < C; ++c) vals[10 + c] = fmaf(w, g[k][4 + c], vals[10 + c]);
                        if (e[k].raw < a.alpha_max) {
                            // sigma = p1^2 + p2^2, p1 = m00 dx, p2 = m10 dx + m11 dy; d(dx)/du = -1;
                            // d sigma / d(conic a, b, c) = (dx^2/2, dx dy, dy^2/2)
                            const float gsig = -dalpha * e[k].raw;
                            vals[0] -= 2.f * gsig * (e[k].p1 * g1.x + e[k].p2 * g1.y);
                            vals[1] -= 2.f * gsig * (e[k].p2 * g1.z);
                            vals[2] += 0.5f * gsig * e[k].dx * e[k].dx;
                            vals[3] += gsig * e[k].dx * e[k].dy;
                            vals[4] += 0.5f * gsig * e[k].dy * e[k].dy;
                            vals[5] += dalpha * e[k].G;
                        }
                    }
                }
                warp_transpose_reduce<NV>(vals, lane);
                const uint32_t rec = s_rec[j];
                const uint32_t gi = rec - rec_base;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const int idx = lane * PER + q;
                    if (idx < 7)
                        atomicAdd(a.g2d + 8 * (size_t)rec + idx, vals[q]);
                    else if (idx < 10)
                        atomicAdd(a.g_rgb + 3 * (size_t)gi + (idx - 7), vals[q]);
                    else if (idx < NRAW)
                        atomicAdd(a.g_sem + (size_t)C * gi + (idx - 10), vals[q]);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------

template <int C>
inline size_t fwd_smem(int batch) {
    return (size_t)batch * (3 * 16 + 4 * (4 + C));
}
template <int C>
inline size_t bwd_smem(int batch) {
    return fwd_smem<C>(batch) + (size_t)batch * 4;
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
    const int threads = a.tile_w * a.tile_h / PPT;
    const size_t smem = backward ? bwd_smem<C>(a.batch) : fwd_smem<C>(a.batch);
    const void *fn = backward ? (const void *)raster_bwd_kernel<C, PPT> : (const void *)raster_fwd_kernel<C, PPT>;
    static size_t configured[2] = {0, 0};
    if (smem > 48 * 1024 && configured[backward] < smem) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return check_launch("raster smem attribute");
        configured[backward] = smem;
    }
    int grid = a.n_tiles;
    if (a.persistent) {
        grid = resident_grid(fn, threads, smem);
        if (grid > a.n_tiles) grid = a.n_tiles;
        cudaMemsetAsync(a.work_counter, 0, sizeof(int), st);
    }
    if (grid <= 0) return SG_OK;
    if (backward)
        raster_bwd_kernel<C, PPT><<<grid, threads, smem, st>>>(a);
    else
        raster_fwd_kernel<C, PPT><<<grid, threads, smem, st>>>(a);
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
