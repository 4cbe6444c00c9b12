// raster.cu -- tile compositing of RGB, depth and C semantic channels (Eq. 7-9) and its
// adjoint (Sec. III-D backpropagation).
//
// One CTA owns one screen tile (tile_w x tile_h pixels, one pixel per thread) of one
// view-level.  Every view-level of every keyframe is addressed through one global tile
// id, so a single launch renders the whole pyramid of all keyframes; with `persistent`
// set, a grid of resident CTAs pulls tile ids from an atomic work counter.
//
// Forward: the tile's depth-sorted list is walked in batches that the CTA stages into
// shared memory (geometry 24 B + features 4*(4+C) B per Gaussian); each thread then
// composites front to back and stops when T would fall below T_min; a CTA leaves the
// tile as soon as all its threads are done (__syncthreads_count).  Saved per pixel:
// T_final, last (list entries examined up to and including the last contributor) and
// the contributor count.
//
// Backward: the list is walked back to front from the tile's largest `last`.  Each pixel
// rebuilds T by dividing by (1 - alpha) and tracks the scalar a = g . A of the
// background-weighted suffix colour A (only its dot product with the upstream gradient
// g is ever needed), so per Gaussian the work is one (4+C)-long dot product.  The 10+C
// per-Gaussian partial gradients of a warp are summed with a lane-transposed butterfly
// (NV-1 shuffles for NV values) and issued as one warp-wide set of atomics.
#include <cstdio>

#include "raster.cuh"

namespace sg {



// Stages entries [b0, b0 + cnt) of a tile's list.  Per entry:
//   s_geo0 = (ui - px0, vi - py0, uf, vf): integer part of the 2D mean relative to the tile
//            origin (exact in float) and its float fraction,
//   s_geo1 = (m00, m10, m11, opacity),
//   s_geo2 = (u, v, ex, ey): approximate tile-relative mean and conservative half extents of
//            the alpha >= alpha_min region, used only by the warp-level skip test,
// and the 4 + C features.
template <int NF>
__device__ __forceinline__ void load_batch(const RasterArgs &a, int C, int list_start, int b0,
                                           int cnt, int px0, int py0, float4 *s_geo0,
                                           float4 *s_geo1, float4 *s_geo2, float *s_feat,
                                           uint32_t *s_rec, int nthreads) {
    for (int j = threadIdx.x; j < cnt; j += nthreads) {
        const uint32_t rec = a.record[list_start + b0 + j];
        const float4 g0 = a.geo[2 * (size_t)rec];
        const float4 g1 = a.geo[2 * (size_t)rec + 1];
        const uint32_t packed = __float_as_uint(g1.w);
        const float uI = (float)((int)(short)(packed & 0xffffu) - px0);
        const float vI = (float)((int)(short)(packed >> 16) - py0);
        // sigma > thr outside |dx| > sqrt(thr)/m00 and |dy| > sqrt(thr (1 + (m10/m00)^2))/m11;
        // thr + 1e-3 and the 1% / 0.05 px margins keep the test strictly conservative
        const float thr = logf(g0.w / a.alpha_min) + 1e-3f;
        const float r = g1.y / g1.x;
        const float ex = sqrtf(thr) / g1.x * 1.01f + 0.05f;
        const float ey = sqrtf(thr * (1.f + r * r)) / g1.z * 1.01f + 0.05f;
        s_geo0[j] = make_float4(uI, vI, g0.x, g0.y);
        s_geo1[j] = make_float4(g1.x, g1.y, g1.z, g0.w);
        s_geo2[j] = make_float4(uI + g0.x, vI + g0.y, ex, ey);
        const uint32_t gi = rec % (uint32_t)a.N;
        float *f = s_feat + (size_t)j * NF;
        f[0] = a.rgb[3 * (size_t)gi];
        f[1] = a.rgb[3 * (size_t)gi + 1];
        f[2] = a.rgb[3 * (size_t)gi + 2];
        f[3] = g0.z;  // depth (camera z of the mean, Eq. 8)
        const float4 *s4 = reinterpret_cast<const float4 *>(a.sem + (size_t)gi * C);
        float4 *f4 = reinterpret_cast<float4 *>(f + 4);
#pragma unroll
        for (int k = 0; k < C / 4; ++k) f4[k] = s4[k];
        if (s_rec) s_rec[j] = rec;
    }
}

__device__ __forceinline__ int next_item(const RasterArgs &a, int &s_item) {
    if (!a.persistent) return blockIdx.x;
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
    __syncthreads();
    return s_item;
}

// Thread -> pixel map: each warp owns an 8 x 4 sub-tile, so that a Gaussian's footprint
// touches few warps and whole warps can skip it with one uniform test.
struct WarpTile {
    int lx, ly;        // pixel relative to the tile origin
    float cxw, cyw;    // centre of the warp's 8 x 4 sub-tile
    __device__ WarpTile(int tile_w) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int warps_x = tile_w >> 3;
        const int wx = (warp % warps_x) * 8, wy = (warp / warps_x) * 4;
        lx = wx + (lane & 7);
        ly = wy + (lane >> 3);
        cxw = wx + 3.5f;
        cyw = wy + 1.5f;
    }
    // true if no pixel of the warp's sub-tile can reach alpha_min (g2 = u, v, ex, ey)
    __device__ __forceinline__ bool misses(const float4 &g2) const {
        return fabsf(g2.x - cxw) > g2.z + 3.5f || fabsf(g2.y - cyw) > g2.w + 1.5f;
    }
};

template <int C>
__global__ void __launch_bounds__(kMaxTileThreads) raster_fwd_kernel(RasterArgs a) {
    constexpr int NF = 4 + C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int batch = a.batch;
    float4 *s_geo0 = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_geo1 = s_geo0 + batch;
    float4 *s_geo2 = s_geo1 + batch;
    float *s_feat = reinterpret_cast<float *>(s_geo2 + batch);
    const int nthreads = a.tile_w * a.tile_h;
    const WarpTile wt(a.tile_w);
    const float fx = (float)wt.lx, fy = (float)wt.ly;
    for (int iter = 0;; ++iter) {
        if (!a.persistent && iter > 0) break;
        const int item = next_item(a, s_item);
        if (item >= a.n_tiles) break;
        const int v = find_view(a.views, a.n_views, item);
        const sg_view &vw = a.views[v];
        const int local = item - vw.tile_offset;
        const int px0 = (local % vw.tiles_x) * a.tile_w, py0 = (local / vw.tiles_x) * a.tile_h;
        const int px = px0 + wt.lx, py = py0 + wt.ly;
        const bool inside = px < vw.W && py < vw.H;
        const int2 range = a.ranges[item];
        const int n = range.y - range.x;
        float acc[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) acc[k] = 0.f;
        float T = 1.f;
        int last = 0, nc = 0;
        bool done = !inside;
        for (int b0 = 0; b0 < n; b0 += batch) {
            if (__syncthreads_count(done) == nthreads) break;
            const int cnt = min(batch, n - b0);
            load_batch<NF>(a, C, range.x, b0, cnt, px0, py0, s_geo0, s_geo1, s_geo2, s_feat, nullptr,
                           nthreads);
            __syncthreads();
            if (__all_sync(SG_FULL_MASK, done)) continue;
            for (int j = 0; j < cnt; ++j) {
                if (wt.misses(s_geo2[j])) continue;  // warp-uniform
                if (done) continue;
                const float4 g0 = s_geo0[j];
                const float4 g1 = s_geo1[j];
                AlphaEval e;
                if (!eval_alpha(fx - g0.x, fy - g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, a.alpha_max,
                                a.alpha_min, e))
                    continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, e.alpha));
                if (Tn < a.T_min) {
                    done = true;
                    continue;
                }
                const float w = e.alpha * T;
                const float4 *f4 = reinterpret_cast<const float4 *>(s_feat + (size_t)j * NF);
#pragma unroll
                for (int k = 0; k < NF / 4; ++k) {
                    const float4 f = f4[k];
                    acc[4 * k + 0] = fmaf(w, f.x, acc[4 * k + 0]);
                    acc[4 * k + 1] = fmaf(w, f.y, acc[4 * k + 1]);
                    acc[4 * k + 2] = fmaf(w, f.z, acc[4 * k + 2]);
                    acc[4 * k + 3] = fmaf(w, f.w, acc[4 * k + 3]);
                }
                T = Tn;
                last = b0 + j + 1;
                ++nc;
            }
        }
        if (inside) {
            const size_t HW = (size_t)vw.W * vw.H;
            const size_t p = (size_t)py * vw.W + px;
            const size_t p0 = (size_t)vw.pixel_offset;
            a.img_rgb[3 * p0 + p] = acc[0] + T * a.bg0;
            a.img_rgb[3 * p0 + HW + p] = acc[1] + T * a.bg1;
            a.img_rgb[3 * p0 + 2 * HW + p] = acc[2] + T * a.bg2;
            a.img_depth[p0 + p] = acc[3];
#pragma unroll
            for (int k = 0; k < C; ++k) a.img_sem[(size_t)C * p0 + k * HW + p] = acc[4 + k];
            a.T_final[p0 + p] = T;
            a.last[p0 + p] = last;
            a.n_contrib[p0 + p] = nc;
        }
        __syncthreads();
    }
}

template <int X>
struct NextPow2 {
    static constexpr int v = X <= 32 ? 32 : (X <= 64 ? 64 : (X <= 128 ? 128 : 256));
};

template <int C>
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
    const int nthreads = a.tile_w * a.tile_h;
    const int lane = threadIdx.x & 31;
    const WarpTile wt(a.tile_w);
    const float fx = (float)wt.lx, fy = (float)wt.ly;
    for (int iter = 0;; ++iter) {
        if (!a.persistent && iter > 0) break;
        const int item = next_item(a, s_item);
        if (item >= a.n_tiles) break;
        const int v = find_view(a.views, a.n_views, item);
        const sg_view &vw = a.views[v];
        const int local = item - vw.tile_offset;
        const int px0 = (local % vw.tiles_x) * a.tile_w, py0 = (local / vw.tiles_x) * a.tile_h;
        const int px = px0 + wt.lx, py = py0 + wt.ly;
        const bool inside = px < vw.W && py < vw.H;
        const int2 range = a.ranges[item];
        const size_t HW = (size_t)vw.W * vw.H;
        const size_t p = (size_t)py * vw.W + px;
        const size_t p0 = (size_t)vw.pixel_offset;
        float g[NF];
        float T = 1.f, acc_a = 0.f;
        int my_last = 0;
        if (inside) {
            g[0] = a.dL_rgb[3 * p0 + p];
            g[1] = a.dL_rgb[3 * p0 + HW + p];
            g[2] = a.dL_rgb[3 * p0 + 2 * HW + p];
            g[3] = a.dL_depth[p0 + p];
#pragma unroll
            for (int k = 0; k < C; ++k) g[4 + k] = a.dL_sem[(size_t)C * p0 + k * HW + p];
            T = a.T_final[p0 + p];
            my_last = a.last[p0 + p];
            acc_a = g[0] * a.bg0 + g[1] * a.bg1 + g[2] * a.bg2;
        } else {
#pragma unroll
            for (int k = 0; k < NF; ++k) g[k] = 0.f;
        }
        const int warp_last = __reduce_max_sync(SG_FULL_MASK, my_last);
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
            load_batch<NF>(a, C, range.x, b0, cnt, px0, py0, s_geo0, s_geo1, s_geo2, s_feat, s_rec,
                           nthreads);
            __syncthreads();
            const int jmax = min(cnt, warp_last - b0);  // warp-uniform
            for (int j = jmax - 1; j >= 0; --j) {
                if (wt.misses(s_geo2[j])) continue;  // warp-uniform
                const float4 g0 = s_geo0[j];
                const float4 g1 = s_geo1[j];
                const int pos = b0 + j;
                AlphaEval e;
                const bool contributed =
                    pos < my_last && eval_alpha(fx - g0.x, fy - g0.y, g0.z, g0.w, g1.x, g1.y, g1.z,
                                                g1.w, a.alpha_max, a.alpha_min, e);
                if (!__any_sync(SG_FULL_MASK, contributed)) continue;
                float vals[NV];
#pragma unroll
                for (int k = 0; k < NV; ++k) vals[k] = 0.f;
                if (contributed) {
                    T = __fdiv_rn(T, __fsub_rn(1.f, e.alpha));  // transmittance before this Gaussian
                    const float4 *f4 = reinterpret_cast<const float4 *>(s_feat + (size_t)j * NF);
                    float gf = 0.f;
#pragma unroll
                    for (int k = 0; k < NF / 4; ++k) {
                        const float4 f = f4[k];
                        gf = fmaf(g[4 * k + 0], f.x, gf);
                        gf = fmaf(g[4 * k + 1], f.y, gf);
                        gf = fmaf(g[4 * k + 2], f.z, gf);
                        gf = fmaf(g[4 * k + 3], f.w, gf);
                    }
                    const float dalpha = T * (gf - acc_a);
                    acc_a = e.alpha * gf + (1.f - e.alpha) * acc_a;
                    const float w = e.alpha * T;
                    vals[6] = w * g[3];
                    vals[7] = w * g[0];
                    vals[8] = w * g[1];
                    vals[9] = w * g[2];
#pragma unroll
                    for (int k = 0; k < C; ++k) vals[10 + k] = w * g[4 + k];
                    if (e.raw < a.alpha_max) {
                        // sigma = p1^2 + p2^2, p1 = m00 dx, p2 = m10 dx + m11 dy; d(dx)/du = -1.
                        // Conic gradients: d sigma / d(a, b, c) = (dx^2/2, dx dy, dy^2/2).
                        const float gsig = -dalpha * e.raw;
                        vals[0] = -2.f * gsig * (e.p1 * g1.x + e.p2 * g1.y);
                        vals[1] = -2.f * gsig * (e.p2 * g1.z);
                        vals[2] = 0.5f * gsig * e.dx * e.dx;
                        vals[3] = gsig * e.dx * e.dy;
                        vals[4] = 0.5f * gsig * e.dy * e.dy;
                        vals[5] = dalpha * e.G;
                    }
                }
                warp_transpose_reduce<NV>(vals, lane);
                const uint32_t rec = s_rec[j];
                const uint32_t gi = rec % (uint32_t)a.N;
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int idx = lane * PER + k;
                    if (idx < 7)
                        atomicAdd(a.g2d + 8 * (size_t)rec + idx, vals[k]);
                    else if (idx < 10)
                        atomicAdd(a.g_rgb + 3 * (size_t)gi + (idx - 7), vals[k]);
                    else if (idx < NRAW)
                        atomicAdd(a.g_sem + (size_t)C * gi + (idx - 10), vals[k]);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------

template <int C>
static size_t fwd_smem(int batch) {
    return (size_t)batch * (3 * 16 + 4 * (4 + C));
}
template <int C>
static size_t bwd_smem(int batch) {
    return fwd_smem<C>(batch) + (size_t)batch * 4;
}

static int resident_grid(const void *fn, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

template <int C>
static sg_status launch_raster_t(RasterArgs &a, bool backward, cudaStream_t st) {
    const int threads = a.tile_w * a.tile_h;
    const size_t smem = backward ? bwd_smem<C>(a.batch) : fwd_smem<C>(a.batch);
    const void *fn = backward ? (const void *)raster_bwd_kernel<C> : (const void *)raster_fwd_kernel<C>;
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
        raster_bwd_kernel<C><<<grid, threads, smem, st>>>(a);
    else
        raster_fwd_kernel<C><<<grid, threads, smem, st>>>(a);
    count_launches(1);
    return check_launch(backward ? "raster_bwd" : "raster_fwd");
}

sg_status launch_raster(RasterArgs &a, int C, bool backward, cudaStream_t st) {
    switch (C) {
        case 4: return launch_raster_t<4>(a, backward, st);
        case 8: return launch_raster_t<8>(a, backward, st);
        case 16: return launch_raster_t<16>(a, backward, st);
        case 32: return launch_raster_t<32>(a, backward, st);
        case 40: return launch_raster_t<40>(a, backward, st);
        default:
            set_error("unsupported semantic width C=%d (supported: 4, 8, 16, 32, 40)", C);
            return SG_ERR_INVALID_ARG;
    }
}

bool raster_supports(int C) { return C == 4 || C == 8 || C == 16 || C == 32 || C == 40; }

}  // namespace sg
