// tiles.cu -- per-tile depth-sorted instance lists (the sorted set N of Eq. 7-9).
//
// Pipeline (all counts stay on the device, so the whole sequence can be captured in a
// CUDA graph with a fixed launch shape):
//   1. compact:  visible records r (non-empty tile rectangle) -> (depth bits, r), in r order
//   2. sort:     stable LSD radix sort by the 32 float32 depth bits (depths are > z_near > 0
//                so their bit patterns order like the values); ties keep record order
//   3. emit:     the slots are the tile rows of each record's rectangle, record after
//                record in depth order (a prefix of the row counts numbers them); for each
//                slot the span of the record's alpha >= alpha_min region within the row (a
//                float32 computation) gives the contiguous run of tiles it reaches; a
//                counting pass, split evenly over the slots, and a scan give the offsets, and
//                an emission pass writes (global tile id, r) for those tiles, row-major
//   4. sort:     stable LSD radix sort of the instances by global tile id (only the bits
//                n_tiles needs), which keeps the (depth, record) order inside each tile
//   5. ranges:   [start, end) of every tile
//   6. order:    (when requested) the tile ids by descending half-octave bucket of their list
//                length, one stable counting pass: the compositing kernels' work order
// The result equals sorting all kept instances by (tile, depth bits, record id).  Every radix
// pass is three kernels: per-block digit histograms, per-digit scans over the blocks, and
// a stable scatter that ranks equal digits inside a block by warp match + prefix counts.
#include <cstdio>

#include <algorithm>

#include "sg_common.cuh"

namespace sg {

constexpr int kScanThreads = 256;
// Widest digit of the tile sort.  Each pass scatters a block's instances over 2^digit runs
// of the output; with 9-bit digits (512 runs per block) the partly written output lines no
// longer stay in L2 and the pass reads and writes twice its bytes in DRAM (measured), so 17 or
// 18 bits of tile id sort in three passes of 6 bits rather than two of 9 and 8.
constexpr int kTileDigitBits = 8;

__device__ __forceinline__ void block_range(int n, int G, int b, int &beg, int &end) {
    const int tiles = (n + kScanThreads - 1) / kScanThreads;
    const int per = (tiles + G - 1) / G;
    beg = min(n, b * per * kScanThreads);
    end = min(n, beg + per * kScanThreads);
}

// Exclusive block scan of one value per thread (blockDim == kScanThreads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &total) {
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(SG_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = kScanThreads / 32;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(SG_FULL_MASK, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) s_warp[lane] = wi - w;
        if (lane == nw - 1) s_warp[nw] = wi;
    }
    __syncthreads();
    const uint32_t res = incl - v + s_warp[warp];
    total = s_warp[kScanThreads / 32];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------------------
// Device-wide exclusive scan (reduce / scan block sums / apply) with a device-side count.
// ---------------------------------------------------------------------------------------

struct VisibleCount {  // 1 if the record's tile rectangle is non-empty
    const uint2 *rect;
    __device__ uint32_t operator()(int i) const {
        const uint2 r = rect[i];
        return r.x != r.y ? 1u : 0u;
    }
};

__device__ __forceinline__ uint32_t rect_tiles(uint2 r) {
    const uint32_t tx0 = r.x & 0xffffu, ty0 = r.x >> 16, tx1 = r.y & 0xffffu, ty1 = r.y >> 16;
    return (tx1 > tx0 && ty1 > ty0) ? (tx1 - tx0) * (ty1 - ty0) : 0u;
}

__device__ __forceinline__ uint32_t rect_rows(uint2 r) {
    const uint32_t ty0 = r.x >> 16, ty1 = r.y >> 16;
    return rect_tiles(r) ? ty1 - ty0 : 0u;
}

struct SortedRowCount {  // tile rows of the rectangle of the record at sorted position i
    const uint2 *rect;
    const uint32_t *rec;
    __device__ uint32_t operator()(int i) const { return rect_rows(rect[rec[i]]); }
};

template <class F>
__global__ void scan_reduce_kernel(F f, const int *n_ptr, int n_host, uint32_t *bsum, int G) {
    pdl_begin();
    const int n = n_ptr ? *n_ptr : n_host;
    int beg, end;
    block_range(n, G, blockIdx.x, beg, end);
    uint32_t s = 0;
    for (int i = beg + threadIdx.x; i < end; i += kScanThreads) s += f(i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(SG_FULL_MASK, s, o);
    __shared__ uint32_t sw[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += sw[w];
        bsum[blockIdx.x] = t;
    }
}

// One block: exclusive scan of G block sums (G <= 4096); writes the grand total.
__global__ void scan_blocks_kernel(uint32_t *bsum, int G, int *total) {
    pdl_begin();
    uint32_t run = 0;
    for (int base = 0; base < G; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < G ? bsum[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, tot);
        if (i < G) bsum[i] = ex + run;
        run += tot;
    }
    if (threadIdx.x == 0) *total = (int)run;
}

// Apply for the compaction: write (depth bits, record) of every visible record.  Each thread
// takes 8 consecutive records per round (two 16-byte loads of their rectangles when the
// array is 16-byte aligned), so a round of the block covers 2048 records with one block scan
// and all of its loads in flight together.
constexpr int kCompactPerThread = 8;
__global__ void compact_apply_kernel(const uint2 *__restrict__ rect, const float4 *__restrict__ geo,
                                     int n, const uint32_t *__restrict__ boff, int G,
                                     uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    pdl_begin();
    constexpr int E = kCompactPerThread;
    int beg, end;
    block_range(n, G, blockIdx.x, beg, end);
    const bool vec = (reinterpret_cast<uintptr_t>(rect) & 15u) == 0;
    uint32_t run = boff[blockIdx.x];
    for (int base = beg; base < end; base += kScanThreads * E) {
        const int i0 = base + (int)threadIdx.x * E;  // a multiple of 8 (beg is one of 256)
        uint2 r[E];
        if (vec && i0 + E <= end) {
            const uint4 *p4 = reinterpret_cast<const uint4 *>(rect + i0);
#pragma unroll
            for (int q = 0; q < E / 2; ++q) {
                const uint4 w = p4[q];
                r[2 * q] = make_uint2(w.x, w.y);
                r[2 * q + 1] = make_uint2(w.z, w.w);
            }
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) r[q] = i0 + q < end ? rect[i0 + q] : make_uint2(0, 0);
        }
        uint32_t f = 0, bits = 0;
#pragma unroll
        for (int q = 0; q < E; ++q)
            if (r[q].x != r[q].y) {
                bits |= 1u << q;
                ++f;
            }
        float dep[E];
#pragma unroll
        for (int q = 0; q < E; ++q) dep[q] = ((bits >> q) & 1u) ? geo[2 * (size_t)(i0 + q)].z : 0.f;
        uint32_t tot;
        uint32_t o = run + block_exclusive_scan(f, tot);
#pragma unroll
        for (int q = 0; q < E; ++q)
            if ((bits >> q) & 1u) {
                key[o] = __float_as_uint(dep[q]);
                val[o] = (uint32_t)(i0 + q);
                ++o;
            }
        run += tot;
    }
}

// The columns of a tile row that the record's alpha >= alpha_min region reaches.  The
// projection wrote the half extent ex = sqrt(2 thr s00) 1.002 + 0.01 with
// thr = ln(o / alpha_min) + 1e-3 and m00 = 1 / sqrt(2 s00), so
// thr' = ((ex - 0.01) (1 / 1.002) m00)^2 recovers the threshold from the record (to float
// rounding, far inside its 1e-3 margin).  Within the band dy in [y0, y1] of the row's pixel
// centres, the ellipse sigma = (m00 dx)^2 + (m10 dx + m11 dy)^2 <= thr' spans dx in
// [xl, xr]: with A = m00^2 + m10^2, B = m10 m11, C = m11^2 and p = m00 m11 (A C - B^2 = p^2),
// the band is cut to |dy| <= sqrt(A thr') / p, the right edge (s - B dy) / A with
// s = sqrt(A thr' - (p dy)^2) is largest at dy = -B (sqrt(thr' C) / p) / C and the left edge
// (-B dy - s) / A smallest at the opposite dy, each clamped to the band.  A tile is kept when
// its pixel-centre columns [X0, X1] meet [xl, xr]; the kept tiles of a row are contiguous.
// Every step is one correctly rounded float32 operation (square roots and divisions
// included) in a fixed order with no contraction, so the decision is reproducible bit for
// bit.  Returns false when the band misses the ellipse.
struct RowSpan {
    float xl, xr;  // extent of the footprint in the band, relative to the mean
    float uf;      // fraction of the mean
    int ui;        // integer part of the mean
};
// The band-independent part of the rule: the mean and the ellipse's constants.
struct Footprint {
    float uf, vf;            // fractions of the mean
    int ui, vi;              // integer parts of the mean
    float A, B, Cq, p, At;   // A thr' = At
    float dymax, dyr;        // |dy| bound; dy of the right edge's maximum
};
__device__ __forceinline__ Footprint footprint(const float4 g0, const float4 g1, float ex) {
    Footprint f;
    const uint32_t packed = __float_as_uint(g1.w);
    f.ui = (int)(short)(packed & 0xffffu);
    f.vi = (int)(short)(packed >> 16);
    f.uf = g0.x;
    f.vf = g0.y;
    const float m00 = g1.x, m10 = g1.y, m11 = g1.z;
    const float t = __fmul_rn(__fmul_rn(__fsub_rn(ex, 0x1.47ae14p-7f /* float(0.01) */), 0x1.fefa62p-1f /* float(1/1.002) */),
                              m00);
    const float thr = __fmul_rn(t, t);
    f.A = __fadd_rn(__fmul_rn(m00, m00), __fmul_rn(m10, m10));
    f.B = __fmul_rn(m10, m11);
    f.Cq = __fmul_rn(m11, m11);
    f.p = __fmul_rn(m00, m11);
    f.dymax = __fdiv_rn(__fsqrt_rn(__fmul_rn(f.A, thr)), f.p);
    const float dxmax = __fdiv_rn(__fsqrt_rn(__fmul_rn(thr, f.Cq)), f.p);
    f.dyr = -__fdiv_rn(__fmul_rn(f.B, dxmax), f.Cq);
    f.At = __fmul_rn(f.A, thr);
    return f;
}
// The span of the footprint within the band of pixel-centre rows [Y0, Y1].
__device__ __forceinline__ bool band_span(const Footprint &f, int Y0, int Y1, RowSpan &rs) {
    rs.ui = f.ui;
    rs.uf = f.uf;
    const float y0 = __fsub_rn((float)(Y0 - f.vi), f.vf), y1 = __fsub_rn((float)(Y1 - f.vi), f.vf);
    const float yb0 = fmaxf(y0, -f.dymax), yb1 = fminf(y1, f.dymax);
    if (!(yb0 <= yb1)) return false;
    auto s_of = [&](float dy) {
        const float q = __fmul_rn(f.p, dy);
        return __fsqrt_rn(fmaxf(__fsub_rn(f.At, __fmul_rn(q, q)), 0.f));
    };
    const float dr = fminf(yb1, fmaxf(yb0, f.dyr));
    const float dl = fminf(yb1, fmaxf(yb0, -f.dyr));
    rs.xr = __fdiv_rn(__fsub_rn(s_of(dr), __fmul_rn(f.B, dr)), f.A);
    rs.xl = __fdiv_rn(__fsub_rn(-__fmul_rn(f.B, dl), s_of(dl)), f.A);
    return true;
}
// The same rule in one pass (the band-independent constants after the early exit), for the
// lists without half masks; identical operations, so identical results.
__device__ __forceinline__ bool row_span(const float4 g0, const float4 g1, float ex, int Y0, int Y1, RowSpan &rs) {
    const uint32_t packed = __float_as_uint(g1.w);
    rs.ui = (int)(short)(packed & 0xffffu);
    rs.uf = g0.x;
    const int vi = (int)(short)(packed >> 16);
    const float m00 = g1.x, m10 = g1.y, m11 = g1.z;
    const float t = __fmul_rn(__fmul_rn(__fsub_rn(ex, 0x1.47ae14p-7f /* float(0.01) */), 0x1.fefa62p-1f /* float(1/1.002) */),
                              m00);
    const float thr = __fmul_rn(t, t);
    const float A = __fadd_rn(__fmul_rn(m00, m00), __fmul_rn(m10, m10));
    const float B = __fmul_rn(m10, m11);
    const float Cq = __fmul_rn(m11, m11);
    const float p = __fmul_rn(m00, m11);
    const float y0 = __fsub_rn((float)(Y0 - vi), g0.y), y1 = __fsub_rn((float)(Y1 - vi), g0.y);
    const float dymax = __fdiv_rn(__fsqrt_rn(__fmul_rn(A, thr)), p);
    const float yb0 = fmaxf(y0, -dymax), yb1 = fminf(y1, dymax);
    if (!(yb0 <= yb1)) return false;
    const float dxmax = __fdiv_rn(__fsqrt_rn(__fmul_rn(thr, Cq)), p);
    const float dyr = -__fdiv_rn(__fmul_rn(B, dxmax), Cq);
    const float At = __fmul_rn(A, thr);
    auto s_of = [&](float dy) {
        const float q = __fmul_rn(p, dy);
        return __fsqrt_rn(fmaxf(__fsub_rn(At, __fmul_rn(q, q)), 0.f));
    };
    const float dr = fminf(yb1, fmaxf(yb0, dyr));
    const float dl = fminf(yb1, fmaxf(yb0, -dyr));
    rs.xr = __fdiv_rn(__fsub_rn(s_of(dr), __fmul_rn(B, dr)), A);
    rs.xl = __fdiv_rn(__fsub_rn(-__fmul_rn(B, dl), s_of(dl)), A);
    return true;
}
// does the row's footprint [xl, xr] meet the pixel-centre columns [X0, X1]?
__device__ __forceinline__ bool span_meets(const RowSpan &rs, int X0, int X1) {
    return __fsub_rn((float)(X1 - rs.ui), rs.uf) >= rs.xl && __fsub_rn((float)(X0 - rs.ui), rs.uf) <= rs.xr;
}

// The kept tile columns [a, b) of a row within [tx0, tx1): the tiles whose pixel-centre
// columns meet the span.  Both halves of span_meets are monotone in the column (the left test
// turns true once, the right test turns false once; each is a correctly rounded subtraction
// of an increasing integer), so a is the first column passing the left test and b the first
// failing the right one.  Each is estimated from the span and then moved to the exact
// boundary by the tests themselves (a step or two), so the result equals a walk over every
// column of the rectangle.
__device__ __forceinline__ void span_run(const RowSpan &rs, int tx0, int tx1, int tile_w, int W, int &a, int &b) {
    auto left = [&](int tx) {  // the tile's last pixel-centre column reaches xl
        return __fsub_rn((float)(min(tx * tile_w + tile_w - 1, W - 1) - rs.ui), rs.uf) >= rs.xl;
    };
    auto right = [&](int tx) {  // the tile's first pixel-centre column is within xr
        return __fsub_rn((float)(tx * tile_w - rs.ui), rs.uf) <= rs.xr;
    };
    const float ca = ((float)rs.ui + rs.uf + rs.xl - (float)(tile_w - 1)) / (float)tile_w;
    a = !(ca > (float)tx0) ? tx0 : (!(ca < (float)tx1) ? tx1 : (int)ceilf(ca));  // (NaN: tx0)
    while (a > tx0 && left(a - 1)) --a;
    while (a < tx1 && !left(a)) ++a;
    const float cb = ((float)rs.ui + rs.uf + rs.xr) / (float)tile_w + 1.f;
    b = !(cb > (float)a) ? a : (!(cb < (float)tx1) ? tx1 : (int)floorf(cb));
    while (b > a && !right(b - 1)) --b;
    while (b < tx1 && right(b)) ++b;
    if (b < a) b = a;
}

// With half masks, the kept tiles [a, a + cnt) of a (record, tile row) slot and which halves
// of each tile they may reach (without them the rule above runs once on the tile row's band
// of pixel-centre rows [Y0, Y1]).  The band splits into a top half [Y0, Y0 + tile_h / 2)
// and a bottom half (clamped to the image), the rule runs on each, and a tile is kept when
// its columns meet either half's span.  The two runs [a0, b0), [a1, b1) of one convex
// footprint overlap (their spans cover the whole band's span), so the kept tiles are the
// contiguous run [a, b) = their hull.  half packs the runs relative to a, one byte each
// (a0 - a, b0 - a, a1 - a, b1 - a), or is kHalfAll when the run is longer than 255 tiles
// (every tile then marked as reaching both halves, a conservative superset).
constexpr uint32_t kHalfAll = 0xffffffffu;
struct SlotRun {
    int a, cnt;
    uint32_t half;
};
__device__ __forceinline__ SlotRun slot_run(const float4 g0, const float4 g1, float ex, int Y0, int Y1, int tile_h,
                                            int tx0, int tx1, int tile_w, int W) {
    RowSpan rs;
    const Footprint f = footprint(g0, g1, ex);
    const int Yh = Y0 + tile_h / 2;
    int a0 = tx1, b0 = tx1, a1 = tx1, b1 = tx1;
    if (band_span(f, Y0, min(Yh - 1, Y1), rs)) span_run(rs, tx0, tx1, tile_w, W, a0, b0);
    if (Yh <= Y1 && band_span(f, Yh, Y1, rs)) span_run(rs, tx0, tx1, tile_w, W, a1, b1);
    const bool e0 = b0 <= a0, e1 = b1 <= a1;
    SlotRun r;
    if (e0 && e1) {
        r.a = tx1;
        r.cnt = 0;
        r.half = 0u;
        return r;
    }
    if (e0) a0 = b0 = a1;
    if (e1) a1 = b1 = a0;
    r.a = min(a0, a1);
    r.cnt = max(b0, b1) - r.a;
    r.half = r.cnt > 255 ? kHalfAll
                         : (uint32_t)(a0 - r.a) | ((uint32_t)(b0 - r.a) << 8) | ((uint32_t)(a1 - r.a) << 16) |
                               ((uint32_t)(b1 - r.a) << 24);
    return r;
}
// Half mask (bit 0 top, bit 1 bottom) of the q-th tile of a slot's run.
__device__ __forceinline__ uint32_t half_mask(uint32_t half, uint32_t q) {
    if (half == kHalfAll) return 3u;
    const uint32_t top = q >= (half & 0xffu) && q < ((half >> 8) & 0xffu);
    const uint32_t bot = q >= ((half >> 16) & 0xffu) && q < (half >> 24);
    return top | (bot << 1);
}

// The (record, tile row) slots: the tile rows of every depth-sorted record's rectangle,
// record after record; P[i] is the first slot of sorted record i.  The two culling passes
// split the S slots evenly over their Gc blocks (a multiple of 256 slots each), so that the
// few near records with huge rectangles do not serialise one warp.
__device__ __forceinline__ uint32_t slot_block_size(uint32_t S, int Gc) {
    const uint32_t chunks = (S + kScanThreads - 1) / kScanThreads;
    const uint32_t per = (chunks + (uint32_t)Gc - 1) / (uint32_t)Gc;
    return (per > 0 ? per : 1u) * kScanThreads;
}

// P[i] = boff[block] + exclusive scan of the rectangle row counts, and for every block of the
// slot partition the record that owns its first slot.
__global__ void slot_prefix_kernel(const uint2 *__restrict__ rect, const uint32_t *__restrict__ rec,
                                   const int *__restrict__ m_ptr, const uint32_t *__restrict__ boff, int G,
                                   const int *__restrict__ s_ptr, int Gc, uint32_t *__restrict__ P,
                                   uint32_t *__restrict__ first_rec) {
    pdl_begin();
    const int n = *m_ptr;
    const uint64_t per = slot_block_size((uint32_t)*s_ptr, Gc);
    int beg, end;
    block_range(n, G, blockIdx.x, beg, end);
    uint32_t run = boff[blockIdx.x];
    for (int base = beg; base < end; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const uint32_t c = i < end ? rect_rows(rect[rec[i]]) : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(c, tot);
        if (i < end) {
            const uint64_t p = run + ex;
            P[i] = (uint32_t)p;
            for (uint64_t b = (p + per - 1) / per; b * per < p + c && b < (uint64_t)Gc; ++b) first_rec[b] = (uint32_t)i;
        }
        run += tot;
    }
}

// The culling passes over the slot partition.  Thread t of a 256-slot chunk takes slot
// s = c0 + t: its record is found by a binary search over the prefixes of the (at most 256)
// records that can own the chunk, staged in shared memory; the row's footprint span gives
// the contiguous run of kept tile columns.
//   COUNT: adds up the kept tiles of the block's slots (kbsum[block]); when the slots fit the
//          slot cache (S <= capacity), also stores each slot's first kept tile and count.
//   EMIT:  writes (global tile id, record) for the kept tiles, column by column, at
//          kbsum[block] (the scanned block offset) plus the block's exclusive scan of the
//          kept counts, i.e. in (record, row, column) order; the runs come from the slot
//          cache when the count pass filled it, else from the same span computation.
// HALVES: the rule runs per half tile row (slot_run) and the emitted records carry each
// tile's half mask in bits 30-31.
template <bool EMIT, bool HALVES>
__global__ void __launch_bounds__(kScanThreads, 6) cull_pass_kernel(const uint2 *__restrict__ rect, const float4 *__restrict__ geo,
                                 const float2 *__restrict__ ext, const uint32_t *__restrict__ rec,
                                 const int *__restrict__ m_ptr, const int *__restrict__ s_ptr,
                                 const uint32_t *__restrict__ P, const uint32_t *__restrict__ first_rec, int Gc,
                                 int N, const sg_view *__restrict__ views, int n_views, int tile_w, int tile_h,
                                 uint32_t *__restrict__ kbsum, uint32_t *__restrict__ tkey, uint32_t *__restrict__ tval,
                                 uint32_t *__restrict__ slot_tf, uint32_t *__restrict__ slot_cnt,
                                 uint32_t *__restrict__ slot_half, int capacity, uint32_t *__restrict__ status) {
    pdl_begin();
    __shared__ uint32_t s_P[kScanThreads];
    __shared__ uint32_t s_ex[EMIT ? kScanThreads : 1], s_tf[EMIT ? kScanThreads : 1], s_or[EMIT ? kScanThreads : 1],
        s_hf[EMIT && HALVES ? kScanThreads : 1];
    __shared__ int s_next;
    __shared__ int4 s_vw[SG_MAX_VIEWS];  // (W, H, tile_offset, tiles_x) of each view-level
    for (int v = threadIdx.x; v < n_views; v += kScanThreads)
        s_vw[v] = make_int4(views[v].W, views[v].H, views[v].tile_offset, views[v].tiles_x);
    const int n = *m_ptr;
    const uint32_t S = (uint32_t)*s_ptr;
    const uint64_t per = slot_block_size(S, Gc);
    const uint64_t s0 = (uint64_t)blockIdx.x * per;
    const uint64_t s1 = min((uint64_t)S, s0 + per);
    const bool cached = S <= (uint32_t)capacity;  // the slot cache holds every slot
    uint32_t kept = 0;
    uint32_t run = EMIT ? kbsum[blockIdx.x] : 0u;
    bool overflow = false;
    int ic = s0 < s1 ? (int)first_rec[blockIdx.x] : 0;
    for (uint64_t c0 = s0; c0 < s1; c0 += kScanThreads) {  // block-uniform trip count
        const int j = ic + (int)threadIdx.x;
        s_P[threadIdx.x] = j < n ? P[j] : 0xffffffffu;
        __syncthreads();
        const uint32_t s = (uint32_t)(c0 + threadIdx.x);
        uint32_t cnt = 0, orec = 0, tfirst = 0, half = 0;
        int k = 0;
        if (c0 + threadIdx.x < s1) {
            int lo = 0, hi = kScanThreads - 1;  // the last k with s_P[k] <= s (s_P[0] <= c0)
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_P[mid] <= s) lo = mid; else hi = mid - 1;
            }
            k = lo;
            orec = rec[ic + k];
        }
        if (EMIT && cached) {
            if (c0 + threadIdx.x < s1) {
                tfirst = __ldcs(slot_tf + s);
                cnt = __ldcs(slot_cnt + s);
                if (HALVES) half = __ldcs(slot_half + s);
            }
        } else if (c0 + threadIdx.x < s1) {
            const uint2 rc = rect[orec];
            const int tx0 = (int)(rc.x & 0xffffu), tx1 = (int)(rc.y & 0xffffu);
            const int ty = (int)(rc.x >> 16) + (int)(s - s_P[k]);
            const int4 vw = s_vw[orec / (uint32_t)N];
            const int Y0 = ty * tile_h;
            const int Y1 = min(Y0 + tile_h - 1, vw.y - 1);
            int tx_a = tx1;
            if constexpr (HALVES) {
                const SlotRun sr = slot_run(geo[2 * (size_t)orec], geo[2 * (size_t)orec + 1], ext[orec].x, Y0, Y1,
                                            tile_h, tx0, tx1, tile_w, vw.x);
                cnt = (uint32_t)sr.cnt;
                half = sr.half;
                tx_a = sr.a;
            } else {
                RowSpan rs;
                if (row_span(geo[2 * (size_t)orec], geo[2 * (size_t)orec + 1], ext[orec].x, Y0, Y1, rs)) {
                    // the kept columns are contiguous
                    int tb;
                    span_run(rs, tx0, tx1, tile_w, vw.x, tx_a, tb);
                    cnt = (uint32_t)(tb - tx_a);
                    if (!cnt) tx_a = tx1;
                }
            }
            tfirst = (uint32_t)vw.z + (uint32_t)ty * (uint32_t)vw.w + (uint32_t)tx_a;
            if (!EMIT && cached) {
                slot_tf[s] = tfirst;
                slot_cnt[s] = cnt;
                if (HALVES) slot_half[s] = half;
            }
        }
        if (!EMIT) {
            kept += cnt;
        } else {
            // the chunk's instances [run, run + tot): consecutive threads write consecutive
            // instances, each finding its slot by a binary search over the slots' offsets
            uint32_t tot;
            const uint32_t ex = block_exclusive_scan(cnt, tot);
            s_ex[threadIdx.x] = ex;
            s_tf[threadIdx.x] = tfirst;
            s_or[threadIdx.x] = orec;
            if (HALVES) s_hf[threadIdx.x] = half;
            __syncthreads();
            for (uint32_t o = threadIdx.x; o < tot; o += kScanThreads) {
                int lo = 0, hi = kScanThreads - 1;  // the last slot t with s_ex[t] <= o
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_ex[mid] <= o) lo = mid; else hi = mid - 1;
                }
                const uint32_t g = run + o;
                if (g < (uint32_t)capacity) {
                    const uint32_t q = o - s_ex[lo];
                    tkey[g] = s_tf[lo] + q;
                    // (with halves, records are below 2^30: checked by the caller)
                    tval[g] = HALVES ? s_or[lo] | (half_mask(s_hf[lo], q) << 30) : s_or[lo];
                } else {
                    overflow = true;
                }
            }
            run += tot;
        }
        // the next chunk starts in the record that owns this chunk's last slot
        if (threadIdx.x == kScanThreads - 1) s_next = ic + k;
        __syncthreads();
        ic = s_next;
    }
    if (!EMIT) {
        uint32_t tot;
        block_exclusive_scan(kept, tot);
        if (threadIdx.x == 0) kbsum[blockIdx.x] = tot;
    }
    if (overflow) atomicOr(status, SG_STATUS_CAPACITY);
}

// ---------------------------------------------------------------------------------------
// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits (or fewer).
// ---------------------------------------------------------------------------------------

// Key sources of the radix sort: pairs held in arrays, or the tiles' list lengths.
struct ArrayPairs {
    const uint32_t *k, *v;
    // each pair is read once per kernel: evict-first loads, which leave L2 to the scatter's
    // partly written output lines
    __device__ uint32_t key(int i) const { return __ldcs(k + i); }
    __device__ uint32_t val(int i) const { return __ldcs(v + i); }
};
// key = 63 - bucket of the tile's instance count n (bucket 0 for n = 0, else
// 1 + 2 floor(log2 n) + the bit below the leading one): descending length, 6 bits
struct TileLengthKeys {
    const int2 *ranges;
    __device__ uint32_t key(int i) const {
        const int2 r = ranges[i];
        const uint32_t n = (uint32_t)max(r.y - r.x, 0);
        if (n == 0) return 63u;
        const int lz = 31 - __clz(n);
        const uint32_t sub = lz >= 1 ? (n >> (lz - 1)) & 1u : 0u;
        return 63u - (1u + 2u * (uint32_t)lz + sub);
    }
    __device__ uint32_t val(int i) const { return (uint32_t)i; }
};

// Radix digits of one pass: up to 8 bits (256 buckets) or 9 bits (512 buckets); each of
// the 256 threads of a block owns ND / 256 consecutive buckets.
template <class Src, int ND>
__global__ void rs_hist_kernel(Src src, const int *__restrict__ n_ptr, int cap, int shift, uint32_t mask,
                               uint32_t *__restrict__ hist, int G) {
    pdl_begin();
    constexpr int DPT = ND / kScanThreads;
    __shared__ uint32_t h[ND];
#pragma unroll
    for (int q = 0; q < DPT; ++q) h[threadIdx.x * DPT + q] = 0;
    __syncthreads();
    const int n = n_ptr ? min(*n_ptr, cap) : cap;
    int beg, end;
    block_range(n, G, blockIdx.x, beg, end);
    for (int i = beg + threadIdx.x; i < end; i += kScanThreads)
        atomicAdd(&h[(src.key(i) >> shift) & mask], 1u);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < DPT; ++q) hist[(threadIdx.x * DPT + q) * G + blockIdx.x] = h[threadIdx.x * DPT + q];
}

// Block d: exclusive scan of digit d's per-block counts; totals[d] = digit d's count.
__global__ void rs_digit_scan_kernel(uint32_t *__restrict__ hist, uint32_t *__restrict__ totals, int G) {
    pdl_begin();
    const int d = blockIdx.x;
    uint32_t run = 0;
    for (int base = 0; base < G; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < G ? hist[d * G + i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, tot);
        if (i < G) hist[d * G + i] = ex + run;
        run += tot;
    }
    if (threadIdx.x == 0) totals[d] = run;
}

// Exclusive scan over ND buckets held DPT per thread (consecutive), block-wide.
template <int DPT>
__device__ __forceinline__ void bucket_exclusive_scan(const uint32_t (&v)[DPT], uint32_t (&ex)[DPT]) {
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) sum += v[q];
    uint32_t tot;
    uint32_t run = block_exclusive_scan(sum, tot);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        ex[q] = run;
        run += v[q];
    }
}

// Scatter of one digit pass.  Each block walks its input range in chunks of 256 IPT
// elements; warp w owns the chunk's elements [32 IPT w, 32 IPT (w + 1)), lane l element
// 32 it + l of them.  Ranking needs no block barrier per element row: every warp ranks its
// own elements against a warp-private digit count (warp match_any + the lanes below), one
// block pass turns the per-warp counts into per-digit offsets, the chunk is reordered by
// digit in shared memory, and consecutive threads store consecutive elements of one digit
// run (coalesced stores instead of one scattered sector per element).
template <int ND>
__host__ __device__ constexpr int scatter_ipt() { return 12; }

template <class Src, int ND>
__global__ void __launch_bounds__(kScanThreads, 4) rs_scatter_kernel(
    Src src, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const int *__restrict__ n_ptr, int cap, int shift, uint32_t mask,
    const uint32_t *__restrict__ hist, const uint32_t *__restrict__ totals, int G) {
    pdl_begin();
    constexpr int kWarps = kScanThreads / 32;
    constexpr int DPT = ND / kScanThreads;  // digits per thread: tid * DPT + q
    constexpr int IPT = scatter_ipt<ND>();
    constexpr int CH = kScanThreads * IPT;
    __shared__ uint32_t run[ND];            // global position of the next element of each digit
    __shared__ uint32_t loc[ND];            // first slot of each digit in the reordered chunk
    __shared__ uint32_t wcnt[kWarps][ND];   // per-warp digit counts, then per-warp offsets
    __shared__ uint32_t skey[CH], sval[CH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // digit base = exclusive scan of the digit totals (+ this block's offset)
    {
        uint32_t t[DPT], ex[DPT];
#pragma unroll
        for (int q = 0; q < DPT; ++q) t[q] = totals[tid * DPT + q];
        bucket_exclusive_scan<DPT>(t, ex);
#pragma unroll
        for (int q = 0; q < DPT; ++q) run[tid * DPT + q] = ex[q] + hist[(tid * DPT + q) * G + blockIdx.x];
    }
    const int n = n_ptr ? min(*n_ptr, cap) : cap;
    int beg, end;
    block_range(n, G, blockIdx.x, beg, end);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t *wc = wcnt[warp];
    for (int cbase = beg; cbase < end; cbase += CH) {
#pragma unroll
        for (int q = 0; q < ND / 32; ++q) wc[32 * q + lane] = 0;
        const int wbase = cbase + 32 * IPT * warp;
        uint32_t key[IPT], val[IPT], rank[IPT];
        // all of the warp's loads first (their latencies overlap), then the ranking
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            const int i = wbase + 32 * it + lane;
            const bool valid = i < end;
            key[it] = valid ? src.key(i) : 0u;
            val[it] = valid ? src.val(i) : 0u;
        }
        __syncwarp();
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            const bool valid = wbase + 32 * it + lane < end;
            const uint32_t d = valid ? ((key[it] >> shift) & mask) : (uint32_t)ND;
            const uint32_t peers = __match_any_sync(SG_FULL_MASK, d);
            const uint32_t below = __popc(peers & lt_mask);
            rank[it] = valid ? wc[d] + below : 0u;
            __syncwarp();
            if (valid && below == 0) wc[d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive offsets of the warps, the chunk's count, and (block scan)
        // the digit's first slot in the reordered chunk
        uint32_t cnt[DPT], ex[DPT];
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid * DPT + q;
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wcnt[w][d];
                wcnt[w][d] = s;
                s += c;
            }
            cnt[q] = s;
        }
        bucket_exclusive_scan<DPT>(cnt, ex);
#pragma unroll
        for (int q = 0; q < DPT; ++q) loc[tid * DPT + q] = ex[q];
        __syncthreads();
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            if (wbase + 32 * it + lane < end) {
                const uint32_t d = (key[it] >> shift) & mask;
                const uint32_t li = loc[d] + wc[d] + rank[it];
                skey[li] = key[it];
                sval[li] = val[it];
            }
        }
        __syncthreads();
        const int cn = min(CH, end - cbase);
        for (int j = tid; j < cn; j += kScanThreads) {
            const uint32_t k = skey[j];
            const uint32_t d = (k >> shift) & mask;
            const uint32_t pos = run[d] + ((uint32_t)j - loc[d]);
            if (kout) kout[pos] = k;
            vout[pos] = sval[j];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < DPT; ++q) run[tid * DPT + q] += cnt[q];
        // (the next chunk's first block barrier orders these updates before their reads)
    }
}

// Sorts n (device count, clamped to cap) pairs on bits [0, bits) from (kin, vin) into
// (kout, vout) using (ktmp, vtmp) as ping-pong; kin/vin are not modified.  The bits are
// split into the fewest passes of at most max_bits (<= 9) bits, as evenly as possible.
static void radix_sort(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                       uint32_t *ktmp, uint32_t *vtmp, const int *n_ptr, int cap, int bits,
                       uint32_t *hist, uint32_t *totals, int G, cudaStream_t st, int max_bits) {
    const int passes = (bits + max_bits - 1) / max_bits;
    const uint32_t *ks = kin, *vs = vin;
    int shift = 0;
    for (int p = 0; p < passes; ++p) {
        const int nb = (bits - shift + (passes - p) - 1) / (passes - p);
        const uint32_t mask = (1u << nb) - 1u;
        uint32_t *kd = ((passes - 1 - p) % 2 == 0) ? kout : ktmp;
        uint32_t *vd = ((passes - 1 - p) % 2 == 0) ? vout : vtmp;
        const ArrayPairs src{ks, vs};
        if (nb > 8) {
            launch_pdl(rs_hist_kernel<ArrayPairs, 512>, G, kScanThreads, 0, st, src, n_ptr, cap, shift, mask, hist, G);
            launch_pdl(rs_digit_scan_kernel, 512, kScanThreads, 0, st, hist, totals, G);
            launch_pdl(rs_scatter_kernel<ArrayPairs, 512>, G, kScanThreads, 0, st, src, kd, vd, n_ptr, cap, shift, mask,
                       hist, totals, G);
        } else {
            launch_pdl(rs_hist_kernel<ArrayPairs, 256>, G, kScanThreads, 0, st, src, n_ptr, cap, shift, mask, hist, G);
            launch_pdl(rs_digit_scan_kernel, 256, kScanThreads, 0, st, hist, totals, G);
            launch_pdl(rs_scatter_kernel<ArrayPairs, 256>, G, kScanThreads, 0, st, src, kd, vd, n_ptr, cap, shift, mask,
                       hist, totals, G);
        }
        count_launches(3);
        ks = kd;
        vs = vd;
        shift += nb;
    }
}

__global__ void clamp_count_kernel(const int *in, int cap, int *out) {
    pdl_begin();
    *out = min(*in, cap);
}

// [start, end) of every tile by binary search in the sorted tile ids ((0, 0) for a tile with
// no instance): one thread per tile, no prior zeroing.
__device__ __forceinline__ int lower_bound_u32(const uint32_t *__restrict__ a, int n, uint32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__global__ void ranges_kernel(const uint32_t *__restrict__ tile, const int *__restrict__ k_ptr, int n_tiles,
                              int2 *__restrict__ ranges) {
    pdl_begin();
    const int K = *k_ptr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
        const int lo = lower_bound_u32(tile, K, (uint32_t)t);
        const int hi = lower_bound_u32(tile, K, (uint32_t)t + 1u);
        ranges[t] = lo < hi ? make_int2(lo, hi) : make_int2(0, 0);
    }
}

// ---------------------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------------------

struct TileWorkspace {
    uint32_t *dkey_in, *dval_in, *dkey_out, *dval_out, *dkey_tmp, *dval_tmp;
    uint32_t *slot0;      // first (record, tile row) slot of each depth-sorted record
    uint32_t *first_rec;  // record owning the first slot of each block of the slot partition
    uint32_t *kbsum;      // kept instances per block of the slot partition, then their offsets
    uint32_t *tkey_in, *tval_in, *tkey_tmp, *tval_tmp;
    uint32_t *bsum, *hist, *totals;
    int *counts;  // [0] visible records M, [1] K clamped
};

static int sort_grid() {
    static int G = 0;
    if (!G) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        G = sms > 0 ? 4 * sms : 512;
        if (G > 4096) G = 4096;
    }
    return G;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t tile_ws_layout(int64_t R, int32_t cap, int G, TileWorkspace *ws, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    const size_t r4 = (size_t)R * 4, c4 = (size_t)cap * 4;
    TileWorkspace w{};
    w.dkey_in = (uint32_t *)take(r4);
    w.dval_in = (uint32_t *)take(r4);
    w.dkey_out = (uint32_t *)take(r4);
    w.dval_out = (uint32_t *)take(r4);
    w.dkey_tmp = (uint32_t *)take(r4);
    w.dval_tmp = (uint32_t *)take(r4);
    w.slot0 = (uint32_t *)take(r4);
    w.first_rec = (uint32_t *)take((size_t)4 * G * 4);  // the slot partition has 4 G blocks
    w.kbsum = (uint32_t *)take((size_t)4 * G * 4);

    w.tkey_in = (uint32_t *)take(c4);
    w.tval_in = (uint32_t *)take(c4);
    w.tkey_tmp = (uint32_t *)take(c4);
    w.tval_tmp = (uint32_t *)take(c4);
    w.bsum = (uint32_t *)take((size_t)4 * G * 4);  // up to 4 G blocks (the emission grid)
    w.hist = (uint32_t *)take((size_t)G * 512 * 4);
    w.totals = (uint32_t *)take(512 * 4);
    w.counts = (int *)take(4 * sizeof(int));
    if (ws) *ws = w;
    return off;
}

size_t tile_lists_workspace_size(int64_t R, int32_t cap) {
    return tile_ws_layout(R, cap, sort_grid(), nullptr, nullptr);
}

sg_status launch_build_tile_lists(const sg_projected *proj, int N, int n_views,
                                  const sg_view *views, int n_tiles, int tile_w, int tile_h, sg_tile_lists *lists,
                                  void *workspace, size_t ws_bytes, uint32_t *status,
                                  cudaStream_t st) {
    const int G = sort_grid();
    const int64_t R = (int64_t)N * n_views;
    TileWorkspace w;
    const size_t need = tile_ws_layout(R, lists->capacity, G, &w, (char *)workspace);
    if (ws_bytes < need) {
        set_error("build_tile_lists: workspace %zu bytes < %zu needed", ws_bytes, need);
        return SG_ERR_CAPACITY;
    }
    const uint2 *rect = reinterpret_cast<const uint2 *>(proj->rect);
    const float4 *geo = reinterpret_cast<const float4 *>(proj->geo);
    // 1. compaction of visible records (count -> counts[0])
    launch_pdl(scan_reduce_kernel<VisibleCount>, G, kScanThreads, 0, st, VisibleCount{rect}, nullptr, (int)R, w.bsum, G);
    launch_pdl(scan_blocks_kernel, 1, kScanThreads, 0, st, w.bsum, G, w.counts + 0);
    launch_pdl(compact_apply_kernel, G, kScanThreads, 0, st, rect, geo, (int)R, w.bsum, G, w.dkey_in, w.dval_in);
    // 2. depth sort (32 bits).  Its input (the visible records) is a small fraction of R, so it
    // runs on a grid of about 2048 elements per block for R / 4, between G / 4 and G.
    const int Gd = (int)std::min<int64_t>(G, std::max<int64_t>(G / 4, R / (4 * 2048)));
    radix_sort(w.dkey_in, w.dval_in, w.dkey_out, w.dval_out, w.dkey_tmp, w.dval_tmp, w.counts + 0,
               (int)R, 32, w.hist, w.totals, Gd, st, 8);
    // 3. emission in depth order (K -> lists->count)
    // The emission runs on a finer grid for large inputs (up to 4 G blocks, about one per 2048
    // records): its blocks own ranges of depth-sorted records, and the near (large) ones,
    // which emit most of the instances, come first.
    const int Ge = (int)std::min<int64_t>(4 * G, std::max<int64_t>(G, R / 2048));
    // slots: the rectangle tile rows of the records in depth order
    const float2 *ext = reinterpret_cast<const float2 *>(proj->ext);
    launch_pdl(scan_reduce_kernel<SortedRowCount>, Ge, kScanThreads, 0, st, SortedRowCount{rect, w.dval_out},
               w.counts + 0, 0, w.bsum, Ge);
    launch_pdl(scan_blocks_kernel, 1, kScanThreads, 0, st, w.bsum, Ge, w.counts + 2);
    const int Gc = 4 * G;  // blocks of the slot partition (each walks a few 256-slot chunks)
    const bool halves = lists->half_masks != 0;  // records carry half masks
    launch_pdl(slot_prefix_kernel, Ge, kScanThreads, 0, st, rect, w.dval_out, w.counts + 0, w.bsum, Ge,
               w.counts + 2, Gc, w.slot0, w.first_rec);
    // culling, evenly over the slots: kept counts, their offsets, emission (the tile sort's
    // ping-pong buffers and the output tile ids, all free until the sort, hold the slot cache)
    const auto count_pass = halves ? cull_pass_kernel<false, true> : cull_pass_kernel<false, false>;
    const auto emit_pass = halves ? cull_pass_kernel<true, true> : cull_pass_kernel<true, false>;
    launch_pdl(count_pass, Gc, kScanThreads, 0, st, rect, geo, ext, w.dval_out, w.counts + 0, w.counts + 2, w.slot0,
               w.first_rec, Gc, N, views, n_views, tile_w, tile_h, w.kbsum, (uint32_t *)nullptr,
               (uint32_t *)nullptr, w.tkey_tmp, w.tval_tmp, lists->tile, lists->capacity, status);
    launch_pdl(scan_blocks_kernel, 1, kScanThreads, 0, st, w.kbsum, Gc, lists->count);
    launch_pdl(emit_pass, Gc, kScanThreads, 0, st, rect, geo, ext, w.dval_out, w.counts + 0, w.counts + 2, w.slot0,
               w.first_rec, Gc, N, views, n_views, tile_w, tile_h, w.kbsum, w.tkey_in, w.tval_in, w.tkey_tmp,
               w.tval_tmp, lists->tile, lists->capacity, status);
    // 4. stable sort by tile id
    int bits = 1;
    while ((1ll << bits) < (long long)n_tiles) ++bits;
    radix_sort(w.tkey_in, w.tval_in, lists->tile, lists->record, w.tkey_tmp, w.tval_tmp,
               lists->count, lists->capacity, bits, w.hist, w.totals, G, st, kTileDigitBits);
    // 5. tile ranges
    launch_pdl(clamp_count_kernel, 1, 1, 0, st, lists->count, lists->capacity, w.counts + 1);
    launch_pdl(ranges_kernel, (n_tiles + kScanThreads - 1) / kScanThreads, kScanThreads, 0, st, lists->tile,
               w.counts + 1, n_tiles, reinterpret_cast<int2 *>(lists->ranges));
    count_launches(3 + 6 + 2);  // compaction, slots + culling + emission, clamp + ranges
    // 6. work order: one stable counting pass over the 6-bit length keys
    if (lists->order) {
        const TileLengthKeys src{reinterpret_cast<const int2 *>(lists->ranges)};
        launch_pdl(rs_hist_kernel<TileLengthKeys, 256>, G, kScanThreads, 0, st, src, nullptr, n_tiles, 0, 63u, w.hist, G);
        launch_pdl(rs_digit_scan_kernel, 256, kScanThreads, 0, st, w.hist, w.totals, G);
        launch_pdl(rs_scatter_kernel<TileLengthKeys, 256>, G, kScanThreads, 0, st, src, nullptr, reinterpret_cast<uint32_t *>(lists->order),
                                                      nullptr, n_tiles, 0, 63u, w.hist, w.totals, G);
        count_launches(3);
    }
    return check_launch("build_tile_lists");
}

}  // namespace sg
