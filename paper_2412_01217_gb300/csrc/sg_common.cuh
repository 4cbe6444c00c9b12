// sg_common.cuh -- device helpers shared by the sm_103a kernels of the pyramid splatting
// library.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/sg.h"

#define SG_FULL_MASK 0xffffffffu

namespace sg {

// Largest tile: 32x8 or 16x16 pixels = 256 threads per CTA.
constexpr int kMaxTileThreads = 256;

struct Float3 {
    float x, y, z;
};

// ----------------------------------------------------------------------------------------
// alpha of one Gaussian at one pixel (Eq. 3 with the anisotropic 2D covariance S).  The
// exponent sigma = 1/2 d^T S^{-1} d is evaluated in its conditional (Schur complement)
// form  sigma = (m00 dx)^2 + (m10 dx + m11 dy)^2  with m00 = 1/sqrt(2 s00),
// m10 = -s01/sqrt(2 s00 det), m11 = sqrt(s00/(2 det)): a sum of squares, so no
// cancellation for elongated footprints, and 7 flops.  The forward and backward kernels
// must take bit-identical skip/stop decisions, so every rounding step is spelled out with
// _rn intrinsics (no compiler contraction can differ between kernels).
// ----------------------------------------------------------------------------------------
struct AlphaEval {
    float dx, dy;  // pixel - mean2D
    float p1, p2;  // m00 dx, m10 dx + m11 dy
    float G;       // exp(-sigma)
    float raw;     // o * G
    float alpha;   // min(alpha_max, raw)
};

// (px - ui) and (py - vi) are exact integers held in floats, (uf, vf) the float fractions of
// the 2D mean: dx = (px - ui) - uf is the correctly rounded offset, whatever the tile.
__device__ __forceinline__ bool eval_alpha(float px_ui, float py_vi, float uf, float vf, float m00,
                                           float m10, float m11, float o, float alpha_max,
                                           float alpha_min, AlphaEval &e) {
    e.dx = __fsub_rn(px_ui, uf);
    e.dy = __fsub_rn(py_vi, vf);
    e.p1 = __fmul_rn(m00, e.dx);
    e.p2 = __fmaf_rn(m10, e.dx, __fmul_rn(m11, e.dy));
    const float sigma = __fmaf_rn(e.p2, e.p2, __fmul_rn(e.p1, e.p1));
    if (!(sigma >= 0.f)) return false;
    e.G = __expf(-sigma);
    e.raw = __fmul_rn(o, e.G);
    e.alpha = fminf(alpha_max, e.raw);
    return e.alpha >= alpha_min;
}

// ---- double-float (unevaluated sum hi + lo of two floats) helpers --------------------
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_add_f(DF a, float b) {
    DF s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return two_sum(s.hi, s.lo);
}
// (a.hi + a.lo) * f, f a float
__device__ __forceinline__ DF df_mul_f(DF a, float f) {
    DF p = two_prod(a.hi, f);
    p.lo = __fmaf_rn(a.lo, f, p.lo);
    return two_sum(p.hi, p.lo);
}
// a / b for double-floats (one Newton-style correction of the float quotient)
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q0 = __fdiv_rn(a.hi, b.hi);
    const DF p = two_prod(q0, b.hi);
    float r = __fsub_rn(a.hi, p.hi);
    r = __fsub_rn(r, p.lo);
    r = __fadd_rn(r, a.lo);
    r = __fmaf_rn(-q0, b.lo, r);
    const float q1 = __fdiv_rn(r, b.hi);
    return two_sum(q0, q1);
}

// a*b - c*d with one rounding error (Kahan's algorithm with FMA).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = c * d;
    const float err = __fmaf_rn(-c, d, w);
    const float dop = __fmaf_rn(a, b, -w);
    return dop + err;
}

// ----------------------------------------------------------------------------------------
// TF32 tensor-core products with FP32-level accuracy: x = hi + lo with hi = x with its 13
// low mantissa bits cleared and lo = x - hi (exact); a*b ~ hi*hi + hi*lo + lo*hi keeps about
// 22 mantissa bits of every product (the dropped lo*lo term is below 2^-22 relative).
// mma.m16n8k8 fragments (gid = lane / 4, tig = lane % 4):
//   A (16 x 8): a0 (gid, tig), a1 (gid + 8, tig), a2 (gid, tig + 4), a3 (gid + 8, tig + 4)
//   B (8 x 8):  b0 (tig, gid), b1 (tig + 4, gid)
//   D (16 x 8): d0 (gid, 2 tig), d1 (gid, 2 tig + 1), d2 (gid + 8, 2 tig), d3 (gid + 8, 2 tig + 1)
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    const uint32_t h = __float_as_uint(x) & 0xffffe000u;
    hi = h;
    lo = __float_as_uint(x - __uint_as_float(h));
}

// (no side effects: not volatile, so the compiler may schedule other work around it)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// a * b with both split (3 MMAs, small terms first)
__device__ __forceinline__ void mma_tf32x3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, ah, bh0, bh1);
}

// Two float additions to consecutive, 8-byte aligned addresses in one vector reduction.
__device__ __forceinline__ void red_add_v2(float *addr, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};\n" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// ----------------------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of one iteration are launched with
// launch_pdl() (programmatic stream serialisation), and every kernel starts with
// pdl_begin(): griddepcontrol.wait, which returns once the grids it depends on have completed
// and their writes are visible (at once when the launch has no such dependency).  Nothing
// before it touches global memory, so the ordering is that of plain stream order; the
// launch of each kernel is prepared while its predecessor runs.  (Letting dependents start
// early with griddepcontrol.launch_dependents was measured slower: their waiting blocks take
// SM slots from the running kernel.)
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ int find_view(const sg_view *views, int n_views, int tile) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_offset <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Sets `bit` in *status when `bad` holds for any active lane of the warp (one atomic per
// warp).  Safe in divergent code: only the lanes that reach it take part.
__device__ __forceinline__ void flag_status(bool bad, uint32_t *status, uint32_t bit) {
    const uint32_t m = __ballot_sync(__activemask(), bad);
    if (m && (threadIdx.x & 31) == (uint32_t)(__ffs(m) - 1)) atomicOr(status, bit);
}

__device__ __forceinline__ uint32_t pack16(int a, int b) {
    return (uint32_t)a | ((uint32_t)b << 16);
}

}  // namespace sg

// Internal launch helpers (defined in api.cu / the kernel files).
namespace sg {
void set_error(const char *fmt, ...);
void count_launches(int n);  // kernel launches issued by the library (diagnostics)
sg_status check_launch(const char *what);
}  // namespace sg
