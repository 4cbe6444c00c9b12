// tc_gemm.cuh -- a BF16 GEMM on the 5th-generation tensor cores (tcgen05) for sm_103a.
//
//   D[M x N] = alpha * A[M x K] * B[N x K]^T   (A, B bf16 with K contiguous, D fp32 in TMEM)
//
// One CTA of 4 warps computes a 128 x BN tile.  Operand tiles of 128 x 64 (A) and BN x 64
// (B) are staged into shared memory in one of two K-major layouts:
//  - TMA (the default): one thread issues two cp.async.bulk.tensor loads per stage (tensor
//    maps with 128-byte swizzle: each 128-byte row of 64 bf16 holds its 16-byte chunks XOR-
//    permuted by the row index mod 8, 8-row groups 1 KiB apart), whose completion is counted
//    in bytes on the stage's "full" mbarrier; the MMA descriptors use the matching
//    128-byte-swizzle layout and step 32 bytes along K per K=16 MMA.
//  - cp.async (the fallback): all threads copy 16-byte chunks into the no-swizzle layout:
//    8-row x 16-byte core matrices stored as contiguous 128-byte blocks, the 8 core matrices
//    of one 8-row group along K contiguous (leading byte offset 128 B), 8-row groups 1 KiB
//    apart (stride byte offset 1024 B).
// One elected thread issues four K=16 tcgen05.mma.kind::f16 per stage and tcgen05.commit
// arrives on the stage's "empty" mbarrier when those MMAs have read the stage, which releases
// it for the next refill (STAGES-deep pipeline).  The accumulator lives in TMEM (128 lanes x BN fp32 columns);
// the epilogue reads it back with tcgen05.ld.32x32b (warp w owns lanes 32w..32w+31, one
// output row per thread) and applies bias / ReLU / ReLU-mask before storing bf16 (row-major
// and/or transposed) or fp32 (stored, or atomically added for split-K).
//
// Every mbarrier wait is bounded: after kSpinLimit polls the CTA records SG_STATUS_TIMEOUT
// in the caller's status word, waits (bounded again) for its issued MMAs, frees its TMEM
// and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "sg_common.cuh"

#define SG_STATUS_TIMEOUT_BIT 4u

namespace sg {
namespace tc {

constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok;
}
// Bounded wait for the phase with the given parity; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Instruction descriptor of kind::f16: D fp32 (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Shared-memory matrix descriptor, no swizzle: start address >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// The same for a K-major tile in the 128-byte swizzle layout (layout type 2 at bits 61-63):
// 8-row groups 1 KiB apart (stride byte offset), leading byte offset unused (1); the tile base
// is 1 KiB aligned, and saddr may step by 32 bytes along K inside the 128-byte swizzle row.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// mbarrier arrive that also announces `bytes` of asynchronous (TMA) transfer to wait for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// 2-D tiled TMA load of the box at (x = inner coordinate, y) into shared memory; completion is
// counted on bar.  x must be a multiple of 8 bf16 elements (16 bytes).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

struct GemmParams {
    const __nv_bfloat16 *A;
    long long lda;  // M x K
    const __nv_bfloat16 *B;
    long long ldb;  // N x K
    int M, N, K;    // K % 64 == 0
    int k_per_split;  // multiple of 64; grid.z = ceil(K / k_per_split)
    float alpha;
    const float *bias;  // N, or null
    int relu;
    const __nv_bfloat16 *mask;  // keep D where mask > 0 (M x N), or null
    long long ldmask;
    __nv_bfloat16 *out_bf16;  // M x N row-major, or null
    long long ld_bf16;
    __nv_bfloat16 *out_bf16_t;  // N x M (transposed), or null
    long long ld_bf16_t;
    float *out_f32;  // M x N (or N x M if f32_transposed), or null
    long long ld_f32;
    int f32_transposed;
    int f32_atomic;  // 1: atomicAdd (split-K / accumulation), 0: store
    uint32_t *status;
    // failure-detection self-test: before its main loop the CTA waits on a barrier that
    // nothing arrives on, bounded by probe_polls polls; 0 = no such wait
    uint32_t probe_polls;
};

template <int BN, int STAGES, bool TMA>
__global__ void __launch_bounds__(128, 2) gemm_kernel(const GemmParams p, const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "BN");
    constexpr int A_BYTES = 128 * 64 * 2;
    constexpr int B_BYTES = BN * 64 * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzled tiles are 1 KiB aligned");
    constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    constexpr uint32_t IDESC = idesc_bf16_f32(128, BN);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ uint64_t bars[STAGES];  // "empty": the stage's MMAs have read it
    __shared__ uint64_t full[STAGES];  // "full": the stage's TMA bytes have landed (TMA mode)
    __shared__ uint64_t probe_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_timeout;
    __shared__ int s_issued;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int k_begin = blockIdx.z * p.k_per_split;
    const int k_end = min(p.K, k_begin + p.k_per_split);
    const int nk = k_end > k_begin ? (k_end - k_begin) / 64 : 0;
    uint32_t sbase = smem_addr(smem_raw);
    sbase = (sbase + 1023u) & ~1023u;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bars[s], 1);
            mbar_init(&full[s], 1);
        }
        mbar_init(&probe_bar, 1);
        s_timeout = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(&tmem_base_s), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    if (p.probe_polls) {
        // phase 0 of probe_bar never completes: the wait gives up after probe_polls polls
        if (tid == 0 && !mbar_wait(&probe_bar, 0, p.probe_polls)) {
            s_timeout = 1;
            if (p.status) atomicOr(p.status, SG_STATUS_TIMEOUT_BIT);
        }
        __syncthreads();
    }

    int issued = 0;  // MMA batches committed
    if constexpr (TMA) {
        // one thread streams the operands (TMA) and issues the MMAs; a stage is refilled once
        // the MMAs that read it have committed
        if (tid == 0 && !s_timeout) {
            auto load_stage = [&](int kc, int s) {
                const uint32_t a_s = sbase + s * STAGE_BYTES, b_s = a_s + A_BYTES;
                const int k0 = k_begin + kc * 64;
                mbar_arrive_expect_tx(&full[s], (uint32_t)STAGE_BYTES);
                tma_load_2d(a_s, &tmA, k0, m0, &full[s]);
                tma_load_2d(b_s, &tmB, k0, n0, &full[s]);
            };
            int loaded = 0;  // stages whose loads were issued
            for (int s = 0; s < STAGES - 1 && s < nk; ++s) load_stage(s, s), ++loaded;
            bool ok = true;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int s = kc % STAGES;
                if (!mbar_wait(&full[s], (kc / STAGES) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a_s = sbase + s * STAGE_BYTES, b_s = a_s + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_bf16(tmem, sdesc_sw128(a_s + kk * 32), sdesc_sw128(b_s + kk * 32), IDESC,
                             (kc > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&bars[s]);
                issued = kc + 1;
                const int nxt = kc + STAGES - 1;
                if (nxt < nk) {
                    const int ns = nxt % STAGES;
                    // the stage held chunk nxt - STAGES (= kc - 1): wait until its MMAs read it
                    if (nxt >= STAGES && !mbar_wait(&bars[ns], ((nxt - STAGES) / STAGES) & 1)) { ok = false; break; }
                    load_stage(nxt, ns);
                    ++loaded;
                }
            }
            if (!ok) {
                s_timeout = 1;
                if (p.status) atomicOr(p.status, SG_STATUS_TIMEOUT_BIT);
                // let every issued TMA load land before the CTA may exit (bounded)
                for (int c = issued; c < loaded; ++c) mbar_wait(&full[c % STAGES], (c / STAGES) & 1);
            }
            s_issued = issued;
        }
        __syncthreads();
        issued = s_issued;
    } else {
    auto load_stage = [&](int kc, int s) {
        const int k0 = k_begin + kc * 64;
        const uint32_t a_s = sbase + s * STAGE_BYTES, b_s = a_s + A_BYTES;
        for (int i = tid; i < 128 * 8; i += 128) {
            const int r = i >> 3, c = i & 7;
            const int gm = m0 + r;
            const bool ok = gm < p.M;
            const __nv_bfloat16 *src = p.A + (long long)(ok ? gm : 0) * p.lda + k0 + c * 8;
            cp_async16(a_s + (r >> 3) * 1024 + c * 128 + (r & 7) * 16, src, ok);
        }
        for (int i = tid; i < BN * 8; i += 128) {
            const int r = i >> 3, c = i & 7;
            const int gn = n0 + r;
            const bool ok = gn < p.N;
            const __nv_bfloat16 *src = p.B + (long long)(ok ? gn : 0) * p.ldb + k0 + c * 8;
            cp_async16(b_s + (r >> 3) * 1024 + c * 128 + (r & 7) * 16, src, ok);
        }
    };

    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % STAGES;
        cp_async_wait<STAGES - 2>();
        fence_proxy_async();
        __syncthreads();
        if (s_timeout) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a_s = sbase + s * STAGE_BYTES, b_s = a_s + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, sdesc(a_s + kk * 256, 128, 1024), sdesc(b_s + kk * 256, 128, 1024), IDESC,
                         (kc > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&bars[s]);
        }
        issued = kc + 1;
        const int nxt = kc + STAGES - 1;
        if (nxt < nk) {
            const int ns = nxt % STAGES;
            if (nxt >= STAGES) {
                // the stage held chunk nxt - STAGES (= kc - 1): wait until its MMAs read it
                if (!mbar_wait(&bars[ns], ((nxt - STAGES) / STAGES) & 1)) {
                    s_timeout = 1;
                    if (p.status) atomicOr(p.status, SG_STATUS_TIMEOUT_BIT);
                }
            }
            if (!s_timeout) load_stage(nxt, ns);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    }
    bool done = true;
    if (issued > 0) {
        const int last = issued - 1;
        done = mbar_wait(&bars[last % STAGES], (last / STAGES) & 1);
        if (!done && p.status) atomicOr(p.status, SG_STATUS_TIMEOUT_BIT);
    }
    tc_fence_after();
    __syncthreads();
    const bool write = done && !s_timeout;
    const int row = warp * 32 + lane;
    const int gm = m0 + row;
    if (write) {
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            tmem_ld_wait();
            if (gm >= p.M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int gn = n0 + c0 + j;
                if (gn >= p.N) continue;
                float v = issued > 0 ? p.alpha * __uint_as_float(r[j]) : 0.f;
                if (p.bias) v += p.bias[gn];
                if (p.relu) v = fmaxf(v, 0.f);
                if (p.mask && !(__bfloat162float(p.mask[(long long)gm * p.ldmask + gn]) > 0.f)) v = 0.f;
                if (p.out_bf16) p.out_bf16[(long long)gm * p.ld_bf16 + gn] = __float2bfloat16_rn(v);
                if (p.out_bf16_t) p.out_bf16_t[(long long)gn * p.ld_bf16_t + gm] = __float2bfloat16_rn(v);
                if (p.out_f32) {
                    float *dst = p.f32_transposed ? p.out_f32 + (long long)gn * p.ld_f32 + gm
                                                  : p.out_f32 + (long long)gm * p.ld_f32 + gn;
                    if (p.f32_atomic) {
                        if (issued > 0) atomicAdd(dst, v);
                    } else {
                        *dst = v;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

template <int BN, int STAGES>
constexpr size_t gemm_smem_bytes() {  // (both staging modes)
    return (size_t)STAGES * (128 * 64 * 2 + BN * 64 * 2) + 1024;
}

}  // namespace tc
}  // namespace sg
