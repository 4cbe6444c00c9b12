// mlp.cu -- the learned Gaussian initializer (not in the paper): a 3-layer BF16 MLP with
// FP32 accumulation, 2048 (2009 used) -> 128 -> 128 -> 32 (20 used), trained and run by
// the tcgen05 GEMM of tc_gemm.cuh.
//
// Forward (per batch of B rows, B % 128 == 0):
//   H1 = relu(X W1^T + b1)      A = X [B][2048],  B-operand = W1 [128][2048]
//   H2 = relu(H1 W2^T + b2)     A = H1 [B][128],  B-operand = W2 [128][128]
//   Y  = H2 W3^T + b3           A = H2 [B][128],  B-operand = W3 [32][128]
// Backward of L = sum_o w_o mean_b (Y - T)^2:
//   dY = 2 w (Y - T) / B                               (CUDA cores)
//   dW3^T = H2^T dY   (K = B)   A = H2t [128][B],  B-operand = dYt [32][B]
//   dH2 = (dY W3) * [H2 > 0]    A = dY [B][64],    B-operand = W3t [128][64]
//   dW2^T = H1^T dH2  (K = B)   A = H1t [128][B],  B-operand = dH2t [128][B]
//   dH1 = (dH2 W2) * [H1 > 0]   A = dH2 [B][128],  B-operand = W2t [128][128]
//   dW1 = dH1^T X     (K = B)   A = dH1t [128][B], B-operand = Xt [2048][B]
// Every operand is K-major: the epilogues write the transposed copies (H1t, H2t, dYt,
// dH2t, dH1t) the later GEMMs need, and the patch extractor writes X and Xt.  The K = B
// reductions are split over CTAs and atomically added into the FP32 gradients.
#include <cstdio>
#include <cstring>

#include "tc_gemm.cuh"

namespace sg {

using bf16 = __nv_bfloat16;

// cuTensorMapEncodeTiled from the driver, found through the runtime's entry-point query (the
// library links only the runtime).  NULL when the driver does not provide it.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
        cudaGetLastError();
    }
    return fn;
}

// Tensor map of a rows x K bf16 operand (K contiguous, leading dimension ld elements) read in
// boxes of 64 (K) x box_rows with the 128-byte swizzle; rows beyond `rows` read as zero.
static bool make_operand_map(CUtensorMap *map, const bf16 *base, long long rows, long long K, long long ld,
                             int box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STAGES, bool TMA>
static sg_status launch_gemm_kernel(const tc::GemmParams &p, int splits, const CUtensorMap &ma,
                                    const CUtensorMap &mb, cudaStream_t st) {
    constexpr size_t smem = tc::gemm_smem_bytes<BN, STAGES>();
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(tc::gemm_kernel<BN, STAGES, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return check_launch("gemm smem attribute");
        attr = true;
    }
    const dim3 grid((p.M + 127) / 128, (p.N + BN - 1) / BN, splits);
    tc::gemm_kernel<BN, STAGES, TMA><<<grid, 128, smem, st>>>(p, ma, mb);
    count_launches(1);
    return check_launch("tcgen05 gemm");
}

template <int BN, int STAGES>
static sg_status launch_gemm_t(const tc::GemmParams &p, int splits, cudaStream_t st) {
    // operands staged by TMA (tensor maps, 128-byte swizzle); by cp.async only when the driver
    // offers no tensor-map encoder
    CUtensorMap ma, mb;
    if (make_operand_map(&ma, p.A, p.M, p.K, p.lda, 128) &&
        make_operand_map(&mb, p.B, p.N, p.K, p.ldb, BN))
        return launch_gemm_kernel<BN, STAGES, true>(p, splits, ma, mb, st);
    memset(&ma, 0, sizeof(ma));
    memset(&mb, 0, sizeof(mb));
    return launch_gemm_kernel<BN, STAGES, false>(p, splits, ma, mb, st);
}

// Chooses the tile width from N and splits K so that the grid covers the SMs.
sg_status launch_gemm(tc::GemmParams p, cudaStream_t st, int max_splits = 64) {
    if (p.K % 64 != 0 || p.M <= 0 || p.N <= 0 || p.K <= 0) {
        set_error("gemm: need M, N > 0 and K a positive multiple of 64 (M=%d N=%d K=%d)", p.M, p.N, p.K);
        return SG_ERR_INVALID_ARG;
    }
    const int BN = p.N <= 32 ? 32 : (p.N <= 128 ? 128 : 256);
    const int tiles = ((p.M + 127) / 128) * ((p.N + BN - 1) / BN);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int splits = 1;
    if (p.f32_atomic && p.out_f32 && !p.out_bf16 && !p.out_bf16_t && !p.relu && !p.mask) {
        const int kch = p.K / 64;
        splits = (sms + tiles - 1) / tiles;
        if (splits > kch) splits = kch;
        if (splits > max_splits) splits = max_splits;
        if (splits < 1) splits = 1;
    }
    const int kch = p.K / 64;
    const int per = (kch + splits - 1) / splits;
    p.k_per_split = per * 64;
    splits = (kch + per - 1) / per;
    if (splits > 1 && p.bias) {
        set_error("gemm: bias with split-K is not supported");
        return SG_ERR_INVALID_ARG;
    }
    switch (BN) {
        case 32: return launch_gemm_t<32, 4>(p, splits, st);
        // 3 stages of 32 KiB: two CTAs per SM keep twice the operand bytes in flight
        // (layer 1 at 65536 rows: 133 -> 107 us against 4 stages and one CTA)
        case 128: return launch_gemm_t<128, 3>(p, splits, st);
        default: return launch_gemm_t<256, 3>(p, splits, st);
    }
}

static tc::GemmParams gemm_params(const bf16 *A, long long lda, const bf16 *B, long long ldb, int M, int N,
                                  int K, uint32_t *status) {
    tc::GemmParams p{};
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb;
    p.M = M; p.N = N; p.K = K;
    p.alpha = 1.f;
    p.status = status;
    return p;
}

// ---------------------------------------------------------------------------------------
// small CUDA-core kernels of the MLP
// ---------------------------------------------------------------------------------------

// fp32 [rows][cols] -> bf16 [rows][cols] and bf16 [cols][ld_t] transposed (zero columns of
// the transposed copy beyond rows are left untouched: the caller zeroes them once)
__global__ void pack_weight_kernel(const float *__restrict__ W, int rows, int cols, bf16 *__restrict__ Wb,
                                   bf16 *__restrict__ Wt, int ld_t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    const bf16 v = __float2bfloat16_rn(W[i]);
    if (Wb) Wb[i] = v;
    if (Wt) Wt[(long long)c * ld_t + r] = v;
}

// dY = 2 w_o (Y - T) / B (bf16, [B][64] with columns >= 32 zero, and [32][B]); loss += sum
__global__ void mse_head_kernel(const float *__restrict__ Y, const float *__restrict__ T,
                                const float *__restrict__ w, int B, bf16 *__restrict__ dY,
                                bf16 *__restrict__ dYt, float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over B * 64
    float l = 0.f;
    if (i < B * 64) {
        const int b = i / 64, o = i % 64;
        float g = 0.f;
        if (o < 32) {
            const float d = Y[(long long)b * 32 + o] - T[(long long)b * 32 + o];
            l = w[o] * d * d / (float)B;
            g = 2.f * w[o] * d / (float)B;
            dYt[(long long)o * B + b] = __float2bfloat16_rn(g);
        }
        dY[(long long)b * 64 + o] = __float2bfloat16_rn(g);
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(SG_FULL_MASK, l, off);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// out[r] += sum_c M[r][c] for a bf16 [rows][cols] matrix (one CTA per row)
__global__ void row_sum_kernel(const bf16 *__restrict__ M, int cols, float *__restrict__ out) {
    const int r = blockIdx.x;
    float s = 0.f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += __bfloat162float(M[(long long)r * cols + c]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(SG_FULL_MASK, s, off);
    __shared__ float sw[32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
        out[r] += t;
    }
}

}  // namespace sg

using namespace sg;

#define MLP_REQUIRE(cond, ...)         \
    do {                               \
        if (!(cond)) {                 \
            set_error(__VA_ARGS__);    \
            return SG_ERR_INVALID_ARG; \
        }                              \
    } while (0)
#define MLP_TRY(expr)                 \
    do {                              \
        const sg_status _s = (expr);  \
        if (_s != SG_OK) return _s;   \
    } while (0)

extern "C" {

sg_status sg_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int32_t M, int32_t N,
                       int32_t K, float *D, int64_t ldd, int32_t accumulate, uint32_t *status,
                       sg_stream_t stream) {
    MLP_REQUIRE(A && B && D, "gemm: NULL operand");
    MLP_REQUIRE(M > 0 && N > 0 && K > 0 && K % 64 == 0, "gemm: need M, N > 0 and K %% 64 == 0");
    MLP_REQUIRE(lda % 8 == 0 && ldb % 8 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0,
                "gemm: operands need 16-byte aligned rows");
    tc::GemmParams p = gemm_params((const bf16 *)A, lda, (const bf16 *)B, ldb, M, N, K, status);
    p.out_f32 = D;
    p.ld_f32 = ldd;
    p.f32_atomic = accumulate ? 1 : 0;
    return launch_gemm(p, (cudaStream_t)stream);
}

sg_status sg_gemm_bf16_timeout_probe(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int32_t M,
                                     int32_t N, int32_t K, float *D, int64_t ldd, uint32_t polls,
                                     uint32_t *status, sg_stream_t stream) {
    MLP_REQUIRE(A && B && D, "gemm: NULL operand");
    MLP_REQUIRE(M > 0 && N > 0 && K > 0 && K % 64 == 0, "gemm: need M, N > 0 and K %% 64 == 0");
    MLP_REQUIRE(lda % 8 == 0 && ldb % 8 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0,
                "gemm: operands need 16-byte aligned rows");
    MLP_REQUIRE(polls >= 1 && polls <= (1u << 20), "timeout probe: polls must be in [1, 2^20]");
    tc::GemmParams p = gemm_params((const bf16 *)A, lda, (const bf16 *)B, ldb, M, N, K, status);
    p.out_f32 = D;
    p.ld_f32 = ldd;
    p.probe_polls = polls;
    return launch_gemm(p, (cudaStream_t)stream);
}

sg_status sg_mlp_pack_weights(const float *W1, const float *W2, const float *W3, uint16_t *W1b, uint16_t *W2b,
                              uint16_t *W3b, uint16_t *W2t, uint16_t *W3t, sg_stream_t stream) {
    MLP_REQUIRE(W1 && W2 && W3 && W1b && W2b && W3b && W2t && W3t, "pack_weights: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    pack_weight_kernel<<<(SG_MLP_HIDDEN * SG_MLP_IN + 255) / 256, 256, 0, st>>>(W1, SG_MLP_HIDDEN, SG_MLP_IN,
                                                                                 (bf16 *)W1b, nullptr, 0);
    pack_weight_kernel<<<(SG_MLP_HIDDEN * SG_MLP_HIDDEN + 255) / 256, 256, 0, st>>>(
        W2, SG_MLP_HIDDEN, SG_MLP_HIDDEN, (bf16 *)W2b, (bf16 *)W2t, SG_MLP_HIDDEN);
    pack_weight_kernel<<<(SG_MLP_OUT * SG_MLP_HIDDEN + 255) / 256, 256, 0, st>>>(
        W3, SG_MLP_OUT, SG_MLP_HIDDEN, (bf16 *)W3b, (bf16 *)W3t, 64);
    count_launches(3);
    return check_launch("mlp_pack_weights");
}

sg_status sg_mlp_forward(const sg_mlp *net, const uint16_t *X, int32_t B, sg_mlp_acts *acts, uint32_t *status,
                         sg_stream_t stream) {
    MLP_REQUIRE(net && X && acts && acts->H1 && acts->H2 && acts->Y, "mlp_forward: NULL argument");
    MLP_REQUIRE(B > 0 && B % 128 == 0, "mlp_forward: B = %d must be a positive multiple of 128", B);
    cudaStream_t st = (cudaStream_t)stream;
    const int H = SG_MLP_HIDDEN;
    tc::GemmParams p = gemm_params((const bf16 *)X, SG_MLP_IN, (const bf16 *)net->W1, SG_MLP_IN, B, H, SG_MLP_IN,
                                   status);
    p.bias = net->b1; p.relu = 1;
    p.out_bf16 = (bf16 *)acts->H1; p.ld_bf16 = H;
    p.out_bf16_t = (bf16 *)acts->H1t; p.ld_bf16_t = B;
    MLP_TRY(launch_gemm(p, st));
    p = gemm_params((const bf16 *)acts->H1, H, (const bf16 *)net->W2, H, B, H, H, status);
    p.bias = net->b2; p.relu = 1;
    p.out_bf16 = (bf16 *)acts->H2; p.ld_bf16 = H;
    p.out_bf16_t = (bf16 *)acts->H2t; p.ld_bf16_t = B;
    MLP_TRY(launch_gemm(p, st));
    p = gemm_params((const bf16 *)acts->H2, H, (const bf16 *)net->W3, H, B, SG_MLP_OUT, H, status);
    p.bias = net->b3;
    p.out_f32 = acts->Y; p.ld_f32 = SG_MLP_OUT;
    return launch_gemm(p, st);
}

sg_status sg_mlp_backward(const sg_mlp *net, const uint16_t *Xt, const float *target, const float *out_weight,
                          int32_t B, sg_mlp_acts *acts, sg_mlp_grads *grads, float *loss, uint32_t *status,
                          sg_stream_t stream) {
    MLP_REQUIRE(net && Xt && target && out_weight && acts && grads && loss, "mlp_backward: NULL argument");
    MLP_REQUIRE(acts->H1t && acts->H2t && acts->dY && acts->dYt && acts->dH2 && acts->dH2t && acts->dH1t,
                "mlp_backward: activation buffers are NULL");
    MLP_REQUIRE(grads->W1 && grads->W2 && grads->W3 && grads->b1 && grads->b2 && grads->b3,
                "mlp_backward: gradient buffers are NULL");
    MLP_REQUIRE(B > 0 && B % 128 == 0, "mlp_backward: B = %d must be a positive multiple of 128", B);
    cudaStream_t st = (cudaStream_t)stream;
    const int H = SG_MLP_HIDDEN, O = SG_MLP_OUT;
    mse_head_kernel<<<(B * 64 + 255) / 256, 256, 0, st>>>(acts->Y, target, out_weight, B, (bf16 *)acts->dY,
                                                          (bf16 *)acts->dYt, loss);
    count_launches(1);
    // dW3 [32][128] += (H2^T dY)^T
    tc::GemmParams p = gemm_params((const bf16 *)acts->H2t, B, (const bf16 *)acts->dYt, B, H, O, B, status);
    p.out_f32 = grads->W3; p.ld_f32 = H; p.f32_transposed = 1; p.f32_atomic = 1;
    MLP_TRY(launch_gemm(p, st));
    // dH2 = (dY W3) * [H2 > 0]
    p = gemm_params((const bf16 *)acts->dY, 64, (const bf16 *)net->W3t, 64, B, H, 64, status);
    p.mask = (const bf16 *)acts->H2; p.ldmask = H;
    p.out_bf16 = (bf16 *)acts->dH2; p.ld_bf16 = H;
    p.out_bf16_t = (bf16 *)acts->dH2t; p.ld_bf16_t = B;
    MLP_TRY(launch_gemm(p, st));
    // dW2 [128][128] += (H1^T dH2)^T
    p = gemm_params((const bf16 *)acts->H1t, B, (const bf16 *)acts->dH2t, B, H, H, B, status);
    p.out_f32 = grads->W2; p.ld_f32 = H; p.f32_transposed = 1; p.f32_atomic = 1;
    MLP_TRY(launch_gemm(p, st));
    // dH1 = (dH2 W2) * [H1 > 0], transposed copy only
    p = gemm_params((const bf16 *)acts->dH2, H, (const bf16 *)net->W2t, H, B, H, H, status);
    p.mask = (const bf16 *)acts->H1; p.ldmask = H;
    p.out_bf16_t = (bf16 *)acts->dH1t; p.ld_bf16_t = B;
    MLP_TRY(launch_gemm(p, st));
    // dW1 [128][2048] += dH1^T X
    p = gemm_params((const bf16 *)acts->dH1t, B, (const bf16 *)Xt, B, H, SG_MLP_IN, B, status);
    p.out_f32 = grads->W1; p.ld_f32 = SG_MLP_IN; p.f32_atomic = 1;
    MLP_TRY(launch_gemm(p, st));
    // bias gradients: row sums of the transposed copies
    row_sum_kernel<<<O, 256, 0, st>>>((const bf16 *)acts->dYt, B, grads->b3);
    row_sum_kernel<<<H, 256, 0, st>>>((const bf16 *)acts->dH2t, B, grads->b2);
    row_sum_kernel<<<H, 256, 0, st>>>((const bf16 *)acts->dH1t, B, grads->b1);
    count_launches(3);
    return check_launch("mlp_backward");
}

}  // extern "C"
