// Tensor-core (tcgen05) Abel GEMMs for sm_103a.
//
// The Abel step of the method (arXiv:1106.0463, Eq. 2.5 evaluated by the
// quadrature of Sec. 2 after Eq. 2.14) is, for a batch of sampled functions,
// the dense product  G[b, j] = sum_k F[b, k] A[j, k]  (rows j = 0..M/2 of the
// grid y_j = 2 pi j/M, K Chebyshev-Lobatto samples).  Its result is
// differenced and scaled by (2n+1) in the FFT stage, which turns white
// rounding noise in G into errors ~ (2N/sqrt(M)) times larger in c_n; FP32
// accumulation of the whole product therefore cannot meet 1e-6.
//
// LEG_SPLIT_FP16 (three-slice split, six products, three accumulators):
//   each operand row is scaled by a power of two (the operator by its L1
//   norm, the input by its max-norm) and split into FP16 slices
//     a = A0 + 2^-9 A1 + 2^-18 A2s,   f = F0 + 2^-9 F1 + 2^-18 F2s,
//   where A0 lies on a 2^-14 grid and F0 on a 2^-9 grid.  Every product
//   A0*F0 is then a multiple of 2^-23 and every partial sum of them is below
//   2 in magnitude, so accumulator 0 (A0 F0) is EXACT in FP32 whatever the
//   accumulation order of the tensor core.  Accumulator 1 (A1 F0 + A0 F1,
//   weight 2^-9) and accumulator 2 (A1 F1 + A2s F0 + A0 F2s, weight 2^-18)
//   carry terms small enough that their FP32 rounding stays below the
//   target.  The epilogue forms G = 2^(e_b + e_j) (acc0 + 2^-9 acc1 +
//   2^-18 acc2) as a double-float pair for the double-float FFT.
// LEG_BF16: one BF16 product into one FP32 accumulator (FP32 G).
//
// Kernel structure (one 128 x 128 output tile per CTA, 192 threads):
//   warp 0 lane 0  TMA producer: per 64-wide K block, loads the operand tiles
//                  (128 rows x 64 FP16, 128-byte swizzle) into a stage and
//                  arms the stage's full barrier with the byte count;
//   warp 1         allocates TMEM (3 x 128 columns); lane 0 issues the
//                  tcgen05.mma instructions (M=128, N=128, K=16 each) and
//                  commits each stage back to the producer;
//   warps 2..5     epilogue: tcgen05.ld of the accumulators (each warp owns
//                  the 32 TMEM lanes of its quadrant), combination, stores.
// Every wait is bounded by a cycle limit; on expiry the kernel records
// LEG_ERR_TIMEOUT in the plan's status word, drains its own TMA copies and
// MMAs (again bounded), releases TMEM and returns.
#include <stdio.h>

#include "leg_fft.cuh"
#include "leg_internal.cuh"
#include "leg_sm100.cuh"

namespace {

constexpr int TILE_M = 128;   // functions per tile (TMEM lanes)
constexpr int TILE_N = 128;   // output columns per tile
constexpr int TILE_K = 64;    // K per stage: one 128-byte swizzle row of FP16
constexpr int TILE_BYTES = TILE_M * TILE_K * 2;   // 16 KB (TILE_M == TILE_N)
constexpr long long DRAIN_LIMIT = 4000000000LL;   // cycles, teardown waits

template <int NPROD> struct TcCfg;
template <> struct TcCfg<6> {
    static constexpr int NPLANES = 3;       // per operand
    static constexpr int STAGES = 2;
    static constexpr uint32_t TMEM_COLS = 512;
};
template <> struct TcCfg<1> {
    static constexpr int NPLANES = 1;
    static constexpr int STAGES = 4;
    static constexpr uint32_t TMEM_COLS = 128;
};

template <int NPROD>
constexpr size_t tc_smem_bytes()
{
    return (size_t)TcCfg<NPROD>::STAGES * 2 * TcCfg<NPROD>::NPLANES * TILE_BYTES + 1024;
}

struct TcMaps {
    CUtensorMap x[3];   // input planes   (B x Kp)
    CUtensorMap w[3];   // operator planes (rows x Kp)
};

// OUT_DF: store G as a double-float pair (float2); else a float.
template <int NPROD, bool OUT_DF>
__global__ void __launch_bounds__(192, 1) tc_gemm_kernel(const __grid_constant__ TcMaps maps, int B, int rows,
                                                         int nkb, const int *__restrict__ xexp,
                                                         const int *__restrict__ wexp, void *__restrict__ out,
                                                         int ldo, int *status, long long wait_limit)
{
    using Cfg = TcCfg<NPROD>;
    constexpr int NP = Cfg::NPLANES;
    constexpr int STAGE_BYTES = 2 * NP * TILE_BYTES;
    constexpr uint32_t IDESC = sm100::idesc_f16(TILE_M, TILE_N, NPROD == 1 ? 1 : 0);

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[Cfg::STAGES];
    __shared__ __align__(8) uint64_t empty_bar[Cfg::STAGES];
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ uint32_t tmem_slot;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = blockIdx.x * TILE_N, b0 = blockIdx.y * TILE_M;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            sm100::mbar_init(&full_bar[s], 1);
            sm100::mbar_init(&empty_bar[s], 1);
        }
        sm100::mbar_init(&acc_bar, 1);
        sm100::fence_mbar_init();
        for (int p = 0; p < NP; ++p) {
            sm100::prefetch_tmap(&maps.x[p]);
            sm100::prefetch_tmap(&maps.w[p]);
        }
    }
    if (warp == 1) {
        sm100::tmem_alloc(&tmem_slot, Cfg::TMEM_COLS);
        sm100::tc_fence_before();
    }
    __syncthreads();
    sm100::tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % Cfg::STAGES;
            const uint32_t ph = (kb / Cfg::STAGES) & 1;
            if (!sm100::mbar_wait(&empty_bar[s], ph ^ 1, wait_limit)) {
                atomicOr(status, 1);
                break;
            }
            unsigned char *st = smem + s * STAGE_BYTES;
            sm100::mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
            for (int p = 0; p < NP; ++p)
                sm100::tma_load_2d(st + p * TILE_BYTES, &maps.x[p], &full_bar[s], kb * TILE_K, b0);
            for (int p = 0; p < NP; ++p)
                sm100::tma_load_2d(st + (NP + p) * TILE_BYTES, &maps.w[p], &full_bar[s], kb * TILE_K, j0);
            issued = kb + 1;
        }
        // drain: the last issued copy of every stage has landed before exit
        const int first = issued > Cfg::STAGES ? issued - Cfg::STAGES : 0;
        for (int kb = first; kb < issued; ++kb)
            sm100::mbar_wait(&full_bar[kb % Cfg::STAGES], (kb / Cfg::STAGES) & 1, DRAIN_LIMIT);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % Cfg::STAGES;
            const uint32_t ph = (kb / Cfg::STAGES) & 1;
            if (!sm100::mbar_wait(&full_bar[s], ph, wait_limit)) {
                atomicOr(status, 1);
                break;
            }
            sm100::tc_fence_after();
            const uint32_t st = sm100::smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < TILE_K / 16; ++kk) {
                const uint32_t koff = kk * 32;   // 16 FP16 = 32 bytes along K
                const bool first = (kb == 0 && kk == 0);
                auto X = [&](int p) { return sm100::desc_k_sw128(st + p * TILE_BYTES + koff); };
                auto W = [&](int p) { return sm100::desc_k_sw128(st + (NP + p) * TILE_BYTES + koff); };
                if constexpr (NPROD == 1) {
                    sm100::mma_f16(tmem, X(0), W(0), IDESC, first ? 0u : 1u);
                } else {
                    const uint32_t a1 = tmem + TILE_N, a2 = tmem + 2 * TILE_N;
                    sm100::mma_f16(tmem, X(0), W(0), IDESC, first ? 0u : 1u);   // F0 A0
                    sm100::mma_f16(a1, X(0), W(1), IDESC, first ? 0u : 1u);     // F0 A1
                    sm100::mma_f16(a1, X(1), W(0), IDESC, 1u);                  // F1 A0
                    sm100::mma_f16(a2, X(1), W(1), IDESC, first ? 0u : 1u);     // F1 A1
                    sm100::mma_f16(a2, X(0), W(2), IDESC, 1u);                  // F0 A2s
                    sm100::mma_f16(a2, X(2), W(0), IDESC, 1u);                  // F2s A0
                }
            }
            sm100::mma_commit(&empty_bar[s]);
        }
        sm100::mma_commit(&acc_bar);   // also drains any MMA in flight on abort
        sm100::mbar_wait(&acc_bar, 0, DRAIN_LIMIT);
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;                    // TMEM lane quadrant of this warp
        const int b = b0 + q * 32 + lane;
        if (!sm100::mbar_wait(&acc_bar, 0, wait_limit)) atomicOr(status, 1);
        sm100::tc_fence_after();
        const int eb = (xexp != nullptr && b < B) ? xexp[b] : 0;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < TILE_N; c0 += 32) {
            float a0[32], a1[32], a2[32];
            sm100::tmem_ld_32x32b_x32(lane_addr + c0, a0);
            if constexpr (NPROD == 6) {
                sm100::tmem_ld_32x32b_x32(lane_addr + TILE_N + c0, a1);
                sm100::tmem_ld_32x32b_x32(lane_addr + 2 * TILE_N + c0, a2);
            }
            sm100::tmem_ld_wait();
            if (b >= B) continue;
            const int jb = j0 + c0;
            if constexpr (OUT_DF) {
                float2 *o = static_cast<float2 *>(out) + (size_t)b * ldo + jb;
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    float2 r[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = jb + i + u;
                        const int e = eb + ((j < rows) ? wexp[j] : 0);
                        float t = fmaf(a2[i + u], 0x1p-18f, a1[i + u] * 0x1p-9f);
                        dfl sum = df_two_sum(a0[i + u], t);
                        r[u] = make_float2(ldexpf(sum.hi, e), ldexpf(sum.lo, e));
                    }
                    if (jb + i + 1 < rows) {
                        *reinterpret_cast<float4 *>(o + i) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
                    } else if (jb + i < rows) {
                        o[i] = r[0];
                    }
                }
            } else {
                float *o = static_cast<float *>(out) + (size_t)b * ldo + jb;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int j = jb + i;
                    if (j >= rows) break;
                    float v;
                    if constexpr (NPROD == 6) {
                        float t = fmaf(a2[i], 0x1p-18f, a1[i] * 0x1p-9f);
                        v = ldexpf(a0[i] + t, eb + wexp[j]);
                    } else {
                        v = a0[i];
                    }
                    o[i] = v;
                }
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) sm100::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------- input split
// One CTA per row: power-of-two scale 2^e >= max|x|, then
//   xs = x 2^-e,  X0 = round(xs 2^9) 2^-9,  r1 = (xs - X0) 2^9,  X1 = fp16(r1),
//   r2 = (r1 - X1) 2^11,  X2s = fp16(r2 / 4).
// Input either FP32 (forward) or a double-float pair (adjoint).
template <class T> __device__ __forceinline__ float hi_of(T v);
template <> __device__ __forceinline__ float hi_of<float>(float v) { return v; }
template <> __device__ __forceinline__ float hi_of<float2>(float2 v) { return v.x; }
template <class T> __device__ __forceinline__ float lo_of(T v);
template <> __device__ __forceinline__ float lo_of<float>(float) { return 0.0f; }
template <> __device__ __forceinline__ float lo_of<float2>(float2 v) { return v.y; }

template <class T>
__global__ void __launch_bounds__(256) split_rows_kernel(const T *__restrict__ x, int ldx, int n, int np,
                                                         __half *__restrict__ X0, __half *__restrict__ X1,
                                                         __half *__restrict__ X2, int *__restrict__ xexp)
{
    const int b = blockIdx.x;
    const T *row = x + (size_t)b * ldx;
    __shared__ float red[8];
    __shared__ int s_e;
    float m = 0.0f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) m = fmaxf(m, fabsf(hi_of(row[k])));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
        int e = 0;
        if (mm > 0.0f) {
            float fr = frexpf(mm, &e);       // mm = fr 2^e, fr in [0.5, 1)
            if (fr == 0.5f) e -= 1;         // scaled |hi| <= 1, hence |X0| <= 1
        }
        s_e = e;
        xexp[b] = e;
    }
    __syncthreads();
    const int e = s_e;
    const size_t o = (size_t)b * np;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        float h = 0.0f, l = 0.0f;
        if (k < n) {
            h = ldexpf(hi_of(row[k]), -e);
            l = ldexpf(lo_of(row[k]), -e);
        }
        float x0 = rintf(h * 512.0f) * (1.0f / 512.0f);
        float r1 = (h - x0) * 512.0f + l * 512.0f;
        __half h1 = __float2half_rn(r1);
        float r2 = (r1 - __half2float(h1)) * 2048.0f;
        X0[o + k] = __float2half_rn(x0);
        X1[o + k] = h1;
        X2[o + k] = __float2half_rn(r2 * 0.25f);
    }
}

__global__ void __launch_bounds__(256) bf16_rows_kernel(const float *__restrict__ x, int n, int np,
                                                        __nv_bfloat16 *__restrict__ X)
{
    const int b = blockIdx.x;
    for (int k = threadIdx.x; k < np; k += blockDim.x)
        X[(size_t)b * np + k] = __float2bfloat16_rn(k < n ? x[(size_t)b * n + k] : 0.0f);
}

// Transposed split planes of the operator for the adjoint GEMM: row k of the
// result is column k of A (j = 0..rows-1, zero-padded to npr), scaled by
// 2^e_k >= sum_j |A[j,k]|, split as in plane_split_kernel.
__global__ void __launch_bounds__(256) split_cols_kernel(const double *__restrict__ A, int rows, int K, int npr,
                                                         __half *__restrict__ T0, __half *__restrict__ T1,
                                                         __half *__restrict__ T2, int *__restrict__ colexp)
{
    const int k = blockIdx.x;
    __shared__ double red[8];
    __shared__ double s_inv;
    double s = 0.0;
    for (int j = threadIdx.x; j < rows; j += blockDim.x) s += fabs(A[(size_t)j * K + k]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        int e = 0;
        if (t > 0.0) {
            double m = frexp(t, &e);
            if (m == 0.5) e -= 1;
        }
        colexp[k] = e;
        s_inv = ldexp(1.0, -e);
    }
    __syncthreads();
    const double inv = s_inv;
    for (int j = threadIdx.x; j < npr; j += blockDim.x) {
        double a = (j < rows) ? A[(size_t)j * K + k] * inv : 0.0;
        double a0;
        if (fabs(a) >= 0.0625) a0 = (double)__double2half(a);
        else a0 = rint(ldexp(a, LEG_SPLIT_ABITS)) * ldexp(1.0, -LEG_SPLIT_ABITS);
        double r1 = ldexp(a - a0, LEG_SPLIT_FBITS);
        __half h1 = __double2half(r1);
        double r2 = ldexp(r1 - (double)h1, 11);
        size_t o = (size_t)k * npr + j;
        T0[o] = __double2half(a0);
        T1[o] = h1;
        T2[o] = __double2half(ldexp(r2, -2));
    }
}

// ---------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiledFn *fn)
{
    static EncodeTiledFn cached = nullptr;
    if (!cached) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return leg_set_error(LEG_ERR_CUDA, "cuTensorMapEncodeTiled entry point not found");
        cached = reinterpret_cast<EncodeTiledFn>(p);
    }
    *fn = cached;
    return LEG_OK;
}

// 2-D map over a [outer x inner] 16-bit array with row stride ld (elements);
// box = 64 (inner) x 128 (outer), 128-byte swizzle, zero fill out of bounds.
int make_map(CUtensorMap *m, const void *base, int inner, int outer, int ld, bool bf16)
{
    EncodeTiledFn enc;
    int rc = get_encoder(&enc);
    if (rc) return rc;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {TILE_K, TILE_M};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return leg_set_error(LEG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return LEG_OK;
}

template <int NPROD, bool OUT_DF>
int launch_tc(const TcMaps &maps, int B, int nrows, int Kp, const int *xexp, const int *wexp, void *out, int ldo,
              int *status, long long limit, cudaStream_t st)
{
    auto kern = tc_gemm_kernel<NPROD, OUT_DF>;
    const size_t smem = tc_smem_bytes<NPROD>();
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((nrows + TILE_N - 1) / TILE_N, (B + TILE_M - 1) / TILE_M);
    kern<<<grid, 192, smem, st>>>(maps, B, nrows, Kp / TILE_K, xexp, wexp, out, ldo, status, limit);
    LEG_LAUNCH_CHECK("tc_gemm_kernel");
    return LEG_OK;
}

}  // namespace

int leg_build_split_transposed(leg_plan *p)
{
    const int npr = leg_round_up(leg_round_up(p->rows, 8), LEG_KPAD);
    for (int s = 0; s < 3; ++s) LEG_CUDA_TRY(cudaMalloc(&p->AhT[s], sizeof(__half) * (size_t)p->K * npr));
    LEG_CUDA_TRY(cudaMalloc(&p->colexp, sizeof(int) * p->K));
    split_cols_kernel<<<p->K, 256>>>(p->A64, p->rows, p->K, npr, p->AhT[0], p->AhT[1], p->AhT[2], p->colexp);
    LEG_LAUNCH_CHECK("split_cols_kernel");
    return LEG_OK;
}

int leg_split_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st)
{
    split_rows_kernel<float><<<B, 256, 0, st>>>(f, p->K, p->K, p->Kp, p->Fh[0], p->Fh[1], p->Fh[2], p->fexp);
    LEG_LAUNCH_CHECK("split_rows_kernel");
    return LEG_OK;
}

int leg_gemm_split_fwd(leg_plan *p, int B, cudaStream_t st)
{
    TcMaps maps;
    int rc;
    for (int s = 0; s < 3; ++s) {
        if ((rc = make_map(&maps.x[s], p->Fh[s], p->Kp, B, p->Kp, false))) return rc;
        if ((rc = make_map(&maps.w[s], p->Ah[s], p->Kp, p->rows, p->Kp, false))) return rc;
    }
    return launch_tc<6, true>(maps, B, p->rows, p->Kp, p->fexp, p->rowexp, p->G, p->ldg, p->status,
                              p->wait_limit, st);
}

int leg_gemm_split_adj(leg_plan *p, void *df, int B, cudaStream_t st)
{
    // Gbar (double-float, B x ldg, rows valid) -> split planes B x npr
    const int npr = leg_round_up(leg_round_up(p->rows, 8), LEG_KPAD);
    split_rows_kernel<float2><<<B, 256, 0, st>>>(static_cast<const float2 *>(p->Gbar), p->ldg, p->rows, npr,
                                                 p->Fh[0], p->Fh[1], p->Fh[2], p->fexp);
    LEG_LAUNCH_CHECK("split_rows_kernel (adjoint)");
    TcMaps maps;
    int rc;
    for (int s = 0; s < 3; ++s) {
        if ((rc = make_map(&maps.x[s], p->Fh[s], npr, B, npr, false))) return rc;
        if ((rc = make_map(&maps.w[s], p->AhT[s], npr, p->K, npr, false))) return rc;
    }
    return launch_tc<6, false>(maps, B, p->K, npr, p->fexp, p->colexp, df, p->K, p->status, p->wait_limit, st);
}

int leg_bf16_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st)
{
    bf16_rows_kernel<<<B, 256, 0, st>>>(f, p->K, p->Kp, p->Fbf);
    LEG_LAUNCH_CHECK("bf16_rows_kernel");
    return LEG_OK;
}

int leg_gemm_bf16_fwd(leg_plan *p, int B, cudaStream_t st)
{
    TcMaps maps;
    int rc;
    if ((rc = make_map(&maps.x[0], p->Fbf, p->Kp, B, p->Kp, true))) return rc;
    if ((rc = make_map(&maps.w[0], p->Abf, p->Kp, p->rows, p->Kp, true))) return rc;
    maps.x[1] = maps.x[2] = maps.x[0];
    maps.w[1] = maps.w[2] = maps.w[0];
    return launch_tc<1, false>(maps, B, p->rows, p->Kp, nullptr, nullptr, p->G, p->ldg, p->status,
                               p->wait_limit, st);
}

// Variants of the split forward launchers that take their buffers explicitly
// (used by leg_forward_noalloc, whose buffers live in a static device array).
int leg_split_prepare_input_into(const leg_plan *p, const float *f, int B, __half *const planes[3], int *fexp,
                                 cudaStream_t st)
{
    split_rows_kernel<float><<<B, 256, 0, st>>>(f, p->K, p->K, p->Kp, planes[0], planes[1], planes[2], fexp);
    LEG_LAUNCH_CHECK("split_rows_kernel");
    return LEG_OK;
}

int leg_gemm_split_fwd_into(leg_plan *p, int B, __half *const planes[3], const int *fexp, float2 *G, int ldg,
                            cudaStream_t st)
{
    TcMaps maps;
    int rc;
    for (int s = 0; s < 3; ++s) {
        if ((rc = make_map(&maps.x[s], planes[s], p->Kp, B, p->Kp, false))) return rc;
        if ((rc = make_map(&maps.w[s], p->Ah[s], p->Kp, p->rows, p->Kp, false))) return rc;
    }
    return launch_tc<6, true>(maps, B, p->rows, p->Kp, fexp, p->rowexp, G, ldg, p->status, p->wait_limit, st);
}
