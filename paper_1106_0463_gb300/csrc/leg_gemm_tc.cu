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
// LEG_SPLIT_FP16 (three-slice split, eight products, four accumulators):
//   each operand row is scaled by a power of two (the operator by its L1
//   norm, the input by its max-norm) and split into FP16 slices
//     a = A0 + 2^-7 A1 + 2^-14 A2s,   f = F0 + 2^-7 F1 + 2^-14 F2s,
//   where A0 lies on a 2^-16 grid and F0 on a 2^-7 grid.  Every product
//   A0*F0 is then a multiple of 2^-23 and every partial sum of them is below
//   2 in magnitude, so accumulator 0 (A0 F0) is EXACT in FP32 whatever the
//   accumulation order or truncation of the tensor core.  Accumulators 1-3
//   hold the terms of weight 2^-7 (A1 F0 + A0 F1), 2^-14 (A1 F1 + A2s F0 +
//   A0 F2s) and 2^-21 (A2s F1 + F2s A1); their FP32 rounding stays below the
//   target, and only terms of weight 2^-28 (A2s F2s) are dropped.  The
//   epilogue forms G = 2^(e_b + e_j) (acc0 + 2^-7 acc1 + 2^-14 acc2 +
//   2^-21 acc3) as a double-float pair for the double-float FFT.
// LEG_BF16: one BF16 product into one FP32 accumulator (FP32 G).
//
// Kernel structure (one 128 x 128 output tile per CTA, 320 threads):
//   warp 0 lane 0  TMA producer: per 32-wide K block, loads the operand tiles
//                  (128 rows x 32 FP16, 64-byte swizzle) into one of four
//                  stages and arms the stage's full barrier with the byte count;
//   warp 1         allocates TMEM (4 x 128 columns); lane 0 issues the
//                  tcgen05.mma instructions (M=128, N=128, K=16 each) and
//                  commits each stage back to the producer;
//   warps 2..9     epilogue: tcgen05.ld of the accumulators (each warp reads
//                  the 32 TMEM lanes of its quadrant, half of the columns),
//                  combination, stores.
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
constexpr int TILE_K = 32;    // K per stage: one 64-byte swizzle row of FP16
constexpr int TILE_BYTES = TILE_M * TILE_K * 2;   // 8 KB (TILE_M == TILE_N)
constexpr int EPI_WARPS = 16; // four warps per TMEM lane quadrant, 32 columns each
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int THREADS = 64 + EPI_THREADS;
constexpr long long DRAIN_LIMIT = 4000000000LL;   // cycles, teardown waits

template <int NPROD> struct TcCfg;
template <> struct TcCfg<8> {
    static constexpr int NPLANES = 3;       // per operand
    static constexpr int STAGES = 4;
    static constexpr uint32_t TMEM_COLS = 512;
};
template <> struct TcCfg<1> {
    static constexpr int NPLANES = 1;
    static constexpr int STAGES = 8;
    static constexpr uint32_t TMEM_COLS = 128;
};

template <int NPROD>
constexpr size_t tc_smem_bytes()
{
    return (size_t)TcCfg<NPROD>::STAGES * 2 * TcCfg<NPROD>::NPLANES * TILE_BYTES + 1024;
}

}  // namespace

// One GEMM problem: out[b, j] = sum_k X[b, k] W[j, k] for b < B, j < rows,
// with X and W given as FP16/BF16 planes through TMA maps.
struct TcProblem {
    CUtensorMap x[3];        // input planes   (B x Kp)
    CUtensorMap w[3];        // operator planes (rows x Kp)
    const int *xexp;         // per-row power-of-two scales of X (or null)
    const int *wexp;         // per-row scales of W (or null)
    void *out;               // float2 (double-float) or float, row stride ldo
    int ldo, B, rows, nkb;   // nkb = Kp / TILE_K
    int ntj;                 // tiles along j: ceil(rows / TILE_N)
    int tile0;               // first global tile index of this problem (grouped launches)
};

namespace {

// Tile t of a launch: its problem and its (b0, j0).
__device__ __forceinline__ const TcProblem &tile_problem(const TcProblem &single, const TcProblem *multi,
                                                         int nprob, int t, int &b0, int &j0)
{
    const TcProblem *pr = &single;
    int lt = t;
    if (multi) {
        int p = 0;
        while (p + 1 < nprob && t >= multi[p + 1].tile0) ++p;
        pr = &multi[p];
        lt = t - pr->tile0;
    }
    b0 = (lt / pr->ntj) * TILE_M;
    j0 = (lt % pr->ntj) * TILE_N;
    return *pr;
}

// Persistent kernel: CTA c processes tiles c, c + gridDim.x, ...  OUT_DF: G
// as a double-float pair (float2); else a float.  `single` describes the
// problem of a plain launch (multi == nullptr); grouped launches pass an
// array of problems whose tiles are numbered consecutively.
template <int NPROD, bool OUT_DF>
__global__ void __launch_bounds__(THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcProblem single,
                                                         const TcProblem *__restrict__ multi, int nprob,
                                                         int ntiles, int *status, long long wait_limit)
{
    using Cfg = TcCfg<NPROD>;
    constexpr int NP = Cfg::NPLANES;
    constexpr int STAGE_BYTES = 2 * NP * TILE_BYTES;
    constexpr uint32_t IDESC = sm100::idesc_f16(TILE_M, TILE_N, NPROD == 1 ? 1 : 0);

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));   // swizzle atoms need 512 B
    __shared__ __align__(8) uint64_t full_bar[Cfg::STAGES];
    __shared__ __align__(8) uint64_t empty_bar[Cfg::STAGES];
    __shared__ __align__(8) uint64_t acc_full;    // MMA -> epilogue: accumulators of a tile are final
    __shared__ __align__(8) uint64_t acc_empty;   // epilogue -> MMA: accumulators have been read
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            sm100::mbar_init(&full_bar[s], 1);
            sm100::mbar_init(&empty_bar[s], 1);
        }
        sm100::mbar_init(&acc_full, 1);
        sm100::mbar_init(&acc_empty, EPI_THREADS);
        sm100::mbar_init(&drain_bar, 1);
        s_abort = 0;
        sm100::fence_mbar_init();
        if (!multi) {
            for (int p = 0; p < NP; ++p) {
                sm100::prefetch_tmap(&single.x[p]);
                sm100::prefetch_tmap(&single.w[p]);
            }
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
        uint32_t it = 0;   // stage-ring position, continues across tiles
        for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x) {
            int b0, j0;
            const TcProblem &pr = tile_problem(single, multi, nprob, t, b0, j0);
            const int nkb = pr.nkb;
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % Cfg::STAGES;
                const uint32_t ph = (it / Cfg::STAGES) & 1;
                if (!sm100::mbar_wait(&empty_bar[s], ph ^ 1, wait_limit)) {
                    ok = false;
                    break;
                }
                unsigned char *st = smem + s * STAGE_BYTES;
                sm100::mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
                for (int p = 0; p < NP; ++p)
                    sm100::tma_load_2d(st + p * TILE_BYTES, &pr.x[p], &full_bar[s], kb * TILE_K, b0);
                for (int p = 0; p < NP; ++p)
                    sm100::tma_load_2d(st + (NP + p) * TILE_BYTES, &pr.w[p], &full_bar[s], kb * TILE_K, j0);
            }
            if (!ok) {
                atomicOr(status, 1);
                s_abort = 1;
                break;
            }
        }
        // drain: the last copy issued into every stage has landed before exit
        const uint32_t first = it > (uint32_t)Cfg::STAGES ? it - Cfg::STAGES : 0;
        for (uint32_t i = first; i < it; ++i)
            sm100::mbar_wait(&full_bar[i % Cfg::STAGES], (i / Cfg::STAGES) & 1, DRAIN_LIMIT);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        uint32_t it = 0;
        int ti = 0;
        for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x, ++ti) {
            int b0, j0;
            const TcProblem &pr = tile_problem(single, multi, nprob, t, b0, j0);
            const int nkb = pr.nkb;
            bool ok = sm100::mbar_wait(&acc_empty, (ti & 1) ^ 1, wait_limit);   // previous tile drained
            sm100::tc_fence_after();
            for (int kb = 0; ok && kb < nkb; ++kb, ++it) {
                const int s = it % Cfg::STAGES;
                const uint32_t ph = (it / Cfg::STAGES) & 1;
                if (!sm100::mbar_wait(&full_bar[s], ph, wait_limit)) {
                    ok = false;
                    break;
                }
                sm100::tc_fence_after();
                const uint32_t st = sm100::smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                for (int kk = 0; kk < TILE_K / 16; ++kk) {
                    const uint32_t koff = kk * 32;   // 16 FP16 = 32 bytes along K
                    const uint32_t acc = (kb == 0 && kk == 0) ? 0u : 1u;
                    auto X = [&](int p) { return sm100::desc_k_sw64(st + p * TILE_BYTES + koff); };
                    auto W = [&](int p) { return sm100::desc_k_sw64(st + (NP + p) * TILE_BYTES + koff); };
                    if constexpr (NPROD == 1) {
                        sm100::mma_f16(tmem, X(0), W(0), IDESC, acc);
                    } else {
                        const uint32_t a1 = tmem + TILE_N, a2 = tmem + 2 * TILE_N, a3 = tmem + 3 * TILE_N;
                        sm100::mma_f16(tmem, X(0), W(0), IDESC, acc);   // F0 A0   (weight 1)
                        sm100::mma_f16(a1, X(0), W(1), IDESC, acc);     // F0 A1   (2^-s)
                        sm100::mma_f16(a1, X(1), W(0), IDESC, 1u);      // F1 A0
                        sm100::mma_f16(a2, X(1), W(1), IDESC, acc);     // F1 A1   (2^-2s)
                        sm100::mma_f16(a2, X(0), W(2), IDESC, 1u);      // F0 A2s
                        sm100::mma_f16(a2, X(2), W(0), IDESC, 1u);      // F2s A0
                        sm100::mma_f16(a3, X(1), W(2), IDESC, acc);     // F1 A2s  (2^-3s)
                        sm100::mma_f16(a3, X(2), W(1), IDESC, 1u);      // F2s A1
                    }
                }
                sm100::mma_commit(&empty_bar[s]);
            }
            if (!ok) {
                atomicOr(status, 1);
                s_abort = 1;
                break;
            }
            sm100::mma_commit(&acc_full);
        }
        // every MMA issued by this thread has completed before TMEM is released
        sm100::mma_commit(&drain_bar);
        sm100::mbar_wait(&drain_bar, 0, DRAIN_LIMIT);
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;                        // TMEM lane quadrant of this warp
        const int c0 = ((warp - 2) >> 2) * 32;         // this warp's 32 columns
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + c0;
        int ti = 0;
        for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x, ++ti) {
            int b0, j0;
            const TcProblem &pr = tile_problem(single, multi, nprob, t, b0, j0);
            if (!sm100::mbar_wait(&acc_full, ti & 1, wait_limit)) {
                atomicOr(status, 1);
                s_abort = 1;
                break;
            }
            sm100::tc_fence_after();
            float a0[32], a1[32];
            sm100::tmem_ld_32x32b_x32(lane_addr, a0);
            if constexpr (NPROD == 8) {
                // fold the small accumulators: a1 <- 2^-s acc1 + 2^-2s acc2 + 2^-3s acc3
                constexpr float W1 = 1.0f / (float)(1 << LEG_SPLIT_FBITS);
                sm100::tmem_ld_32x32b_x32(lane_addr + TILE_N, a1);
                sm100::tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < 32; h += 16) {
                    float tq[16];
                    sm100::tmem_ld_32x32b_x16(lane_addr + 2 * TILE_N + h, tq);
                    sm100::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) a1[h + i] = fmaf(tq[i], W1 * W1, a1[h + i] * W1);
                    sm100::tmem_ld_32x32b_x16(lane_addr + 3 * TILE_N + h, tq);
                    sm100::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) a1[h + i] = fmaf(tq[i], W1 * W1 * W1, a1[h + i]);
                }
            } else {
                sm100::tmem_ld_wait();
            }
            // accumulators read: the MMA warp may start the next tile
            sm100::tc_fence_before();
            sm100::mbar_arrive(&acc_empty);

            const int b = b0 + q * 32 + lane;
            if (b >= pr.B) continue;
            const int jb = j0 + c0;
            const int rows = pr.rows;
            const int eb = (pr.xexp != nullptr) ? pr.xexp[b] : 0;
            if constexpr (OUT_DF) {
                float2 *o = static_cast<float2 *>(pr.out) + (size_t)b * pr.ldo + jb;
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    float2 r[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = jb + i + u;
                        const int e = eb + ((j < rows) ? pr.wexp[j] : 0);
                        dfl sum = df_two_sum(a0[i + u], a1[i + u]);
                        r[u] = make_float2(ldexpf(sum.hi, e), ldexpf(sum.lo, e));
                    }
                    if (jb + i + 1 < rows) {
                        *reinterpret_cast<float4 *>(o + i) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
                    } else if (jb + i < rows) {
                        o[i] = r[0];
                    }
                }
            } else {
                float *o = static_cast<float *>(pr.out) + (size_t)b * pr.ldo + jb;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int j = jb + i;
                    if (j >= rows) break;
                    if constexpr (NPROD == 8) o[i] = ldexpf(a0[i] + a1[i], eb + pr.wexp[j]);
                    else o[i] = a0[i];
                }
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) sm100::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------- input split
// One CTA per row: power-of-two scale 2^e >= max|x|, then with s = LEG_SPLIT_FBITS
//   xs = x 2^-e,  X0 = round(xs 2^s) 2^-s,  r1 = (xs - X0) 2^s,  X1 = fp16(r1),
//   X2s = fp16((r1 - X1) 2^s),   so xs = X0 + 2^-s X1 + 2^-2s X2s.
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
        constexpr float SC = (float)(1 << LEG_SPLIT_FBITS), ISC = 1.0f / SC;
        float x0 = rintf(h * SC) * ISC;
        float r1 = (h - x0) * SC + l * SC;
        __half h1 = __float2half_rn(r1);
        X0[o + k] = __float2half_rn(x0);
        X1[o + k] = h1;
        X2[o + k] = __float2half_rn((r1 - __half2float(h1)) * SC);
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
        if (fabs(a) >= ldexp(1.0, 10 - LEG_SPLIT_ABITS)) a0 = (double)__double2half(a);
        else a0 = rint(ldexp(a, LEG_SPLIT_ABITS)) * ldexp(1.0, -LEG_SPLIT_ABITS);
        double r1 = ldexp(a - a0, LEG_SPLIT_FBITS);
        __half h1 = __double2half(r1);
        size_t o = (size_t)k * npr + j;
        T0[o] = __double2half(a0);
        T1[o] = h1;
        T2[o] = __double2half(ldexp(r1 - (double)h1, LEG_SPLIT_FBITS));
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
// box = 32 (inner) x 128 (outer), 64-byte swizzle, zero fill out of bounds.
int make_map(CUtensorMap *m, const void *base, int inner, int outer, int ld, bool bf16)
{
    EncodeTiledFn enc;
    int rc = get_encoder(&enc);
    if (rc) return rc;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {TILE_K, TILE_M};   // 32 x 16 bit = 64 B rows
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return leg_set_error(LEG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return LEG_OK;
}

template <int NPROD, bool OUT_DF>
int launch_tc(const TcProblem &single, const TcProblem *multi, int nprob, int ntiles, int *status, long long limit,
              cudaStream_t st)
{
    if (ntiles <= 0) return LEG_OK;
    auto kern = tc_gemm_kernel<NPROD, OUT_DF>;
    const size_t smem = tc_smem_bytes<NPROD>();
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    static int num_sms = 0;
    if (!num_sms) {
        int dev = 0;
        LEG_CUDA_TRY(cudaGetDevice(&dev));
        LEG_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    kern<<<grid, THREADS, smem, st>>>(single, multi, nprob, ntiles, status, limit);
    LEG_LAUNCH_CHECK("tc_gemm_kernel");
    return LEG_OK;
}

// A single-problem descriptor; maps over planes with row stride ld.
int make_problem(TcProblem *pr, __half *const xs[3], int xrows, const __half *const ws[3], int wrows, int Kp,
                 const int *xexp, const int *wexp, void *out, int ldo, int B, int rows)
{
    int rc;
    for (int s = 0; s < 3; ++s) {
        if ((rc = make_map(&pr->x[s], xs[s], Kp, xrows, Kp, false))) return rc;
        if ((rc = make_map(&pr->w[s], ws[s], Kp, wrows, Kp, false))) return rc;
    }
    pr->xexp = xexp;
    pr->wexp = wexp;
    pr->out = out;
    pr->ldo = ldo;
    pr->B = B;
    pr->rows = rows;
    pr->nkb = Kp / TILE_K;
    pr->ntj = (rows + TILE_N - 1) / TILE_N;
    pr->tile0 = 0;
    return LEG_OK;
}

int tiles_of(const TcProblem &pr) { return ((pr.B + TILE_M - 1) / TILE_M) * pr.ntj; }

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
    TcProblem pr;
    int rc = make_problem(&pr, p->Fh, B, p->Ah, p->rows, p->Kp, p->fexp, p->rowexp, p->G, p->ldg, B, p->rows);
    if (rc) return rc;
    return launch_tc<8, true>(pr, nullptr, 1, tiles_of(pr), p->status, p->wait_limit, st);
}

int leg_gemm_split_adj(leg_plan *p, void *df, int B, cudaStream_t st)
{
    // Gbar (double-float, B x ldg, rows valid) -> split planes B x npr
    const int npr = leg_round_up(leg_round_up(p->rows, 8), LEG_KPAD);
    split_rows_kernel<float2><<<B, 256, 0, st>>>(static_cast<const float2 *>(p->Gbar), p->ldg, p->rows, npr,
                                                 p->Fh[0], p->Fh[1], p->Fh[2], p->fexp);
    LEG_LAUNCH_CHECK("split_rows_kernel (adjoint)");
    TcProblem pr;
    int rc = make_problem(&pr, p->Fh, B, p->AhT, p->K, npr, p->fexp, p->colexp, df, p->K, B, p->K);
    if (rc) return rc;
    return launch_tc<8, false>(pr, nullptr, 1, tiles_of(pr), p->status, p->wait_limit, st);
}

int leg_bf16_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st)
{
    bf16_rows_kernel<<<B, 256, 0, st>>>(f, p->K, p->Kp, p->Fbf);
    LEG_LAUNCH_CHECK("bf16_rows_kernel");
    return LEG_OK;
}

int leg_gemm_bf16_fwd(leg_plan *p, int B, cudaStream_t st)
{
    TcProblem pr;
    int rc;
    if ((rc = make_map(&pr.x[0], p->Fbf, p->Kp, B, p->Kp, true))) return rc;
    if ((rc = make_map(&pr.w[0], p->Abf, p->Kp, p->rows, p->Kp, true))) return rc;
    pr.x[1] = pr.x[2] = pr.x[0];
    pr.w[1] = pr.w[2] = pr.w[0];
    pr.xexp = pr.wexp = nullptr;
    pr.out = p->G;
    pr.ldo = p->ldg;
    pr.B = B;
    pr.rows = p->rows;
    pr.nkb = p->Kp / TILE_K;
    pr.ntj = (p->rows + TILE_N - 1) / TILE_N;
    pr.tile0 = 0;
    return launch_tc<1, false>(pr, nullptr, 1, tiles_of(pr), p->status, p->wait_limit, st);
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
    TcProblem pr;
    int rc = make_problem(&pr, planes, B, p->Ah, p->rows, p->Kp, fexp, p->rowexp, G, ldg, B, p->rows);
    if (rc) return rc;
    return launch_tc<8, true>(pr, nullptr, 1, tiles_of(pr), p->status, p->wait_limit, st);
}
