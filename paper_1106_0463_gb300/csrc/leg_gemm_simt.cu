// CUDA-core (SIMT) GEMMs of the FP64 and FP32 paths.
//
// Forward (the Abel step, Eq. 2.5 on the y-grid):  G[b, j] = sum_k F[b, k] A[j, k]
// Adjoint (transposed Abel operator):             D[b, k] = sum_j Gb[b, j] A[j, k]
//
// Register-tiled outer-product kernels: a CTA computes a BM x BN tile of the
// output with 256 threads, each owning a TM x TN micro-tile; operand tiles of
// depth BK are staged in shared memory transposed to reduction-major order so
// the inner loop reads contiguous fragments.  Bounds are checked on every
// global access (ragged B, rows and K).  FP64: simt_gemm_kernel; FP32: the
// double-buffered sgemm_kernel below.
#include "leg_internal.cuh"

namespace {

// ADJ = false: A is [n][k] (reduction index k contiguous)   -> forward
// ADJ = true:  A is [k][n] (output index n contiguous)       -> adjoint
template <class T, int BM, int BN, int BK, int TM, int TN, bool ADJ>
__global__ void __launch_bounds__(256) simt_gemm_kernel(
    const T *__restrict__ X, int ldx,      // B x R  (R = reduction length)
    const T *__restrict__ A, int lda,
    T *__restrict__ Y, int ldy,            // B x Nout
    int B, int Nout, int R)
{
    static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
    __shared__ T sX[BK][BM + 1];
    __shared__ T sA[BK][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int b0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int r0 = 0; r0 < R; r0 += BK) {
        // X tile: BM rows x BK reduction, row-major in global (reduction contiguous)
        for (int e = tid; e < BM * BK; e += 256) {
            int m = e / BK, kk = e % BK;
            int gb = b0 + m, gr = r0 + kk;
            sX[kk][m] = (gb < B && gr < R) ? X[(size_t)gb * ldx + gr] : T(0);
        }
        if (!ADJ) {
            // A[n][k]: reduction contiguous
            for (int e = tid; e < BN * BK; e += 256) {
                int n = e / BK, kk = e % BK;
                int gn = n0 + n, gr = r0 + kk;
                sA[kk][n] = (gn < Nout && gr < R) ? A[(size_t)gn * lda + gr] : T(0);
            }
        } else {
            // A[k][n]: output index contiguous
            for (int e = tid; e < BN * BK; e += 256) {
                int kk = e / BN, n = e % BN;
                int gn = n0 + n, gr = r0 + kk;
                sA[kk][n] = (gn < Nout && gr < R) ? A[(size_t)gr * lda + gn] : T(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T xf[TM], af[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) xf[i] = sX[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) af[j] = sA[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(xf[i], af[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gb = b0 + ty * TM + i;
        if (gb >= B) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gn = n0 + tx * TN + j;
            if (gn < Nout) Y[(size_t)gb * ldy + gn] = acc[i][j];
        }
    }
}

// FP32: a CTA computes a 128 x 128 tile (functions x outputs) with 256
// threads of 8 x 8 outputs each, taken as two 4 x 4 blocks 64 apart in each
// direction so that every fragment is one conflict-free float4 read from
// shared memory.  The reduction advances in steps of 16 through two
// shared-memory buffers: the global loads of step s + 1 are in flight while
// the FMAs of step s run, and one barrier per step separates the buffers.
// Row-major operands with the reduction index contiguous are stored
// transposed (padded rows: at most two-way bank conflicts on the stores).
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 16, SG_PAD = 4;

template <bool ADJ>
__global__ void __launch_bounds__(256, 2) sgemm_kernel(const float *__restrict__ X, int ldx,
                                                       const float *__restrict__ A, int lda,
                                                       float *__restrict__ Y, int ldy, int B, int Nout, int R)
{
    __shared__ __align__(16) float sX[2][SG_BK][SG_BM + SG_PAD];
    __shared__ __align__(16) float sA[2][SG_BK][SG_BN + SG_PAD];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int b0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;
    constexpr int PER = SG_BM * SG_BK / 256;   // elements of each operand tile per thread (8)
    float px[PER], pa[PER];

    // element e = tid + 256 i of a 128 x 16 tile stored reduction-minor:
    // row e / 16 = tid / 16 + 16 i, reduction index e % 16 = tid % 16 (a warp
    // reads two 64-byte row pieces); of the adjoint's 16 x 128 A tile:
    // reduction row tid / 128 + 2 i, column tid % 128 (128 contiguous bytes
    // per warp)
    const int lm = tid >> 4, lk = tid & 15;
    const float *xb = X + (size_t)(b0 + lm) * ldx + lk;
    const float *ab = ADJ ? A + (size_t)(tid >> 7) * lda + (n0 + (tid & 127)) : A + (size_t)(n0 + lm) * lda + lk;
    unsigned xok = 0, aok = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        if (b0 + lm + 16 * i < B) xok |= 1u << i;
        if (!ADJ && n0 + lm + 16 * i < Nout) aok |= 1u << i;
    }
    const bool acol = ADJ && n0 + (tid & 127) < Nout;
    auto load = [&](int r0) {
        const bool kin = r0 + lk < R;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            px[i] = (kin && (xok >> i & 1u)) ? xb[(size_t)(16 * i) * ldx + r0] : 0.0f;
            if (!ADJ) {
                pa[i] = (kin && (aok >> i & 1u)) ? ab[(size_t)(16 * i) * lda + r0] : 0.0f;
            } else {
                const int gr = r0 + (tid >> 7) + 2 * i;
                pa[i] = (acol && gr < R) ? ab[(size_t)(r0 + 2 * i) * lda] : 0.0f;
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            sX[buf][lk][lm + 16 * i] = px[i];
            if (!ADJ) sA[buf][lk][lm + 16 * i] = pa[i];
            else sA[buf][(tid >> 7) + 2 * i][tid & 127] = pa[i];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    const int nsteps = (R + SG_BK - 1) / SG_BK;
    load(0);
    store(0);
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        const int cur = s & 1;
        if (s + 1 < nsteps) load((s + 1) * SG_BK);
#pragma unroll
        for (int kk = 0; kk < SG_BK; ++kk) {
            const float4 x0 = *reinterpret_cast<const float4 *>(&sX[cur][kk][ty * 4]);
            const float4 x1 = *reinterpret_cast<const float4 *>(&sX[cur][kk][64 + ty * 4]);
            const float4 a0 = *reinterpret_cast<const float4 *>(&sA[cur][kk][tx * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sA[cur][kk][64 + tx * 4]);
            const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xv[i], av[j], acc[i][j]);
        }
        if (s + 1 < nsteps) store(cur ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gb = b0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (gb >= B) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
            if (gn < Nout) Y[(size_t)gb * ldy + gn] = acc[i][j];
        }
    }
}

template <bool ADJ>
int launch_sgemm(const float *X, int ldx, const float *A, int lda, float *Y, int ldy, int B, int Nout, int R,
                 cudaStream_t st, const char *name)
{
    if (B == 0 || Nout == 0) return LEG_OK;
    dim3 grid((Nout + SG_BN - 1) / SG_BN, (B + SG_BM - 1) / SG_BM);
    sgemm_kernel<ADJ><<<grid, 256, 0, st>>>(X, ldx, A, lda, Y, ldy, B, Nout, R);
    LEG_LAUNCH_CHECK(name);
    return LEG_OK;
}

template <class T, int BM, int BN, int BK, int TM, int TN, bool ADJ>
int launch(const T *X, int ldx, const T *A, int lda, T *Y, int ldy, int B, int Nout, int R,
           cudaStream_t st, const char *name)
{
    if (B == 0 || Nout == 0) return LEG_OK;
    dim3 grid((Nout + BN - 1) / BN, (B + BM - 1) / BM);
    simt_gemm_kernel<T, BM, BN, BK, TM, TN, ADJ><<<grid, 256, 0, st>>>(X, ldx, A, lda, Y, ldy, B, Nout, R);
    LEG_LAUNCH_CHECK(name);
    return LEG_OK;
}

}  // namespace

int leg_gemm_f64_fwd(const double *F, int ldf, const double *A, int lda, double *G, int ldg,
                     int B, int rows, int K, cudaStream_t st)
{
    return launch<double, 64, 64, 16, 4, 4, false>(F, ldf, A, lda, G, ldg, B, rows, K, st,
                                                   "simt_gemm f64 fwd");
}

int leg_gemm_f32_fwd(const float *F, int ldf, const float *A, int lda, float *G, int ldg,
                     int B, int rows, int K, cudaStream_t st)
{
    return launch_sgemm<false>(F, ldf, A, lda, G, ldg, B, rows, K, st, "sgemm f32 fwd");
}

int leg_gemm_f64_adj(const double *Gb, int ldg, const double *A, int lda, double *D, int ldd,
                     int B, int rows, int K, cudaStream_t st)
{
    return launch<double, 64, 64, 16, 4, 4, true>(Gb, ldg, A, lda, D, ldd, B, K, rows, st,
                                                  "simt_gemm f64 adj");
}

int leg_gemm_f32_adj(const float *Gb, int ldg, const float *A, int lda, float *D, int ldd,
                     int B, int rows, int K, cudaStream_t st)
{
    return launch_sgemm<true>(Gb, ldg, A, lda, D, ldd, B, K, rows, st, "sgemm f32 adj");
}
