// CUDA-core (SIMT) GEMMs of the FP64 and FP32 paths.
//
// Forward (the Abel step, Eq. 2.5 on the y-grid):  G[b, j] = sum_k F[b, k] A[j, k]
// Adjoint (transposed Abel operator):             D[b, k] = sum_j Gb[b, j] A[j, k]
//
// Register-tiled outer-product kernels: a CTA computes a BM x BN tile of the
// output with 256 threads, each owning a TM x TN micro-tile; operand tiles of
// depth BK are staged in shared memory transposed to reduction-major order so
// the inner loop reads contiguous fragments.  Bounds are checked on every
// global access (ragged B, rows and K).
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
    return launch<float, 128, 128, 8, 8, 8, false>(F, ldf, A, lda, G, ldg, B, rows, K, st,
                                                   "simt_gemm f32 fwd");
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
    return launch<float, 128, 128, 8, 8, 8, true>(Gb, ldg, A, lda, D, ldd, B, K, rows, st,
                                                  "simt_gemm f32 adj");
}
