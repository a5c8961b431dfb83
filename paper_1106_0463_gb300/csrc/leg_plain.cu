// The plain method (arXiv:1106.0463, Sec. 2, the quadrature paragraph after
// Eq. 2.14): the Abel integral of a closed-form f evaluated at the quadrature
// points themselves,
//     g_j = sum_q w_q f(x_jq),   1 - x_jq = 2 sin^2(pi j / M) (1 - tau_q^2),
// for the rows j = 0..M/2 of the grid y_j = 2 pi j / M, in FP64.  The result
// feeds the same FFT stage as the sampled path.  Families: the generating
// function (Eq. 2.2), e^{ax}, |x|^alpha (the test function of Table 1, whose
// coefficients Eq. 2.15 gives in closed form), and Chebyshev series given by
// coefficients.
#include "leg_internal.cuh"

namespace {

__device__ __forceinline__ double closed_form(int family, double par, double omx)
{
    if (family == LEG_FAMILY_GENFN) {
        // (1 - 2 x t + t^2)^(-1/2) with x = 1 - omx:  (1 - t)^2 + 2 t omx
        double om = 1.0 - par;
        return rsqrt(om * om + 2.0 * par * omx);
    }
    if (family == LEG_FAMILY_ABSPOW) {
        // |x|^alpha (Table 1: alpha = 3/2); |x| = |1 - omx|, 0^alpha = 0
        const double ax = fabs(1.0 - omx);
        return ax > 0.0 ? pow(ax, par) : 0.0;
    }
    // exp(a x)
    return exp(par * (1.0 - omx));
}

__global__ void plain_g_kernel(int M, int Q, int family, const double *__restrict__ params,
                               const double *__restrict__ omt2, const double *__restrict__ wq,
                               double *__restrict__ G, int ldg)
{
    const int b = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > M / 2) return;
    const double par = params[b];
    const double s = sinpi((double)j / (double)M);
    const double u = 2.0 * s * s;
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) acc += wq[q] * closed_form(family, par, u * omt2[q]);
    G[(size_t)b * ldg + j] = acc;
}

// f(x) = sum_{m < Kc} coef[m] T_m(x) by Clenshaw's recurrence in FP64,
//   b_k = coef_k + 2 x b_{k+1} - b_{k+2} (k = Kc-1 .. 1),  f = coef_0 + x b_1 - b_2,
// with the function's coefficients staged in shared memory.
__global__ void plain_g_cheb_kernel(int M, int Q, const double *__restrict__ coef, int Kc,
                                    const double *__restrict__ omt2, const double *__restrict__ wq,
                                    double *__restrict__ G, int ldg)
{
    extern __shared__ double cs[];
    const int b = blockIdx.y;
    for (int k = threadIdx.x; k < Kc; k += blockDim.x) cs[k] = coef[(size_t)b * Kc + k];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > M / 2) return;
    const double s = sinpi((double)j / (double)M);
    const double u = 2.0 * s * s;
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) {
        const double x = 1.0 - u * omt2[q];
        double b1 = 0.0, b2 = 0.0;
        for (int k = Kc - 1; k >= 1; --k) {
            const double t = fma(2.0 * x, b1, cs[k] - b2);
            b2 = b1;
            b1 = t;
        }
        acc += wq[q] * fma(x, b1, cs[0] - b2);
    }
    G[(size_t)b * ldg + j] = acc;
}

}  // namespace

int leg_plain_g_cheb(const leg_plan *p, const double *coef, int Kc, int B, double *G, int ldg, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const size_t smem = sizeof(double) * (size_t)Kc;
    if (smem > 48 * 1024)
        LEG_CUDA_TRY(cudaFuncSetAttribute(plain_g_cheb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((p->rows + 127) / 128, B);
    plain_g_cheb_kernel<<<grid, 128, smem, st>>>(p->M, p->Q, coef, Kc, p->omt2, p->wq, G, ldg);
    LEG_LAUNCH_CHECK("plain_g_cheb_kernel");
    return LEG_OK;
}

int leg_plain_g(const leg_plan *p, int family, const double *params, int B, double *G, int ldg,
                cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    dim3 grid((p->rows + 127) / 128, B);
    plain_g_kernel<<<grid, 128, 0, st>>>(p->M, p->Q, family, params, p->omt2, p->wq, G, ldg);
    LEG_LAUNCH_CHECK("plain_g_kernel");
    return LEG_OK;
}
