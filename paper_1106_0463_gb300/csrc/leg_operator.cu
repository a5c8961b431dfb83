// Plan-time construction of the Abel-interpolation operator (FP64) and of the
// per-dtype operand planes derived from it.
//
// Method (arXiv:1106.0463, Theorem 1, Eq. 2.5 and the quadrature paragraph
// after Eq. 2.14): on the grid y_j = 2 pi j / M the Abel-type integral
//     phi(y) = int_{cos y}^1 f(x) / sqrt(2 (x - cos y)) dx
// becomes, with x = cos y + s^2 and s = sqrt(2)|sin(y/2)| tau,
//     phi(y) = 2 |sin(y/2)| g(y),   g(y) = int_0^1 f(1 - 2 sin^2(y/2)(1 - tau^2)) dtau,
// and g is taken by Gauss-Legendre in tau.  With f given at the K
// Chebyshev-Lobatto nodes x_k = cos(pi k/(K-1)) and read through its
// barycentric interpolant, g_j = sum_k A[j,k] f_k with
//     A[j,k] = sum_q w_q l_k(x_jq),   1 - x_jq = 2 sin^2(pi j/M) (1 - tau_q^2).
// Rows j and M-j coincide (g is even: the symmetry Eq. 2.12), so only rows
// j = 0..M/2 are built.  Differences x - x_k are formed as
// (1 - x_k) - (1 - x_jq) with 1 - x_k = 2 sin^2(pi k / (2(K-1))), which keeps
// full relative accuracy next to x = 1 (y -> 0).
#include <math.h>
#include <stdio.h>

#include "leg_internal.cuh"

namespace {

// --- Gauss-Legendre rule on [-1,1], FP64, Newton on the three-term recurrence.
__device__ void legendre_pn_pnm1(int n, double x, double &pn, double &pnm1)
{
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    pn = (n == 0) ? 1.0 : p1;
    pnm1 = (n == 0) ? 0.0 : p0;
}

// Nodes in descending order x[0] > x[1] > ...; only the nonnegative half is
// needed by the tau rules, i = 0..(n+1)/2-1.
__global__ void gauss_legendre_half_kernel(int n, double *x, double *w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (n + 1) / 2) return;
    double z;
    if (2 * i + 1 == n) {
        z = 0.0;   // middle node of an odd rule
    } else {
        z = cospi((4.0 * i + 3.0) / (4.0 * n + 2.0));
        for (int it = 0; it < 60; ++it) {
            double pn, pm;
            legendre_pn_pnm1(n, z, pn, pm);
            double dp = n * (z * pn - pm) / ((z - 1.0) * (z + 1.0));
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) <= 1e-16 * (1.0 + fabs(z))) break;
        }
    }
    double pn, pm;
    legendre_pn_pnm1(n, z, pn, pm);
    double dp = n * (z * pn - pm) / ((z - 1.0) * (z + 1.0));
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z) * (1.0 + z) * dp * dp);
}

// tau rule on [0,1]: nonnegative half of a 2Q-point rule (sym) or a Q-point
// rule mapped affinely (literal).  Writes tau_q, w_q, 1 - tau_q^2.
__global__ void tau_rule_kernel(int Q, int literal, const double *xh, const double *wh,
                                double *omt2, double *wq)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    double tau, w;
    if (!literal) {
        tau = xh[q];          // q-th largest root of the 2Q-point rule (all positive)
        w = wh[q];
    } else {
        // Q-point rule: node t_q (descending list holds the nonnegative half;
        // the negative half is its mirror).
        int half = (Q + 1) / 2;
        double t = (q < half) ? xh[q] : -xh[Q - 1 - q];
        double wt = (q < half) ? wh[q] : wh[Q - 1 - q];
        tau = 0.5 * (t + 1.0);
        w = 0.5 * wt;
    }
    omt2[q] = (1.0 - tau) * (1.0 + tau);
    wq[q] = w;
}

__global__ void cl_node_kernel(int K, double *omxk, double *lam)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double s = sinpi(k / (2.0 * (K - 1)));
    omxk[k] = 2.0 * s * s;
    double l = (k & 1) ? -1.0 : 1.0;
    if (k == 0 || k == K - 1) l *= 0.5;
    lam[k] = l;
}

// One CTA per operator row j.  Pass 1 (one warp per quadrature point q):
// barycentric denominator S_q = sum_k lam_k / (x_jq - x_k), or the index of
// the node that x_jq hits exactly.  Pass 2 (one thread per k):
// A[j,k] = lam_k sum_q (w_q / S_q) / (x_jq - x_k), hits contributing w_q.
__global__ void __launch_bounds__(256) abel_operator_kernel(
    int M, int K, int Q, const double *__restrict__ omt2, const double *__restrict__ wq,
    const double *__restrict__ omxk, const double *__restrict__ lam, double *__restrict__ A)
{
    extern __shared__ double sh[];
    double *coef = sh;                        // Q: w_q / S_q
    int *hit = reinterpret_cast<int *>(sh + Q);   // Q: exact node hit or -1
    __shared__ double s_u;

    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
        double s = sinpi((double)j / (double)M);
        s_u = 2.0 * s * s;                     // 1 - cos(y_j) = 2 sin^2(y_j/2)
    }
    __syncthreads();
    const double u = s_u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

    for (int q = warp; q < Q; q += nwarp) {
        const double omx = __dmul_rn(u, omt2[q]);
        double s = 0.0;
        int h = -1;
        for (int k = lane; k < K; k += 32) {
            double d = __dsub_rn(omxk[k], omx);          // x_jq - x_k
            if (d == 0.0) h = k;
            else s += lam[k] / d;
        }
        for (int off = 16; off > 0; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            h = max(h, __shfl_xor_sync(0xffffffffu, h, off));
        }
        if (lane == 0) {
            hit[q] = h;
            coef[q] = (h >= 0) ? wq[q] : wq[q] / s;
        }
    }
    __syncthreads();

    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double xk = omxk[k];
        double acc = 0.0, acc_hit = 0.0;
        for (int q = 0; q < Q; ++q) {
            const int h = hit[q];
            if (h >= 0) {
                if (h == k) acc_hit += coef[q];
            } else {
                acc += coef[q] / __dsub_rn(xk, __dmul_rn(u, omt2[q]));
            }
        }
        A[(size_t)j * K + k] = lam[k] * acc + acc_hit;
    }
}

// --- per-dtype planes --------------------------------------------------------
__global__ void plane_f32_kernel(const double *A, float *A32, size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) A32[i] = (float)A[i];
}

__global__ void plane_bf16_kernel(const double *A, int K, int Kp, __nv_bfloat16 *Ab)
{
    const int j = blockIdx.x;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x)
        Ab[(size_t)j * Kp + k] = __float2bfloat16_rn(k < K ? (float)A[(size_t)j * K + k] : 0.0f);
}

// Split-FP16 planes of row j.  Row scale 2^e_j >= sum_k |A[j,k]| (so the
// scaled row has L1 norm <= 1).  With a = A[j,k] / 2^e_j, s = fbits and
// abits = LEG_SPLIT_GRID - s:
//   A0 = a rounded to FP16 but never finer than 2^-abits (a fixed-point
//        grid for small |a|, ordinary FP16 rounding above),
//   r1 = (a - A0) 2^s,  A1 = fp16(r1),  A2s = fp16((r1 - A1) 2^s),
// so a = A0 + 2^-s A1 + 2^-2s A2s up to the FP16 rounding of A2s.
__global__ void plane_split_kernel(const double *A, int K, int Kp, __half *A0p, __half *A1p,
                                   __half *A2p, int *rowexp, int fbits)
{
    const int abits = LEG_SPLIT_GRID - fbits;
    const int j = blockIdx.x;
    __shared__ double red[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) s += fabs(A[(size_t)j * K + k]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) {
            int e = 0;
            if (s > 0.0) {
                double m = frexp(s, &e);       // s = m 2^e, m in [0.5, 1)
                if (m == 0.5) e -= 1;          // exact power of two
            }
            red[0] = ldexp(1.0, -e);
            rowexp[j] = e;
        }
    }
    __syncthreads();
    const double inv = red[0];
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double a = (k < K) ? A[(size_t)j * K + k] * inv : 0.0;
        double a0;
        if (fabs(a) >= ldexp(1.0, 10 - abits)) a0 = (double)__double2half(a);   // FP16 ulp >= grid
        else a0 = rint(ldexp(a, abits)) * ldexp(1.0, -abits);
        double r1 = ldexp(a - a0, fbits);
        __half h1 = __double2half(r1);
        __half h2 = __double2half(ldexp(r1 - (double)h1, fbits));
        size_t o = (size_t)j * Kp + k;
        A0p[o] = __double2half(a0);
        A1p[o] = h1;
        A2p[o] = h2;
    }
}

// out[c * ldo + r] = in[r * ldi + c] for r < R, c < C (32 x 32 tiles, 32 x 8 threads).
__global__ void transpose_f64_kernel(const double *__restrict__ in, int ldi, double *__restrict__ out, int ldo,
                                     int R, int C)
{
    __shared__ double t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[(size_t)r * ldi + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * ldo + r] = t[threadIdx.x][i];
    }
}

void transpose_f64(const double *in, int ldi, double *out, int ldo, int R, int C)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    transpose_f64_kernel<<<grid, block>>>(in, ldi, out, ldo, R, C);
}

// e^{2 pi i n / M} for n < M, then (entries M .. M + M/4 - 1) the compact copy
// e^{2 pi i q / (M/4)} = entry 4q, which the register-tiled FFT passes read
// (their twiddle indices are multiples of 4: a table a quarter the size).
__global__ void twiddle_kernel(int M, double2 *t64, float2 *t32, float4 *tdf)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= M + M / 4) return;
    const int m = n < M ? n : 4 * (n - M);
    double s, c;
    sincospi(2.0 * m / M, &s, &c);
    t64[n] = make_double2(c, s);
    t32[n] = make_float2((float)c, (float)s);
    float ch = (float)c, sh = (float)s;
    tdf[n] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
}

}  // namespace

int leg_build_twiddles(leg_plan *p)
{
    const size_t n = (size_t)p->M + p->M / 4;   // the full table and its compact copy
    LEG_CUDA_TRY(leg_dev_malloc(&p->tw64, sizeof(double2) * n));
    LEG_CUDA_TRY(leg_dev_malloc(&p->tw32, sizeof(float2) * n));
    LEG_CUDA_TRY(leg_dev_malloc(&p->twdf, sizeof(float4) * n));
    twiddle_kernel<<<(int)((n + 255) / 256), 256>>>(p->M, p->tw64, p->tw32, p->twdf);
    LEG_LAUNCH_CHECK("twiddle_kernel");
    return LEG_OK;
}

int leg_build_operator(leg_plan *p)
{
    const int K = p->K, Q = p->Q, rows = p->rows;
    const int literal = (p->flags & LEG_FLAG_TAU_LITERAL) ? 1 : 0;
    const int n_rule = literal ? Q : 2 * Q;
    const int n_half = (n_rule + 1) / 2;

    double *xh = nullptr, *wh = nullptr, *omxk = nullptr, *lam = nullptr;
    auto cleanup = [&]() {
        leg_dev_free(xh); leg_dev_free(wh); leg_dev_free(omxk); leg_dev_free(lam);
    };
#define LEG_TRY_CLEAN(expr)                                                         \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            cleanup();                                                              \
            return leg_set_error(_e == cudaErrorMemoryAllocation ? LEG_ERR_OOM : LEG_ERR_CUDA, \
                                 std::string(#expr) + ": " + cudaGetErrorString(_e));         \
        }                                                                           \
    } while (0)

    LEG_TRY_CLEAN(leg_dev_malloc(&xh, sizeof(double) * n_half));
    LEG_TRY_CLEAN(leg_dev_malloc(&wh, sizeof(double) * n_half));
    LEG_TRY_CLEAN(leg_dev_malloc(&p->omt2, sizeof(double) * Q));
    LEG_TRY_CLEAN(leg_dev_malloc(&p->wq, sizeof(double) * Q));
    double *omt2 = p->omt2, *wq = p->wq;
    LEG_TRY_CLEAN(leg_dev_malloc(&omxk, sizeof(double) * K));
    LEG_TRY_CLEAN(leg_dev_malloc(&lam, sizeof(double) * K));
    LEG_TRY_CLEAN(leg_dev_malloc(&p->A64, sizeof(double) * (size_t)rows * K));

    gauss_legendre_half_kernel<<<(n_half + 127) / 128, 128>>>(n_rule, xh, wh);
    tau_rule_kernel<<<(Q + 127) / 128, 128>>>(Q, literal, xh, wh, omt2, wq);
    cl_node_kernel<<<(K + 255) / 256, 256>>>(K, omxk, lam);
    size_t smem = (size_t)Q * (sizeof(double) + sizeof(int));
    LEG_TRY_CLEAN(cudaFuncSetAttribute(abel_operator_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    abel_operator_kernel<<<rows, 256, smem>>>(p->M, K, Q, omt2, wq, omxk, lam, p->A64);
    LEG_TRY_CLEAN(cudaGetLastError());
    cleanup();
#undef LEG_TRY_CLEAN
    return leg_build_planes(p);
}

// LEG_FLAG_COLLAPSED: L = R A (N x K, FP64), row n of L giving c_n of Eq. 2.4
// with the twist of Eq. 2.5 from the K samples.  Column k of L is the plan's
// FP64 transform (twist, first difference, (2n+1)) of column k of A, so the
// columns of A are transposed into rows, transformed as a batch of K
// "functions", and the result transposed back.
int leg_build_collapsed(leg_plan *p)
{
    const int K = p->K, rows = p->rows, N = p->N;
    const int ldt = leg_round_up(rows, 8);
    double *AT = nullptr, *LT = nullptr;
    auto fail = [&](cudaError_t e, const char *what) {
        leg_dev_free(AT);
        leg_dev_free(LT);
        return leg_set_error(e == cudaErrorMemoryAllocation ? LEG_ERR_OOM : LEG_ERR_CUDA,
                             std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = leg_dev_malloc(&AT, sizeof(double) * (size_t)K * ldt)) != cudaSuccess) return fail(e, "collapsed operator");
    if ((e = leg_dev_malloc(&LT, sizeof(double) * (size_t)K * N)) != cudaSuccess) return fail(e, "collapsed operator");
    if ((e = leg_dev_malloc(&p->L64, sizeof(double) * (size_t)N * K)) != cudaSuccess)
        return fail(e, "collapsed operator");
    if ((e = cudaMemset(AT, 0, sizeof(double) * (size_t)K * ldt)) != cudaSuccess) return fail(e, "collapsed operator");
    transpose_f64(p->A64, K, AT, ldt, rows, K);
    int rc = leg_fft_forward_f64(p, AT, ldt, LT, K, 0);
    if (rc) {
        leg_dev_free(AT);
        leg_dev_free(LT);
        return rc;
    }
    transpose_f64(LT, N, p->L64, K, K, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "collapsed operator");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "collapsed operator");
    leg_dev_free(AT);
    leg_dev_free(LT);
    return LEG_OK;
}

// Operand planes of the plan's dtype, derived from the FP64 operator (A, or
// L = R A for collapsed plans).
int leg_build_planes(leg_plan *p)
{
    const int K = p->K;
    const bool col = p->collapsed();
    if (col && !p->L64) {
        int rc = leg_build_collapsed(p);
        if (rc) return rc;
    }
    const double *S = col ? p->L64 : p->A64;
    const int rows = col ? p->N : p->rows;
    p->grows = rows;
    auto cleanup = []() {};
#define LEG_TRY_CLEAN(expr)                                                         \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            cleanup();                                                              \
            return leg_set_error(_e == cudaErrorMemoryAllocation ? LEG_ERR_OOM : LEG_ERR_CUDA, \
                                 std::string(#expr) + ": " + cudaGetErrorString(_e));         \
        }                                                                           \
    } while (0)
    if (p->dtype == LEG_F32) {
        size_t n = (size_t)rows * K;
        LEG_TRY_CLEAN(leg_dev_malloc(&p->A32, sizeof(float) * n));
        plane_f32_kernel<<<(unsigned)((n + 255) / 256), 256>>>(S, p->A32, n);
    } else if (p->dtype == LEG_BF16) {
        LEG_TRY_CLEAN(leg_dev_malloc(&p->Abf, sizeof(__nv_bfloat16) * (size_t)rows * p->Kp));
        plane_bf16_kernel<<<rows, 256>>>(S, K, p->Kp, p->Abf);
    } else if (p->dtype == LEG_SPLIT_FP16) {
        const size_t plane = (size_t)rows * p->Kp;
        LEG_TRY_CLEAN(leg_dev_malloc(&p->Ah[0], sizeof(__half) * 3 * plane));
        p->Ah[1] = p->Ah[0] + plane;
        p->Ah[2] = p->Ah[0] + 2 * plane;
        LEG_TRY_CLEAN(leg_dev_malloc(&p->rowexp, sizeof(int) * rows));
        plane_split_kernel<<<rows, 256>>>(S, K, p->Kp, p->Ah[0], p->Ah[1], p->Ah[2], p->rowexp, p->fbits);
        LEG_TRY_CLEAN(cudaGetLastError());
        int rc2 = leg_build_split_transposed(p);
        if (rc2) {
            cleanup();
            return rc2;
        }
    }
    LEG_TRY_CLEAN(cudaGetLastError());
    LEG_TRY_CLEAN(cudaDeviceSynchronize());
    // row 0 (y = 0: every quadrature point is x = 1, the node k = 0) is a00 e_0
    if (p->dtype == LEG_SPLIT_FP16 && !col)
        LEG_TRY_CLEAN(cudaMemcpy(&p->a00, p->A64, sizeof(double), cudaMemcpyDeviceToHost));
#undef LEG_TRY_CLEAN
    return LEG_OK;
}
