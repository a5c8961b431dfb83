/*
 * FP64 CPU oracle for the Legendre-coefficient method of De Micheli & Viano,
 * "A new and efficient method for the computation of Legendre coefficients"
 * (arXiv:1106.0463).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header or table with the CUDA library.
 *
 * Independent routes to the coefficients c_n of f(x) = sum_n c_n P_n(x):
 *
 *   Route 1 (plain definition, Eq. 2.3):
 *       c_n = (n + 1/2) * integral_{-1}^{1} f(x) P_n(x) dx,
 *     evaluated by a Gauss-Legendre rule, with P_n from the three-term
 *     recurrence that follows from the generating function (Eq. 2.2).
 *
 *   Route 2 (the paper's method: Theorem 1, Eq. 2.4 and Eq. 2.5, then the
 *   quadrature + FFT recipe of Sec. 2 after Eq. 2.14), written step by step:
 *     - y-grid: y_j = -pi + 2 pi j / M, j = 0..M-1 (the interval [-pi, pi)
 *       of Eq. 2.4, trapezoid rule on a periodic integrand);
 *     - the Abel-type integral of Eq. 2.14,
 *           phi(y) = int_{cos y}^{1} f(x) / sqrt(2 (x - cos y)) dx,
 *       under the change of variable x = cos y + s^2, s = s_max * tau,
 *       s_max = sqrt(2) |sin(y/2)|, which removes the endpoint singularity:
 *           phi(y) = 2 |sin(y/2)| * int_0^1 f(1 - 2 sin^2(y/2) (1 - tau^2)) dtau,
 *       the tau-integral taken by Gauss-Legendre;
 *     - fhat(y) = eps(y) e^{i y/2} phi(y) / (2 pi i)   (Eq. 2.5);
 *     - a_n = (2 pi / M) sum_j fhat(y_j) e^{i n y_j}    (Eq. 2.4, trapezoid),
 *       as a direct O(M N) sum (no FFT), and c_n = (2n+1) a_n.
 *
 *   Route 3 (the half-range sine form, Eq. 2.13 with phi of Eq. 2.14):
 *       c_n = (2/pi) (n + 1/2) int_0^pi phi(y) sin((n + 1/2) y) dy
 *     on y_j = pi j / L, j = 0..L, by the trapezoid rule, phi from the same
 *     substitution as route 2, the sine sum written out directly.
 *
 *   Route 1 transposed (or_coeffs_quadrature_T, or_cl_barycentric_T): the
 *   adjoint df = L^T v of the route-1 map on sampled inputs, for checks of
 *   the library's adjoint at sizes where explicit operators are too large.
 *
 * Sampled inputs are values f_k at the Chebyshev-Lobatto nodes
 * x_k = cos(pi k / (K-1)), k = 0..K-1 (x_0 = 1 down to x_{K-1} = -1), and are
 * evaluated elsewhere through the barycentric interpolant on those nodes,
 * with the differences x - x_k formed as (1 - x_k) - (1 - x) so that points
 * next to x = 1 (y -> 0) keep their relative accuracy.
 *
 * Pins: see tests/test_oracle.py (closed forms of Eq. 2.2, Eq. 2.15 / Table 1,
 * P_m -> delta, e^{ax}, Parseval, symmetry Eq. 2.12, sine form Eq. 2.13,
 * brute-force high-precision quadrature, adjoint identities).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1, 1]: nodes ascending, weights.                 */
/* Newton's method on P_n, with P_n and P_n' from the three-term recurrence  */
/* (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}; weights 2 / ((1-x^2) P_n'(x)^2). */
/* ------------------------------------------------------------------------ */
static void legendre_pair(int n, double x, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

void or_gauss_legendre(int n, double *x, double *w)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < (n + 1) / 2; ++i) {
        /* i-th largest root; classical initial guess */
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn, pm, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, z, &pn, &pm);
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16 * (1.0 + fabs(z))) break;
        }
        legendre_pair(n, z, &pn, &pm);
        dp = n * (z * pn - pm) / (z * z - 1.0);
        double wt = 2.0 / ((1.0 - z) * (1.0 + z) * dp * dp);
        /* ascending order: largest root goes last */
        x[n - 1 - i] = z;
        w[n - 1 - i] = wt;
        x[i] = -z;
        w[i] = wt;
    }
    if (n % 2 == 1) {   /* middle node is exactly 0 */
        double pn, pm;
        int m = n / 2;
        legendre_pair(n, 0.0, &pn, &pm);
        double dp = n * (0.0 * pn - pm) / (0.0 - 1.0);
        x[m] = 0.0;
        w[m] = 2.0 / (dp * dp);
    }
}

/* ------------------------------------------------------------------------ */
/* The rule for int_0^1 h(tau) dtau used on the Abel integral.               */
/*   sym = 1: the nonnegative half of a 2Q-point Gauss-Legendre rule on      */
/*            [-1,1] (the integrand is even in s, hence in tau): Q distinct  */
/*            nodes, weights summing to 1.                                   */
/*   sym = 0: a Q-point Gauss-Legendre rule mapped affinely onto [0,1].       */
/* Also returns 1 - tau^2 accurately as (1 - tau)(1 + tau).                   */
/* ------------------------------------------------------------------------ */
void or_tau_rule(int Q, int sym, double *tau, double *wt, double *one_minus_tau2)
{
    if (sym) {
        double *x = (double *)malloc(sizeof(double) * 2 * Q);
        double *w = (double *)malloc(sizeof(double) * 2 * Q);
        or_gauss_legendre(2 * Q, x, w);
        for (int q = 0; q < Q; ++q) {
            tau[q] = x[Q + q];
            wt[q] = w[Q + q];
        }
        free(x);
        free(w);
    } else {
        double *x = (double *)malloc(sizeof(double) * Q);
        double *w = (double *)malloc(sizeof(double) * Q);
        or_gauss_legendre(Q, x, w);
        for (int q = 0; q < Q; ++q) {
            tau[q] = 0.5 * (x[q] + 1.0);
            wt[q] = 0.5 * w[q];
        }
        free(x);
        free(w);
    }
    for (int q = 0; q < Q; ++q)
        one_minus_tau2[q] = (1.0 - tau[q]) * (1.0 + tau[q]);
}

/* ------------------------------------------------------------------------ */
/* P_n(x_i), n = 0..N-1, for npts points: P[n * npts + i].                    */
/* ------------------------------------------------------------------------ */
void or_legendre_table(int N, int npts, const double *x, double *P)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < npts; ++i) {
        double p0 = 1.0, p1 = x[i];
        if (N > 0) P[i] = 1.0;
        if (N > 1) P[(size_t)npts + i] = p1;
        for (int n = 1; n + 1 < N; ++n) {
            double p2 = ((2.0 * n + 1.0) * x[i] * p1 - n * p0) / (n + 1.0);
            P[(size_t)(n + 1) * npts + i] = p2;
            p0 = p1;
            p1 = p2;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Route 1: c_n = (n + 1/2) sum_i wts_i f(x_i) P_n(x_i)   (Eq. 2.3).         */
/* fvals: B x npts row-major; c: B x N row-major.                             */
/* ------------------------------------------------------------------------ */
void or_coeffs_quadrature(int N, int npts, const double *x, const double *wts,
                          int B, const double *fvals, double *c)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)N * npts);
    or_legendre_table(N, npts, x, P);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        const double *fb = fvals + (size_t)b * npts;
        for (int n = 0; n < N; ++n) {
            const double *Pn = P + (size_t)n * npts;
            double s = 0.0;
            for (int i = 0; i < npts; ++i) s += wts[i] * fb[i] * Pn[i];
            c[(size_t)b * N + n] = (n + 0.5) * s;
        }
    }
    free(P);
}

/* ------------------------------------------------------------------------ */
/* Barycentric interpolation on the K Chebyshev-Lobatto nodes.                */
/* Evaluation points are given through omx = 1 - x.  Second-form weights      */
/* lambda_k = (-1)^k, halved at k = 0 and k = K-1.  An evaluation point that  */
/* coincides with a node returns that node's value.                           */
/* f: B x K, out: B x npts.                                                   */
/* ------------------------------------------------------------------------ */
void or_cl_barycentric(int K, int B, const double *f, int npts, const double *omx, double *out)
{
    double *omxk = (double *)malloc(sizeof(double) * K);
    double *lam = (double *)malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        double s = sin(M_PI * k / (2.0 * (K - 1)));
        omxk[k] = 2.0 * s * s;              /* 1 - cos(pi k/(K-1)) */
        lam[k] = (k % 2 == 0) ? 1.0 : -1.0;
    }
    lam[0] *= 0.5;
    lam[K - 1] *= 0.5;
    #pragma omp parallel
    {
        double *t = (double *)malloc(sizeof(double) * K);
        #pragma omp for schedule(dynamic, 8)
        for (int i = 0; i < npts; ++i) {
            int hit = -1;
            double den = 0.0;
            for (int k = 0; k < K; ++k) {
                double d = omxk[k] - omx[i];        /* = x - x_k */
                if (d == 0.0) { hit = k; break; }
                t[k] = lam[k] / d;
                den += t[k];
            }
            for (int b = 0; b < B; ++b) {
                const double *fb = f + (size_t)b * K;
                double v;
                if (hit >= 0) {
                    v = fb[hit];
                } else {
                    double num = 0.0;
                    for (int k = 0; k < K; ++k) num += t[k] * fb[k];
                    v = num / den;
                }
                out[(size_t)b * npts + i] = v;
            }
        }
        free(t);
    }
    free(omxk);
    free(lam);
}

/* ------------------------------------------------------------------------ */
/* Route 2, step 1: the Abel quadrature points.                               */
/*   y_j = -pi + 2 pi j / M,  1 - x_jq = 2 sin^2(y_j/2) (1 - tau_q^2).        */
/* omx: M x Q.                                                                */
/* ------------------------------------------------------------------------ */
void or_abel_points(int M, int Q, int sym, double *omx, double *wq)
{
    double *tau = (double *)malloc(sizeof(double) * Q);
    double *omt2 = (double *)malloc(sizeof(double) * Q);
    or_tau_rule(Q, sym, tau, wq, omt2);
    for (int j = 0; j < M; ++j) {
        double y = -M_PI + 2.0 * M_PI * j / M;
        double s = sin(0.5 * y);
        double u = 2.0 * s * s;
        for (int q = 0; q < Q; ++q) omx[(size_t)j * Q + q] = u * omt2[q];
    }
    free(tau);
    free(omt2);
}

/* ------------------------------------------------------------------------ */
/* Route 2, step 2: phi(y_j) = 2 |sin(y_j/2)| sum_q w_q f(x_jq)   (Eq. 2.14  */
/* after the substitution).  fq: B x M x Q, phi: B x M.                       */
/* ------------------------------------------------------------------------ */
void or_abel_phi(int M, int Q, int B, const double *fq, const double *wq, double *phi)
{
    #pragma omp parallel for schedule(static)
    for (int b = 0; b < B; ++b) {
        for (int j = 0; j < M; ++j) {
            double y = -M_PI + 2.0 * M_PI * j / M;
            const double *row = fq + ((size_t)b * M + j) * Q;
            double g = 0.0;
            for (int q = 0; q < Q; ++q) g += wq[q] * row[q];
            phi[(size_t)b * M + j] = 2.0 * fabs(sin(0.5 * y)) * g;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Route 2, step 3: fhat(y) = eps(y) e^{iy/2} phi(y) / (2 pi i)  (Eq. 2.5),   */
/* a_n = (2 pi / M) sum_j fhat(y_j) e^{i n y_j}  (Eq. 2.4),  c_n = (2n+1) a_n. */
/* Direct sum, no FFT.  phi: B x M; c_re, c_im: B x N.                        */
/* ------------------------------------------------------------------------ */
void or_abel_coeffs(int N, int M, int B, const double *phi, double *c_re, double *c_im)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        /* per-function private copies of the twisted samples */
        double *hr = (double *)malloc(sizeof(double) * M);
        double *hi = (double *)malloc(sizeof(double) * M);
        for (int j = 0; j < M; ++j) {
            double y = -M_PI + 2.0 * M_PI * j / M;
            double eps = (y > 0.0) ? 1.0 : ((y < 0.0) ? -1.0 : 0.0);
            /* eps e^{iy/2} / (2 pi i) = eps (cos(y/2) + i sin(y/2)) * (-i) / (2 pi) */
            double er = eps * sin(0.5 * y) / (2.0 * M_PI);
            double ei = -eps * cos(0.5 * y) / (2.0 * M_PI);
            double p = phi[(size_t)b * M + j];
            hr[j] = er * p;
            hi[j] = ei * p;
        }
        for (int n = 0; n < N; ++n) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < M; ++j) {
                /* e^{i n y_j}; angle reduced exactly through the integer n*j mod M */
                long long r = ((long long)n * j) % M;
                double ang = 2.0 * M_PI * (double)r / M - M_PI * (double)(n % 2);
                double cr = cos(ang), ci = sin(ang);
                sr += hr[j] * cr - hi[j] * ci;
                si += hr[j] * ci + hi[j] * cr;
            }
            double scale = (2.0 * n + 1.0) * 2.0 * M_PI / M;
            c_re[(size_t)b * N + n] = scale * sr;
            c_im[(size_t)b * N + n] = scale * si;
        }
        free(hr);
        free(hi);
    }
}

/* ------------------------------------------------------------------------ */
/* Explicit operators for the adjoint checks (small sizes only).             */
/* Abel-interpolation operator on the y-grid of route 2, with the factor      */
/* 2|sin(y/2)| of phi included:  phi = Aphi f,   Aphi: M x K,                 */
/*   Aphi[j,k] = 2|sin(y_j/2)| sum_q w_q l_k(x_jq).                           */
/* ------------------------------------------------------------------------ */
void or_abel_operator(int M, int K, int Q, int sym, double *Aphi)
{
    double *omx = (double *)malloc(sizeof(double) * (size_t)M * Q);
    double *wq = (double *)malloc(sizeof(double) * Q);
    or_abel_points(M, Q, sym, omx, wq);
    double *I = (double *)calloc((size_t)K * K, sizeof(double));
    for (int k = 0; k < K; ++k) I[(size_t)k * K + k] = 1.0;
    /* basis functions l_k at every quadrature point: L[k, (j,q)] */
    double *Lk = (double *)malloc(sizeof(double) * (size_t)K * M * Q);
    or_cl_barycentric(K, K, I, M * Q, omx, Lk);
    for (int j = 0; j < M; ++j) {
        double y = -M_PI + 2.0 * M_PI * j / M;
        double s2 = 2.0 * fabs(sin(0.5 * y));
        for (int k = 0; k < K; ++k) {
            const double *row = Lk + (size_t)k * M * Q + (size_t)j * Q;
            double a = 0.0;
            for (int q = 0; q < Q; ++q) a += wq[q] * row[q];
            Aphi[(size_t)j * K + k] = s2 * a;
        }
    }
    free(omx);
    free(wq);
    free(I);
    free(Lk);
}

/* Real part of the twist + DFT of route 2 as a matrix: c = R phi, R: N x M. */
void or_twisted_dft_matrix(int N, int M, double *R)
{
    double *e = (double *)calloc(M, sizeof(double));
    double *cre = (double *)malloc(sizeof(double) * N);
    double *cim = (double *)malloc(sizeof(double) * N);
    for (int j = 0; j < M; ++j) {
        memset(e, 0, sizeof(double) * M);
        e[j] = 1.0;
        or_abel_coeffs(N, M, 1, e, cre, cim);
        for (int n = 0; n < N; ++n) R[(size_t)n * M + j] = cre[n];
    }
    free(e);
    free(cre);
    free(cim);
}

/* ------------------------------------------------------------------------ */
/* Route 3: the half-range sine form of the coefficients (Eq. 2.13, with phi */
/* of Eq. 2.14), obtained in the paper from the symmetry Eq. 2.12:           */
/*   c_n = (2/pi) (n + 1/2) int_0^pi phi(y) sin((n + 1/2) y) dy,             */
/* on the grid y_j = pi j / L, j = 0..L, by the trapezoid rule (end points   */
/* at half weight), phi from the same substitution as route 2:               */
/*   phi(y) = 2 sin(y/2) int_0^1 f(1 - 2 sin^2(y/2)(1 - tau^2)) dtau.        */
/* Step 1: the quadrature points, omx: (L+1) x Q.                            */
/* ------------------------------------------------------------------------ */
void or_sine_points(int L, int Q, int sym, double *omx, double *wq)
{
    double *tau = (double *)malloc(sizeof(double) * Q);
    double *omt2 = (double *)malloc(sizeof(double) * Q);
    or_tau_rule(Q, sym, tau, wq, omt2);
    for (int j = 0; j <= L; ++j) {
        double s = sin(0.5 * M_PI * j / L);
        double u = 2.0 * s * s;
        for (int q = 0; q < Q; ++q) omx[(size_t)j * Q + q] = u * omt2[q];
    }
    free(tau);
    free(omt2);
}

/* Step 2: phi(y_j) = 2 sin(y_j/2) sum_q w_q f(x_jq), y_j in [0, pi].        */
/* fq: B x (L+1) x Q, phi: B x (L+1).                                        */
void or_sine_phi(int L, int Q, int B, const double *fq, const double *wq, double *phi)
{
    #pragma omp parallel for schedule(static)
    for (int b = 0; b < B; ++b) {
        for (int j = 0; j <= L; ++j) {
            const double *row = fq + ((size_t)b * (L + 1) + j) * Q;
            double g = 0.0;
            for (int q = 0; q < Q; ++q) g += wq[q] * row[q];
            phi[(size_t)b * (L + 1) + j] = 2.0 * sin(0.5 * M_PI * j / L) * g;
        }
    }
}

/* Step 3: the sine sum of Eq. 2.13, direct (no fast transform).             */
/* phi: B x (L+1); c: B x N.                                                 */
void or_sine_coeffs(int N, int L, int B, const double *phi, double *c)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        const double *pb = phi + (size_t)b * (L + 1);
        for (int n = 0; n < N; ++n) {
            double s = 0.0;
            for (int j = 0; j <= L; ++j) {
                /* sin((n + 1/2) pi j / L) = sin(pi (2n+1) j / (2L)); the     */
                /* angle is reduced exactly through the integer (2n+1) j mod 4L */
                long long r = ((long long)(2 * n + 1) * j) % (4LL * L);
                double w = (j == 0 || j == L) ? 0.5 : 1.0;
                s += w * pb[j] * sin(M_PI * (double)r / (2.0 * L));
            }
            c[(size_t)b * N + n] = (2.0 / M_PI) * (n + 0.5) * (M_PI / L) * s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Route 1 transposed, for checks of the adjoint df = L^T v of sampled      */
/* inputs.  Route 1 on CL samples is c = P (W (B f)), with B the barycentric */
/* interpolation to the Gauss points, W the Gauss weights and                */
/* P[n, i] = (n + 1/2) P_n(x_i) (Eq. 2.3).  Its transpose is applied in two */
/* steps:                                                                    */
/*   u_i = wts_i sum_n (n + 1/2) v_n P_n(x_i)        (or_coeffs_quadrature_T) */
/*   df_k = sum_i l_k(x_i) u_i                       (or_cl_barycentric_T)    */
/* v: B x N, u: B x npts.                                                    */
/* ------------------------------------------------------------------------ */
void or_coeffs_quadrature_T(int N, int npts, const double *x, const double *wts,
                            int B, const double *v, double *u)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)N * npts);
    or_legendre_table(N, npts, x, P);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        const double *vb = v + (size_t)b * N;
        double *ub = u + (size_t)b * npts;
        for (int i = 0; i < npts; ++i) ub[i] = 0.0;
        for (int n = 0; n < N; ++n) {
            const double *Pn = P + (size_t)n * npts;
            const double a = (n + 0.5) * vb[n];
            for (int i = 0; i < npts; ++i) ub[i] += a * Pn[i];
        }
        for (int i = 0; i < npts; ++i) ub[i] *= wts[i];
    }
    free(P);
}

/* df[b, k] = sum_i l_k(x_i) u[b, i], x_i given by omx = 1 - x_i; the same   */
/* barycentric weights and node-hit rule as or_cl_barycentric.               */
void or_cl_barycentric_T(int K, int B, const double *u, int npts, const double *omx, double *df)
{
    double *omxk = (double *)malloc(sizeof(double) * K);
    double *lam = (double *)malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        double s = sin(M_PI * k / (2.0 * (K - 1)));
        omxk[k] = 2.0 * s * s;
        lam[k] = (k % 2 == 0) ? 1.0 : -1.0;
    }
    lam[0] *= 0.5;
    lam[K - 1] *= 0.5;
    memset(df, 0, sizeof(double) * (size_t)B * K);
    #pragma omp parallel
    {
        double *t = (double *)malloc(sizeof(double) * K);
        double *acc = (double *)calloc((size_t)B * K, sizeof(double));
        #pragma omp for schedule(dynamic, 8)
        for (int i = 0; i < npts; ++i) {
            int hit = -1;
            double den = 0.0;
            for (int k = 0; k < K; ++k) {
                double d = omxk[k] - omx[i];
                if (d == 0.0) { hit = k; break; }
                t[k] = lam[k] / d;
                den += t[k];
            }
            for (int b = 0; b < B; ++b) {
                double ui = u[(size_t)b * npts + i];
                double *ab = acc + (size_t)b * K;
                if (hit >= 0) {
                    ab[hit] += ui;
                } else {
                    for (int k = 0; k < K; ++k) ab[k] += (t[k] / den) * ui;
                }
            }
        }
        #pragma omp critical
        {
            for (size_t e = 0; e < (size_t)B * K; ++e) df[e] += acc[e];
        }
        free(acc);
        free(t);
    }
    free(omxk);
    free(lam);
}
