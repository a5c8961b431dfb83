"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Every check compares the oracle with something other than itself: values
printed in the paper (Table 1), closed forms (Eq. 2.2, Eq. 2.15, e^{ax}, the
Dirichlet-Murphy pair behind Eq. 2.6), identities (Parseval, the sine form
Eq. 2.13, the symmetry Eq. 2.12), library routines (numpy/scipy) on special
cases, and 30-digit mpmath quadrature.  Chosen so that a dropped term, a
wrong sign or index, or a transposed operand in either route fails one.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sp
from numpy.polynomial.chebyshev import chebval
from numpy.polynomial.legendre import leggauss

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- building blocks
def test_gauss_legendre_matches_library_small(oracle):
    for n in (1, 2, 3, 7, 16, 33):
        x, w = oracle.gauss_legendre(n)
        X, W = leggauss(n)
        assert np.allclose(x, X, atol=1e-15, rtol=0)
        assert np.allclose(w, W, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [5, 64, 513, 2049])
def test_gauss_legendre_polynomial_exactness(oracle, n):
    x, w = oracle.gauss_legendre(n)
    assert np.all(np.diff(x) > 0)
    for p in sorted({0, 1, 2, min(10, 2 * n - 2), 2 * n - 2, 2 * n - 1}):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * x ** p) - exact) < 2e-15 * max(1, n / 100)


@pytest.mark.parametrize("sym", [True, False])
def test_tau_rule_integrates_even_polynomials(oracle, sym):
    Q = 9
    tau, w, omt2 = oracle.tau_rule(Q, sym)
    assert np.all((tau > 0) & (tau < 1))
    assert np.allclose(omt2, 1 - tau ** 2, atol=1e-15)
    # symmetric rule: exact to degree 4Q-1 in tau for even integrands;
    # literal rule: exact to degree 2Q-1
    top = 4 * Q - 2 if sym else 2 * Q - 2
    for p in range(0, top + 1, 2):
        assert abs(np.sum(w * tau ** p) - 1.0 / (p + 1)) < 1e-15


def test_legendre_table_matches_scipy(oracle):
    x = np.linspace(-1, 1, 37)
    P = oracle.legendre_table(40, x)
    for n in (0, 1, 2, 5, 39):
        assert np.allclose(P[n], sp.eval_legendre(n, x), atol=1e-13)


def test_barycentric_reproduces_polynomials_and_nodes(oracle):
    rng = np.random.default_rng(3)
    K = 65
    coef = rng.standard_normal((2, K)) * 0.9 ** np.arange(K)
    xk, omxk = oracle.cl_nodes(K)
    fk = np.stack([chebval(xk, c) for c in coef])
    xe = np.concatenate([rng.uniform(-1, 1, 50), [1.0, -1.0, xk[7]]])
    out = oracle.cl_barycentric(fk, 1.0 - xe)
    ref = np.stack([chebval(xe, c) for c in coef])
    assert np.allclose(out, ref, atol=1e-13)
    # exact node hit returns the sample itself
    assert out[0, -1] == fk[0, 7] and out[1, -3] == fk[1, 0]
    assert np.allclose(omxk, 1 - xk, atol=1e-16)


# ---------------------------------------------------------------- route 1 (Eq. 2.3)
def test_route1_generating_function(oracle):
    # Eq. 2.2: sum P_n t^n = (1 - 2xt + t^2)^(-1/2)  =>  c_n = t^n
    for t in (0.5, -0.7, 0.9):
        c = oracle.coeffs_direct(60, 400, f=lambda x: (1 - 2 * x * t + t * t) ** -0.5)[0]
        assert np.max(np.abs(c - t ** np.arange(60))) < 1e-13


def test_route1_legendre_polynomial_gives_delta(oracle):
    for m in (0, 1, 7, 30):
        c = oracle.coeffs_direct(40, 64, f=lambda x: sp.eval_legendre(m, x))[0]
        e = np.zeros(40)
        e[m] = 1.0
        assert np.max(np.abs(c - e)) < 1e-13


def test_route1_exponential(oracle):
    # int_{-1}^{1} e^{ax} P_n dx = 2 i_n(a)  =>  c_n = (2n+1) i_n(a)
    for a in (-3.0, 0.5, 20.0):
        N = 60
        c = oracle.coeffs_direct(N, 300, f=lambda x: np.exp(a * x))[0]
        n = np.arange(N)
        ref = (2 * n + 1) * sp.spherical_in(n, a)
        assert np.max(np.abs(c - ref)) < 1e-13 * np.max(np.abs(ref))


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_abs_x_3_2.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, t, c = line.split()
                rows.append((int(n), t, c))
    return rows


def _eq_2_15(n, alpha=Fraction(3, 2)):
    """Closed form Eq. 2.15 for |x|^alpha, as an exact rational."""
    if n % 2:
        return Fraction(0)
    if n == 0:
        return 1 / (alpha + 1)
    num = Fraction(2 * n + 1)
    for i in range(n // 2):
        num *= alpha - 2 * i
    den = Fraction(1)
    for i in range(n // 2 + 1):
        den *= alpha + 1 + 2 * i
    return num / den


def test_table1_true_column_is_eq_2_15():
    for n, true_s, _ in _table1():
        assert abs(float(_eq_2_15(n)) - float(true_s)) < 1e-19 + 1e-16 * abs(float(true_s))


def test_route1_reproduces_table1_true_column(oracle):
    # |x|^{3/2}: split at 0 and substitute x = w^2, so the integrand is a
    # polynomial in w and Gauss-Legendre on [0,1] is exact.
    N = 32
    nw = N + 4
    t, om = oracle.gauss_legendre(nw)
    w = 0.5 * (t + 1)
    om = 0.5 * om
    x = np.concatenate([w ** 2, -(w ** 2)])
    wts = np.concatenate([2 * w * om, 2 * w * om])
    fv = np.concatenate([w ** 3, w ** 3])
    c = oracle.coeffs_quadrature(N, x, wts, fv)[0]
    for n, true_s, _ in _table1():
        assert abs(c[n] - float(true_s)) < 2e-14
    assert np.max(np.abs(c[1::2])) < 1e-15


def test_route1_against_mpmath_bruteforce(oracle):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    gam = 0.5   # rational test family (1+x)/(gamma^2+x^2), Sec. 2 last paragraph
    f = lambda x: (1 + x) / (gam * gam + x * x)
    N = 12
    c = oracle.coeffs_direct(N, 600, f=f)[0]
    for n in range(N):
        ref = (n + mpmath.mpf(1) / 2) * mpmath.quad(
            lambda x: (1 + x) / (mpmath.mpf(gam) ** 2 + x * x) * mpmath.legendre(n, x), [-1, 0, 1])
        assert abs(c[n] - float(ref)) < 1e-12


# ---------------------------------------------------------------- route 2 (Thm 1)
@pytest.mark.parametrize("sym", [True, False])
def test_route2_plain_method_generating_function(oracle, sym):
    # plain method, N=64, M=256, Q=32, t=0.5 must give c_n = 0.5^n to 1e-12
    cfg = workloads.CONFIGS["genfn_plain_n64"]
    t = cfg["t"]
    cr, ci = oracle.coeffs_abel(cfg["N"], cfg["M"], cfg["Q"], sym=sym,
                                f=lambda omx: (1 - 2 * (1 - omx) * t + t * t) ** -0.5,
                                return_imag=True)
    assert np.max(np.abs(cr[0] - t ** np.arange(cfg["N"]))) < 1e-12
    assert np.max(np.abs(ci)) < 1e-12


def test_route2_abel_step_of_legendre_polynomial(oracle):
    # For f = P_m the Abel integral has the closed form (Dirichlet-Murphy pair
    # behind Eq. 2.6): phi(y) = 2 sin((m + 1/2)|y|) / (2m + 1).
    M = 128
    for m in (0, 1, 5, 20):
        Q = m // 2 + 2
        omx, wq = oracle.abel_points(M, Q, True)
        fq = sp.eval_legendre(m, 1 - omx)[None]
        phi = oracle.abel_phi(fq, wq)[0]
        y = -np.pi + 2 * np.pi * np.arange(M) / M
        ref = 2 * np.sin((m + 0.5) * np.abs(y)) / (2 * m + 1)
        assert np.max(np.abs(phi - ref)) < 1e-14


def test_route2_legendre_polynomial_gives_delta(oracle):
    N, M = 24, 128
    for m in (0, 3, 23):
        cr, ci = oracle.coeffs_abel(N, M, 16, f=lambda omx: sp.eval_legendre(m, 1 - omx),
                                    return_imag=True)
        e = np.zeros(N)
        e[m] = 1.0
        assert np.max(np.abs(cr[0] - e)) < 1e-13
        assert np.max(np.abs(ci)) < 1e-13


def test_route2_sine_form_eq_2_13(oracle):
    # c_n = (2/pi)(n+1/2) int_0^pi phi(y) sin((n+1/2) y) dy, trapezoid on the
    # same grid, must equal the Eq. 2.4/2.5 route (symmetry Eq. 2.12).
    N, M, Q = 40, 256, 24
    rng = np.random.default_rng(7)
    K = 33
    coef = rng.standard_normal(K) * 0.8 ** np.arange(K)
    xk, _ = oracle.cl_nodes(K)
    fk = chebval(xk, coef)[None]
    omx, wq = oracle.abel_points(M, Q, True)
    fq = oracle.cl_barycentric(fk, omx.ravel()).reshape(1, M, Q)
    phi = oracle.abel_phi(fq, wq)[0]
    cr = oracle.abel_coeffs(N, phi[None])[0][0]
    y = -np.pi + 2 * np.pi * np.arange(M) / M
    pos = np.arange(M // 2, M)           # y in [0, pi)
    yy = np.concatenate([y[pos], [np.pi]])
    ph = np.concatenate([phi[pos], [phi[0]]])   # phi(pi) = phi(-pi)
    wt = np.full(yy.size, 2 * np.pi / M)
    wt[0] *= 0.5
    wt[-1] *= 0.5
    n = np.arange(N)
    sine = (2 / np.pi) * (n + 0.5) * (np.sin(np.outer(n + 0.5, yy)) @ (wt * ph))
    assert np.max(np.abs(sine - cr)) < 1e-13


def test_route2_symmetry_eq_2_12_phi_even(oracle):
    # phi(-y) = phi(y) on the grid, the real form of fhat(y) = -e^{iy} fhat(-y)
    M, Q = 64, 8
    omx, wq = oracle.abel_points(M, Q, True)
    fq = np.exp(0.7 * (1 - omx))[None]
    phi = oracle.abel_phi(fq, wq)[0]
    j = np.arange(1, M)
    assert np.max(np.abs(phi[j] - phi[M - j])) < 1e-15


def test_route2_exact_for_polynomials_equals_route1(oracle):
    # degree d = K-1 polynomial, M > N + d, exact tau rule: discretisation
    # error vanishes and both routes agree to rounding.
    rng = np.random.default_rng(11)
    K, N, M = 65, 48, 128
    coef = rng.standard_normal((3, K)) * 0.95 ** np.arange(K)
    xk, _ = oracle.cl_nodes(K)
    fk = np.stack([chebval(xk, c) for c in coef])
    c2, ci = oracle.coeffs_abel(N, M, oracle.exact_tau_points(K), f_cl=fk, return_imag=True)
    c1 = oracle.coeffs_direct(N, (K + N) // 2 + 2, f_cl=fk)
    assert np.max(np.abs(c2 - c1)) < 1e-13 * np.max(np.abs(c1))
    assert np.max(np.abs(ci)) < 1e-13 * np.max(np.abs(c1))
    # and route 1 on the interpolant equals the closed-form Chebyshev series
    c1b = oracle.coeffs_direct(N, 80, f=lambda x: np.stack([chebval(x, c) for c in coef]))
    assert np.max(np.abs(c1 - c1b)) < 1e-13 * np.max(np.abs(c1))


def test_route2_parseval(oracle):
    # int f^2 = sum 2 c_n^2 / (2n+1) for a polynomial of degree < N
    rng = np.random.default_rng(5)
    K, N, M = 33, 40, 128
    coef = rng.standard_normal(K) * 0.9 ** np.arange(K)
    xk, _ = oracle.cl_nodes(K)
    c = oracle.coeffs_abel(N, M, oracle.exact_tau_points(K), f_cl=chebval(xk, coef)[None])[0]
    X, W = leggauss(100)
    lhs = np.sum(W * chebval(X, coef) ** 2)
    rhs = np.sum(2 * c ** 2 / (2 * np.arange(N) + 1))
    assert abs(lhs - rhs) < 1e-12 * lhs


def test_route2_exponential_and_mpmath(oracle):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    N, M, Q = 14, 256, 40
    a = 2.5
    c = oracle.coeffs_abel(N, M, Q, f=lambda omx: np.exp(a * (1 - omx)))[0]
    for n in range(N):
        ref = (n + mpmath.mpf(1) / 2) * mpmath.quad(lambda x: mpmath.exp(a * x) * mpmath.legendre(n, x), [-1, 1])
        assert abs(c[n] - float(ref)) < 1e-13


def test_route2_table1_converges(oracle):
    # |x|^{3/2} has a kink at 0: route 2 converges algebraically in Q; at
    # M=1024, Q=512 it is within 1e-6 of the true column of Table 1 (the
    # paper's own M, Q are not stated, so its "computed" column is not pinned).
    rows = _table1()
    c = oracle.coeffs_abel(32, 1024, 512, f=lambda omx: np.abs(1 - omx) ** 1.5)[0]
    err = max(abs(c[n] - float(t)) for n, t, _ in rows)
    assert err < 1e-6


# ---------------------------------------------------------------- explicit operators
def test_explicit_operators_reproduce_route2(oracle):
    rng = np.random.default_rng(2)
    K, N, M, Q = 17, 12, 32, 9
    A = oracle.abel_operator(M, K, Q, True)
    R = oracle.twisted_dft_matrix(N, M)
    f = rng.standard_normal((4, K))
    c = oracle.coeffs_abel(N, M, Q, f_cl=f)
    assert np.max(np.abs(f @ (R @ A).T - c)) < 1e-13
    # columns of A applied to Legendre samples reproduce the D4 closed form
    xk, _ = oracle.cl_nodes(K)
    m = 6
    phi = A @ sp.eval_legendre(m, xk)
    y = -np.pi + 2 * np.pi * np.arange(M) / M
    assert np.max(np.abs(phi - 2 * np.sin((m + 0.5) * np.abs(y)) / (2 * m + 1))) < 1e-14


# ---------------------------------------------------------------- route 3 (Eq. 2.13)
@pytest.mark.parametrize("sym", [True, False])
def test_route3_plain_method_generating_function(oracle, sym):
    # the sine form of Eq. 2.13 on [0, pi]: c_n = 0.5^n to 1e-12 at the plain
    # method's sizes (Eq. 2.2)
    cfg = workloads.CONFIGS["genfn_plain_n64"]
    t = cfg["t"]
    c = oracle.coeffs_sine(cfg["N"], cfg["M"], cfg["Q"], sym=sym,
                           f=lambda omx: (1 - 2 * (1 - omx) * t + t * t) ** -0.5)[0]
    assert np.max(np.abs(c - t ** np.arange(cfg["N"]))) < 1e-12


def test_route3_phi_of_legendre_polynomial(oracle):
    # Eq. 2.14 for f = P_m on [0, pi]: phi(y) = 2 sin((m + 1/2) y) / (2m + 1)
    L = 64
    for m in (0, 2, 9, 31):
        Q = m // 2 + 2
        omx, wq = oracle.sine_points(L, Q, True)
        phi = oracle.sine_phi(sp.eval_legendre(m, 1 - omx)[None], wq)[0]
        y = np.pi * np.arange(L + 1) / L
        assert np.max(np.abs(phi - 2 * np.sin((m + 0.5) * y) / (2 * m + 1))) < 1e-14


def test_route3_legendre_polynomial_gives_delta(oracle):
    N, M = 24, 128
    for m in (0, 5, 23):
        c = oracle.coeffs_sine(N, M, 16, f=lambda omx: sp.eval_legendre(m, 1 - omx))[0]
        e = np.zeros(N)
        e[m] = 1.0
        assert np.max(np.abs(c - e)) < 1e-13


def test_route3_exponential(oracle):
    # c_n = (2n+1) i_n(a) for e^{ax}
    N, M, Q = 40, 256, 40
    for a in (-4.0, 1.5):
        c = oracle.coeffs_sine(N, M, Q, f=lambda omx: np.exp(a * (1 - omx)))[0]
        n = np.arange(N)
        ref = (2 * n + 1) * sp.spherical_in(n, a)
        assert np.max(np.abs(c - ref)) < 1e-13 * np.max(np.abs(ref))


def test_route3_equals_route2_on_sampled_inputs(oracle):
    # the half-range sine form and the full-range Fourier sum are the same
    # discrete map (symmetry Eq. 2.12 on the grid): route 3 = route 2 to
    # rounding on random series at non-exact (M, Q)
    rng = np.random.default_rng(17)
    K, N, M, Q = 97, 60, 256, 20
    coef = rng.standard_normal((3, K)) * 0.93 ** np.arange(K)
    xk, _ = oracle.cl_nodes(K)
    fk = np.stack([chebval(xk, c) for c in coef])
    c2 = oracle.coeffs_abel(N, M, Q, f_cl=fk)
    c3 = oracle.coeffs_sine(N, M, Q, f_cl=fk)
    assert np.max(np.abs(c3 - c2)) < 1e-13 * np.max(np.abs(c2))


def test_route3_table1_converges(oracle):
    # |x|^{3/2}: at M = 1024, Q = 512 within 1e-6 of Table 1's true column
    rows = _table1()
    c = oracle.coeffs_sine(32, 1024, 512, f=lambda omx: np.abs(1 - omx) ** 1.5)[0]
    assert max(abs(c[n] - float(t)) for n, t, _ in rows) < 1e-6
    assert np.max(np.abs(c[1::2])) < 1e-6


# ---------------------------------------------------------------- route 1 transposed
def test_adjoint_direct_dot_product_identity(oracle):
    # <L f, v> = <f, L^T v> with L f from route 1 (Eq. 2.3) on CL samples
    rng = np.random.default_rng(21)
    for K, N, Qo in ((9, 5, 12), (65, 48, 60), (129, 100, 120)):
        f = rng.standard_normal((3, K))
        v = rng.standard_normal((3, N))
        c = oracle.coeffs_direct(N, Qo, f_cl=f)
        df = oracle.adjoint_direct(Qo, K, v)
        lhs = np.sum(c * v, axis=1)
        rhs = np.sum(f * df, axis=1)
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(c) @ np.abs(v).T)


def test_adjoint_direct_equals_explicit_route2_transpose(oracle):
    # exact configuration (M > N + K - 1, exact tau rule): the explicit route-2
    # operators give the same map, so (R A)^T v equals route 1 transposed
    rng = np.random.default_rng(22)
    K, N, M = 17, 12, 32
    Q = oracle.exact_tau_points(K)
    A = oracle.abel_operator(M, K, Q, True)
    R = oracle.twisted_dft_matrix(N, M)
    v = rng.standard_normal((4, N))
    ref = v @ (R @ A)
    df = oracle.adjoint_direct((K + N) // 2 + 2, K, v)
    assert np.max(np.abs(df - ref)) < 1e-12 * np.max(np.abs(ref))
