"""ctypes front end of the FP64 CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.

Routes (De Micheli & Viano, arXiv:1106.0463):

* :func:`coeffs_direct` -- route 1, the plain definition Eq. 2.3,
  c_n = (n + 1/2) int f P_n, by Gauss-Legendre quadrature.
* :func:`coeffs_abel` -- route 2, the paper's method: the Abel-type transform
  of Eq. 2.5 sampled on y_j = -pi + 2 pi j / M, the singularity removed by
  x = cos y + s^2 and the s-integral taken by Gauss-Legendre (Sec. 2, the
  paragraph after Eq. 2.14), then the Fourier sum of Eq. 2.4 written out
  directly (no FFT).
* :func:`coeffs_sine` -- route 3, the half-range sine form Eq. 2.13 with phi
  of Eq. 2.14 on y_j = pi j / L, j = 0..L (L = M/2), trapezoid rule, the
  sine sum written out directly.
* :func:`adjoint_direct` -- route 1 transposed: df = L^T v for sampled
  inputs, for checks of the adjoint.

Sampled inputs are values at the Chebyshev-Lobatto nodes
x_k = cos(pi k / (K-1)), k = 0..K-1, read through their barycentric
interpolant.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, p = ctypes.c_int, _dp
            sig = {
                "or_gauss_legendre": [i, p, p],
                "or_tau_rule": [i, i, p, p, p],
                "or_legendre_table": [i, i, p, p],
                "or_coeffs_quadrature": [i, i, p, p, i, p, p],
                "or_cl_barycentric": [i, i, p, i, p, p],
                "or_abel_points": [i, i, i, p, p],
                "or_abel_phi": [i, i, i, p, p, p],
                "or_abel_coeffs": [i, i, i, p, p, p],
                "or_abel_operator": [i, i, i, i, p],
                "or_twisted_dft_matrix": [i, i, p],
                "or_sine_points": [i, i, i, p, p],
                "or_sine_phi": [i, i, i, p, p, p],
                "or_sine_coeffs": [i, i, i, p, p],
                "or_coeffs_quadrature_T": [i, i, p, p, i, p, p],
                "or_cl_barycentric_T": [i, i, p, i, p, p],
            }
            for name, argt in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = argt
                fn.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Building blocks
# --------------------------------------------------------------------------
def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (nodes ascending, weights)."""
    x = np.empty(n)
    w = np.empty(n)
    _load().or_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def tau_rule(Q: int, sym: bool = True):
    """Rule for int_0^1 h(tau) dtau on the Abel integral (Sec. 2 after Eq. 2.14).

    sym=True: nonnegative half of a 2Q-point Gauss-Legendre rule (the
    integrand is even in s); sym=False: Q-point rule mapped onto [0, 1].
    Returns (tau, w, 1 - tau^2).
    """
    tau = np.empty(Q)
    w = np.empty(Q)
    omt2 = np.empty(Q)
    _load().or_tau_rule(Q, int(bool(sym)), _ptr(tau), _ptr(w), _ptr(omt2))
    return tau, w, omt2


def legendre_table(N: int, x) -> np.ndarray:
    """P_n(x_i) for n < N by the three-term recurrence; shape (N, len(x))."""
    x = _f64(x)
    P = np.empty((N, x.size))
    _load().or_legendre_table(N, x.size, _ptr(x), _ptr(P))
    return P


def coeffs_quadrature(N: int, x, wts, fvals) -> np.ndarray:
    """Eq. 2.3 on a given rule: c_n = (n + 1/2) sum_i wts_i f_i P_n(x_i)."""
    x, wts = _f64(x), _f64(wts)
    fvals = _f64(np.atleast_2d(fvals))
    B = fvals.shape[0]
    c = np.empty((B, N))
    _load().or_coeffs_quadrature(N, x.size, _ptr(x), _ptr(wts), B, _ptr(fvals), _ptr(c))
    return c


def cl_nodes(K: int):
    """Chebyshev-Lobatto nodes x_k = cos(pi k/(K-1)) and 1 - x_k = 2 sin^2(pi k/(2(K-1)))."""
    k = np.arange(K)
    return np.cos(np.pi * k / (K - 1)), 2.0 * np.sin(np.pi * k / (2.0 * (K - 1))) ** 2


def cl_barycentric(f_cl, omx) -> np.ndarray:
    """Barycentric interpolant of CL samples f_cl (B x K) at points given by 1 - x."""
    f_cl = _f64(np.atleast_2d(f_cl))
    omx = _f64(omx).ravel()
    B, K = f_cl.shape
    out = np.empty((B, omx.size))
    _load().or_cl_barycentric(K, B, _ptr(f_cl), omx.size, _ptr(omx), _ptr(out))
    return out


def abel_points(M: int, Q: int, sym: bool = True):
    """1 - x_jq = 2 sin^2(y_j/2)(1 - tau_q^2) on y_j = -pi + 2 pi j/M; shape (M, Q); and w_q."""
    omx = np.empty((M, Q))
    wq = np.empty(Q)
    _load().or_abel_points(M, Q, int(bool(sym)), _ptr(omx), _ptr(wq))
    return omx, wq


def abel_phi(fq, wq) -> np.ndarray:
    """phi(y_j) = 2|sin(y_j/2)| sum_q w_q f(x_jq)  (Eq. 2.14 after substitution); fq: (B, M, Q)."""
    fq = _f64(fq)
    B, M, Q = fq.shape
    phi = np.empty((B, M))
    _load().or_abel_phi(M, Q, B, _ptr(fq), _ptr(_f64(wq)), _ptr(phi))
    return phi


def abel_coeffs(N: int, phi):
    """Eq. 2.5 twist and Eq. 2.4 Fourier sum, direct: returns (Re c_n, Im c_n), shape (B, N)."""
    phi = _f64(np.atleast_2d(phi))
    B, M = phi.shape
    cr = np.empty((B, N))
    ci = np.empty((B, N))
    _load().or_abel_coeffs(N, M, B, _ptr(phi), _ptr(cr), _ptr(ci))
    return cr, ci


# --------------------------------------------------------------------------
# Routes
# --------------------------------------------------------------------------
def coeffs_direct(N: int, Qo: int, *, f=None, f_cl=None) -> np.ndarray:
    """Route 1 (Eq. 2.3) with a Qo-point Gauss-Legendre rule.

    Either ``f`` (a vectorised closed form of x, returning an array (B, npts)
    or (npts,)) or ``f_cl`` (B x K samples at CL nodes, read through the
    barycentric interpolant) gives the function values.
    """
    x, w = gauss_legendre(Qo)
    if f_cl is not None:
        fv = cl_barycentric(f_cl, 1.0 - x)
    else:
        fv = np.atleast_2d(f(x))
    return coeffs_quadrature(N, x, w, fv)


def abel_g_points(M: int, Q: int, sym: bool = True):
    """Quadrature points of route 2 (1 - x_jq) and weights."""
    return abel_points(M, Q, sym)


def coeffs_abel(N: int, M: int, Q: int, *, sym: bool = True, f=None, f_cl=None,
                return_imag: bool = False):
    """Route 2: the paper's method with a direct Fourier sum (Eqs. 2.4, 2.5, 2.14).

    ``f`` is a closed form evaluated at the quadrature points (the plain
    method), given as a function of (1 - x) through ``f(omx)``; ``f_cl`` are
    CL samples read through the barycentric interpolant.
    """
    omx, wq = abel_points(M, Q, sym)
    if f_cl is not None:
        f_cl = np.atleast_2d(f_cl)
        fq = cl_barycentric(f_cl, omx.ravel()).reshape(f_cl.shape[0], M, Q)
    else:
        fq = np.asarray(f(omx), dtype=np.float64)
        fq = fq.reshape(-1, M, Q)
    phi = abel_phi(fq, wq)
    cr, ci = abel_coeffs(N, phi)
    return (cr, ci) if return_imag else cr


def abel_operator(M: int, K: int, Q: int, sym: bool = True) -> np.ndarray:
    """Explicit A_phi (M x K): phi = A_phi f for CL samples f (route 2 grid)."""
    A = np.empty((M, K))
    _load().or_abel_operator(M, K, Q, int(bool(sym)), _ptr(A))
    return A


def twisted_dft_matrix(N: int, M: int) -> np.ndarray:
    """Explicit R (N x M): Re c = R phi (Eq. 2.5 twist + Eq. 2.4 sum)."""
    R = np.empty((N, M))
    _load().or_twisted_dft_matrix(N, M, _ptr(R))
    return R


def sine_points(L: int, Q: int, sym: bool = True):
    """1 - x_jq = 2 sin^2(y_j/2)(1 - tau_q^2) on y_j = pi j / L, j = 0..L; shape (L+1, Q); and w_q."""
    omx = np.empty((L + 1, Q))
    wq = np.empty(Q)
    _load().or_sine_points(L, Q, int(bool(sym)), _ptr(omx), _ptr(wq))
    return omx, wq


def sine_phi(fq, wq) -> np.ndarray:
    """phi(y_j) = 2 sin(y_j/2) sum_q w_q f(x_jq) on [0, pi] (Eq. 2.14); fq: (B, L+1, Q)."""
    fq = _f64(fq)
    B, L1, Q = fq.shape
    phi = np.empty((B, L1))
    _load().or_sine_phi(L1 - 1, Q, B, _ptr(fq), _ptr(_f64(wq)), _ptr(phi))
    return phi


def sine_coeffs(N: int, phi) -> np.ndarray:
    """Eq. 2.13 by the trapezoid rule on y_j = pi j / L, direct sine sum; phi: (B, L+1)."""
    phi = _f64(np.atleast_2d(phi))
    B, L1 = phi.shape
    c = np.empty((B, N))
    _load().or_sine_coeffs(N, L1 - 1, B, _ptr(phi), _ptr(c))
    return c


def coeffs_sine(N: int, M: int, Q: int, *, sym: bool = True, f=None, f_cl=None) -> np.ndarray:
    """Route 3: the half-range sine form (Eqs. 2.13, 2.14) on L = M/2 intervals of [0, pi].

    ``f`` is a closed form of (1 - x) evaluated at the quadrature points (the
    plain method); ``f_cl`` are CL samples read through the barycentric
    interpolant."""
    L = M // 2
    omx, wq = sine_points(L, Q, sym)
    if f_cl is not None:
        f_cl = np.atleast_2d(f_cl)
        fq = cl_barycentric(f_cl, omx.ravel()).reshape(f_cl.shape[0], L + 1, Q)
    else:
        fq = np.asarray(f(omx), dtype=np.float64).reshape(-1, L + 1, Q)
    return sine_coeffs(N, sine_phi(fq, wq))


def adjoint_direct(Qo: int, K: int, v) -> np.ndarray:
    """df = L^T v for the route-1 map on K CL samples with a Qo-point Gauss rule:
    u_i = w_i sum_n (n + 1/2) v_n P_n(x_i), then df_k = sum_i l_k(x_i) u_i.
    v: (B, N); returns (B, K)."""
    v = _f64(np.atleast_2d(v))
    B, N = v.shape
    x, w = gauss_legendre(Qo)
    u = np.empty((B, Qo))
    _load().or_coeffs_quadrature_T(N, Qo, _ptr(x), _ptr(w), B, _ptr(v), _ptr(u))
    omx = _f64(1.0 - x)
    df = np.empty((B, K))
    _load().or_cl_barycentric_T(K, B, _ptr(u), Qo, _ptr(omx), _ptr(df))
    return df


def exact_tau_points(K: int) -> int:
    """Distinct tau nodes of the symmetric rule that integrates the degree-(K-1)
    interpolant exactly: the integrand is a polynomial of degree 2(K-1) in tau,
    and a 2Q-point rule is exact to degree 4Q-1, so Q = ceil(K/2)."""
    return (K + 1) // 2
