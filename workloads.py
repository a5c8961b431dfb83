"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds input generation only -- none of the method's arithmetic --
so that both the CUDA path and the FP64 oracle can be fed the same data
without sharing code.  The paper's experiments use unnamed test functions
("polynomials, exponential/hyperbolic functions, rational functions", Sec. 2,
last paragraph) and no public dataset; these families stand in for them.

Sampled inputs are values at the Chebyshev-Lobatto nodes
x_k = cos(pi k/(K-1)), k = 0..K-1, computed in FP64 and rounded to FP32.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

SEED_BASE = 1106046300

# Problem sizes of the five workloads (name -> dict).  "rho" is the range of
# the decay rate of the random Chebyshev series.
CONFIGS = {
    "genfn_plain_n64": dict(N=64, M=256, Q=32, t=0.5),
    "cheb_b4096_k1025_n512_m2048": dict(B=4096, K=1025, N=512, M=2048, rho=(0.80, 0.99)),
    "cheb_b256_k8193_n4096_m16384": dict(B=256, K=8193, N=4096, M=16384, rho=(0.95, 0.999)),
    "ragged_10000": dict(count=10000, Nmin=32, Nmax=8192),
    "cheb_b1024_k4097_n2048_m8192": dict(B=1024, K=4097, N=2048, M=8192, rho=(0.80, 0.99)),
}
CONFIG_INDEX = {name: i for i, name in enumerate(CONFIGS)}


def rng_for(name_or_index, salt: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with SEED_BASE + config index (+ salt)."""
    idx = CONFIG_INDEX[name_or_index] if isinstance(name_or_index, str) else int(name_or_index)
    return np.random.Generator(np.random.PCG64(SEED_BASE + idx + 1000 * salt))


def cl_points(K: int) -> np.ndarray:
    return np.cos(np.pi * np.arange(K) / (K - 1))


def chebyshev_values(coef: np.ndarray) -> np.ndarray:
    """Values at the K CL nodes of sum_m coef[..., m] T_m(x), FP64.

    T_m(x_k) = cos(pi m k/(K-1)), so the values are a type-1 DCT of the
    coefficients (interior terms halved for scipy's normalisation).
    """
    coef = np.atleast_2d(np.asarray(coef, dtype=np.float64))
    a = coef.copy()
    a[:, 1:-1] *= 0.5
    return scipy.fft.dct(a, type=1, axis=-1)


def random_chebyshev(B: int, K: int, rho_range, rng: np.random.Generator):
    """B random series sum_{m<K} g_m rho^m T_m(x), g_m ~ N(0,1), rho ~ U(rho_range).

    Returns (f32 values B x K, FP64 coefficients B x K, rho B).
    """
    rho = rng.uniform(rho_range[0], rho_range[1], size=B)
    g = rng.standard_normal((B, K))
    coef = g * rho[:, None] ** np.arange(K)[None, :]
    vals = chebyshev_values(coef)
    return vals.astype(np.float32), coef, rho


def workload_inputs(name: str, B: int | None = None, salt: int = 0):
    """FP32 CL samples of a sampled workload.

    Always draws the whole configured batch, so that the first B rows are the
    same functions whatever B is requested."""
    cfg = CONFIGS[name]
    rng = rng_for(name, salt)
    f32, coef, rho = random_chebyshev(cfg["B"], cfg["K"], cfg["rho"], rng)
    return f32 if B is None else f32[:B]


def loss_weights(N: int, rng: np.random.Generator):
    """Weights w_n ~ U(0,1) and targets c*_n ~ N(0,1) 0.97^n of the quadratic loss."""
    w = rng.uniform(0.0, 1.0, size=N)
    target = rng.standard_normal(N) * 0.97 ** np.arange(N)
    return w, target


def ragged_spec(count: int, rng: np.random.Generator, Nmin: int = 32, Nmax: int = 8192):
    """Per-function family (0 genfn, 1 exp, 2 chebyshev), parameter and N_i.

    N_i is log-uniform in [Nmin, Nmax]; a third of the functions are
    (1 - 2xt + t^2)^(-1/2) with t ~ U(0.1, 0.95), a third exp(a x) with
    a ~ U(-20, 20), a third random decaying Chebyshev series.
    """
    fam = np.arange(count) % 3
    rng.shuffle(fam)
    par = np.where(fam == 0, rng.uniform(0.1, 0.95, count),
                   np.where(fam == 1, rng.uniform(-20.0, 20.0, count),
                            rng.uniform(0.80, 0.99, count)))
    n = np.exp(rng.uniform(np.log(Nmin), np.log(Nmax), count))
    n = np.clip(np.floor(n).astype(np.int64), Nmin, Nmax)
    return fam.astype(np.int32), par, n


def bucket_of(n: int) -> int:
    """Size bucket of a function needing n coefficients: next power of two >= n."""
    return 1 << int(np.ceil(np.log2(max(int(n), 1))))


def bucket_sizes(Nb: int):
    """(N, M, K, Q) of the plan of bucket Nb: M = 4N, K = min(2N, 1024) + 1,
    Q = max(32, N/8) Gauss nodes per y-point."""
    return Nb, 4 * Nb, min(2 * Nb, 1024) + 1, max(32, Nb // 8)


def ragged_layout(fam, par, n, rng: np.random.Generator):
    """Packed layout of a ragged batch.

    Returns a dict with the bucket list (sorted N_b), per-function bucket
    index, K, input/output offsets, and the Chebyshev coefficients (FP64,
    g_m rho^m, g_m ~ N(0,1)) of the functions of that family.
    """
    Nb = np.array([bucket_of(v) for v in n])
    buckets = sorted(set(Nb.tolist()))
    bidx = np.array([buckets.index(v) for v in Nb], dtype=np.int32)
    K = np.array([bucket_sizes(v)[2] for v in Nb], dtype=np.int32)
    in_off = np.concatenate([[0], np.cumsum(K)[:-1]]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    coef_off = np.zeros(len(n), dtype=np.int64)
    coefs = []
    pos = 0
    for i in range(len(n)):
        if fam[i] == 2:
            coef_off[i] = pos
            g = rng.standard_normal(K[i]) * par[i] ** np.arange(K[i])
            coefs.append(g)
            pos += K[i]
    coef = np.concatenate(coefs) if coefs else np.zeros(1)
    return dict(buckets=buckets, bidx=bidx, K=K, in_off=in_off, out_off=out_off, coef_off=coef_off,
                coef=coef, n_in=int(K.sum()), n_out=int(np.sum(n)))


def closed_form_samples(fam: int, par: float, K: int, coef=None) -> np.ndarray:
    """FP64 values of one closed-form function at its K CL nodes (host reference)."""
    k = np.arange(K)
    omx = 2.0 * np.sin(np.pi * k / (2.0 * (K - 1))) ** 2
    x = np.cos(np.pi * k / (K - 1))
    if fam == 0:
        return ((1.0 - par) ** 2 + 2.0 * par * omx) ** -0.5
    if fam == 1:
        return np.exp(par * x)
    return chebyshev_values(coef)[0]
