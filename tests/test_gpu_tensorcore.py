"""Parity of the tensor-core (tcgen05) paths with the FP64 CPU oracle.

LEG_SPLIT_FP16 must stay within 1e-6 of the oracle (relative to max|c| per
function); LEG_BF16 is a single BF16 product and is held to 5e-2.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

SMALL = [
    (40, 128, 97, 0, 37),
    (64, 256, 129, 20, 130),
    (31, 64, 33, 5, 3),
    (4, 8, 2, 1, 5),
    (128, 256, 65, 0, 1),
    (200, 512, 300, 0, 260),   # three function tiles, ragged rows/K
    (8192, 32768, 65, 0, 3),   # largest grid (M = 32768)
]


@pytest.fixture(scope="module")
def leg():
    import paper_1106_0463_gb300 as leg
    assert torch.cuda.is_available()
    return leg


def relerr(c, ref):
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    ref = np.atleast_2d(ref)
    return float(np.max(np.max(np.abs(c - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def cheb_inputs(B, K, rho=(0.8, 0.99), seed=0):
    f32, _, _ = workloads.random_chebyshev(B, K, rho, np.random.default_rng(seed))
    return f32


@pytest.mark.parametrize("N,M,K,Q,B", SMALL)
def test_split_forward_matches_route2(leg, oracle, N, M, K, Q, B):
    plan = leg.Plan(N, M, K, Q, leg.SPLIT_FP16)
    f = cheb_inputs(B, K, seed=N + K)
    c = plan.forward(torch.from_numpy(f).cuda())
    plan.status()
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f.astype(np.float64))
    assert relerr(c.double().cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("N,M,K,Q,B", SMALL[:3])
def test_bf16_forward_matches_route2(leg, oracle, N, M, K, Q, B):
    plan = leg.Plan(N, M, K, Q, leg.BF16)
    f = cheb_inputs(B, K, seed=N + K)
    c = plan.forward(torch.from_numpy(f).cuda())
    plan.status()
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f.astype(np.float64))
    assert relerr(c.double().cpu().numpy(), ref) < 5e-2


def test_split_backward_is_the_transpose(leg, oracle):
    N, M, K, Q, B = 24, 64, 33, 9, 5
    plan = leg.Plan(N, M, K, Q, leg.SPLIT_FP16)
    L = oracle.twisted_dft_matrix(N, M) @ oracle.abel_operator(M, K, Q, True)
    v = np.random.default_rng(1).standard_normal((B, N)).astype(np.float32)
    df = plan.backward(torch.from_numpy(v).cuda())
    plan.status()
    assert relerr(df.double().cpu().numpy(), v.astype(np.float64) @ L) < 1e-6


@pytest.mark.parametrize("dt,tol", [(3, 1e-6), (0, 1e-11)])
def test_largest_k_polynomial_input_is_exact(leg, oracle, dt, tol):
    """K = 16385 samples (513 K blocks of the GEMM) of polynomials of degree
    1000 with M > N + degree and the exact tau rule: the method has no
    discretisation error, so the GPU meets the plain definition (route 1)."""
    N, M, K, B, deg = 512, 2048, 16385, 5, 1000
    rng = np.random.default_rng(11)
    coef = np.zeros((B, K))
    coef[:, :deg + 1] = rng.standard_normal((B, deg + 1)) * 0.995 ** np.arange(deg + 1)
    f = workloads.chebyshev_values(coef)
    plan = leg.Plan(N, M, K, 0, dt)
    io = np.float64 if dt == leg.F64 else np.float32
    fi = f.astype(io)
    c = plan.forward(torch.from_numpy(fi).cuda())
    plan.status()
    ref = oracle.coeffs_direct(N, (deg + N) // 2 + 4, f_cl=fi.astype(np.float64))
    assert relerr(c.double().cpu().numpy(), ref) < tol


def test_degenerate_inputs(leg, oracle):
    """All-zero rows give zero coefficients (no NaN from the zero scale), a
    constant gives c_0 only, and inputs near 1e30 and 1e-30 keep their
    relative accuracy through the per-function power-of-two scales."""
    N, M, K = 40, 128, 97
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    base = cheb_inputs(2, K, seed=5)
    f = np.stack([np.zeros(K), np.full(K, 3.25), base[0] * 1e30, base[1] * 1e-30]).astype(np.float32)
    c = plan.forward(torch.from_numpy(f).cuda()).double().cpu().numpy()
    plan.status()
    assert np.all(np.isfinite(c))
    assert np.all(c[0] == 0.0)
    assert abs(c[1, 0] - 3.25) < 1e-6 * 3.25 and np.max(np.abs(c[1, 1:])) < 1e-6 * 3.25
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f[2:].astype(np.float64))
    assert relerr(c[2:], ref) < 1e-6


@pytest.mark.parametrize("N,M,K,B", [(512, 2048, 2049, 600), (2048, 8192, 1025, 160), (256, 1024, 4097, 1000)])
def test_partial_wave_shapes_match_oracle(leg, oracle, N, M, K, B):
    """Shapes whose GEMM tiles leave the last wave of CTA pairs partly empty
    (and a ragged last function tile): the forward against the oracle, and
    the backward GEMM through <L f, v> = <f, L^T v>."""
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f = cheb_inputs(B, K, seed=B)
    c = plan.forward(torch.from_numpy(f).cuda())
    plan.status()
    sample = np.random.default_rng(B).choice(B, 6, replace=False)
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f[sample].astype(np.float64))
    assert relerr(c.double().cpu().numpy()[sample], ref) < 1e-6
    v = np.random.default_rng(1).standard_normal((B, N)).astype(np.float32)
    df = plan.backward(torch.from_numpy(v).cuda())
    plan.status()
    lhs = np.sum(c.double().cpu().numpy() * v.astype(np.float64), axis=1)      # <L f, v> per function
    rhs = np.sum(f.astype(np.float64) * df.double().cpu().numpy(), axis=1)     # <f, L^T v>
    scale = np.sqrt(np.sum(c.double().cpu().numpy() ** 2, 1) * np.sum(v.astype(np.float64) ** 2, 1))
    assert np.max(np.abs(lhs - rhs) / scale) < 2e-6
