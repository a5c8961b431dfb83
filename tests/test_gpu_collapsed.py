"""Collapsed plans (LEG_FLAG_COLLAPSED): c = L f with L = R A multiplied out
at plan time, one GEMM per forward and one transposed GEMM per backward.

The map is the same as Theorem 1's (Eq. 2.4 with the twist of Eq. 2.5 and the
Abel operator of the quadrature after Eq. 2.14), so the oracle is the same:
route 2 for the forward, the oracle's explicit R A for the operator and its
transpose.  Tolerances as for the uncollapsed paths (FP64 1e-11, split-FP16
1e-6, FP32 3e-4).
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def leg():
    import paper_1106_0463_gb300 as leg
    assert torch.cuda.is_available()
    return leg


def relerr(c, ref):
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    ref = np.atleast_2d(ref)
    return float(np.max(np.max(np.abs(c - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def forward(leg, plan, f_np):
    f = torch.from_numpy(f_np.astype(np.float64 if plan.dtype == leg.F64 else np.float32)).cuda()
    c = plan.forward(f)
    plan.status()
    return c.double().cpu().numpy()


# B, K, N, M: one tile with ragged edges; several row tiles (N > 256) and
# function tiles with a ragged tail; K not a multiple of the 64-wide padding
SIZES = [(37, 97, 40, 128), (300, 257, 300, 1024), (129, 1025, 512, 2048)]


@pytest.mark.parametrize("B,K,N,M", SIZES)
@pytest.mark.parametrize("dt,tol", [(3, 1e-6), (0, 1e-11), (1, 3e-4), (2, 5e-2)])
def test_collapsed_forward_matches_oracle(leg, oracle, B, K, N, M, dt, tol):
    Q = oracle.exact_tau_points(K)
    f32, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(B + K))
    plan = leg.Plan(N, M, K, 0, dt, flags=leg.FLAG_COLLAPSED)
    c = forward(leg, plan, f32)
    ref = oracle.coeffs_abel(N, M, Q, f_cl=f32.astype(np.float64))
    assert relerr(c, ref) < tol


def test_collapsed_equals_uncollapsed(leg):
    B, K, N, M = 64, 257, 128, 512
    f32, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(5))
    a = forward(leg, leg.Plan(N, M, K, 0, leg.SPLIT_FP16), f32)
    b = forward(leg, leg.Plan(N, M, K, 0, leg.SPLIT_FP16, flags=leg.FLAG_COLLAPSED), f32)
    assert relerr(b, a) < 5e-7


def test_collapsed_operator_is_r_times_a(leg, oracle):
    """Applying the FP64 collapsed plan to the unit vectors e_k gives column k
    of L; the oracle's explicit R A (route-2 grid) must agree to rounding."""
    N, M, K, Q = 24, 64, 33, 9
    plan = leg.Plan(N, M, K, Q, leg.F64, flags=leg.FLAG_COLLAPSED)
    eye = np.eye(K)
    Lt = forward(leg, plan, eye)                     # row k = column k of L
    L = oracle.twisted_dft_matrix(N, M) @ oracle.abel_operator(M, K, Q, True)
    assert np.max(np.abs(Lt.T - L)) < 1e-12 * np.max(np.abs(L))


@pytest.mark.parametrize("dt,tol", [(3, 1e-6), (0, 1e-12), (1, 1e-5)])
def test_collapsed_backward_is_the_transpose(leg, oracle, dt, tol):
    N, M, K, Q, B = 40, 128, 97, 20, 11
    plan = leg.Plan(N, M, K, Q, dt, flags=leg.FLAG_COLLAPSED)
    L = oracle.twisted_dft_matrix(N, M) @ oracle.abel_operator(M, K, Q, True)
    v = np.random.default_rng(2).standard_normal((B, N))
    vt = torch.from_numpy(v if dt == 0 else v.astype(np.float32)).cuda()
    df = plan.backward(vt)
    plan.status()
    ref = (v if dt == 0 else v.astype(np.float32).astype(np.float64)) @ L
    assert relerr(df.double().cpu().numpy(), ref) < tol


def test_collapsed_full_size_sampled(leg, oracle):
    """B=4096, K=1025, N=512, M=2048, the default launch: 16 sampled functions."""
    cfg = workloads.CONFIGS["cheb_b4096_k1025_n512_m2048"]
    B, K, N, M = cfg["B"], cfg["K"], cfg["N"], cfg["M"]
    f32 = workloads.workload_inputs("cheb_b4096_k1025_n512_m2048")
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16, flags=leg.FLAG_COLLAPSED)
    c = forward(leg, plan, f32)
    assert np.isfinite(c).all()
    sample = np.random.default_rng(9).choice(B, 16, replace=False)
    ref = oracle.coeffs_abel(N, M, oracle.exact_tau_points(K), f_cl=f32[sample].astype(np.float64))
    assert relerr(c[sample], ref) < 1e-6


def test_collapsed_plans_are_refused_where_unsupported(leg):
    plan = leg.Plan(40, 128, 97, 0, leg.SPLIT_FP16, flags=leg.FLAG_COLLAPSED)
    f = torch.zeros((3, 97), dtype=torch.float32, device="cuda")
    c = torch.empty((3, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(leg.LegError) as err:
        plan.forward_noalloc(f, c)
    assert err.value.code == 4 and "COLLAPSED" in str(err.value)   # LEG_ERR_UNSUPPORTED
    with pytest.raises(leg.LegError):
        leg.Ragged([plan], np.zeros(1, np.int32), np.array([40]), np.array([0]), np.array([0]))
