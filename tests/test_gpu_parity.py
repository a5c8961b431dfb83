"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (max over the batch of max_n |c - c_ref| / max_n |c_ref|):
  LEG_F64         1e-11  (FP64 throughout; rounding only)
  LEG_F32         3e-4   (FP32 GEMM + FP32 FFT: the (2n+1) factor amplifies
                          white FP32 rounding by ~(2N) / sqrt(M))
  LEG_SPLIT_FP16  1e-6   (the split path's target)
  LEG_BF16        5e-2   (one BF16 product; reported, not a precision path)
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 3e-4, 2: 5e-2, 3: 1e-6}


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
    rng = np.random.default_rng(seed)
    f32, _, _ = workloads.random_chebyshev(B, K, rho, rng)
    return f32


def run_forward(leg, plan, f_np):
    f = torch.from_numpy(f_np.astype(np.float64 if plan.dtype == leg.F64 else np.float32)).cuda()
    c = plan.forward(f)
    torch.cuda.synchronize()
    return c.double().cpu().numpy()


# ------------------------------------------------------------------ plain method
def test_plain_method_generating_function(leg, oracle):
    cfg = workloads.CONFIGS["genfn_plain_n64"]
    plan = leg.Plan(cfg["N"], cfg["M"], 2, cfg["Q"], leg.F64)
    t = torch.tensor([cfg["t"], -0.3, 0.9], dtype=torch.float64, device="cuda")
    c = plan.plain_forward(leg.FAMILY_GENFN, t).cpu().numpy()
    n = np.arange(cfg["N"])
    assert np.max(np.abs(c[0] - 0.5 ** n)) < 1e-12
    for i, tv in enumerate(t.cpu().numpy()):
        ref = oracle.coeffs_abel(cfg["N"], cfg["M"], cfg["Q"],
                                 f=lambda omx: (1 - 2 * (1 - omx) * tv + tv * tv) ** -0.5)[0]
        assert np.max(np.abs(c[i] - ref)) < 1e-13


def test_plain_method_exponential(leg, oracle):
    N, M, Q = 48, 256, 24
    plan = leg.Plan(N, M, 2, Q, leg.F64)
    a = np.array([-20.0, -1.5, 0.0, 7.0])
    c = plan.plain_forward(leg.FAMILY_EXP, torch.tensor(a, device="cuda")).cpu().numpy()
    for i, av in enumerate(a):
        ref = oracle.coeffs_abel(N, M, Q, f=lambda omx: np.exp(av * (1 - omx)))[0]
        assert relerr(c[i], ref) < 1e-12


def test_plain_method_chebyshev_series(leg, oracle):
    """The third ragged family on the plain path: f = sum_m g_m rho^m T_m
    evaluated at the quadrature points (Clenshaw) against route 2 with the same
    closed form (numpy's chebval), and, the rule being exact for degree 40 and
    M > N + 40, against the exact Legendre coefficients of route 1."""
    N, M, Q, Kc = 48, 256, 24, 41
    plan = leg.Plan(N, M, 2, Q, leg.F64)
    rng = np.random.default_rng(31)
    coef = np.array([rng.standard_normal(Kc) * r ** np.arange(Kc) for r in (0.5, 0.9, 0.99)])
    c = plan.plain_forward_cheb(torch.tensor(coef, device="cuda")).cpu().numpy()
    plan.status()
    for i in range(coef.shape[0]):
        ref = oracle.coeffs_abel(N, M, Q, f=lambda omx: np.polynomial.chebyshev.chebval(1 - omx, coef[i]))[0]
        assert relerr(c[i], ref) < 1e-12
        exact = oracle.coeffs_direct(N, 64, f=lambda x: np.polynomial.chebyshev.chebval(x, coef[i]))[0]
        assert relerr(c[i], exact) < 1e-12
    with pytest.raises(leg.LegError):
        plan.plain_forward_cheb(torch.zeros((1, 16385 + 1), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("sym", [True, False])
def test_plain_method_literal_and_symmetric_rules(leg, oracle, sym):
    N, M, Q = 32, 128, 11
    plan = leg.Plan(N, M, 2, Q, leg.F64, 0 if sym else leg.FLAG_TAU_LITERAL)
    t = 0.8
    c = plan.plain_forward(leg.FAMILY_GENFN, torch.tensor([t], dtype=torch.float64, device="cuda"))
    ref = oracle.coeffs_abel(N, M, Q, sym=sym, f=lambda omx: (1 - 2 * (1 - omx) * t + t * t) ** -0.5)[0]
    assert np.max(np.abs(c.cpu().numpy()[0] - ref)) < 1e-13


# ------------------------------------------------------------------ sampled path
SMALL = [
    # (N, M, K, Q, B): several GEMM tiles, ragged tails in B, rows and K
    (40, 128, 97, 0, 37),
    (64, 256, 129, 20, 130),
    (31, 64, 33, 5, 3),
    (4, 8, 2, 1, 5),        # degenerate: smallest grid, linear f
    (128, 256, 65, 0, 1),   # N = M/2
    (8192, 32768, 65, 0, 3),   # largest grid: M = 32768, N = M/4
]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("N,M,K,Q,B", SMALL[:5])
def test_forward_matches_route2(leg, oracle, dtype, N, M, K, Q, B):
    plan = leg.Plan(N, M, K, Q, dtype)
    f = cheb_inputs(B, K, seed=N + K)
    c = run_forward(leg, plan, f)
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f.astype(np.float64))
    assert relerr(c, ref) < TOL[dtype]


def test_forward_f64_largest_grid(leg, oracle):
    N, M, K, Q, B = SMALL[5]
    plan = leg.Plan(N, M, K, Q, leg.F64)
    f = cheb_inputs(B, K, seed=7)
    c = run_forward(leg, plan, f)
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f.astype(np.float64))
    assert relerr(c, ref) < 1e-11


def test_plain_method_largest_grid(leg):
    N, M, Q = 8192, 32768, 1024
    plan = leg.Plan(N, M, 2, Q, leg.F64)
    t = torch.tensor([0.95, 0.5], dtype=torch.float64, device="cuda")
    c = plan.plain_forward(leg.FAMILY_GENFN, t).cpu().numpy()
    n = np.arange(N)
    # aliasing of the trapezoid rule is ~t^(M - N) (negligible); FP64 rounding,
    # amplified by (2n+1) up to n = 8191, stays within the FP64 tolerance
    assert np.max(np.abs(c[1] - 0.5 ** n)) < 1e-11
    assert np.max(np.abs(c[0] - 0.95 ** n)) < 1e-9


def test_forward_f64_exact_config_equals_route1(leg, oracle):
    # polynomial input of degree K-1 with M > N + K - 1 and the exact tau rule:
    # the method has no discretisation error, so the GPU meets the plain definition
    N, M, K, B = 96, 512, 257, 9
    plan = leg.Plan(N, M, K, 0, leg.F64)
    f = cheb_inputs(B, K, seed=3).astype(np.float64)
    c = run_forward(leg, plan, f)
    ref = oracle.coeffs_direct(N, (K + N) // 2 + 4, f_cl=f)
    assert relerr(c, ref) < 1e-11


@pytest.mark.parametrize("dtype", [0, 1])
def test_backward_is_the_transpose(leg, oracle, dtype):
    N, M, K, Q, B = 24, 64, 33, 9, 5
    plan = leg.Plan(N, M, K, Q, dtype)
    # explicit L = R A on the oracle's grid
    A = oracle.abel_operator(M, K, Q, True)
    R = oracle.twisted_dft_matrix(N, M)
    L = R @ A
    rng = np.random.default_rng(1)
    v = rng.standard_normal((B, N))
    tdt = torch.float64 if dtype == 0 else torch.float32
    vd = torch.tensor(v, dtype=tdt, device="cuda")
    df = plan.backward(vd).double().cpu().numpy()
    ref = (v.astype(np.float32).astype(np.float64) if dtype else v) @ L
    assert relerr(df, ref) < (1e-11 if dtype == 0 else 1e-4)


def test_backward_dot_product_identity_f64(leg):
    N, M, K, B = 200, 512, 301, 4
    plan = leg.Plan(N, M, K, 0, leg.F64)
    g = torch.Generator(device="cpu").manual_seed(0)
    f = torch.randn(B, K, dtype=torch.float64, generator=g).cuda()
    v = torch.randn(B, N, dtype=torch.float64, generator=g).cuda()
    lhs = (plan.forward(f) * v).sum(1)
    rhs = (f * plan.backward(v)).sum(1)
    assert torch.allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * float(lhs.abs().max()))


def test_autograd_function_f64(leg):
    N, M, K, B = 16, 64, 17, 3
    plan = leg.Plan(N, M, K, 0, leg.F64)
    f = torch.randn(B, K, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.rand(N, dtype=torch.float64, device="cuda")
    target = torch.randn(N, dtype=torch.float64, device="cuda")
    loss = (w * (leg.legendre(f, plan) - target) ** 2).sum()
    loss.backward()
    # central differences (the loss is quadratic: no truncation error)
    h = 1e-3
    d = torch.randn_like(f)
    with torch.no_grad():
        lp = (w * (plan.forward(f + h * d) - target) ** 2).sum()
        lm = (w * (plan.forward(f - h * d) - target) ** 2).sum()
    fd = (lp - lm) / (2 * h)
    assert abs(float(fd) - float((f.grad * d).sum())) < 1e-9 * max(1.0, abs(float(fd)))


# ------------------------------------------------------------------ edges and errors
def test_empty_batch_is_a_noop(leg):
    plan = leg.Plan(16, 64, 17, 0, leg.F32)
    f = torch.empty((0, 17), dtype=torch.float32, device="cuda")
    c = plan.forward(f)
    assert c.shape == (0, 16)


def test_argument_errors(leg):
    with pytest.raises(leg.LegError) as e:
        leg.Plan(64, 100, 33)
    assert e.value.code == 1
    plan = leg.Plan(16, 64, 17, 0, leg.F32)
    with pytest.raises(ValueError):
        plan.forward(torch.zeros((2, 16), dtype=torch.float32, device="cuda"))
