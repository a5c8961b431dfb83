"""The half-range sine form of the coefficients (Eq. 2.13 with phi of Eq. 2.14)
as the forward transform (LEG_FLAG_SINE_FORM / LEG_TRANSFORM_SINE), against
the oracle's route 3 (the sine sum written out directly on [0, pi]) and
route 2 (the full-range Fourier sum of Eq. 2.4), element by element.

Tolerances (relative to max|c| per function): FP64 1e-11 (1e-12 for the
plain method), split-FP16 1e-6, FP32 3e-4 -- those of the real-even route.
The second workload is the test function of Table 1, f = |x|^{3/2}, on the
plain method at several (M, Q): parity against route 3 at the same (M, Q),
and the method error against the true column of Table 1 (Eq. 2.15) reported.
"""
import os

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


def table1_true():
    """n -> true c_n of |x|^{3/2} (Table 1, tests/golden)."""
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1_abs_x_3_2.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, t, _ = line.split()
                out[int(n)] = float(t)
    return out


def relerr(c, ref):
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    return float(np.max(np.max(np.abs(c - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def run(leg, plan, f_np):
    dt = torch.float64 if plan.dtype == leg.F64 else torch.float32
    c = plan.forward(torch.from_numpy(f_np).to(device="cuda", dtype=dt))
    plan.status()
    return c.double().cpu().numpy()


TOL = {"F64": 1e-11, "SPLIT_FP16": 1e-6, "F32": 3e-4, "BF16": 5e-2}


@pytest.mark.parametrize("dtype_name", ["F64", "SPLIT_FP16", "F32", "BF16"])
def test_sine_form_sampled_inputs(leg, oracle, dtype_name):
    # several function tiles and a ragged tail (B = 300); non-exact Q so that
    # the parity is against the method's own discretisation (route 3)
    N, M, K, Q, B = 256, 1024, 257, 100, 300
    rng = np.random.default_rng(1300)
    f, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), rng)
    dt = getattr(leg, dtype_name)
    plan = leg.Plan(N, M, K, Q, dt, flags=leg.FLAG_SINE_FORM)
    assert plan.transform == leg.TRANSFORM_SINE
    c = run(leg, plan, f)
    sample = np.array([0, 1, 127, 128, 150, 255, 256, 298, 299])
    ref3 = oracle.coeffs_sine(N, M, Q, f_cl=f[sample].astype(np.float64))
    ref2 = oracle.coeffs_abel(N, M, Q, f_cl=f[sample].astype(np.float64))
    e3, e2 = relerr(c[sample], ref3), relerr(c[sample], ref2)
    print(dtype_name, "sine form vs route 3", e3, "vs route 2", e2)
    assert e3 < TOL[dtype_name] and e2 < TOL[dtype_name]


@pytest.mark.parametrize("M", [256, 512, 2048, 8192, 32768])
def test_sine_form_every_length_f64_and_split(leg, oracle, M):
    N, K = M // 4, 129
    B = 5
    rng = np.random.default_rng(M)
    f, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.95), rng)
    Q = oracle.exact_tau_points(K)
    ref = oracle.coeffs_sine(N, M, Q, f_cl=f.astype(np.float64))
    base = leg.Plan(N, M, K, 0, leg.F64, flags=leg.FLAG_SINE_FORM)
    split = leg.Plan.like(base, leg.SPLIT_FP16)
    assert split.transform == leg.TRANSFORM_SINE
    e64, esp = relerr(run(leg, base, f), ref), relerr(run(leg, split, f), ref)
    print("M", M, "f64", e64, "split", esp)
    assert e64 < 1e-11 and esp < 1e-6


def test_sine_form_equals_real_even_route(leg):
    # the same discrete map: FP64 results agree to rounding, on the plan and
    # through leg_plan_set_transform
    N, M, K, B = 512, 2048, 1025, 64
    f, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(5))
    plan = leg.Plan(N, M, K, 0, leg.F64)
    assert plan.transform == leg.TRANSFORM_REG
    c_reg = run(leg, plan, f)
    plan.set_transform(leg.TRANSFORM_SINE)
    c_sine = run(leg, plan, f)
    plan.set_transform(leg.TRANSFORM_STOCKHAM)
    c_stk = run(leg, plan, f)
    scale = np.max(np.abs(c_reg), axis=1, keepdims=True)
    assert np.max(np.abs(c_sine - c_reg) / scale) < 1e-12
    assert np.max(np.abs(c_stk - c_reg) / scale) < 1e-12


@pytest.mark.parametrize("M", [2048, 8192, 32768])
def test_radix16_matches_radix8(leg, M):
    """The register-tiled kernels with 16 values per thread (radix-16 passes)
    compute the same map as with 8: FP64 results agree to rounding, split
    results to far below the split path's tolerance, for both transforms.
    FP64 bound: the (2n+1) factor scales the transform's rounding (about
    1e-16 relative to max|g|) by up to 2N = M/2, so two orderings of the same
    sums may differ by ~2e-16 M relative to max|c| (3.3e-12 at M = 32768)."""
    N, K, B = M // 4, 129, 7
    f, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.95), np.random.default_rng(M + 1))
    base = leg.Plan(N, M, K, 0, leg.F64)
    split = leg.Plan.like(base, leg.SPLIT_FP16)
    for plan, tol in ((base, 4e-16 * M), (split, 1e-7)):
        for variant in (leg.TRANSFORM_REG, leg.TRANSFORM_SINE):
            plan.set_transform(variant, 8)
            c8 = run(leg, plan, f)
            plan.set_transform(variant, 16)
            assert plan.transform_radix == 16 and plan.transform == variant
            c16 = run(leg, plan, f)
            scale = np.max(np.abs(c8), axis=1, keepdims=True)
            assert np.max(np.abs(c16 - c8) / scale) < tol, (plan.dtype, variant)


def test_sine_form_plain_method_generating_function(leg):
    cfg = workloads.CONFIGS["genfn_plain_n64"]
    plan = leg.Plan(cfg["N"], cfg["M"], 17, cfg["Q"], leg.F64, flags=leg.FLAG_SINE_FORM)
    c = plan.plain_forward(leg.FAMILY_GENFN, torch.tensor([cfg["t"]], dtype=torch.float64, device="cuda"))
    got = c.cpu().numpy()[0]
    assert np.max(np.abs(got - cfg["t"] ** np.arange(cfg["N"]))) < 1e-12


@pytest.mark.parametrize("M,Q", [(256, 64), (1024, 128), (1024, 512), (4096, 1024)])
def test_table1_abs_x_three_halves_plain_method(leg, oracle, M, Q):
    # f = |x|^{3/2} evaluated at the quadrature points (plain method), sine form
    N = 32
    plan = leg.Plan(N, M, 17, Q, leg.F64, flags=leg.FLAG_SINE_FORM)
    c = plan.plain_forward(leg.FAMILY_ABSPOW, torch.tensor([1.5, 2.5], dtype=torch.float64, device="cuda"))
    got = c.cpu().numpy()
    for row, alpha in enumerate((1.5, 2.5)):
        ref = oracle.coeffs_sine(N, M, Q, f=lambda omx: np.abs(1 - omx) ** alpha)[0]
        assert np.max(np.abs(got[row] - ref)) < 1e-12 * np.max(np.abs(ref))
    # the method error against Table 1's true column (Eq. 2.15) shrinks with Q
    err = max(abs(got[0][n] - t) for n, t in table1_true().items())
    print("M", M, "Q", Q, "max |c_n - true c_n| over Table 1", err)
    if Q >= 512:
        assert err < 1e-6


def test_sine_form_ragged_batch(leg, oracle):
    # the bucket plans take the sine form; parity against route 3 per bucket
    rng = np.random.default_rng(31)
    fam, par, n = workloads.ragged_spec(240, rng, 32, 1024)
    lay = workloads.ragged_layout(fam, par, n, rng)
    plans = []
    for Nb in lay["buckets"]:
        p = leg.Plan(*workloads.bucket_sizes(Nb), dtype=leg.SPLIT_FP16)
        if p.M >= 256:
            p.set_transform(leg.TRANSFORM_SINE)
        plans.append(p)
    batch = leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"])
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    f = torch.empty(lay["n_in"], dtype=torch.float32, device="cuda")
    leg.sample_cl(dev(fam, torch.int32), dev(par, torch.float64), dev(lay["K"], torch.int32),
                  dev(lay["in_off"], torch.int64), f, coef=dev(lay["coef"], torch.float64),
                  coef_off=dev(lay["coef_off"], torch.int64))
    c = torch.full((lay["n_out"],), float("nan"), dtype=torch.float32, device="cuda")
    batch.forward(f, c)
    batch.forward(f, c)
    torch.cuda.synchronize()
    batch.status()
    f_host, c_host = f.cpu().numpy(), c.cpu().numpy()
    worst = 0.0
    for b, Nb in enumerate(lay["buckets"]):
        N, M, K, Q = workloads.bucket_sizes(Nb)
        idx = np.where(lay["bidx"] == b)[0]
        for i in (idx[0], idx[-1]):
            fk = f_host[lay["in_off"][i]:lay["in_off"][i] + K].astype(np.float64)
            ref = oracle.coeffs_sine(N, M, Q, f_cl=fk[None])[0][:n[i]]
            got = c_host[lay["out_off"][i]:lay["out_off"][i] + n[i]]
            worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    print("ragged sine form worst", worst)
    assert worst < 1e-6


def test_sine_form_argument_checks(leg):
    with pytest.raises(leg.LegError) as e:
        leg.Plan(16, 128, 17, 0, leg.F64, flags=leg.FLAG_SINE_FORM)
    assert e.value.code == 4   # M < 256
    with pytest.raises(leg.LegError) as e:
        leg.Plan(16, 256, 17, 0, leg.F64, flags=leg.FLAG_SINE_FORM | leg.FLAG_COLLAPSED)
    assert e.value.code == 1
    p = leg.Plan(16, 128, 17, 0, leg.F64)
    with pytest.raises(leg.LegError):
        p.set_transform(leg.TRANSFORM_SINE)
    with pytest.raises(leg.LegError):
        p.set_transform(7)
    with pytest.raises(leg.LegError):
        p.set_transform(leg.TRANSFORM_REG, 32)


# ---------------------------------------------------------------- the adjoint
@pytest.mark.parametrize("dtype_name,tol", [("F64", 1e-11), ("SPLIT_FP16", 1e-6)])
def test_sine_form_adjoint_is_the_transpose(leg, oracle, dtype_name, tol):
    # leg_backward on a sine-form plan against the explicit L = R A of the
    # oracle's route 2 on the same grid
    N, M, K, Q, B = 64, 256, 65, 17, 5
    plan = leg.Plan(N, M, K, Q, getattr(leg, dtype_name), flags=leg.FLAG_SINE_FORM)
    L = oracle.twisted_dft_matrix(N, M) @ oracle.abel_operator(M, K, Q, True)
    v = np.random.default_rng(3).standard_normal((B, N))
    if dtype_name != "F64":
        v = v.astype(np.float32).astype(np.float64)
    dt = torch.float64 if dtype_name == "F64" else torch.float32
    df = plan.backward(torch.tensor(v, dtype=dt, device="cuda")).double().cpu().numpy()
    plan.status()
    assert relerr(df, v @ L) < tol


@pytest.mark.parametrize("M", [256, 2048, 8192, 32768])
def test_sine_form_adjoint_at_every_length(leg, oracle, M):
    # FP64: both transform kernels' backward passes against the oracle's
    # route 1 transposed (the configuration is exact, M > N + K - 1).  The
    # (2n+1) weights, up to 2N = M/2, carry the kernels' rounding into the
    # result, so the bound grows with M (8e-15 M; measured at M = 32768: the
    # real-even adjoint 1.1e-10, the sine form 2.1e-11).  Split FP16: the two
    # kernels agree to the split GEMM's resolution (up to M = 8192: with K = 65
    # and N = M/4 the transposed GEMM sums rows whose result cancels to a
    # degree-64 polynomial, and its relative error grows with N/K)
    N, K, B = M // 4, 65, 6
    g = torch.Generator(device="cpu").manual_seed(M)
    v = torch.randn(B, N, generator=g, dtype=torch.float64)
    ref = oracle.adjoint_direct((K + N) // 2 + 4, K, v.numpy())
    plan = leg.Plan(N, M, K, 0, leg.F64)
    for tr in (leg.TRANSFORM_REG, leg.TRANSFORM_SINE):
        plan.set_transform(tr)
        d = plan.backward(v.cuda()).cpu().numpy()
        plan.status()
        assert relerr(d, ref) < 8e-15 * M, (tr, relerr(d, ref))
    if M <= 8192:
        plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
        v32 = v.float().cuda()
        plan.set_transform(leg.TRANSFORM_REG)
        d_reg = plan.backward(v32).double().cpu().numpy()
        plan.set_transform(leg.TRANSFORM_SINE)
        d_sine = plan.backward(v32).double().cpu().numpy()
        plan.status()
        scale = np.max(np.abs(d_reg), axis=1, keepdims=True)
        assert np.max(np.abs(d_sine - d_reg) / scale) < 1e-7


def test_sine_form_dot_product_identity_f64(leg):
    # <L f, v> = <f, L^T v> with the sine-form forward and its adjoint
    N, M, K, B = 1024, 4096, 513, 4
    plan = leg.Plan(N, M, K, 0, leg.F64, flags=leg.FLAG_SINE_FORM)
    g = torch.Generator(device="cpu").manual_seed(9)
    f = torch.randn(B, K, dtype=torch.float64, generator=g).cuda()
    v = torch.randn(B, N, dtype=torch.float64, generator=g).cuda()
    lhs = (plan.forward(f) * v).sum(1)
    rhs = (f * plan.backward(v)).sum(1)
    assert torch.allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * float(lhs.abs().max()))
