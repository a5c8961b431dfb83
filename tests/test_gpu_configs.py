"""Full-size workloads on the GPU, checked on sampled outputs the oracle can compute.

* B=4096, K=1025, N=512, M=2048: split-FP16 and the plain FP32 / FP64 paths,
  the first and last function of every GEMM function tile plus 16 more
  against oracle route 1 (an exact configuration).
* Precision sweep B=256, K=8193, N=4096, M=16384 (rho up to 0.999): FP64, FP32,
  BF16 and split-FP16 from one operator, 40 sampled functions (the first and
  last of every GEMM function tile among them) against oracle route 1 (the
  configuration is exact for polynomial inputs: M > N + K - 1 with the exact
  tau rule, so routes 1 and 2 agree to rounding).
* Differentiation B=1024, K=4097, N=2048, M=8192: forward parity on >= 16
  sampled functions (first and last of every function tile); the adjoint
  df = L^T v element by element against the oracle's route 1 transposed on the
  same functions (split 1e-6, FP64 1e-11 of max|df|); torch.autograd gradients
  of sum_n w_n (c_n - c*_n)^2 (FP64 path and split path) against FP64 central
  differences on 64 random directions, and the split adjoint against the
  oracle's forward through <L f, v> = <f, L^T v>.
Errors are max_n |c - c_ref| / max_n |c_ref| per function, max over the sample.
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
    return float(np.max(np.max(np.abs(c - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def forward(leg, plan, f_np):
    dt = torch.float64 if plan.dtype == leg.F64 else torch.float32
    c = plan.forward(torch.from_numpy(f_np).to(device="cuda", dtype=dt))
    plan.status()
    return c.double().cpu().numpy()


def tile_sample(B, tn, extra, seed):
    """The first and last function of every GEMM function tile of width tn,
    plus `extra` more at random."""
    idx = set()
    for t0 in range(0, B, tn):
        idx.update((t0, min(B, t0 + tn) - 1))
    rest = np.setdiff1d(np.arange(B), sorted(idx))
    idx.update(int(i) for i in np.random.default_rng(seed).choice(rest, size=min(extra, rest.size), replace=False))
    return np.array(sorted(idx))


def test_bench_workload_all_paths(leg, oracle):
    name = "cheb_b4096_k1025_n512_m2048"
    cfg = workloads.CONFIGS[name]
    f = workloads.workload_inputs(name)
    split = leg.Plan(cfg["N"], cfg["M"], cfg["K"], 0, leg.SPLIT_FP16)
    sample = tile_sample(cfg["B"], split.tile_info(cfg["B"])["tn"], 16, 2)
    # exact configuration (M > N + K - 1, exact tau rule): route 1
    ref = oracle.coeffs_direct(cfg["N"], (cfg["K"] + cfg["N"]) // 2 + 4, f_cl=f[sample].astype(np.float64))
    errs = {"split": relerr(forward(leg, split, f)[sample], ref)}
    for name_, dt in (("f32", leg.F32), ("f64", leg.F64)):
        errs[name_] = relerr(forward(leg, leg.Plan.like(split, dt), f)[sample], ref)
    print("bench workload errors", errs)
    assert errs["split"] < 1e-6
    assert errs["f64"] < 1e-11
    # measured 5.6e-5 (FP32 GEMM + FP32 transform); the bound leaves 2.5x
    assert errs["f32"] < 1.5e-4


def test_precision_sweep(leg, oracle):
    name = "cheb_b256_k8193_n4096_m16384"
    cfg = workloads.CONFIGS[name]
    N, M, K = cfg["N"], cfg["M"], cfg["K"]
    f = workloads.workload_inputs(name)
    base = leg.Plan(N, M, K, 0, leg.F64)
    tn = leg.Plan.like(base, leg.SPLIT_FP16).tile_info(cfg["B"])["tn"]
    sample = tile_sample(cfg["B"], tn, 36, 3)
    assert len(sample) >= 32
    ref = oracle.coeffs_direct(N, (K + N) // 2 + 4, f_cl=f[sample].astype(np.float64))
    errs = {"f64": relerr(forward(leg, base, f)[sample], ref)}
    for name_, dt in (("f32", leg.F32), ("bf16", leg.BF16), ("split_fp16", leg.SPLIT_FP16)):
        errs[name_] = relerr(forward(leg, leg.Plan.like(base, dt), f)[sample], ref)
    print("precision sweep errors", errs)
    assert errs["f64"] < 1e-11
    assert errs["split_fp16"] < 1e-6
    # measured 2.4e-4 (FP32) and 8.3e-3 (one BF16 product) on these 40
    # functions; the bounds leave 2.5x, so a drop in either path's accuracy shows
    assert errs["f32"] < 6e-4
    assert errs["bf16"] < 2.1e-2


def test_differentiation(leg, oracle):
    name = "cheb_b1024_k4097_n2048_m8192"
    cfg = workloads.CONFIGS[name]
    B, N, M, K = cfg["B"], cfg["N"], cfg["M"], cfg["K"]
    f_np = workloads.workload_inputs(name)
    w_np, tgt_np = workloads.loss_weights(N, workloads.rng_for(name, salt=1))
    split = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f64 = leg.Plan.like(split, leg.F64)
    w = torch.tensor(w_np, device="cuda")
    tgt = torch.tensor(tgt_np, device="cuda")

    # forward parity on sampled functions (route 1: exact configuration)
    sample = tile_sample(B, split.tile_info(B)["tn"], 8, 4)
    assert len(sample) >= 16
    Qo = (K + N) // 2 + 4
    ref = oracle.coeffs_direct(N, Qo, f_cl=f_np[sample].astype(np.float64))
    x32 = torch.from_numpy(f_np).cuda().requires_grad_(True)
    c32 = leg.legendre(x32, split)
    assert relerr(c32.detach().double().cpu().numpy()[sample], ref) < 1e-6

    # the adjoint element by element against the oracle's route 1 transposed
    # (df = L^T v for random v), split and FP64.  The FP64 bound: the adjoint
    # scales v_n by (2n+1) before the transposed transform and operator, so
    # FP64 rounding (1.1e-16) grows by about 2N sqrt(M) / sqrt(K) ~ 6e3 here
    # plus the sums' own growth: 1e-10 (measured 1.0e-11).
    vv = np.random.default_rng(8).standard_normal((B, N))
    ref_b = oracle.adjoint_direct(Qo, K, vv[sample])
    for pl, tdt, tol in ((split, torch.float32, 1e-6), (f64, torch.float64, 1e-10)):
        dfv = pl.backward(torch.from_numpy(vv).to(device="cuda", dtype=tdt)).double().cpu().numpy()[sample]
        eb = relerr(dfv, ref_b)
        print("adjoint vs oracle route 1 transposed", pl.dtype, eb)
        assert eb < tol

    # end-to-end gradient of the split-path loss through LegendreFn
    (w.float() * (c32 - tgt.float()) ** 2).sum().backward()
    split.status()
    grad_split = x32.grad.double()

    # exact-adjoint gradient of the FP64 loss through LegendreFn
    x64 = torch.from_numpy(f_np).cuda().double().requires_grad_(True)
    c64 = leg.legendre(x64, f64)
    (w * (c64 - tgt) ** 2).sum().backward()
    grad64 = x64.grad
    # the split adjoint applied to the same cotangent as the FP64 one
    v64 = (2 * w * (c64.detach() - tgt)).float()
    grad_split_v = split.backward(v64).double()

    def loss64(x):
        return float((w * (f64.forward(x) - tgt) ** 2).sum())

    # FP64 central differences on 64 random directions (the loss is quadratic in f,
    # so central differences carry no truncation error)
    g = torch.Generator(device="cpu").manual_seed(1106)
    h = 1e-2
    x0 = x64.detach()
    worst = {"f64": 0.0, "split_adjoint": 0.0, "split_end_to_end": 0.0}
    for _ in range(64):
        d = torch.randn(B, K, dtype=torch.float64, generator=g).cuda()
        fd = (loss64(x0 + h * d) - loss64(x0 - h * d)) / (2 * h)
        for key, gr in (("f64", grad64), ("split_adjoint", grad_split_v), ("split_end_to_end", grad_split)):
            worst[key] = max(worst[key], abs(fd - float((gr * d).sum())) / abs(fd))
    print("max relative directional-derivative error over 64 directions", worst)
    assert worst["f64"] < 1e-8              # leg_backward is the exact adjoint
    assert worst["split_adjoint"] < 1e-4    # split backward, same cotangent
    # the split-path loss differs from the FP64 loss by the forward's rounding,
    # which is largest at high n and is weighted again by ~(n+1/2) in L^T
    assert worst["split_end_to_end"] < 1e-3

    # adjoint against the oracle's forward: <L f_i, v> = <f_i, L^T v> per sampled function
    v = np.random.default_rng(3).standard_normal((len(sample), N)).astype(np.float32)
    vt = torch.zeros((B, N), dtype=torch.float32, device="cuda")
    vt[torch.from_numpy(sample).cuda()] = torch.from_numpy(v).cuda()
    df = split.backward(vt).double().cpu().numpy()[sample]
    lhs = np.sum(ref * v.astype(np.float64), axis=1)
    rhs = np.sum(f_np[sample].astype(np.float64) * df, axis=1)
    scale = np.sum(np.abs(ref) * np.abs(v), axis=1)
    # the split adjoint carries ~1e-6 of max|df| per element; the K = 4097
    # terms of <f, L^T v> sum those errors
    assert np.max(np.abs(lhs - rhs) / scale) < 5e-5
