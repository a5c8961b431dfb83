"""Allocation failures injected on the host.

With LEG_FAULT_ALLOC = k the k-th device allocation the library attempts
after the variable takes that value fails on the host without allocating (no
kernel ever sees a bad pointer).  For every entry point that allocates, the
sweep k = 1, 2, ... makes each of its allocations fail in turn: the call must
return LEG_ERR_OOM, leave the device's free memory where it was once the
objects of the failed call are gone, and the next call without the fault must
succeed (with the same results as before).
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

SLACK = 2 << 20   # free-memory granularity of the driver (the library's own count is compared exactly)


@pytest.fixture(scope="module")
def leg():
    import paper_1106_0463_gb300 as leg
    assert torch.cuda.is_available()
    return leg


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def settle(leg):
    """Collect the plans and batches earlier tests left to the garbage
    collector (their memory returns to the device), then the library's count."""
    import gc
    gc.collect()
    torch.cuda.synchronize()
    return leg.memory_info()


def sweep(leg, monkeypatch, attempt, max_k=100):
    """attempt() under LEG_FAULT_ALLOC = 1, 2, ... until it succeeds; returns
    (number of allocations the call makes, the successful result).  After
    every failed attempt the library holds exactly what it held before."""
    held = settle(leg)
    base = free_bytes()
    for k in range(1, max_k):
        monkeypatch.setenv("LEG_FAULT_ALLOC", str(k))
        try:
            obj = attempt()
        except leg.LegError as e:
            assert e.code == 2, (k, str(e))   # LEG_ERR_OOM
            assert settle(leg) == held, (k, held, leg.memory_info())
            assert abs(free_bytes() - base) <= SLACK, (k, base - free_bytes())
            continue
        monkeypatch.delenv("LEG_FAULT_ALLOC")
        return k - 1, obj
    raise AssertionError("the call never succeeded")


@pytest.mark.parametrize("dtype_name,flags", [("SPLIT_FP16", 0), ("F64", 0), ("BF16", 0), ("F32", 0),
                                              ("SPLIT_FP16", 2)])
def test_plan_create_fails_cleanly(leg, monkeypatch, dtype_name, flags):
    dt = getattr(leg, dtype_name)
    leg.Plan(64, 256, 65, 0, dt, flags=flags).close()   # loads the kernels once
    held = settle(leg)
    base = free_bytes()
    n, plan = sweep(leg, monkeypatch, lambda: leg.Plan(64, 256, 65, 0, dt, flags=flags))
    assert n >= 3
    plan.close()
    assert leg.memory_info() == held
    assert abs(free_bytes() - base) <= SLACK
    like = leg.Plan(64, 256, 65, 0, leg.F64)
    held = settle(leg)
    base = free_bytes()
    n, p2 = sweep(leg, monkeypatch, lambda: leg.Plan.like(like, dt))
    assert n >= 2
    p2.close()
    assert leg.memory_info() == held
    assert abs(free_bytes() - base) <= SLACK


@pytest.mark.parametrize("dtype_name", ["SPLIT_FP16", "F64", "BF16"])
def test_workspace_growth_fails_cleanly(leg, monkeypatch, dtype_name):
    dt = getattr(leg, dtype_name)
    N, M, K, B = 128, 512, 129, 40
    f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(9))
    io = torch.float64 if dt == leg.F64 else torch.float32
    f = torch.from_numpy(f_np).to(device="cuda", dtype=io)
    c = torch.empty((B, N), dtype=io, device="cuda")
    ref = leg.Plan(N, M, K, 0, dt).forward(f).clone()
    plan = leg.Plan(N, M, K, 0, dt)
    n, _ = sweep(leg, monkeypatch, lambda: plan.forward(f, c))
    assert n >= 1
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
    if dt != leg.BF16:   # backward grows no further buffers after the forward's
        dc = torch.ones((B, N), dtype=io, device="cuda")
        plan.backward(dc)
        plan.status()


def test_forward_host_fails_cleanly(leg, monkeypatch):
    N, M, K, B = 128, 512, 129, 24
    f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(10))
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    ref = plan.forward(torch.from_numpy(f_np).cuda()).cpu()
    f_host = torch.from_numpy(f_np)            # pageable: the staged path allocates device copies
    c_host = torch.empty((B, N), dtype=torch.float32)
    plan2 = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    plan2.reserve(B)   # the plan's own workspace first: the sweep covers the call's device copies
    n, _ = sweep(leg, monkeypatch, lambda: plan2.forward_host(f_host, c_host))
    assert n >= 1
    assert torch.equal(c_host, ref)


def test_plain_method_scratch_fails_cleanly(leg, monkeypatch):
    # an FP32 plan's G holds 4-byte values: the FP64 plain method takes a
    # stream-ordered allocation for its G (after the plan's workspace)
    plan = leg.Plan(64, 256, 17, 32, leg.F32)
    plan.reserve(2)   # the plan's own workspace first: the sweep covers the call's G
    params = torch.tensor([0.5, 0.3], dtype=torch.float64, device="cuda")
    ref = leg.Plan(64, 256, 17, 32, leg.F64).plain_forward(leg.FAMILY_GENFN, params)
    n, c = sweep(leg, monkeypatch, lambda: plan.plain_forward(leg.FAMILY_GENFN, params))
    assert n >= 1
    torch.cuda.synchronize()
    assert torch.allclose(c, ref, rtol=0, atol=1e-14)


def test_ragged_fails_cleanly(leg, monkeypatch):
    rng = np.random.default_rng(12)
    fam, par, n = workloads.ragged_spec(90, rng, 32, 256)
    lay = workloads.ragged_layout(fam, par, n, rng)
    plans = [leg.Plan(*workloads.bucket_sizes(Nb), dtype=leg.SPLIT_FP16) for Nb in lay["buckets"]]
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    f = torch.empty(lay["n_in"], dtype=torch.float32, device="cuda")
    leg.sample_cl(dev(fam, torch.int32), dev(par, torch.float64), dev(lay["K"], torch.int32),
                  dev(lay["in_off"], torch.int64), f, coef=dev(lay["coef"], torch.float64),
                  coef_off=dev(lay["coef_off"], torch.int64))
    ref = torch.empty(lay["n_out"], dtype=torch.float32, device="cuda")
    leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"]).forward(f, ref)
    held = settle(leg)
    k, batch = sweep(leg, monkeypatch, lambda: leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"]))
    assert k >= 3 * len(lay["buckets"])
    c = torch.empty_like(ref)
    batch.forward(f, c)
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
    batch.close()
    assert settle(leg) == held
    # the one-call form: its cached batch is built inside the call
    arrays = (dev(lay["bidx"], torch.int32), dev(n, torch.int32), dev(lay["in_off"], torch.int64),
              dev(lay["out_off"], torch.int64))
    c2 = torch.empty_like(ref)
    k, _ = sweep(leg, monkeypatch, lambda: leg.forward_ragged(plans, *arrays, f, c2))
    assert k >= 3 * len(lay["buckets"])
    torch.cuda.synchronize()
    assert torch.equal(c2, ref)
    assert leg.memory_info() != held       # the cached one-call batch
    for p in plans:                         # destroying a plan drops the cached batches that use it
        p.close()
    n_after, _ = settle(leg)
    assert n_after < held[0]
