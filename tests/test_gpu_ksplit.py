"""Balanced K split of the forward split-FP16 GEMM (leg_plan_set_ksplit).

Every resident CTA pair takes an equal share of the (tile, K block) work; a
tile cut between pairs leaves up to three partial outputs, which the
transform adds while it stages each row of G.  Checked element by element:
K split against whole tiles (the same products, summed in another order:
within 1e-7 of max|c|), both against the oracle (route 1 on exact
configurations, 1e-6), graph replays bit for bit, batch sizes that change the
segmentation between calls (the parts a tile lacks must read as zero), and
the host-buffer path.
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


def fwd(leg, plan, f):
    c = plan.forward(f)
    plan.status()
    return c.double().cpu().numpy()


# (N, M, K, B) at 128-function tiles: one partial wave (48 tiles for 76
# pairs), a barely started second wave (80 tiles), a ragged last function
# tile (42 tiles); each pair's share is at least half a tile's K depth, so no
# tile is cut into more than three parts
SHAPES = [(2048, 8192, 2049, 384), (512, 2048, 1025, 2500), (256, 1024, 513, 2600)]


@pytest.mark.parametrize("N,M,K,B", SHAPES)
@pytest.mark.parametrize("transform", ["REG", "SINE"])
def test_ksplit_matches_whole_tiles_and_oracle(leg, oracle, N, M, K, B, transform):
    rng = np.random.default_rng(N + B)
    f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), rng)
    f = torch.from_numpy(f_np).cuda()
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    plan.set_transform(getattr(leg, "TRANSFORM_" + transform))
    plan.set_ksplit(leg.KSPLIT_OFF)
    assert plan.ksplit_info(B)["parts"] == 1
    whole = fwd(leg, plan, f)
    plan.set_ksplit(leg.KSPLIT_ON)
    info = plan.ksplit_info(B)
    assert info["parts"] >= 2, info
    outs = [fwd(leg, plan, f) for _ in range(3)]   # direct, captured, replayed
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    split = outs[0]
    scale = np.max(np.abs(whole), axis=1, keepdims=True)
    assert np.max(np.abs(split - whole) / scale) < 1e-7
    idx = np.unique(np.array([0, 1, B // 3, B // 2, B - 2, B - 1]))
    ref = oracle.coeffs_direct(N, (K + N) // 2 + 4, f_cl=f_np[idx].astype(np.float64))
    e = relerr(split[idx], ref)
    print("ksplit", N, M, K, B, transform, info, "vs oracle", e)
    assert e < 1e-6


def fresh_plan(leg, like):
    p = leg.Plan.like(like, leg.SPLIT_FP16)
    p.set_ksplit(leg.KSPLIT_ON)
    return p


def test_ksplit_segmentation_changes_between_calls(leg):
    """Batch sizes that cut the tiles differently, in turn on one plan: each
    result equals that of a fresh plan (parts a tile lacks stay zero)."""
    N, M, K = 2048, 8192, 2049
    f_np, _, _ = workloads.random_chebyshev(520, K, (0.8, 0.99), np.random.default_rng(5))
    f = torch.from_numpy(f_np).cuda()
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    plan.set_ksplit(leg.KSPLIT_ON)
    plan.reserve(520)
    for B in (384, 520, 300, 520, 17, 384):
        got = fwd(leg, plan, f[:B].contiguous())
        ref = fwd(leg, fresh_plan(leg, plan), f[:B].contiguous())
        assert np.array_equal(got, ref), B


def test_ksplit_host_buffers(leg):
    N, M, K, B = 2048, 8192, 2049, 384
    f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(6))
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    plan.set_ksplit(leg.KSPLIT_ON)
    ref = fwd(leg, plan, torch.from_numpy(f_np).cuda())
    for pin in (False, True):   # pageable: copies in pieces; pinned: read in place
        fh = torch.from_numpy(f_np)
        if pin:
            fh = fh.pin_memory()
        got = plan.forward_host(fh).double().numpy()
        assert np.array_equal(got, ref), pin


def test_ksplit_modes_and_arguments(leg):
    plan = leg.Plan(512, 2048, 1025, 0, leg.SPLIT_FP16)
    assert plan.ksplit_info(4096)["mode"] == leg.KSPLIT_AUTO
    with pytest.raises(leg.LegError):
        plan.set_ksplit(3)
    plan.set_transform(leg.TRANSFORM_STOCKHAM)
    plan.set_ksplit(leg.KSPLIT_ON)
    assert plan.ksplit_info(2500)["parts"] == 1   # the Stockham transform does not add parts
