"""leg_plan_autotune: the chosen launch parameters leave results unchanged,
and the tuning cache (LEG_TUNE_CACHE) is written and reused."""
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


@pytest.mark.parametrize("dtype_name,N,M,K,B", [("SPLIT_FP16", 512, 2048, 1025, 600), ("F64", 128, 512, 129, 64)])
def test_autotune_keeps_results(leg, tmp_path, monkeypatch, dtype_name, N, M, K, B):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LEG_TUNE_CACHE", str(cache))
    dt = getattr(leg, dtype_name)
    plan = leg.Plan(N, M, K, 0, dt)
    rng = np.random.default_rng(K)
    f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), rng)
    tdt = torch.float64 if dt == leg.F64 else torch.float32
    f = torch.from_numpy(f_np).to(device="cuda", dtype=tdt)
    ref = plan.forward(f).clone()
    choice = plan.autotune(f)
    assert choice["fft"] in (leg.TRANSFORM_REG, leg.TRANSFORM_STOCKHAM, leg.TRANSFORM_SINE)
    assert plan.transform == choice["fft"] and plan.transform_radix in (8, 16)
    if dt == leg.SPLIT_FP16:
        assert choice["tn"] == 0 or (64 <= choice["tn"] <= 128 and choice["tn"] % 16 == 0)
    out = plan.forward(f)
    plan.status()
    scale = ref.abs().max(1).values
    err = float(((out - ref).abs().max(1).values / scale).max())
    # the tile width does not change results; the transform kernels differ by rounding
    assert err < (1e-12 if dt == leg.F64 else 1e-7), err
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and lines[0].split()[1] == str(choice["tn"])
    # a second plan with the same key takes the stored choice without timing
    plan2 = leg.Plan(N, M, K, 0, dt)
    assert plan2.autotune(f) == choice
    assert plan2.transform_radix == plan.transform_radix
    assert len(cache.read_text().strip().splitlines()) == 1
