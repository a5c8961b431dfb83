"""leg_forward replays a CUDA graph of its launches from the third call with
the same buffers and launch parameters on.  The replay must give the same
coefficients as direct launches (leg_forward_profiled never uses the graph),
follow new input contents, and be rebuilt when the buffers, the batch, the
workspace or a launch parameter change.  A call made while the caller's own
stream is being captured joins the caller's graph instead.
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


def inputs(B, K, seed):
    f, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(seed))
    return torch.from_numpy(f).cuda()


def direct(plan, f):
    c = torch.empty((f.shape[0], plan.N), dtype=torch.float32, device="cuda")
    plan.forward_profiled(f, c)
    return c


@pytest.mark.parametrize("flags", [0, 2])
def test_graph_replay_matches_direct_launches(leg, flags):
    N, M, K, B = 64, 256, 129, 300
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16, flags=flags)
    f = inputs(B, K, 1)
    c = torch.empty((B, N), device="cuda")
    for _ in range(4):                       # direct, capture, replay, replay
        c.fill_(float("nan"))
        plan.forward(f, c)
        assert torch.equal(c, direct(plan, f))
    f.copy_(inputs(B, K, 2))                 # same buffer, new contents
    plan.forward(f, c)
    assert torch.equal(c, direct(plan, f))
    c2 = torch.full_like(c, float("nan"))    # new output buffer: c must stay as it was
    keep = c.clone()
    for _ in range(3):
        plan.forward(f, c2)
    assert torch.equal(c2, keep) and torch.equal(c, keep)
    plan.set_tile(64)                        # launch parameter changed
    for _ in range(3):
        plan.forward(f, c)
    assert torch.equal(c, direct(plan, f))
    plan.reserve(4 * B)                      # workspace reallocated
    for _ in range(3):
        plan.forward(f, c)
    assert torch.equal(c, direct(plan, f))
    fb = inputs(B // 2, K, 3)                # another batch size
    cb = torch.empty((B // 2, N), device="cuda")
    for _ in range(3):
        plan.forward(fb, cb)
    assert torch.equal(cb, direct(plan, fb))
    plan.status()


def test_forward_inside_a_caller_capture(leg):
    N, M, K, B = 64, 256, 129, 100
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f = inputs(B, K, 4)
    c = torch.empty((B, N), device="cuda")
    plan.forward(f, c)
    plan.forward(f, c)
    ref = direct(plan, f)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.forward(f, c)
    torch.cuda.current_stream().wait_stream(s)
    c.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
    plan.status()
