"""leg_forward_batches: batches one after another, pipelined for split-FP16
plans (batch b's split and GEMM on a high-priority stream, batch b-1's
transform on a low-priority one, the GEMM results alternating between two
G-sized workspaces).  Every batch must equal leg_forward on it bit for bit,
whatever the number of batches, the batch size, the transform kernel, and for
the plans that take the plain loop (FP64, collapsed); the backward pass, whose
workspace the pipeline borrows, must be unaffected.
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


def batches(nb, B, K, seed, dtype=torch.float32):
    f, _, _ = workloads.random_chebyshev(nb * B, K, (0.8, 0.99), np.random.default_rng(seed))
    return torch.from_numpy(f).to(dtype).view(nb, B, K).cuda()


@pytest.mark.parametrize("transform", ["sine", "reg"])
def test_batches_equal_forward(leg, transform):
    N, M, K = 384, 1024, 513
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    plan.set_transform(leg.TRANSFORM_SINE if transform == "sine" else leg.TRANSFORM_REG)
    for nb, B in ((1, 40), (2, 300), (3, 37), (6, 129)):
        f = batches(nb, B, K, nb * 1000 + B)
        c = torch.full((nb, B, N), float("nan"), device="cuda")
        plan.forward_batches(f, c)
        for b in range(nb):
            ref = plan.forward(f[b].contiguous())
            assert torch.equal(c[b], ref), (nb, B, b)
    plan.status()


def test_batches_headline_shape(leg):
    """The headline shape (K = 8193, M = 16384, 256 functions per batch):
    three pipelined batches against leg_forward on each."""
    N, M, K, B, nb = 4096, 16384, 8193, 256, 3
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f = batches(nb, B, K, 5)
    c = plan.forward_batches(f)
    for b in range(nb):
        assert torch.equal(c[b], plan.forward(f[b].contiguous())), b
    plan.status()


@pytest.mark.parametrize("dt,flags", [(0, 0), (3, 2), (1, 0)])
def test_batches_other_plans_loop(leg, dt, flags):
    N, M, K, B, nb = 96, 256, 129, 50, 3
    plan = leg.Plan(N, M, K, 0, dt, flags=flags)
    f = batches(nb, B, K, 11, plan.io_dtype)
    c = plan.forward_batches(f)
    for b in range(nb):
        assert torch.equal(c[b], plan.forward(f[b].contiguous())), b


def test_backward_unaffected_by_the_pipeline(leg):
    N, M, K, B = 256, 1024, 513, 64
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    dc = torch.randn(B, N, device="cuda")
    before = plan.backward(dc).clone()
    plan.forward_batches(batches(4, B, K, 21))
    assert torch.equal(plan.backward(dc), before)


def test_batches_argument_errors(leg):
    plan = leg.Plan(32, 128, 33, 0, leg.SPLIT_FP16)
    f = torch.zeros((2, 4, 33), device="cuda")
    c = torch.zeros((2, 4, 32), device="cuda")
    assert leg._lib.leg_forward_batches(plan._h, f.data_ptr(), c.data_ptr(), 4, -1, None) == 1
    assert leg._lib.leg_forward_batches(plan._h, f.data_ptr(), c.data_ptr(), 4, 0, None) == 0
    with pytest.raises(ValueError):
        plan.forward_batches(f[0])


@pytest.mark.parametrize("pinned", [True, False])
def test_host_batches_equal_forward(leg, pinned):
    """leg_forward_host_batches: pinned buffers take the pipeline with staged
    input copies and in-place output writes, pageable ones the loop of
    leg_forward_host; both equal leg_forward on each batch bit for bit,
    including calls queued back to back without synchronising."""
    N, M, K = 256, 1024, 513
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    for nb, B in ((2, 64), (5, 37), (3, 300)):
        fd = batches(nb, B, K, 300 + nb * B)
        refs = [plan.forward(fd[b].contiguous()).cpu() for b in range(nb)]
        fh = fd.cpu()
        ch = torch.full((nb, B, N), float("nan"))
        if pinned:
            fh, ch = fh.pin_memory(), ch.pin_memory()
        plan.forward_host_batches(fh, ch, sync=False)
        plan.forward_host_batches(fh, ch)
        for b in range(nb):
            assert torch.equal(ch[b], refs[b]), (nb, B, b)
    plan.status()


def test_host_batches_fp64_loop(leg):
    N, M, K, B, nb = 64, 256, 65, 20, 3
    plan = leg.Plan(N, M, K, 0, leg.F64)
    fd = batches(nb, B, K, 17, torch.float64)
    c = plan.forward_host_batches(fd.cpu().pin_memory())
    for b in range(nb):
        assert torch.equal(c[b], plan.forward(fd[b].contiguous()).cpu()), b


def test_batches_profiled_equal_and_timed(leg):
    """The profiled pipeline gives the same coefficients and positive stage
    times (the GEMM longer than the split at this shape)."""
    N, M, K, B, nb = 512, 2048, 1025, 256, 4
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f = batches(nb, B, K, 31)
    c = torch.empty((nb, B, N), device="cuda")
    ms = plan.forward_batches_profiled(f, c)
    assert all(t > 0 for t in ms) and ms[1] > ms[0], ms
    for b in range(nb):
        assert torch.equal(c[b], plan.forward(f[b].contiguous())), b


def test_batches_inside_a_caller_capture(leg):
    """On a stream being captured the batches run through leg_forward in
    turn, so their launches join the caller's graph; a replay gives every
    batch's coefficients."""
    N, M, K, B, nb = 128, 512, 257, 60, 3
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f = batches(nb, B, K, 51)
    c = torch.empty((nb, B, N), device="cuda")
    plan.reserve(B)
    refs = [plan.forward(f[b].contiguous()).clone() for b in range(nb)]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.forward_batches(f, c)
    torch.cuda.current_stream().wait_stream(s)
    c.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for b in range(nb):
        assert torch.equal(c[b], refs[b]), b
    plan.status()


def test_host_batches_single_batch(leg):
    N, M, K, B = 128, 512, 257, 33
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    fd = batches(1, B, K, 61)
    c = plan.forward_host_batches(fd.cpu().pin_memory())
    assert torch.equal(c[0], plan.forward(fd[0].contiguous()).cpu())


def test_batches_small_transform_length(leg):
    """M = 128 (the shared-memory Stockham transform) through the pipeline."""
    N, M, K = 32, 128, 65
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    f = batches(5, 70, K, 71)
    c = plan.forward_batches(f)
    for b in range(5):
        assert torch.equal(c[b], plan.forward(f[b].contiguous())), b
