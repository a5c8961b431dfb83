"""leg_forward_host: the forward pass on host buffers, with the copies
overlapped with the computation, gives leg_forward's coefficients bit for bit
(every kernel computes each function on its own, so the pieces the batch is
copied and transformed in cannot change a result).  Checked for the split-FP16
plan (Abel GEMM + transform), the collapsed split plan and the FP64 plan, with
batches that do not divide into the four pieces, pinned and pageable host
memory, and calls of growing and shrinking size on one plan.
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


def inputs(B, K, seed, dtype=torch.float32):
    f, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(seed))
    return torch.from_numpy(f).to(dtype)


@pytest.mark.parametrize("dt,flags", [(3, 0), (3, 2), (0, 0)])
def test_forward_host_equals_forward(leg, dt, flags):
    N, M, K = 200, 512, 257
    plan = leg.Plan(N, M, K, 0, dt, flags=flags)
    io = plan.io_dtype
    for B, pinned in ((301, True), (3, False), (1026, True), (5, True)):
        f = inputs(B, K, B, io)
        ref = plan.forward(f.cuda())
        torch.cuda.synchronize()
        fh = f.pin_memory() if pinned else f.clone()
        ch = torch.full((B, N), float("nan"), dtype=io)
        if pinned:
            ch = ch.pin_memory()
        out = plan.forward_host(fh, ch)
        assert out.data_ptr() == ch.data_ptr()
        assert torch.equal(ch, ref.cpu()), (B, pinned)
    plan.status()


def test_forward_host_full_size_matches_oracle(leg, oracle):
    cfg = workloads.CONFIGS["cheb_b4096_k1025_n512_m2048"]
    B, K, N, M = cfg["B"], cfg["K"], cfg["N"], cfg["M"]
    f = torch.from_numpy(workloads.workload_inputs("cheb_b4096_k1025_n512_m2048")).pin_memory()
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    c = plan.forward_host(f).numpy().astype(np.float64)
    sample = np.random.default_rng(3).choice(B, 8, replace=False)
    ref = oracle.coeffs_abel(N, M, oracle.exact_tau_points(K), f_cl=f.numpy()[sample].astype(np.float64))
    err = np.max(np.max(np.abs(c[sample] - ref), 1) / np.max(np.abs(ref), 1))
    assert err < 1e-6


def test_forward_host_registered_and_staged_paths_agree(leg):
    """Pinned tensors are mapped host memory (read in place by the kernels);
    pageable tensors go through the staged copies; both give leg_forward's
    coefficients bit for bit, including for the collapsed plan."""
    N, M, K, B = 128, 512, 257, 777
    for flags in (0, 2):
        plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16, flags=flags)
        f = inputs(B, K, 9)
        ref = plan.forward(f.cuda()).cpu()
        pinned = plan.forward_host(f.pin_memory(), torch.empty((B, N)).pin_memory())
        staged = plan.forward_host(f.clone(), torch.empty((B, N)))
        assert torch.equal(pinned, ref) and torch.equal(staged, ref)
        plan.status()


def test_forward_host_rejects_device_tensors(leg):
    plan = leg.Plan(16, 64, 17, 0, leg.SPLIT_FP16)
    with pytest.raises(ValueError):
        plan.forward_host(torch.zeros((2, 17), device="cuda"))


@pytest.mark.parametrize("dt", [3, 2])
def test_host_overlap_stream_of_batches(leg, dt):
    """With the host overlap on, each call's input copy waits only for the
    previous user of its staging buffer: a stream of calls queued without
    synchronising (distinct inputs and outputs, sizes that grow and shrink)
    still gives every batch leg_forward's coefficients bit for bit, and so do
    calls after the overlap is switched off again."""
    N, M, K = 160, 512, 257
    plan = leg.Plan(N, M, K, 0, dt)
    plan.set_host_overlap(True)
    sizes = (37, 301, 301, 5, 301, 128, 1, 301)
    fs = [inputs(B, K, 40 + i).pin_memory() for i, B in enumerate(sizes)]
    refs = []
    for f in fs:
        refs.append(plan.forward(f.cuda()).cpu())
    torch.cuda.synchronize()
    for rnd in range(2):
        cs = [torch.full((f.shape[0], N), float("nan")).pin_memory() for f in fs]
        for f, c in zip(fs, cs):
            plan.forward_host(f, c, sync=False)
        torch.cuda.synchronize()
        for i, (c, ref) in enumerate(zip(cs, refs)):
            assert torch.equal(c, ref), (rnd, i)
    plan.set_host_overlap(False)
    c = plan.forward_host(fs[1], torch.empty((sizes[1], N)).pin_memory())
    assert torch.equal(c, refs[1])
    plan.status()


def test_host_overlap_reuses_one_input_buffer(leg):
    """The caller refills one pinned input buffer between synchronised calls:
    every call reads the contents it was made with."""
    N, M, K, B = 128, 512, 257, 200
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    plan.set_host_overlap(True)
    fh = torch.empty((B, K)).pin_memory()
    ch = torch.empty((B, N)).pin_memory()
    for seed in range(5):
        f = inputs(B, K, 70 + seed)
        ref = plan.forward(f.cuda()).cpu()
        fh.copy_(f)
        plan.forward_host(fh, ch)
        assert torch.equal(ch, ref), seed
    with pytest.raises(RuntimeError):
        leg._check(leg._lib.leg_plan_set_host_overlap(plan._h, 2))
