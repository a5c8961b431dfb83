"""leg_forward_noalloc: the split-FP16 forward pass for callers that must not
allocate device memory at call time (a framework that owns the whole device
budget through its own pool, or a latency-critical caller that cannot take
cudaMalloc's host blocking).  Its intermediates live in the library's static
64 MiB device array.

Checked through the C ABI against leg_forward on two calls in a row: the same
kernels on the same input, so the results must be identical bit for bit.
Also: the largest batch that fits the array (its G region ends 3 KB before the
array's end), the first batch that does not, and the plans it refuses.  This
file is collected last on purpose.
"""
import ctypes

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


def _abi(leg):
    lib = ctypes.CDLL(leg.library_path())
    fn = lib.leg_forward_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    lib.leg_last_error.restype = ctypes.c_char_p
    return lib, fn


def _call(fn, plan, f, c, B, stream=None):
    return fn(plan._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(c.data_ptr()), B,
              ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)


def need_bytes(B, Kp, ldg):
    """Scratch of a batch: seven FP16 input planes, the per-function scales and
    G (double-float pairs), each region rounded up to 256 bytes."""
    a = lambda x: (x + 255) // 256 * 256
    return 7 * a(2 * B * Kp) + a(4 * B) + a(8 * B * ldg)


@pytest.mark.parametrize("N,M,K,B", [(40, 128, 97, 37), (512, 2048, 1025, 300)])
def test_noalloc_matches_leg_forward_twice(leg, N, M, K, B):
    lib, fn = _abi(leg)
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    rng = np.random.default_rng(K)
    stream = torch.cuda.current_stream()
    for call in range(2):   # two calls in a row, different inputs
        f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), rng)
        f = torch.from_numpy(f_np).cuda()
        ref = plan.forward(f)
        c = torch.full((B, N), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        held = leg.memory_info()
        assert _call(fn, plan, f, c, B, stream) == 0, lib.leg_last_error()
        torch.cuda.synchronize()
        assert leg.memory_info() == held   # the library allocated nothing
        if call == 1:
            # no device memory was taken by the call (the first call may load the module)
            assert torch.cuda.mem_get_info()[0] == free0
        plan.status()
        assert torch.equal(c, ref)


def test_noalloc_largest_batch_that_fits(leg):
    lib, fn = _abi(leg)
    N, M, K = 512, 2048, 1025
    plan = leg.Plan(N, M, K, 0, leg.SPLIT_FP16)
    Kp, ldg = 1056, 1056
    cap = 64 << 20
    B = 2888
    assert need_bytes(B, Kp, ldg) <= cap < need_bytes(B + 1, Kp, ldg)
    f_np, _, _ = workloads.random_chebyshev(B, K, (0.8, 0.99), np.random.default_rng(77))
    f = torch.from_numpy(f_np).cuda()
    ref = plan.forward(f)
    c = torch.full((B, N), float("nan"), dtype=torch.float32, device="cuda")
    assert _call(fn, plan, f, c, B) == 0, lib.leg_last_error()
    torch.cuda.synchronize()
    plan.status()
    assert torch.equal(c, ref)
    c1 = torch.zeros((B + 1, N), dtype=torch.float32, device="cuda")
    f1 = torch.zeros((B + 1, K), dtype=torch.float32, device="cuda")
    assert _call(fn, plan, f1, c1, B + 1) == 1
    assert "scratch" in lib.leg_last_error().decode()


def test_noalloc_rejects_batches_beyond_the_scratch(leg):
    lib, fn = _abi(leg)
    plan = leg.Plan(512, 2048, 1025, 0, leg.SPLIT_FP16)
    B = 8192     # needs about 200 MB of scratch; the array holds 64 MiB
    f = torch.zeros((B, 1025), dtype=torch.float32, device="cuda")
    c = torch.zeros((B, 512), dtype=torch.float32, device="cuda")
    assert _call(fn, plan, f, c, B) == 1
    msg = lib.leg_last_error().decode()
    assert "scratch" in msg and "67108864" in msg


def test_noalloc_rejects_other_plans(leg):
    lib, fn = _abi(leg)
    f = torch.zeros((2, 17), dtype=torch.float32, device="cuda")
    c = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    assert _call(fn, leg.Plan(16, 64, 17, 0, leg.F32), f, c, 2) == 1
    collapsed = leg.Plan(16, 64, 17, 0, leg.SPLIT_FP16, flags=leg.FLAG_COLLAPSED)
    assert _call(fn, collapsed, f, c, 2) == 4   # LEG_ERR_UNSUPPORTED
