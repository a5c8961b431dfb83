"""Ragged batches: size buckets N_b = 2^ceil(log2 N_i), M = 4 N_b,
K = min(2 N_b, 1024) + 1, Q = max(32, N_b / 8), split-FP16 plans, one grouped
persistent GEMM launch, the forward replayed as a CUDA graph.

Inputs are sampled on the device from closed forms (leg_sample_cl): a third
(1 - 2xt + t^2)^(-1/2), a third e^{ax}, a third random decaying Chebyshev
series.  Parity: sampled functions of every bucket against the oracle at the
bucket's (N, M, K, Q) -- route 2 (the same tau rule), or route 1 where the
bucket is exact (Q >= K/2 and M > N + K - 1) -- within 1e-6 of max|c|.
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


def build(leg, count, Nmin, Nmax, seed):
    rng = np.random.default_rng(seed)
    fam, par, n = workloads.ragged_spec(count, rng, Nmin, Nmax)
    lay = workloads.ragged_layout(fam, par, n, rng)
    plans = [leg.Plan(*workloads.bucket_sizes(Nb), dtype=leg.SPLIT_FP16) for Nb in lay["buckets"]]
    batch = leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"])
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    f = torch.empty(lay["n_in"], dtype=torch.float32, device="cuda")
    leg.sample_cl(dev(fam, torch.int32), dev(par, torch.float64), dev(lay["K"], torch.int32),
                  dev(lay["in_off"], torch.int64), f, coef=dev(lay["coef"], torch.float64),
                  coef_off=dev(lay["coef_off"], torch.int64))
    return fam, par, n, lay, plans, batch, f


def samples_of(lay, f_host, i):
    o, K = lay["in_off"][i], lay["K"][i]
    return f_host[o:o + K].astype(np.float64)


def reference(oracle, lay, Nb, fk):
    N, M, K, Q = workloads.bucket_sizes(Nb)
    if 2 * Q >= K and M > N + K - 1:
        return oracle.coeffs_direct(N, (K + N) // 2 + 4, f_cl=fk[None])[0]
    return oracle.coeffs_abel(N, M, Q, f_cl=fk[None])[0]


def check(leg, oracle, count, Nmin, Nmax, seed, per_bucket):
    fam, par, n, lay, plans, batch, f = build(leg, count, Nmin, Nmax, seed)
    c1 = torch.full((lay["n_out"],), float("nan"), dtype=torch.float32, device="cuda")
    c2 = torch.full((lay["n_out"],), float("nan"), dtype=torch.float32, device="cuda")
    batch.forward(f, c1)       # direct
    batch.forward(f, c2)       # captured graph
    batch.forward(f, c2)       # graph replay
    torch.cuda.synchronize()
    batch.status()
    assert torch.isfinite(c1).all()
    assert torch.equal(c1, c2)
    f_host = f.cpu().numpy()
    c_host = c1.cpu().numpy()
    # the device sampler against the host closed forms (FP64 -> FP32)
    for i in range(0, count, max(1, count // 25)):
        ref = workloads.closed_form_samples(fam[i], par[i], lay["K"][i],
                                            lay["coef"][lay["coef_off"][i]:lay["coef_off"][i] + lay["K"][i]])
        got = samples_of(lay, f_host, i)
        assert np.max(np.abs(got - ref)) <= 2e-7 * np.max(np.abs(ref))
    worst = 0.0
    for b, Nb in enumerate(lay["buckets"]):
        idx = np.where(lay["bidx"] == b)[0][:per_bucket]
        for i in idx:
            ref = reference(oracle, lay, Nb, samples_of(lay, f_host, i))[:n[i]]
            got = c_host[lay["out_off"][i]:lay["out_off"][i] + n[i]]
            worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    print("ragged worst error", worst, "buckets", lay["buckets"])
    assert worst < 1e-6


def test_ragged_small(leg, oracle):
    check(leg, oracle, 300, 32, 1024, 11, per_bucket=2)


def test_ragged_10000(leg, oracle):
    cfg = workloads.CONFIGS["ragged_10000"]
    check(leg, oracle, cfg["count"], cfg["Nmin"], cfg["Nmax"], workloads.SEED_BASE + 3, per_bucket=1)


def test_ragged_inside_a_caller_capture(leg):
    """Called while the caller's stream is capturing, the batch's launches
    (the transforms on their parallel branches included) join the caller's
    graph; replaying it gives the direct launches' coefficients bit for bit."""
    fam, par, n, lay, plans, batch, f = build(leg, 200, 32, 2048, 23)
    ref = torch.empty(lay["n_out"], dtype=torch.float32, device="cuda")
    batch.forward(f, ref)
    torch.cuda.synchronize()
    c = torch.full((lay["n_out"],), float("nan"), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.forward(f, c)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    batch.status()
    assert torch.equal(c, ref)
