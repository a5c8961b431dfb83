"""Ragged batches: size buckets N_b = 2^ceil(log2 N_i), M = 4 N_b,
K = min(2 N_b, 1024) + 1, Q = max(32, N_b / 8), split-FP16 plans, one grouped
persistent GEMM launch, the forward replayed as a CUDA graph.

Inputs are sampled on the device from closed forms (leg_sample_cl): a third
(1 - 2xt + t^2)^(-1/2), a third e^{ax}, a third random decaying Chebyshev
series.  Parity: sampled functions of every bucket against the oracle at the
bucket's (N, M, K, Q) -- route 2 (the same tau rule), or route 1 where the
bucket is exact (Q >= K/2 and M > N + K - 1) -- within 1e-6 of max|c|, on
8 functions of every bucket of the 10,000-function workload (the first and
last of each bucket and one of each family among them).
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


def reference(oracle, Nb, fk):
    """Oracle coefficients of the functions fk (rows) of bucket Nb."""
    N, M, K, Q = workloads.bucket_sizes(Nb)
    if 2 * Q >= K and M > N + K - 1:
        return oracle.coeffs_direct(N, (K + N) // 2 + 4, f_cl=fk)
    return oracle.coeffs_abel(N, M, Q, f_cl=fk)


def sample_bucket(lay, fam, b, per_bucket, rng):
    """Functions of bucket b to check: its first and last, one of each family
    present, the rest drawn at random, per_bucket in all (fewer if the bucket
    is smaller)."""
    idx = np.where(lay["bidx"] == b)[0]
    pick = [idx[0], idx[-1]]
    for fm in range(3):
        of = idx[fam[idx] == fm]
        if of.size:
            pick.append(of[0])
    rest = np.setdiff1d(idx, pick)
    extra = max(0, per_bucket - len(set(pick)))
    if extra and rest.size:
        pick += list(rng.choice(rest, size=min(extra, rest.size), replace=False))
    return np.array(sorted(set(int(i) for i in pick)))


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
    worst, checked = 0.0, 0
    rng = np.random.default_rng(seed + 1)
    for b, Nb in enumerate(lay["buckets"]):
        idx = sample_bucket(lay, fam, b, per_bucket, rng)
        refs = reference(oracle, Nb, np.stack([samples_of(lay, f_host, i) for i in idx]))
        for i, ref in zip(idx, refs):
            ref = ref[:n[i]]
            got = c_host[lay["out_off"][i]:lay["out_off"][i] + n[i]]
            worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
            checked += 1
    print("ragged worst error", worst, "over", checked, "functions; buckets", lay["buckets"])
    assert worst < 1e-6
    return fam, par, n, lay, plans, batch, f, c1


def test_ragged_small(leg, oracle):
    check(leg, oracle, 300, 32, 1024, 11, per_bucket=6)


def test_ragged_10000(leg, oracle):
    """The full ragged workload: 8 functions per bucket (its first and last,
    one of each family), and the one-call form leg_forward_ragged (device
    arrays) against the batch handle, bit for bit."""
    cfg = workloads.CONFIGS["ragged_10000"]
    fam, par, n, lay, plans, batch, f, c1 = check(leg, oracle, cfg["count"], cfg["Nmin"], cfg["Nmax"],
                                                  workloads.SEED_BASE + 3, per_bucket=8)
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    arrays = (dev(lay["bidx"], torch.int32), dev(n, torch.int32), dev(lay["in_off"], torch.int64),
              dev(lay["out_off"], torch.int64))
    for _ in range(3):   # first call builds and caches the batch, then graph capture and replay
        c3 = torch.full_like(c1, float("nan"))
        leg.forward_ragged(plans, *arrays, f, c3)
        torch.cuda.synchronize()
        assert torch.equal(c3, c1)


def test_ragged_one_call_follows_array_contents(leg):
    """The one-call form keys its cached batch on the arrays' contents: new
    contents at the same addresses give a new batch, not a stale one."""
    fam, par, n, lay, plans, batch, f = build(leg, 120, 32, 512, 41)
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    bidx, nt = dev(lay["bidx"], torch.int32), dev(n, torch.int32)
    io, oo = dev(lay["in_off"], torch.int64), dev(lay["out_off"], torch.int64)
    ref = torch.empty(lay["n_out"], dtype=torch.float32, device="cuda")
    batch.forward(f, ref)
    c = torch.full_like(ref, float("nan"))
    leg.forward_ragged(plans, bidx, nt, io, oo, f, c)
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
    # keep fewer coefficients per function, in place in the same tensors
    n2 = np.maximum(1, n // 2)
    out2 = np.concatenate([[0], np.cumsum(n2)[:-1]]).astype(np.int64)
    nt.copy_(dev(n2, torch.int32))
    oo[:] = dev(out2, torch.int64)
    c2 = torch.full((int(n2.sum()),), float("nan"), dtype=torch.float32, device="cuda")
    leg.forward_ragged(plans, bidx, nt, io, oo, f, c2)
    torch.cuda.synchronize()
    r, g = ref.cpu().numpy(), c2.cpu().numpy()
    for i in range(len(n)):
        assert np.array_equal(g[out2[i]:out2[i] + n2[i]], r[lay["out_off"][i]:lay["out_off"][i] + n2[i]])


def test_ragged_autotune_keeps_results(leg, tmp_path, monkeypatch):
    """The timed tile choice of the grouped GEMM leaves every coefficient
    unchanged, is stored in LEG_TUNE_CACHE and reused by a new batch."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LEG_TUNE_CACHE", str(cache))
    fam, par, n, lay, plans, batch, f = build(leg, 600, 32, 4096, 43)
    ref = torch.empty(lay["n_out"], dtype=torch.float32, device="cuda")
    batch.forward(f, ref)
    torch.cuda.synchronize()
    for tn in (128, 96, 64, 16):
        batch.set_tile(tn)
        assert batch.tile_info()["tn"] == tn
        c = torch.full_like(ref, float("nan"))
        batch.forward(f, c)
        torch.cuda.synchronize()
        assert torch.equal(c, ref), tn
    c = torch.empty_like(ref)
    tn = batch.autotune(f, c)
    assert 64 <= tn <= 128 and tn % 16 == 0
    assert torch.equal(c, ref)
    ms = batch.forward_profiled(f, c)
    assert all(v > 0 for v in ms)
    assert torch.equal(c, ref)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and lines[0].startswith("ragged|") and lines[0].split()[1] == str(tn)
    batch2 = leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"])
    assert batch2.tile_info()["tn"] == tn
    batch.status()


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
