"""The split-FP16 path on the hardest members of the input families.

The split's error grows with the transform's amplification (about 2N/sqrt(M)
for white errors in G) and with how little of the input fits in its leading
slice: a peaked function such as (1 - 2xt + t^2)^(-1/2) with t near 1 is
large only near x = 1, so most of its samples keep few bits in F0.  The
largest ragged bucket (N = 8192, M = 32768, K = 1025, Q = 1024) with
t = 0.95 (the top of the ragged family's range) and e^{ax} with |a| = 20
is the worst case of the workloads; the headline plan (N = 512, M = 2048,
K = 1025) is checked on the same families.  Parity: route 2 of the oracle at
the plan's (N, M, K, Q) (the same discrete map, Eqs. 2.4, 2.5 and the
quadrature after Eq. 2.14), within 1e-6 of max|c| per function.
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


def family_samples(K):
    rng = np.random.default_rng(17)
    f = [workloads.closed_form_samples(0, t, K) for t in (0.9, 0.95)]
    f += [workloads.closed_form_samples(1, a, K) for a in (-20.0, 20.0)]
    f.append(workloads.closed_form_samples(2, 0.0, K, rng.standard_normal(K) * 0.99 ** np.arange(K)))
    return np.array(f).astype(np.float32)


def errors(leg, oracle, N, M, K, Q):
    f = family_samples(K)
    plan = leg.Plan(N, M, K, Q, leg.SPLIT_FP16)
    c = plan.forward(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    plan.status()
    ref = oracle.coeffs_abel(N, M, plan.Q, f_cl=f.astype(np.float64))
    c = c.double().cpu().numpy()
    return np.max(np.abs(c - ref), 1) / np.max(np.abs(ref), 1)


def test_largest_ragged_bucket_extremes(leg, oracle):
    e = errors(leg, oracle, *workloads.bucket_sizes(8192))
    print("N=8192 bucket, t=0.9, 0.95, a=-20, 20, rho=0.99:", e)
    assert np.all(e < 1e-6)


def test_headline_plan_extremes(leg, oracle):
    e = errors(leg, oracle, 512, 2048, 1025, 0)
    print("N=512 M=2048 K=1025, t=0.9, 0.95, a=-20, 20, rho=0.99:", e)
    assert np.all(e < 1e-6)
