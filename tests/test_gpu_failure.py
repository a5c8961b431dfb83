"""Failure detection without a GPU fault: the tensor-core kernels bound every
mbarrier wait by a cycle budget.  With a budget of zero cycles the waits of
the MMA and epilogue roles expire at once; the kernel records LEG_ERR_TIMEOUT
in the plan's status word, drains its own TMA copies and MMAs, releases TMEM
and returns.  The context stays usable and a normal call afterwards is exact.
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


def test_expired_wait_sets_timeout_status(leg):
    plan = leg.Plan(40, 128, 97, 0, leg.SPLIT_FP16)
    f_np, _, _ = workloads.random_chebyshev(37, 97, (0.8, 0.99), np.random.default_rng(0))
    f = torch.from_numpy(f_np).cuda()
    ref = plan.forward(f)
    plan.status()                       # clean
    plan.set_wait_limit(0)
    plan.forward(f)
    with pytest.raises(leg.LegError) as e:
        plan.status(reset=True)
    assert e.value.code == 5            # LEG_ERR_TIMEOUT
    plan.set_wait_limit(2_000_000_000)
    c = plan.forward(f)
    plan.status()                       # clean again: the context survived
    assert torch.equal(c, ref)


def test_host_side_argument_errors_launch_nothing(leg):
    plan = leg.Plan(16, 64, 17, 0, leg.SPLIT_FP16)
    with pytest.raises(leg.LegError) as e:
        leg.Plan(16, 64, 17, 0, 7)
    assert e.value.code == 1
    with pytest.raises(ValueError):
        plan.forward(torch.zeros((2, 16), dtype=torch.float32, device="cuda"))
    plan.status()
