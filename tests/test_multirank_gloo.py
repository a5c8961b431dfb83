"""The N > 1 host logic of bench.py on CPU, with two gloo ranks.

The method's functions are independent (each c_n depends on its own f only),
so N processes run N replicas on disjoint batches with no exchange on the data
path: each rank draws its own seeded batch, times its own steps, and the
whole-job rate is all ranks' coefficients over the slowest rank's time.  These
tests run that logic (seeding per rank, max over ranks, whole-job rate) in two
real gloo processes; no GPU is involved.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import workloads

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's batch: the seeded inputs of its own salt
        f = workloads.workload_inputs("cheb_b4096_k1025_n512_m2048", B=4, salt=rank)
        gathered = [torch.zeros(4 * 1025, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(f.astype(np.float64).ravel()))
        # the rank's step time: different on every rank
        t_rank = 10.0 + 7.0 * rank
        t_max = bench.max_over_ranks(torch, dist, t_rank, "cpu")
        rate = bench.whole_job_rate(world, 4096 * 512, t_max)
        out[rank] = (t_max, rate, [g.numpy().copy() for g in gathered])
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0] * world, codes
        return dict(out)


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_batches_and_take_the_slowest_time():
    world = 2
    res = _run(world)
    assert sorted(res) == [0, 1]
    t0, rate0, batches0 = res[0]
    t1, rate1, batches1 = res[1]
    # every rank sees the same slowest step time and the same whole-job rate
    assert t0 == t1 == 17.0
    assert rate0 == rate1 == pytest.approx(world * 4096 * 512 / 17e-3)
    # the ranks' batches are distinct, and each is what its seed gives on its own
    assert not np.array_equal(batches0[0], batches0[1])
    for r in range(world):
        np.testing.assert_array_equal(batches0[r], batches1[r])
        import workloads
        mine = workloads.workload_inputs("cheb_b4096_k1025_n512_m2048", B=4, salt=r)
        np.testing.assert_array_equal(batches0[r], mine.astype(np.float64).ravel())


def test_single_process_rate_is_units_over_time():
    import torch

    import bench
    assert bench.max_over_ranks(torch, None, 3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 4096 * 512, 0.125) == pytest.approx(4096 * 512 / 1.25e-4)
