"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): the
timing reduction takes the slowest rank, the whole-job rate counts every
rank's units, and the reference arm runs on rank 0 alone."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 40.0][rank]
        slow = bench.max_over_ranks(ms, dist)
        dist.barrier()
        q.put((rank, slow, bench.whole_job_rate(world, 1000.0, slow)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, slow, rate in got:
        assert slow == 40.0                             # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 0.040)  # units of both ranks per second


def test_single_process_and_reference_arm_off_rank_0():
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_rate(1, 500.0, 250.0) == pytest.approx(2000.0)

    class Args:
        steps, warmup = 1, 3
    assert bench.run_reference(Args(), rank=1, world=2) == 0   # no work, no line


def test_all_cores_oracle_timing_counts_every_sampled_vertex():
    """The all-cores CPU baseline deals the sampled start vertices to spawned
    processes; with time to finish, their 2-paths add up to the single-process
    walk over all vertices (the oracle's own count of the same loops)."""
    import numpy as np

    import oracle as O
    from paper_1801_00338_gb300 import synth
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)
    dU = np.bincount(g.u, minlength=g.nU).astype(np.float64)
    dV = np.bincount(g.v, minlength=g.nV).astype(np.float64)
    side = 1 if (dU * dU).sum() < (dV * dV).sum() else 0
    n = g.nV if side else g.nU
    val, cores, desc = bench.oracle_sample_all_cores(g, side, budget_s=30.0, cores=2)
    assert cores == 2 and val > 0
    P = O.Prepared(g.u, g.v, g.nU, g.nV, side)
    _, paths = P.count(np.arange(n, dtype=np.uint32))
    P.close()
    assert f"{n} of {n} start vertices" in desc
    assert f" {paths} 2-paths" in desc
