"""bench.py host logic on CPU: the N > 1 cross-rank helpers (world-size-2 gloo
ranks) and the CPU-oracle arm.

bench.py runs one independent compression job per GPU (weak scaling, no
collective in the data path); across ranks it only takes the slowest rank's
time (all-reduce MAX) and reports the whole job's throughput.  These tests
drive exactly those helpers with the gloo backend, two processes, no GPU.
"""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tmax = bench.max_over_ranks(times[rank], dist, "cpu")
        value = bench.job_throughput(world, 5, tmax)
        seed = bench.rank_seed(1000, rank)
        out.put((rank, tmax, value, seed))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_single_rank_helpers():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_throughput(1, 5, 2.5) == pytest.approx(2.0)
    assert bench.rank_seed(7, 0) == 7


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    times = [1.25, 2.0]  # rank 1 is the slow one
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every rank sees the slowest rank's time and the same whole-job throughput
    assert [r[1] for r in res] == [2.0, 2.0]
    assert [r[2] for r in res] == pytest.approx([2 * 5 / 2.0] * 2)
    # the two replicas are independent jobs (distinct test-matrix seeds)
    assert res[0][3] != res[1][3]


def test_oracle_sample_of_the_reference_arm_runs_on_cpu():
    """bench.py's CPU-oracle arm (the reference line and the cpu_baseline key)
    on a small job: a positive throughput estimate, the cores it used, and a
    description of the bounded sample."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import hm_workloads as W
    out = bench.cpu_baseline(W.torus_laplace(n=3000, tol=1e-6, r=32), rows_per_level=5)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] >= 1
    assert out["seconds_estimate"] > 0 and "lower bound" in out["sample"]
