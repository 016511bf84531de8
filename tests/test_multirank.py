"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks.

The method's single-system step does not shard, so N GPUs run N independent
replicas (different seeds); the host logic is what crosses ranks: the
slowest replica's time is the job's, whole-job throughput counts every
replica's steps, each replica draws its own inputs, and only rank 0 runs
the reference arm.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r measured 10 + r ms for the timed steps, 5 - r for steady state
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 7.0], "cpu")
    x, v, L, tag, rg = bench.workload_inputs(seed=rank)
    out.put((rank, got, float(x[:8].sum()), tag[:4].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, g0, s0, t0), (_, g1, s1, t1) = res
    assert g0 == g1 == [11.0, 5.0, 7.0]          # element-wise maximum, identical on every rank
    assert s0 != s1 or t0 != t1                  # replicas draw different inputs


def test_job_rate_and_single_process_fallback():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_rate(4, 200, 100.0) == pytest.approx(8000.0)
    assert bench.max_over_ranks([3.0, 1.5], "cpu") == [3.0, 1.5]  # no process group: unchanged


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0

    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""
