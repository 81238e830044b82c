"""Multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

The bench runs one independent replica per GPU; the only cross-rank steps are
the barrier and the max over ranks of the timed region, and rank 0 alone
prints. These tests run those steps with world_size 2 over gloo."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    m = bench.max_over_ranks(times[rank], world, "cpu")
    out[rank] = (m, bench.job_throughput(10, world, m / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_two_gloo_ranks():
    world = 2
    times = [120.0, 150.0]                      # ms of the timed region per rank
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        m, v = res[r]
        assert m == 150.0                        # every rank sees the slowest rank's time
        assert abs(v - world * 10 / 0.150) < 1e-9


def _ref_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        workload = "fp64_fullbox_32x32x64"
        steps, warmup, cpu_budget, tol = 1, 0, 2.0, 1e-8
    line = bench.reference_arm(A, rank, world)
    out[rank] = None if line is None else line["impl"]
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.slow
def test_reference_arm_runs_on_rank_zero_only():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_ref_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == "reference" and res[1] is None
