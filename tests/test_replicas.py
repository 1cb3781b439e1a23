"""The multi-GPU path of bench.py is replicas: every rank advances its own copy
of the workload and the job's time is the slowest rank's.  These tests run
that host logic as two gloo ranks on the CPU (no GPU involved)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    # per-rank timings differ; every rank must agree on the slowest
    job_ms = bench.max_over_ranks(10.0 + 5.0 * r, w)
    out[r] = (job_ms, bench.whole_job_mlups(1000, 4, w, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of a threaded test process
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # all ranks' node updates (2 x 1000 x 4) over the slowest rank's 15 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    # rank 1 of the reference arm returns before doing any work
    class A:
        n, steps, warmup = 256, 1, 0
    assert bench.run_reference(A()) is None

