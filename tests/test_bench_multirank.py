"""Multi-rank logic of the benchmark on CPU (gloo, two ranks): each rank runs its own replica,
the job time is the slowest rank's, and throughput counts every rank's frames."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, world, "cpu")
    out[rank] = (t, bench.job_throughput(world, 10, t))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_frames():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, 2 * 10 / 2.5)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(1, 20, 0.5) == pytest.approx(40.0)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    # under torchrun the oracle arm runs and prints on rank 0 alone; another rank returns at once
    import argparse
    import time

    import bench
    monkeypatch.setattr(bench, "oracle_setup", lambda f: pytest.fail("rank 1 must not run the oracle"))
    t0 = time.perf_counter()
    bench.run_reference(argparse.Namespace(steps=3, warmup=3, seed=0), 2, 1)
    assert time.perf_counter() - t0 < 1.0 and capsys.readouterr().out == ""
