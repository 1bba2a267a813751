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


def test_clock_sampler_keeps_the_timed_window_and_reports_throttling(monkeypatch):
    """The bench's clock record (read through NVML in a thread): samples outside the timed region
    and one sampling period around it are dropped, the SM clock is their median, and any throttle
    reason seen inside is reported; with no NVML the record says so."""
    import time
    import bench

    class FakeNvml:
        def __init__(self):
            self.calls = 0

        def handle(self, bus, index):
            return "h"

        def sample(self, h):
            self.calls += 1
            slow = ["sw_power_cap"] if self.calls == 3 else []
            return 1900.0 + self.calls, 2032.0, slow

    fake = FakeNvml()
    monkeypatch.setattr(bench, "_nvml", lambda: fake)
    monkeypatch.setattr(bench.ClockSampler, "PERIOD_S", 0.01)
    with bench.ClockSampler(0) as c:
        time.sleep(0.08)
    s = c.summary()
    assert s["samples"] >= 3 and s["sm_max_mhz"] == 2032.0
    assert 1900.0 < s["sm_mhz"] < 1900.0 + fake.calls + 1
    assert s["reasons"] == ["sw_power_cap"]
    early = c.t0 - 1.0  # a sample from well before the region is not counted
    c.rows.insert(0, (early, 100.0, 2032.0, ["hw_slowdown"]))
    assert c.summary()["reasons"] == ["sw_power_cap"] and c.summary()["sm_mhz"] > 1000.0
    monkeypatch.setattr(bench, "_nvml", lambda: None)
    with bench.ClockSampler(0) as c2:
        pass
    assert c2.summary()["reasons"] == ["unavailable"]
