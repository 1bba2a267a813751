#!/usr/bin/env python3
"""G-ICP tracking benchmark on one B300: frames/s of the whole per-frame hot path.

Workload (Replica-shaped single frame): a seeded synthetic 1200x680 depth image
(fx = fy = 600, cx = 599.5, cy = 339.5, depth noise sigma = 1 mm * z^2), stride 2
(~204k source points), registered against a map of ~2.04M Gaussians built from
10 prior views of the same room; initial pose offset 2 deg / 2 cm.  A step is
one frame through the C ABI: depth -> points, source k-NN covariances (plane
regularisation, scale aligning p = 1.5), map-index rebuild, and the
Gauss-Newton loop with per-iteration nearest-neighbour search.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica of
the workload (independent frames, no data-path collective: weak scaling).

The default run's line also carries "workloads": compact records of the other forms of the
path, each measured in the same run: "sharded" (one frame's registration split across the ranks,
one all-gather of 30 float64 sums per Gauss-Newton iteration; strong scaling), and at N = 1
"batch" (64 independent pairs in one persistent launch), "sequence" (the tracking loop with the
paper's keyframe policy over a 120-frame TUM-shaped sequence) and "surrogate" (learned covariances
on their 500-frame held-out sequence, ATE against the plain form on the same run).
--no-workloads skips them; --workload X runs one of them alone at full size.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G-ICP tracking frames/s (1200x680 frame, ~204k points, vs 2.04M-Gaussian map)"
WORKLOAD = "replica-shaped frame: 1200x680 depth, stride 2 (~204k pts), 2.04M-Gaussian map from 10 views, offset 2deg/2cm"
STRIDE, Z_MIN, Z_MAX = 2, 0.1, 10.0
K_NN, EPS, P_ALIGN = 20, 1e-3, 1.5
MAX_DIST, MAX_ITERS, TOL = 0.1, 30, 1e-6
# algorithmic bytes the method must move per unit (the roofline numerators):
BYTES_PER_POINT_ITER = 72      # x 12 + C_s 24 + mu 12 + C_t 24
BYTES_PER_POINT_COV = 40       # read x 12 + z 4, write C 24
BYTES_PER_MAP_GAUSSIAN = 132  # means for the bounds 12, means for the keys 12 + keys 4, one sort pass 4 + 8,
                              # gather: index 4 + mean and cov 36 read, packed 16 + 32 written; cell keys 4
REGSTATE_BYTES = 616 + 4       # registration state record (pose, H, b, cost, iters, status) + point count per frame
L2_FLUSH_BYTES = 256 << 20
GN_BODY_ITERS = 4              # iteration launches per pass of the Gauss-Newton graph (gicp.cu)
# kernels launched per timed step (counted from the ncu launch list of this workload):
LAUNCHES_MAP_REBUILD = 14  # count reset 1, bbox + quantise 1, Morton keys + digit counts 1, radix sort 4,
                           # gather + leaf boxes 1, box levels 3, cell table size/clear/fill 3
LAUNCHES_FRAME = 13        # a1 2 (counts, write), source index 5 (counts, write, gather + leaf boxes, 2 box
                           # levels), k-NN covariances 4 (9x9 window, 25x25 window, tree, reorder), GN seed 1,
                           # GN set-up 1; plus one Gauss-Newton launch per iteration (plain-launch mode: one
                           # more set-up launch)
# DRAM bytes per gicp_iter_kernel launch (read + write, mean over the iterations of one frame of this
# workload, ncu dram__bytes_read.sum + dram__bytes_write.sum), valid for the CUDA sources whose
# SHA-256 is given; reported as null once any of them has changed.
GN_TRAFFIC = {"bytes_per_launch": 28788531,
              "sources_sha256": "9377b331aa02713307c69e0ddddbb5e30eae5f8607f91cf871ff1a794fe2abf4"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["frame", "batch", "sequence", "surrogate", "sharded"], default="frame",
                    help="frame: the tracking step (default); batch: batched registration of independent pairs; "
                         "sequence: the tracking loop with keyframes over a TUM-shaped sequence (latency p50/p99); "
                         "surrogate: the tracking loop with learned covariances on their held-out sequence; "
                         "sharded: one frame's registration split across the ranks")
    ap.add_argument("--no-workloads", action="store_true",
                    help="frame workload only: skip the compact batch / sequence / surrogate / sharded records "
                         "the default run adds to its line")
    ap.add_argument("--frames", type=int, default=None,
                    help="sequence length (default 300 for sequence, 500 for surrogate)")
    ap.add_argument("--pairs", type=int, default=64)
    ap.add_argument("--shape", default=None,
                    help="BUCKET,CELL_M,COOP[,BLOCK]: use this map-index shape, cooperative-walk threshold and "
                         "Gauss-Newton block size instead of the autotuner's choice (e.g. for profiling runs)")
    ap.add_argument("--gn-plain", action="store_true",
                    help="launch each Gauss-Newton iteration as a plain kernel (not a graph node), for "
                         "launch-listing profilers; same results")
    args = ap.parse_args()
    if args.frames is None:
        args.frames = 500 if args.workload == "surrogate" else 300
    return args


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class _Nvml:
    """The few NVML reads the clock sampler needs, through ctypes on the driver's libnvidia-ml
    (read-only queries; nothing is set).  A polling nvidia-smi process slowed this process's own
    CUDA calls (host time per tracked frame +0.2 to +1.4 ms) for a while after it had exited, so
    the clocks are read in-process from a thread instead."""

    CLOCK_SM = 1
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40}

    def __init__(self):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def handle(self, pci_bus_id: str | None, index: int):
        C = self.C
        h = C.c_void_p()
        if pci_bus_id and self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), C.byref(h)) == 0:
            return h
        if self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(h)) == 0:
            return h
        raise RuntimeError("no NVML handle for the device")

    def sample(self, h):
        C = self.C
        sm, mx, bits = C.c_uint(), C.c_uint(), C.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(h, self.CLOCK_SM, C.byref(sm)) != 0 or \
                self.lib.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM, C.byref(mx)) != 0 or \
                self.reasons_fn(h, C.byref(bits)) != 0:
            raise RuntimeError("NVML query failed")
        return float(sm.value), float(mx.value), [k for k, b in self.REASON_BITS.items() if bits.value & b]


_NVML = None


def _nvml():
    """The process's NVML reader, made once (None where NVML cannot be loaded)."""
    global _NVML
    if _NVML is None:
        try:
            _NVML = _Nvml()
        except Exception as e:
            _NVML = False
            print(f"bench: NVML unavailable for clock sampling ({e!r})", file=sys.stderr)
    return _NVML or None


class ClockSampler:
    """SM clock, its maximum and the throttle reasons, sampled every 50 ms by a thread of this
    process (NVML) during the timed region; the summary keeps the samples from the region and one
    sampling period on either side of it."""

    PERIOD_S = 0.05

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []  # (time, sm_mhz, max_mhz, reasons)
        self.t0 = self.t1 = None
        self.thread = None
        self.handle = None
        self.error = None
        nv = _nvml()
        if not nv:
            self.error = "NVML unavailable"
            return
        try:
            import torch
            p = torch.cuda.get_device_properties(gpu_index)
            bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
        except Exception:
            bus = None
        try:
            self.handle = nv.handle(bus, gpu_index)
        except Exception as e:
            self.error = repr(e)

    def _sample(self):
        sm, mx, reasons = _nvml().sample(self.handle)
        self.rows.append((time.time(), sm, mx, reasons))

    def _loop(self):
        while not self.stop:
            try:
                self._sample()
            except Exception as e:
                self.error = f"sample: {e!r}"
                return
            time.sleep(self.PERIOD_S)

    def __enter__(self):
        import threading
        self.stop = False
        if self.handle is not None:
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            deadline = time.time() + 1.0
            while not self.rows and time.time() < deadline:
                time.sleep(0.001)
        self.t0 = time.time()
        return self

    def __exit__(self, *exc):
        self.t1 = time.time()
        if self.thread:
            time.sleep(self.PERIOD_S * 1.2)  # one more sample after the region
            self.stop = True
            self.thread.join(timeout=5)

    def summary(self):
        pad = self.PERIOD_S * 1.5
        rows = [r for r in self.rows if self.t0 - pad <= r[0] <= self.t1 + pad]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "error": self.error}
        return {"sm_mhz": float(np.median([r[1] for r in rows])), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted({x for r in rows for x in r[3]}), "samples": len(rows),
                "period_ms": int(self.PERIOD_S * 1e3), "window_ms": round((self.t1 - self.t0) * 1e3, 1),
                "source": "NVML"}


# the sources the Gauss-Newton kernel's DRAM traffic depends on: the kernel and its search, the index
# it walks and the parameters the library sets for it
GN_SOURCES = ("api.cu", "common.cuh", "gicp.cu", "index.cu", "internal.h", "traverse.cuh")


def sources_sha256() -> str:
    """SHA-256 over the Gauss-Newton kernel's CUDA sources (names and contents, sorted by name)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2403_12550_b300", "csrc")
    for name in sorted(GN_SOURCES):
        h.update(name.encode())
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest of every rank's x (the job's time is its slowest replica's); x itself at N=1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, total_s: float) -> float:
    """Whole-job frames/s: every rank tracks `steps` frames of its own replica in `total_s` (the max)."""
    return world * steps / total_s


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- our arm

def build_map_gpu(g, ctx, f, torch):
    """Map Gaussians from the prior views with the library itself (keyframe insertion path)."""
    intr = f["intr"].as_array()
    cp = g.CovParams(K_NN, EPS, g.PLANE, P_ALIGN)
    means, covs = [], []
    for d, P in zip(f["view_depths"], f["view_poses"]):
        pts, z = g.gsicp_depth_to_points(ctx, torch.from_numpy(d).cuda(), intr, STRIDE, Z_MIN, Z_MAX)
        pts, z = pts.clone(), z.clone()
        c = g.gsicp_source_covariances(ctx, pts, z, cp)
        mw, cw = g.gsicp_transform_gaussians(P, pts, c)
        means.append(mw)
        covs.append(cw)
    return torch.cat(means).contiguous(), torch.cat(covs).contiguous()


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    import paper_2403_12550_b300 as g
    from synth import frame_config2

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    f = frame_config2(args.seed)
    ctx = g.Context()
    if args.gn_plain:
        g.gsicp_ctx_set_gn_launch_mode(ctx, g.GN_PLAIN)
    means, covs = build_map_gpu(g, ctx, f, torch)
    intr = f["intr"].as_array()
    cp = g.CovParams(K_NN, EPS, g.PLANE, P_ALIGN)
    rp = g.RegParams(MAX_DIST, MAX_ITERS, TOL, TOL, 6)
    depth_dev = torch.from_numpy(f["depth"]).cuda()
    # the map index's shape, the context's cooperative-walk threshold and its Gauss-Newton block size,
    # picked by the autotuner on this frame (untimed; every shape and threshold gives the same poses
    # bit for bit; the block size fixes the order of the sums, so poses agree to rounding)
    from paper_2403_12550_b300.autotune import tune_frame
    if args.shape:
        b_, c_, k_, *bs_ = args.shape.split(",")
        tune = dict(bucket=int(b_), cell=float(c_), coop=int(k_), block=int(bs_[0]) if bs_ else 256, ms={},
                    coop_ms={}, block_ms={})
        g.gsicp_ctx_set_coop_walks(ctx, tune["coop"])
        g.gsicp_ctx_set_gn_block(ctx, tune["block"])
    else:
        tune = tune_frame(ctx, depth_dev, intr, STRIDE, Z_MIN, Z_MAX, cp, means, covs, f["T0"], rp,
                          key=f"frame-{f['depth'].shape}-{means.shape[0]}")
    m = g.gsicp_build_map_index(ctx, means, covs, tune["bucket"], tune["cell"])
    n_map = m.size
    depth_host = torch.from_numpy(f["depth"]).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        # a1 -> a2+a3 -> a5-a7 for one frame
        return g.gsicp_track_frame(ctx, depth_dev, intr, STRIDE, Z_MIN, Z_MAX, cp, m, f["T0"], rp)

    def rebuild():
        # a4: rebuild the map index over the map's resident Gaussians (no allocation)
        g.gsicp_map_rebuild(ctx, m)

    # warm-up (also instantiates the Gauss-Newton graph and grows every scratch buffer)
    for _ in range(args.warmup):
        rebuild()
        r = step()
    # ---- end-to-end through the host-buffer entry point (H2D depth + D2H results inside), before
    # the clock-sampled device-timed steps: reading the clocks while this process runs CUDA calls
    # (NVML in a thread, or a polling nvidia-smi) slows those calls for a while afterwards
    e2e_ms = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rebuild()
        rh = g.gsicp_track_frame_host(ctx, depth_host, intr, STRIDE, Z_MIN, Z_MAX, cp, m, f["T0"], rp)
        t1 = time.perf_counter()
        if i > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    assert np.array_equal(rh["T"], r["T"])
    e2e_s = max_over_ranks(sum(e2e_ms) / 1e3, world, "cuda")

    g.gsicp_ctx_set_timing(ctx, True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases, iters, npts = [], [], 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (not timed)
            a, b, c = ev[i]
            a.record(stream)
            torch.cuda.nvtx.range_push("map_rebuild")  # NVTX ranges: profilers can select the phases
            rebuild()                           # a4: map index over 2.04M Gaussians
            torch.cuda.nvtx.range_pop()
            b.record(stream)
            torch.cuda.nvtx.range_push("track_frame")
            r = step()                          # a1 -> a2+a3 -> a5-a7 (synchronises)
            torch.cuda.nvtx.range_pop()
            c.record(stream)
            phases.append(g.gsicp_ctx_phase_times(ctx))
            iters.append(r["iters"])
            npts = r["n_points"]
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    index_ms = [a.elapsed_time(b) for a, b, _ in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, "cuda")
    g.gsicp_ctx_set_timing(ctx, False)

    # ---- roofline of the dominant kernel, from the event-timed phases of the timed steps
    keys = ("depth_to_points", "source_index", "knn_cov", "gauss_newton")
    ph = {k: float(np.mean([p[k] for p in phases])) for k in keys}
    ph["map_index"] = float(np.mean(index_ms))
    it_mean = float(np.mean(iters))
    peak, peak_kind = load_peaks()
    dominant = max(("gauss_newton", "knn_cov", "map_index", "source_index"), key=lambda k: ph[k])
    if dominant == "gauss_newton":
        per_launch_ms = ph["gauss_newton"] / max(it_mean, 1)
        alg = npts * BYTES_PER_POINT_ITER
        kname = "gicp_iter_kernel"
    elif dominant == "knn_cov":
        per_launch_ms, alg, kname = ph["knn_cov"], npts * BYTES_PER_POINT_COV, "knn_cov_kernel"
    elif dominant == "map_index":
        per_launch_ms, alg, kname = ph["map_index"], n_map * BYTES_PER_MAP_GAUSSIAN, "map index build"
    else:
        per_launch_ms, alg, kname = ph["source_index"], npts * 64, "source index build"
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    if kname == "gicp_iter_kernel" and GN_TRAFFIC["bytes_per_launch"] and \
            GN_TRAFFIC["sources_sha256"] == sources_sha256():
        traffic = GN_TRAFFIC["bytes_per_launch"]
    # the Gauss-Newton graph runs its iteration launches GN_BODY_ITERS at a time (the ones after
    # convergence exit at once); in plain-launch mode every frame launches max_iters of them
    launches = int(sum(LAUNCHES_MAP_REBUILD + LAUNCHES_FRAME +
                       (MAX_ITERS + 1 if args.gn_plain else GN_BODY_ITERS * -(-int(it) // GN_BODY_ITERS))
                       for it in iters))
    K = args.steps
    out = {
        "metric": METRIC, "value": job_throughput(world, K, total_s), "unit": "frames/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(npts, n_map, world),
                   "autotuned": {"index_bucket": tune["bucket"], "index_cell_m": tune["cell"],
                                 "coop_walks": tune["coop"], "gn_block": tune["block"],
                                 "frame_ms": {f"{b}/{c * 1e3:g}mm": round(v, 4) for (b, c), v in tune["ms"].items()},
                                 "coop_frame_ms": {str(c): round(v, 4) for c, v in tune["coop_ms"].items()},
                                 "block_frame_ms": {str(c): round(v, 4) for c, v in tune["block_ms"].items()}}},
        "gn_iters_mean": it_mean,
        "point_iters_per_s": world * float(npts) * sum(iters) / total_s,
        "phases_ms": {k: round(v, 4) for k, v in ph.items()},
        "tracking_only_frames_per_s": world * K / (total_s - sum(index_ms) / 1e3),
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": int(alg), "avg_launch_ms": per_launch_ms},
        # the host-buffer call uploads the rows a1 samples: ceil(H / stride) rows of W floats
        "e2e": {"value": job_throughput(world, K, e2e_s), "unit": "frames/s",
                "h2d_bytes_per_step": int(-(-f["depth"].shape[0] // STRIDE) * f["depth"].shape[1] * 4),
                "d2h_bytes_per_step": REGSTATE_BYTES, "ms_p50": round(float(np.median(e2e_ms)), 4),
                "ms_max": round(float(np.max(e2e_ms)), 4)},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(f, args.seed)
    m.close()
    ctx.close()
    if not args.no_workloads:
        out["workloads"] = sub_workloads(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- split registration

SHARD_METRIC = ("split G-ICP registrations/s (one 1200x680 frame, ~204k points, vs 2.04M-Gaussian map; the "
                "frame's points shared by the ranks)")


def measure_sharded(args, world, rank, local, steps: int = 20, warmup: int = 3) -> dict:
    """One registration of the benchmark frame whose points are split across the ranks
    (paper_2403_12550_b300.sharded: per iteration each rank linearises its share, the ranks
    all-gather the 30 sums, every rank solves).  Each rank builds the whole map and the frame's
    covariances once, untimed; a step is one split registration from the frame's start pose,
    timed by CUDA events on the stream (the loop synchronises every iteration), L2 flushed between
    steps.  Beside it, the same registration by gsicp_register on one rank (all points)."""
    import torch
    import torch.distributed as dist

    import paper_2403_12550_b300 as g
    from paper_2403_12550_b300.sharded import register_sharded, share
    from synth import frame_config2

    torch.cuda.set_device(local)
    f = frame_config2(args.seed)
    ctx = g.Context()
    means, covs = build_map_gpu(g, ctx, f, torch)
    m = g.gsicp_build_map_index(ctx, means, covs)
    intr = f["intr"].as_array()
    cp = g.CovParams(K_NN, EPS, g.PLANE, P_ALIGN)
    rp = g.RegParams(MAX_DIST, MAX_ITERS, TOL, TOL, 6)
    pts, _, cs = g.gsicp_frame_covariances(ctx, torch.from_numpy(f["depth"]).cuda(), intr, STRIDE, Z_MIN, Z_MAX, cp)
    pts, cs = pts.clone(), cs.clone()
    sl = share(pts.shape[0], world, rank)
    src, scov = pts[sl].contiguous(), cs[sl].contiguous()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        ms, r = [], None
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return ms, r

    split = lambda: register_sharded(ctx, src, scov, m, f["T0"], rp)
    single = lambda: g.gsicp_register(ctx, pts, cs, m, f["T0"], rp)
    timed(split, warmup)
    timed(single, warmup)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms, r = timed(split, steps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_s = max_over_ranks(sum(ms) / 1e3, world, "cuda")
    ms1, r1 = timed(single, steps)
    out = {
        "metric": SHARD_METRIC, "value": steps / total_s, "unit": "registrations/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": total_s * 1e3 / steps, "higher_is_better": True,
        "scaling": "strong", "dtype": "f32",
        "config": {"workload": f"the benchmark frame ({pts.shape[0]} points) split into {world} contiguous shares "
                               f"of its Morton-unordered point list; map replicated on every rank",
                   "collective": "all-gather of 30 float64 per rank per Gauss-Newton iteration" if world > 1 else
                                 "none (one rank)", "l2": "flushed between timed steps (256 MB write)"},
        "iters": r["iters"], "status": r["status"],
        "single_register": {"value": 1e3 / float(np.mean(ms1)), "unit": "registrations/s",
                            "ms": float(np.mean(ms1)), "iters": r1["iters"]},
        "pose_equals_single": bool(np.array_equal(r["T"], r1["T"])),
        "pose_diff_single": {"rot_rad": rot_angle(r["T"][:3, :3].T @ r1["T"][:3, :3]),
                             "trans_m": float(np.linalg.norm(r["T"][:3, 3] - r1["T"][:3, 3]))},
        "gpu_launches": steps * (int(r["rounds"]) * 2 + 16),
    }
    m.close()
    ctx.close()
    return out


def run_sharded(args, world, rank, local):
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = measure_sharded(args, world, rank, local, steps=args.steps, warmup=args.warmup)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def rot_angle(R) -> float:
    """Rotation angle of R from its antisymmetric part and trace together (atan2): arccos of the
    trace alone reads a common scale error e of nearly orthonormal matrices as sqrt(6 e)."""
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    return float(np.arctan2(0.5 * np.linalg.norm(w), 0.5 * (np.trace(R) - 1.0)))


def _pick(d: dict, keys) -> dict:
    return {k: d[k] for k in keys if k in d}


def sub_workloads(args, world, rank, local) -> dict:
    """Compact records of the other forms of the path, for the default run's line: the split
    registration (any N), and at N = 1 the batched registration, the tracking loop over a
    TUM-shaped sequence and the learned covariances on their held-out sequence (each as its own
    --workload prints it, shortened: fewer timed steps, shorter oracle samples, a 120-frame
    sequence)."""
    import argparse
    short = argparse.Namespace(**{**vars(args), "steps": 20, "warmup": 3})
    common = ("metric", "value", "unit", "ms_per_step", "steps", "dtype", "config", "clocks", "cpu_baseline",
              "roofline", "e2e", "gpu_launches")
    w = {"sharded": _pick(measure_sharded(args, world, rank, local), common + (
        "scaling", "iters", "status", "single_register", "pose_equals_single", "pose_diff_single"))}
    if world == 1:
        w["batch"] = _pick(measure_batch(short, world, rank, local, cpu_sample_s=6.0), common + (
            "point_iters_per_s", "one_by_one", "converged"))
        w["sequence"] = _pick(measure_sequence(short, world, rank, local, 120, cpu_sample_s=8.0), common + (
            "latency_ms", "ate_m", "ate_aligned_m", "ate_first_frames", "keyframes", "mapping_keyframes",
            "map_sizes"))
        w["surrogate"] = _pick(measure_surrogate(short, world, rank, local, 500, cpu_sample_s=6.0), common + (
            "knn_frames_per_s", "latency_ms", "ate_m", "ate_knn_m", "ate_gap_m", "ate_aligned_m",
            "ate_knn_aligned_m", "surrogate_frames", "fell_back", "layer_ms"))
    return w


# ----------------------------------------------------------------------------- the oracle (CPU)

def oracle_setup(f):
    import oracle as orc
    intr = f["intr"].as_array()
    means, covs = [], []
    for d, P in zip(f["view_depths"], f["view_poses"]):
        pts, z = orc.depth_to_points(d, intr, STRIDE, Z_MIN, Z_MAX)
        pts, z = pts.astype(np.float32), z.astype(np.float32)
        c = orc.source_covariances(pts, z, k=K_NN, eps=EPS, reg_mode=orc.PLANE, p=P_ALIGN)["covs"]
        mw, cw = orc.transform_gaussians(P, pts, c)
        means.append(mw)
        covs.append(cw)
    return orc.Map(np.concatenate(means).astype(np.float32), np.concatenate(covs).astype(np.float32))


def workload_config(n_points, map_gaussians, world) -> dict:
    """The workload as both arms of the benchmark state it."""
    return {"workload": WORKLOAD, "n_points": int(n_points), "map_gaussians": int(map_gaussians), "k": K_NN,
            "reg": "plane", "eps": EPS, "p": P_ALIGN, "max_corr_dist": MAX_DIST, "parallelism": f"replicas x{world}",
            "l2": "GPU: flushed between timed steps (256 MB write); the 2.04M-Gaussian map (73 MB packed) is "
                  "re-indexed every step", "step": "a4 map-index rebuild + a1..a7"}


def oracle_frame(f, omap, frac: float = 1.0, seed: int = 0):
    """One step of the workload through the oracle, the same steps the GPU arm times: the map's
    index rebuilt (a4: the k-d tree over the map means), a1, covariances, Gauss-Newton
    registration.  With frac < 1 the registration runs on a seeded random subset of the points.
    Returns (registration result, seconds of a4 + a1 + a2/a3, seconds of the registration, seconds
    of a4 alone)."""
    import oracle as orc
    t0 = time.perf_counter()
    m = orc.Map(omap.means, omap.covs)
    t_index = time.perf_counter() - t0
    pts, z = orc.depth_to_points(f["depth"], f["intr"].as_array(), STRIDE, Z_MIN, Z_MAX)
    pts, z = pts.astype(np.float32), z.astype(np.float32)
    cs = orc.source_covariances(pts, z, k=K_NN, eps=EPS, reg_mode=orc.PLANE, p=P_ALIGN)["covs"]
    if frac < 1.0:
        sel = np.random.default_rng(seed).choice(len(pts), int(frac * len(pts)), replace=False)
        pts, cs = pts[sel], cs[sel]
    t1 = time.perf_counter()
    r = orc.register(pts, cs, m, f["T0"], MAX_DIST, MAX_ITERS, TOL, TOL, 6)
    return r, t1 - t0, time.perf_counter() - t1, t_index


def oracle_threads():
    import oracle as orc
    return orc.threads()


def orc_points(f):
    import oracle as orc
    return orc.depth_to_points(f["depth"], f["intr"].as_array(), STRIDE, Z_MIN, Z_MAX)[0]


def cpu_baseline(f, seed, sample_s: float = 10.0):
    """The oracle on this host's cores: whole steps of the same workload (map-index rebuild, a1,
    covariances, registration), repeated until about ``sample_s`` seconds have passed (at least one)."""
    import oracle as orc
    omap = oracle_setup(f)
    cores = orc.threads()
    frames, t_index, t0 = 0, 0.0, time.perf_counter()
    while True:
        r, _, _, ti = oracle_frame(f, omap)
        frames += 1
        t_index += ti
        dt = time.perf_counter() - t0
        if dt >= sample_s:
            break
    # one more step on a single thread
    orc.set_threads(1)
    try:
        t1 = time.perf_counter()
        oracle_frame(f, omap)
        t_single = time.perf_counter() - t1
    finally:
        orc.set_threads(cores)
    return {"value": frames / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "tracking_only_frames_per_s": frames / (dt - t_index),
            "single_thread": {"value": 1.0 / t_single, "unit": "frames/s", "sample": "1 full step on one thread"},
            "sample": f"{frames} full steps in {dt:.1f} s (each: k-d tree rebuild over the 2.04M map means + a1 + "
                      f"k-NN covariances of ~204k points + {r['iters']} GN iterations), FP64 C oracle with OpenMP "
                      f"over points (the k-d tree build is serial: {1e3 * t_index / frames:.0f} ms a step); the map's "
                      f"Gaussians themselves built once, untimed"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    from synth import frame_config2
    f = frame_config2(args.seed)
    omap = oracle_setup(f)
    _, a, b, _ = oracle_frame(f, omap)
    t_full = a + b
    run_s = 150.0  # seconds of oracle work for the whole run
    frac = min(1.0, run_s / max((args.steps + args.warmup) * t_full, 1e-9))
    for _ in range(max(args.warmup - 1, 0)):
        oracle_frame(f, omap, frac)
    times, iters = [], []
    for i in range(args.steps):
        r, fixed, gn, _ = oracle_frame(f, omap, frac, seed=i)
        times.append(fixed + gn / frac)  # a full step: the registration's time scaled to all points
        iters.append(r["iters"])
    total = sum(times)
    value = args.steps / total
    sample = ("full step per step (k-d tree rebuild over the map means, a1, covariances, registration)" if frac >= 1 else
              f"per step: k-d tree rebuild over the map means, a1 and covariances of the full frame, GN registration "
              f"on a random {frac:.3f} of its points; a step's time is the first part plus the registration's "
              f"time divided by that fraction")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(len(orc_points(f)), len(omap.means), world),
        "gn_iters_mean": float(np.mean(iters)),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": oracle_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- batched registration

BATCH_METRIC = "batched G-ICP registrations/s (independent pairs, 5k-300k points each)"


def batch_launches(n_pts) -> int:
    """Kernels one gsicp_register_batch call launches: the joint Morton order of all sources (bbox
    2, quantise 1, keys 1, radix sort by key 5, cloud keys 1, radix sort by cloud 3, gather 1), the
    seeds 1, the set-up 1 and the persistent kernel 1."""
    return 17 if int(np.sum(n_pts)) > 1 else 3


def measure_batch(args, world, rank, local, cpu_sample_s: float = 15.0) -> dict:
    """Batched registration of `args.pairs` independent pairs (log-uniform 5k-300k points, offsets
    <= 5 deg / 5 cm, plane covariances k = 20 computed on the GPU, maps indexed with the shape the
    autotuner picks); one step = one gsicp_register_batch call over all pairs.  Also times the same
    pairs registered one by one with gsicp_register."""
    import torch

    import paper_2403_12550_b300 as g
    from paper_2403_12550_b300.autotune import tune_index_params
    from synth import batch_config4

    torch.cuda.set_device(local)
    pairs = batch_config4(args.seed + 1000 * rank, n_pairs=args.pairs)
    ctx = g.Context()
    cp = g.CovParams(K_NN, EPS, g.PLANE, 0.0)
    rp = g.RegParams(MAX_DIST, MAX_ITERS, TOL, TOL, 6)
    srcs, scovs, tgts, tcovs = [], [], [], []
    for p in pairs:
        for pts, dst_p, dst_c in ((p["src"], srcs, scovs), (p["tgt"], tgts, tcovs)):
            t = torch.from_numpy(pts).cuda()
            dst_p.append(t)
            dst_c.append(g.gsicp_source_covariances(ctx, t, None, cp).clone())
    T0s = np.stack([np.eye(4)] * len(pairs))
    sample = list(range(0, len(pairs), max(1, len(pairs) // 16)))
    tune = tune_index_params(ctx, [srcs[i] for i in sample], [scovs[i] for i in sample],
                             [tgts[i] for i in sample], [tcovs[i] for i in sample], T0s[sample], rp)
    maps = [g.gsicp_build_map_index(ctx, t, c, tune["bucket"], tune["cell"]) for t, c in zip(tgts, tcovs)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        r = g.gsicp_register_batch(ctx, srcs, scovs, maps, T0s, rp)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            r = g.gsicp_register_batch(ctx, srcs, scovs, maps, T0s, rp)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, world, "cuda")
    # the same pairs one by one
    seq = []
    for i in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(len(pairs)):
            g.gsicp_register(ctx, srcs[k], scovs[k], maps[k], T0s[k], rp)
        b.record(stream)
        b.synchronize()
        seq.append(a.elapsed_time(b) / 1e3)
    seq_s = float(np.mean(seq))
    n_pts = np.array([len(p["src"]) for p in pairs])
    point_iters = float(np.sum(n_pts * r["iters"]))
    K, B = args.steps, len(pairs)
    out = {
        "metric": BATCH_METRIC, "value": world * K * B / total_s, "unit": "registrations/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{B} config-1-style pairs, points log-uniform 5k-300k (total {int(n_pts.sum())}), "
                               f"offsets <= 5 deg / 5 cm, k = 20 plane covariances, T0 = I",
                   "index_bucket": tune["bucket"], "index_cell": tune["cell"],
                   "autotune_ms": {f"{b}/{c}": round(v, 3) for (b, c), v in tune["ms"].items()},
                   "l2": "flushed between timed steps (256 MB write)"},
        "point_iters_per_s": world * K * point_iters / total_s,
        # the whole batch is one persistent launch (plus the joint Morton order and set-up, counted in
        # its time here: a lower bound on the kernel's rate)
        "roofline": {"kernel": "gicp_batch_kernel (whole call)", "bound": "hbm",
                     "achieved": point_iters * BYTES_PER_POINT_ITER / (total_s / K) / 1e9,
                     "peak": load_peaks()[0], "unit": "GB/s",
                     "frac": point_iters * BYTES_PER_POINT_ITER / (total_s / K) / 1e9 / load_peaks()[0],
                     "traffic": None, "peak_source": f"{load_peaks()[1]} hbm_gbs",
                     "algorithmic_bytes_per_launch": int(point_iters * BYTES_PER_POINT_ITER),
                     "avg_launch_ms": total_s * 1e3 / K},
        "one_by_one": {"value": B / seq_s, "unit": "registrations/s", "ms": seq_s * 1e3},
        "converged": int(np.sum((r["status"] == g.OK) & (r["iters"] < MAX_ITERS))),
        "gpu_launches": K * batch_launches(n_pts),
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = batch_cpu_baseline(pairs, cpu_sample_s)
    for m in maps:
        m.close()
    ctx.close()
    return out


def run_batch(args, world, rank, local):
    out = measure_batch(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- tracking sequence

SEQ_METRIC = "tracked frames/s and per-frame latency (640x480 sequence, keyframe appends, tracking loop)"


def batch_cpu_baseline(pairs, sample_s: float = 15.0) -> dict:
    """The oracle on the same pairs, in a seeded random order, until about sample_s seconds of
    registration: each pair's covariances and k-d tree built untimed (as the batched step takes
    them prebuilt), its registration from T0 = I timed.  The whole batch's time is estimated from
    the sample's time per source point (registration cost is linear in the points)."""
    import oracle as orc
    done, reg_s, pts = 0, 0.0, 0
    total = sum(len(p["src"]) for p in pairs)
    for i in np.random.default_rng(0).permutation(len(pairs)):
        p = pairs[i]
        cs = orc.source_covariances(p["src"], k=K_NN, eps=EPS, reg_mode=orc.PLANE)["covs"]
        ct = orc.source_covariances(p["tgt"], k=K_NN, eps=EPS, reg_mode=orc.PLANE)["covs"]
        m = orc.Map(p["tgt"], ct)
        t0 = time.perf_counter()
        orc.register(p["src"], cs, m, np.eye(4), MAX_DIST, MAX_ITERS, TOL, TOL, 6)
        reg_s += time.perf_counter() - t0
        done += 1
        pts += len(p["src"])
        if reg_s >= sample_s:
            break
    batch_s = reg_s * total / pts
    return {"value": len(pairs) / batch_s, "unit": "registrations/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": f"{done} of the {len(pairs)} pairs in a seeded random order ({pts} of {total} source points), "
                      f"registration only ({reg_s:.1f} s); the batch's time scaled from the sample's time per "
                      f"source point; FP64 C oracle with OpenMP over points"}


def sequence_cpu_baseline(seq, frames, sample_s: float = 20.0) -> dict:
    """The oracle's tracking loop (same keyframe policy) over the sequence's frames in order until
    about sample_s seconds of work; every frame's full tracker step is timed.  Also returns the
    number of frames run and the oracle's ATE over them."""
    from oracle.tracker import Tracker as OTracker
    from paper_2403_12550_b300.trajectory import ate_rmse
    trk = OTracker(seq["intr"].as_array(), stride=STRIDE, z_min=Z_MIN, z_max=Z_MAX, k=K_NN, eps=EPS, p=P_ALIGN,
                   max_dist=MAX_DIST, max_iters=MAX_ITERS, tol_rot=TOL, tol_trans=TOL)
    done, el, est = 0, 0.0, []
    for f in range(len(frames)):
        t0 = time.perf_counter()
        T, _ = trk.frame(frames[f], seq["poses"][0] if f == 0 else None)
        el += time.perf_counter() - t0
        est.append(T)
        done += 1
        if el >= sample_s:
            break
    return {"value": done / el, "unit": "frames/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": f"the first {done} of {len(frames)} frames through the oracle's tracking loop ({el:.1f} s; "
                      f"frame 0 builds the first map)", "frames_done": done,
            "ate_first_m": ate_rmse(est, seq["poses"][:done])}


def render_workers() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def measure_sequence(args, world, rank, local, n_frames: int, cpu_sample_s: float = 20.0) -> dict:
    """The tracking loop (gsicp_tracker_frame: a1..a7, keyframe decision, non-overlap appends with
    map-index rebuilds) over a TUM-shaped sequence; per-frame latency is host wall time of each
    call (it synchronises), depth images resident on the device."""
    import torch

    import paper_2403_12550_b300 as g
    from paper_2403_12550_b300.trajectory import ate_rmse, ate_rmse_aligned
    from synth import render_sequence_frames, sequence_config3

    torch.cuda.set_device(local)
    seed = 1 + args.seed
    seq = sequence_config3(seed, n_frames=n_frames)
    frames = render_sequence_frames("config3", seed, n_frames, render_workers())
    depths = [torch.from_numpy(d).cuda() for d in frames]
    intr = seq["intr"].as_array()
    ctx = g.Context()
    cp = g.CovParams(K_NN, EPS, g.PLANE, P_ALIGN)
    rp = g.RegParams(MAX_DIST, MAX_ITERS, TOL, TOL, 6)

    def one_pass():
        trk = g.Tracker(ctx, 2, Z_MIN, Z_MAX, cp, rp)
        lat, est, kinds = [], [], []
        for f, d in enumerate(depths):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            T, info = trk.frame(d, intr, seq["poses"][0] if f == 0 else None)
            lat.append(time.perf_counter() - t0)
            est.append(T)
            kinds.append(info["kind"])
        sizes = trk.map_sizes()
        trk.close()
        return lat, est, kinds, sizes

    for _ in range(max(1, min(args.warmup, 2))):
        one_pass()
    lat, est, kinds, sizes = one_pass()
    lat_ms = np.array(lat[1:]) * 1e3  # frame 0 only builds the first map
    ate = ate_rmse(est, seq["poses"])
    out = {
        "metric": SEQ_METRIC, "value": world * len(lat_ms) / (lat_ms.sum() / 1e3), "unit": "frames/s",
        "n_gpus": world, "steps": len(lat_ms), "warmup": args.warmup, "ms_per_step": float(lat_ms.mean()),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"TUM-shaped sequence seed {seed}: {n_frames} frames 640x480 at 30 Hz, stride 2, "
                               f"keyframes by inlier ratio < 0.85, forced every 30, mapping-only every 10",
                   "k": K_NN, "reg": "plane", "p": P_ALIGN},
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "max": float(lat_ms.max())},
        "ate_m": ate, "ate_aligned_m": ate_rmse_aligned(est, seq["poses"]),
        "keyframes": kinds.count(g.KEYFRAME), "mapping_keyframes": kinds.count(g.MAPPING_KEYFRAME),
        "map_sizes": list(sizes),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = sequence_cpu_baseline(seq, frames, cpu_sample_s)
        # the oracle's tracking loop over the frames it ran, against the GPU's over the same frames
        nf = cb.pop("frames_done")
        cb["ate_m"] = cb.pop("ate_first_m")
        out["ate_first_frames"] = {"frames": nf, "ate_m": ate_rmse(est[:nf], seq["poses"][:nf]),
                                   "oracle_ate_m": cb["ate_m"]}
        out["cpu_baseline"] = cb
    ctx.close()
    return out


def run_sequence(args, world, rank, local):
    out = measure_sequence(args, world, rank, local, args.frames)
    if rank == 0:
        print(json.dumps(out), flush=True)


SURR_METRIC = "G-ICP tracking frames/s with learned covariances (640x480 held-out sequence, per-frame k-NN fallback)"
# floating-point operations of one layer-2 forward per sample pixel (32 x 32 channels x 25 taps, multiply + add)
FLOP_PER_PIXEL_L2 = 2 * 32 * 32 * 25


def surrogate_cpu_baseline(frames, seq, sample_s: float = 15.0) -> dict:
    """The oracle on this host's cores for the learned-covariance workload: per frame the FP64 network
    forward and covariances, then the FP64 registration against a map built from the previous frame
    (its oracle k-NN covariances, in the world frame by the ground-truth pose); frames in order until
    about sample_s of work."""
    import oracle as orc
    from oracle import surrogate as sgo
    from paper_2403_12550_b300 import surrogate as S
    w = S.load_weights()
    intr = seq["intr"].as_array()
    done, t0 = 0, time.perf_counter()
    for f in range(1, len(frames)):
        P, M = sgo.point_grid(frames[f], intr, STRIDE, Z_MIN, Z_MAX)
        P = P.astype(np.float32).astype(np.float64)
        v = sgo.forward(P, M, w)["v"]
        covs, _ = sgo.covariances(v, M, P, EPS, P_ALIGN)
        Pm, Mm = sgo.point_grid(frames[f - 1], intr, STRIDE, Z_MIN, Z_MAX)
        mp_ = Pm[Mm]
        mc = orc.source_covariances(mp_, mp_[:, 2], k=K_NN, eps=EPS, reg_mode=orc.PLANE, p=P_ALIGN)["covs"]
        Tm = seq["poses"][f - 1]
        wm = mp_ @ Tm[:3, :3].T + Tm[:3, 3]
        R = Tm[:3, :3]
        C = np.stack([mc[:, 0], mc[:, 1], mc[:, 2], mc[:, 1], mc[:, 3], mc[:, 4], mc[:, 2], mc[:, 4], mc[:, 5]],
                     1).reshape(-1, 3, 3)
        Cw = R[None] @ C @ R.T[None]
        mcw = np.stack([Cw[:, 0, 0], Cw[:, 0, 1], Cw[:, 0, 2], Cw[:, 1, 1], Cw[:, 1, 2], Cw[:, 2, 2]], 1)
        orc.register(P[M], covs, orc.Map(wm, mcw), seq["poses"][f - 1], MAX_DIST, MAX_ITERS, TOL, TOL, 6)
        done += 1
        if time.perf_counter() - t0 > sample_s:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "frames/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": f"{done} frame(s) of the held-out sequence: FP64 network forward + covariances + registration "
                      f"against a map from the previous frame ({el:.1f} s)"}


def measure_surrogate(args, world, rank, local, n_frames: int, cpu_sample_s: float = 15.0) -> dict:
    """The learned covariance surrogate on its held-out sequence: the tracking loop with the
    surrogate's covariances (per-frame fallback to k-NN when the RMS correspondence residual exceeds
    1.1 x the last k-NN frame's; k-NN calibration every 30 frames; keyframes keep k-NN covariances),
    and the same loop with k-NN covariances for comparison.  frames/s from host wall time per
    gsicp_tracker_frame call (it synchronises), depth images resident on the device; e2e copies each
    frame's depth from pinned host memory inside the loop.  The roofline line is the tensor-core
    layer-2 kernel, timed by the library's per-layer CUDA events on the tracker's stream."""
    import torch

    import paper_2403_12550_b300 as g
    from paper_2403_12550_b300 import surrogate as S
    from paper_2403_12550_b300.trajectory import ate_rmse, ate_rmse_aligned
    from synth import sequence_config5

    torch.cuda.set_device(local)
    n = n_frames
    seq = sequence_config5(args.seed, n_frames=n)
    frames = S.render_sequence(args.seed, n, render_workers())
    depths = [torch.from_numpy(f).cuda() for f in frames]
    host = [torch.from_numpy(f).pin_memory() for f in frames]
    intr = seq["intr"].as_array()
    ctx = g.Context()
    sg = g.Surrogate(S.load_weights())
    sg.set_timing(True)
    cp = g.CovParams(K_NN, EPS, g.PLANE, P_ALIGN)
    rp = g.RegParams(MAX_DIST, MAX_ITERS, TOL, TOL, 6)
    hs, ws = (frames[0].shape[0] + STRIDE - 1) // STRIDE, (frames[0].shape[1] + STRIDE - 1) // STRIDE

    def one_pass(use_sg: bool, e2e: bool = False):
        trk = g.Tracker(ctx, STRIDE, Z_MIN, Z_MAX, cp, rp)
        if use_sg:
            trk.set_surrogate(sg, 1.1, 30, True)
        lat, est, infos, layers = [], [], [], []
        for f in range(n):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d = host[f].cuda(non_blocking=True) if e2e else depths[f]
            T, info = trk.frame(d, intr, seq["poses"][0] if f == 0 else None)
            lat.append(time.perf_counter() - t0)
            est.append(T)
            infos.append(info)
            if use_sg and (info["cov_source"] == 1 or info["fell_back"]):
                layers.append(sg.layer_times())
        trk.close()
        return np.array(lat[1:]) * 1e3, est, infos, np.array(layers)

    for _ in range(max(1, min(args.warmup, 2))):
        one_pass(True)
        one_pass(False)
    with ClockSampler(local) as clk:
        lat_s, est_s, inf_s, layers = one_pass(True)
        lat_k, est_k, inf_k, _ = one_pass(False)
    lat_e, _, _, _ = one_pass(True, e2e=True)

    def ate(est):
        return ate_rmse(est, seq["poses"])

    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1800.0
    l2_ms = float(layers[:, 1].mean()) if len(layers) else float("nan")
    flops = FLOP_PER_PIXEL_L2 * hs * ws
    achieved = flops / (l2_ms * 1e-3) / 1e12
    out = {
        "metric": SURR_METRIC, "value": world * len(lat_s) / (lat_s.sum() / 1e3), "unit": "frames/s",
        "n_gpus": world, "steps": len(lat_s), "warmup": args.warmup, "ms_per_step": float(lat_s.mean()),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"held-out config-5 sequence seed {args.seed}: {n} frames 640x480 at 30 Hz, stride 2, "
                               f"orbit in a config-2-style room none of the 2000 training frames shows",
                   "covariances": "3-layer 5x5 CNN (32 channels, bfloat16 weights and activations, float "
                                  "accumulate); fallback to k-NN at residual ratio 1.1; k-NN calibration every 30 "
                                  "frames; keyframes add k-NN covariances",
                   "k": K_NN, "eps": EPS, "p": P_ALIGN},
        "knn_frames_per_s": world * len(lat_k) / (lat_k.sum() / 1e3),
        "latency_ms": {"p50": float(np.percentile(lat_s, 50)), "p99": float(np.percentile(lat_s, 99)),
                       "knn_p50": float(np.percentile(lat_k, 50)), "knn_p99": float(np.percentile(lat_k, 99))},
        "ate_m": ate(est_s), "ate_knn_m": ate(est_k), "ate_gap_m": ate(est_s) - ate(est_k),
        "ate_aligned_m": ate_rmse_aligned(est_s, seq["poses"]), "ate_knn_aligned_m": ate_rmse_aligned(est_k, seq["poses"]),
        "surrogate_frames": int(sum(i["cov_source"] == 1 for i in inf_s)),
        "fell_back": int(sum(i["fell_back"] for i in inf_s)),
        "layer_ms": {"grid_l1": float(layers[:, 0].mean()), "l2_tensor": l2_ms, "l3_tensor_cov": float(layers[:, 2].mean())}
        if len(layers) else None,
        "roofline": {"kernel": "sg_conv_tc_kernel<32> (layer 2, tcgen05)", "bound": "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": "measured bf16_tflops (burst)", "flop_per_launch": flops, "avg_launch_ms": l2_ms},
        "e2e": {"value": world * len(lat_e) / (lat_e.sum() / 1e3), "unit": "frames/s",
                "h2d_bytes_per_step": int(frames[0].nbytes), "d2h_bytes_per_step": 16 * 8},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = surrogate_cpu_baseline(frames, seq, cpu_sample_s)
    sg.close()
    ctx.close()
    return out


def run_surrogate(args, world, rank, local):
    out = measure_surrogate(args, world, rank, local, args.frames)
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch":
        run_batch(args, world, rank, local)
    elif args.workload == "sequence":
        run_sequence(args, world, rank, local)
    elif args.workload == "surrogate":
        run_surrogate(args, world, rank, local)
    elif args.workload == "sharded":
        run_sharded(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
