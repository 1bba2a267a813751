"""Autotuner for batched registration: times gsicp_register_batch on a sample of the caller's
workload for each candidate shape of the map index (points per BVH leaf, grid cell size) and
returns the fastest.  Results are kept per (device, workload key) for the life of the process.
"""
from __future__ import annotations

import torch

from . import (IndexParams, MapHandle, RegParams, gsicp_build_map_index,  # noqa: F401
               gsicp_register_batch)

# (points per leaf, grid cell in metres)
CANDIDATES = ((16, 0.008), (8, 0.008), (32, 0.008), (16, 0.005), (16, 0.012), (8, 0.005))

_CACHE: dict = {}


def batch_ms(ctx, srcs, scovs, maps, T0s, params: RegParams, reps: int) -> float:
    """Best of `reps` timed gsicp_register_batch calls (after one warm-up for buffers and caches),
    in ms, from CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    gsicp_register_batch(ctx, srcs, scovs, maps, T0s, params)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gsicp_register_batch(ctx, srcs, scovs, maps, T0s, params)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_index_params(ctx, srcs, scovs, tgts, tcovs, T0s, params: RegParams, candidates=CANDIDATES, reps: int = 3,
                      key: str | None = None, timer=batch_ms) -> dict:
    """Returns dict(bucket, cell, ms: {(bucket, cell): best of `reps` batch times in ms}).  The
    maps are built from tgts / tcovs with each candidate shape; srcs / scovs / T0s are the pairs'
    sources, their covariances and start poses (a sample of the real batch is enough).  Ties go to
    the earlier candidate."""
    ck = (torch.cuda.get_device_name(), key) if key is not None else None
    if ck is not None and ck in _CACHE:
        return _CACHE[ck]
    times = {}
    for bucket, cell in candidates:
        maps = [gsicp_build_map_index(ctx, t, c, bucket, cell) for t, c in zip(tgts, tcovs)]
        try:
            times[(bucket, cell)] = timer(ctx, srcs, scovs, maps, T0s, params, reps)
        finally:
            for m in maps:
                m.close()
    bucket, cell = min(times, key=times.get)
    res = dict(bucket=bucket, cell=cell, ms=times)
    if ck is not None:
        _CACHE[ck] = res
    return res
