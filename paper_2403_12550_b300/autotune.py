"""Autotuners: time the library on a sample of the caller's workload for each candidate shape and
return the fastest.  Results are kept per (device, workload key) for the life of the process.

* ``tune_index_params`` (batched registration): the map index's shape (points per BVH leaf, grid
  cell size), timing gsicp_register_batch.
* ``tune_frame`` (one frame tracked against a map): the map index's shape, timing
  gsicp_track_frame, then on the chosen shape the cooperative-walk threshold of the context (how
  many tree walks a warp of 32 source points takes together), then the Gauss-Newton kernel's block
  size (source points per block).

Every candidate returns the same result (the searches are exact), so only time is compared.  The
cell size matters most: a larger cell's 2x2x2 block certifies more nearest-point searches and more
complete candidate lists (fewer tree walks, fewer cache refreshes in later iterations) but costs
more in the scan of the block; where the balance lies depends on the map's density.
"""
from __future__ import annotations

import torch

from . import (IndexParams, MapHandle, RegParams, gsicp_build_map_index,  # noqa: F401
               gsicp_ctx_set_coop_walks, gsicp_ctx_set_gn_block, gsicp_register_batch, gsicp_track_frame)

# (points per leaf, grid cell in metres)
CANDIDATES = ((16, 0.012), (8, 0.012), (32, 0.012), (16, 0.008), (16, 0.005), (8, 0.008))
FRAME_CANDIDATES = ((8, 0.012), (16, 0.012), (8, 0.010), (16, 0.010), (8, 0.013), (16, 0.013), (8, 0.008),
                    (16, 0.008), (8, 0.016))
COOP_CANDIDATES = (4, 2, 8, 0)
BLOCK_CANDIDATES = (256, 128, 384)

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


def frame_ms(ctx, depth, intr, stride, z_min, z_max, cov_params, map_, T0, params: RegParams, reps: int) -> float:
    """Best of `reps` timed gsicp_track_frame calls (after one warm-up), in ms, from CUDA events on
    the current stream."""
    stream = torch.cuda.current_stream()
    gsicp_track_frame(ctx, depth, intr, stride, z_min, z_max, cov_params, map_, T0, params)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gsicp_track_frame(ctx, depth, intr, stride, z_min, z_max, cov_params, map_, T0, params)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_frame(ctx, depth, intr, stride: int, z_min: float, z_max: float, cov_params, means, covs, T0,
               params: RegParams, candidates=FRAME_CANDIDATES, coop_candidates=COOP_CANDIDATES,
               block_candidates=BLOCK_CANDIDATES, reps: int = 3, key: str | None = None, timer=frame_ms) -> dict:
    """Returns dict(bucket, cell, coop, block, ms: {(bucket, cell): ms}, coop_ms: {coop: ms},
    block_ms: {block: ms}) for tracking frames like `depth` (a sample frame, its intrinsics and a1
    settings, start pose T0) against the map Gaussians means / covs.  Each index shape is built,
    timed (best of `reps` frames) and released; then, on the fastest shape, the context's
    cooperative-walk threshold and then its Gauss-Newton block size are timed, each left set to the
    fastest.  Ties go to the earlier candidate."""
    ck = (torch.cuda.get_device_name(), key) if key is not None else None
    if ck is not None and ck in _CACHE:
        res = _CACHE[ck]
        gsicp_ctx_set_coop_walks(ctx, res["coop"])
        gsicp_ctx_set_gn_block(ctx, res["block"])
        return res
    times = {}
    for bucket, cell in candidates:
        m = gsicp_build_map_index(ctx, means, covs, bucket, cell)
        try:
            times[(bucket, cell)] = timer(ctx, depth, intr, stride, z_min, z_max, cov_params, m, T0, params, reps)
        finally:
            m.close()
    bucket, cell = min(times, key=times.get)
    coop_times, block_times = {}, {}
    m = gsicp_build_map_index(ctx, means, covs, bucket, cell)
    try:
        for c in coop_candidates:
            gsicp_ctx_set_coop_walks(ctx, c)
            coop_times[c] = timer(ctx, depth, intr, stride, z_min, z_max, cov_params, m, T0, params, reps)
        coop = min(coop_times, key=coop_times.get)
        gsicp_ctx_set_coop_walks(ctx, coop)
        for bs in block_candidates:
            gsicp_ctx_set_gn_block(ctx, bs)
            block_times[bs] = timer(ctx, depth, intr, stride, z_min, z_max, cov_params, m, T0, params, reps)
    finally:
        m.close()
    block = min(block_times, key=block_times.get)
    gsicp_ctx_set_gn_block(ctx, block)
    res = dict(bucket=bucket, cell=cell, coop=coop, block=block, ms=times, coop_ms=coop_times, block_ms=block_times)
    if ck is not None:
        _CACHE[ck] = res
    return res
