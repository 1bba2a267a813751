"""One G-ICP registration whose source points are split across processes (ranks).

The cost of Eq. (MLE_for_T) (Sec. 3) and its Gauss-Newton system are sums over the
correspondences, so a registration splits by source point: every rank holds the whole map and a
share of the points, linearises its share at the current pose, and the shares' sums add up to the
whole registration's.  Per iteration:

1. each rank runs ``gsicp_shard_linearise``: SHARD_SUMS float64 sums of its share, on its device;
2. the ranks all-gather those rows (one collective of SHARD_SUMS doubles per rank);
3. each rank runs ``gsicp_shard_update`` on the gathered rows: the library sums them in rank order,
   solves in FP64 and updates the pose.

Every rank passes the same rows in the same order, so every rank computes the same bits: the poses
stay identical without a broadcast, and the loop ends on every rank at the same iteration.  The
collective is tiny (SHARD_SUMS x 8 bytes per rank); it is the path's only exchange.

The host loop (``ShardLoop``) takes the three steps as callables, so its control flow can be run
against any implementation of them with the same contract; ``register_sharded`` wires the
library's entry points and ``torch.distributed``.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import (SHARD_RUNNING, SHARD_SUMS, Context, MapHandle, RegParams, gsicp_shard_begin, gsicp_shard_linearise,
               gsicp_shard_update)

__all__ = ["share", "gather_rows", "ShardLoop", "register_sharded"]


def share(n: int, world: int, rank: int) -> slice:
    """Rank `rank`'s contiguous share of n points: [rank n / world, (rank + 1) n / world)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return slice(rank * n // world, (rank + 1) * n // world)


def gather_rows(row: torch.Tensor, group=None) -> torch.Tensor:
    """Every rank's row, stacked in rank order (world x len(row)); a single process gets its own row."""
    row = row.reshape(-1).contiguous()
    if not (dist.is_available() and dist.is_initialized()):
        return row.reshape(1, -1)
    world = dist.get_world_size(group)
    out = torch.empty((world, row.numel()), dtype=row.dtype, device=row.device)
    if world == 1:
        out.copy_(row.reshape(1, -1))
        return out
    dist.all_gather(list(out.unbind(0)), row, group=group)
    return out


class ShardLoop:
    """Linearise -> gather -> update until the update's status leaves SHARD_RUNNING, at most
    max_iters times.

    linearise() -> this rank's row of SHARD_SUMS sums; gather(row) -> the rows of every rank in rank
    order; update(rows) -> a dict with at least "status" (SHARD_*).  Returns the last update's dict
    with "rounds", the number of linearise / gather / update rounds run."""

    def __init__(self, linearise, gather, update):
        self.linearise, self.gather, self.update = linearise, gather, update

    def run(self, max_iters: int) -> dict:
        if max_iters < 1:
            raise ValueError("max_iters must be at least 1")
        out, rounds = None, 0
        while rounds < max_iters:
            rows = self.gather(self.linearise())
            out = self.update(rows)
            rounds += 1
            if out["status"] != SHARD_RUNNING:
                break
        out = dict(out)
        out["rounds"] = rounds
        return out


def register_sharded(ctx: Context, src_share: torch.Tensor, covs_share: torch.Tensor, map_: MapHandle, T0,
                     params: RegParams, group=None) -> dict:
    """Register this rank's share of the source points (n_r x 3 and n_r x 6 CUDA tensors) against its
    copy of the map, together with the other ranks of `group` (every rank calls this with the same
    T0 and params).  Returns dict(status, T, H, iters, cost, inliers, rounds): the same on every rank;
    T, H, cost and inliers are the whole registration's."""
    gsicp_shard_begin(ctx, src_share, covs_share, map_, T0, params)
    partial = torch.empty(SHARD_SUMS, dtype=torch.float64, device=src_share.device)

    def linearise():
        gsicp_shard_linearise(ctx, partial)
        return partial

    return ShardLoop(linearise, lambda row: gather_rows(row, group),
                     lambda rows: gsicp_shard_update(ctx, rows)).run(params.max_iters)
