"""A registration whose source points are split across ranks, on CPU (gloo, two ranks).

The library's host loop (``paper_2403_12550_b300.sharded``: ``share``, ``gather_rows``,
``ShardLoop``) runs with the oracle standing in for the two CUDA entry points: each rank linearises
its share with ``oracle.linearise`` (the 30 sums of the shard contract) and updates with the
oracle's Gauss-Newton step on the rank-ordered sum of the gathered rows.  Eq. (MLE_for_T) (Sec. 3)
is a sum over correspondences, so the split registration must end where the oracle's single
registration does (up to the rounding of the sums' order), and every rank must hold the same pose
bit for bit after every update.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from ._util import config1_inputs

RUNNING, CONVERGED, MAXITER, DEGENERATE = range(4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ut(r, c):
    return r * 6 - (r * (r - 1)) // 2 + (c - r)


def oracle_steps(src, cs, omap, T0, max_dist=0.1, tol=1e-6, min_inliers=6, max_iters=30):
    """linearise / update callables with the shard contract, computed by the oracle."""
    import oracle as orc
    state = {"T": np.array(T0, dtype=np.float64), "it": 0}

    def linearise():
        lo = orc.linearise(src, cs, omap, state["T"], max_dist)
        H = lo["H"]
        row = [H[r, c] for r in range(6) for c in range(r, 6)] + list(lo["b"]) + [lo["cost"], lo["inliers"], 0.0]
        return torch.tensor(row, dtype=torch.float64)

    def update(rows):
        tot = np.zeros(30)
        for r in rows.numpy():  # rank order
            tot = tot + r
        H = np.empty((6, 6))
        for r in range(6):
            for c in range(r, 6):
                H[r, c] = H[c, r] = tot[_ut(r, c)]
        state["it"] += 1
        if tot[28] < min_inliers:
            return dict(status=DEGENERATE, T=state["T"].copy(), iters=state["it"])
        Tn, conv = orc.gn_update(H, tot[21:27], state["T"], tol, tol)
        if conv < 0:
            return dict(status=DEGENERATE, T=state["T"].copy(), iters=state["it"])
        state["T"] = Tn
        status = CONVERGED if conv == 1 else (MAXITER if state["it"] >= max_iters else RUNNING)
        return dict(status=status, T=Tn.copy(), iters=state["it"])

    return linearise, update


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    from paper_2403_12550_b300.sharded import ShardLoop, gather_rows, share
    orc.set_threads(1)
    src, cs, tgt, ct, _ = config1_inputs(1, 2, n=4000)
    sl = share(len(src), world, rank)
    lin, upd = oracle_steps(src[sl], cs[sl], orc.Map(tgt, ct), np.eye(4))
    res = ShardLoop(lin, gather_rows, upd).run(30)
    # every rank's pose, gathered, to compare them bit for bit
    Ts = gather_rows(torch.from_numpy(res["T"].reshape(16).copy()))
    out[rank] = (res["status"], res["iters"], res["rounds"], res["T"], Ts.numpy())
    dist.destroy_process_group()


def test_two_ranks_split_registration_matches_single_and_each_other():
    import oracle as orc
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    (s0, it0, r0, T0, all0), (s1, it1, r1, T1, all1) = res[0], res[1]
    assert s0 == s1 == CONVERGED and it0 == it1 == r0 == r1
    np.testing.assert_array_equal(T0, T1)            # the same bits on every rank
    np.testing.assert_array_equal(all0[0], all0[1])
    src, cs, tgt, ct, _ = config1_inputs(1, 2, n=4000)
    ro = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4))
    assert ro["status"] == orc.OK and ro["iters"] == it0
    np.testing.assert_allclose(T0, ro["T"], rtol=0, atol=1e-9)  # only the sums' order differs


def test_share_covers_every_point_once():
    from paper_2403_12550_b300.sharded import share
    for n in (0, 1, 7, 100, 4097):
        for world in (1, 2, 3, 8):
            idx = np.concatenate([np.arange(n)[share(n, world, r)] for r in range(world)])
            np.testing.assert_array_equal(idx, np.arange(n))
    with pytest.raises(ValueError):
        share(10, 2, 2)


def test_loop_stops_on_the_first_final_status_and_at_max_iters():
    from paper_2403_12550_b300.sharded import ShardLoop
    seq = iter([RUNNING, RUNNING, CONVERGED, RUNNING])
    calls = []
    r = ShardLoop(lambda: torch.zeros(30, dtype=torch.float64), lambda row: row.reshape(1, -1),
                  lambda rows: calls.append(1) or {"status": next(seq)}).run(30)
    assert r["status"] == CONVERGED and r["rounds"] == 3 and len(calls) == 3
    r = ShardLoop(lambda: torch.zeros(30, dtype=torch.float64), lambda row: row.reshape(1, -1),
                  lambda rows: {"status": RUNNING}).run(4)
    assert r["rounds"] == 4
    with pytest.raises(ValueError):
        ShardLoop(None, None, None).run(0)


def test_single_process_gather_is_the_row_itself():
    from paper_2403_12550_b300.sharded import gather_rows
    row = torch.arange(30, dtype=torch.float64)
    g = gather_rows(row)
    assert g.shape == (1, 30) and torch.equal(g[0], row)
