"""A registration whose source points are split across ranks (Sec. 3, Eq. (MLE_for_T): a sum over
correspondences), through the C ABI on one GPU.

One rank: the split registration (begin, then linearise / update until it stops) is the single
registration, so it must equal gsicp_register bit for bit.  Two ranks are emulated by two contexts
on the same GPU, run one after the other (no kernel waits on another): each linearises its share,
the two rows are stacked in rank order as an all-gather would deliver them, and each context
updates from the same rows; both must hold the same pose bit for bit after every update, and the
final pose must meet the oracle's within the pose bar.
"""
import numpy as np
import pytest

import oracle as orc

from ._util import POSE_ROT_TOL, POSE_TRANS_TOL, config1_inputs, config2_inputs, oracle_frame_points, pose_diff

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12550_b300 as g
    return g


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_one_rank_split_registration_is_the_single_registration(g):
    from paper_2403_12550_b300.sharded import register_sharded
    ctx = g.Context()
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    for scene, pose in ((0, 0), (1, 2), (2, 1)):
        src, cs, tgt, ct, _ = config1_inputs(scene, pose)
        m = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
        rs = g.gsicp_register(ctx, cu(src), cu(cs), m, np.eye(4), rp)
        rh = register_sharded(ctx, cu(src), cu(cs), m, np.eye(4), rp)
        np.testing.assert_array_equal(rh["T"], rs["T"])
        np.testing.assert_array_equal(rh["H"], rs["H"])
        assert (rh["iters"], rh["cost"], rh["inliers"]) == (rs["iters"], rs["cost"], rs["inliers"])
        assert rh["rounds"] == rs["iters"]
        assert rh["status"] == (g.SHARD_CONVERGED if rs["iters"] < 30 else g.SHARD_MAXITER)
        m.close()
    ctx.close()


def _two_contexts(g, src, cs, means, covs, T0, rp, world=2):
    from paper_2403_12550_b300.sharded import share
    ctxs = [g.Context() for _ in range(world)]
    maps = [g.gsicp_build_map_index(c, cu(means), cu(covs)) for c in ctxs]
    parts = [torch.empty(g.SHARD_SUMS, dtype=torch.float64, device="cuda") for _ in range(world)]
    for r, c in enumerate(ctxs):
        sl = share(len(src), world, r)
        g.gsicp_shard_begin(c, cu(src[sl]), cu(cs[sl]), maps[r], T0, rp)
    outs = None
    for _ in range(rp.max_iters):
        for r, c in enumerate(ctxs):
            g.gsicp_shard_linearise(c, parts[r])
        rows = torch.stack(parts)  # rank order, as an all-gather delivers them
        outs = [g.gsicp_shard_update(c, rows) for c in ctxs]
        for o in outs[1:]:
            np.testing.assert_array_equal(o["T"], outs[0]["T"])
            assert o["status"] == outs[0]["status"] and o["iters"] == outs[0]["iters"]
        if outs[0]["status"] != g.SHARD_RUNNING:
            break
    for m in maps:
        m.close()
    for c in ctxs:
        c.close()
    return outs[0]


def test_two_ranks_agree_and_meet_the_oracle_config1(g):
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    for scene, pose in ((0, 0), (3, 0)):
        src, cs, tgt, ct, _ = config1_inputs(scene, pose)
        r = _two_contexts(g, src, cs, tgt, ct, np.eye(4), rp)
        ro = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4))
        assert r["status"] == g.SHARD_CONVERGED and ro["status"] == orc.OK
        dr, dt = pose_diff(r["T"], ro["T"])
        assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (dr, dt, r["iters"], ro["iters"])


def test_four_ranks_on_the_full_bench_frame_meet_the_oracle(g):
    """The 1200 x 680 frame (204,000 points) against the 2.04M-Gaussian map, split four ways."""
    f, means, covs = config2_inputs(0)
    pts, z = oracle_frame_points(f["depth"])
    cs = orc.source_covariances(pts, z, k=20, eps=1e-3, reg_mode=orc.PLANE, p=1.5)["covs"].astype(np.float32)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    r = _two_contexts(g, pts, cs, means, covs, f["T0"], rp, world=4)
    ro = orc.register(pts, cs, orc.Map(means, covs), f["T0"], 0.1, 30, 1e-6, 1e-6, 6)
    assert r["status"] == g.SHARD_CONVERGED and ro["status"] == orc.OK
    dr, dt = pose_diff(r["T"], ro["T"])
    assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (dr, dt, r["iters"], ro["iters"])


def test_shard_calls_need_a_begun_registration(g):
    ctx = g.Context()
    part = torch.empty(g.SHARD_SUMS, dtype=torch.float64, device="cuda")
    with pytest.raises(g.GsicpError):
        g.gsicp_shard_linearise(ctx, part)
    with pytest.raises(g.GsicpError):
        g.gsicp_shard_update(ctx, part.reshape(1, -1))
    # another registration on the context ends a begun one
    src, cs, tgt, ct, _ = config1_inputs(0, 0, n=2000)
    m = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    g.gsicp_shard_begin(ctx, cu(src), cu(cs), m, np.eye(4), g.RegParams())
    g.gsicp_shard_linearise(ctx, part)
    g.gsicp_register(ctx, cu(src), cu(cs), m, np.eye(4), g.RegParams())
    with pytest.raises(g.GsicpError):
        g.gsicp_shard_linearise(ctx, part)
    m.close()
    ctx.close()
