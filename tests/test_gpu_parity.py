"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Inputs come from the seeded generators (synth) and, where the method's own
arithmetic is needed to make an input (covariances of a map), from the oracle;
nothing the CUDA library produced is ever fed to the oracle.
"""
import numpy as np
import pytest

import oracle as orc
from synth import (Intrinsics, REPLICA_INTR, add_depth_noise, frame_config2, make_room, random_offset, raycast_depth,
                   circle_poses, const_velocity, sequence_config3, transform_points)

from ._util import (COV_REL_TOL, KNN_TIE_REL, PLANE_GAP_EXCLUDE, POSE_ROT_TOL, POSE_TRANS_TOL, config1_inputs,
                    config2_inputs, cov_rel_err, oracle_frame_points, pose_diff, sym)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12550_b300 as g
    return g


@pytest.fixture(scope="module")
def ctx(g):
    c = g.Context()
    yield c
    c.close()


def cu(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ----------------------------------------------------------------------------- a1

def _depth_case(W, H, seed, dropout=0.02):
    intr = Intrinsics(W, H, 0.5 * W, 0.5 * W, (W - 1) / 2, (H - 1) / 2)
    scene = make_room(seed)
    rng = np.random.default_rng(seed)
    P = circle_poses(rng, scene, 1)[0]
    d = add_depth_noise(raycast_depth(scene, P, intr), rng, 1e-3, dropout=dropout)
    d[rng.random(d.shape) < 0.01] = np.nan
    d[rng.random(d.shape) < 0.01] = 50.0  # beyond z_max
    return intr, d


@pytest.mark.parametrize("W,H,stride", [(1, 1, 1), (37, 23, 1), (64, 48, 2), (101, 77, 3), (1200, 680, 2),
                                        (640, 480, 2), (640, 480, 1)])
def test_depth_to_points_bit_exact(g, ctx, W, H, stride):
    intr, d = _depth_case(W, H, W + H)
    pts_o, z_o = orc.depth_to_points(d, intr.as_array(), stride, 0.1, 10.0)
    pts, z = g.gsicp_depth_to_points(ctx, cu(d), intr.as_array(), stride, 0.1, 10.0)
    assert pts.shape[0] == len(pts_o)
    # each coordinate is the correctly rounded value of the formula on both sides
    np.testing.assert_array_equal(pts.cpu().numpy(), pts_o.astype(np.float32))
    np.testing.assert_array_equal(z.cpu().numpy(), z_o.astype(np.float32))


def test_depth_to_points_empty_and_capacity(g, ctx):
    d = np.full((48, 64), np.nan, dtype=np.float32)
    pts, z = g.gsicp_depth_to_points(ctx, cu(d), [50, 50, 31.5, 23.5], 2, 0.1, 10.0)
    assert pts.shape[0] == 0
    d = np.ones((48, 64), dtype=np.float32)
    small = torch.empty((10, 3), device="cuda")
    with pytest.raises(g.GsicpError) as e:
        g.gsicp_depth_to_points(ctx, cu(d), [50, 50, 31.5, 23.5], 2, 0.1, 10.0, pts_out=small,
                                z_out=torch.empty(10, device="cuda"))
    assert e.value.status == g.ERR_CAPACITY


# ----------------------------------------------------------------------------- a2 + a3

def _check_knn_and_covs(pts, z, mode, p, k, g, ctx, gap_exclude=True):
    ref = orc.source_covariances(pts, z, k=k, eps=1e-3, reg_mode=mode, p=p)
    idx_o, d2_o = orc.KDTree(pts).knn(pts, k)
    params = g.CovParams(k, 1e-3, mode, p)
    covs, knn = g.gsicp_source_covariances(ctx, cu(pts), None if z is None else cu(z), params, want_knn=True)
    covs, knn = covs.cpu().numpy().astype(np.float64), knn.cpu().numpy()
    n = len(pts)
    kk = min(k, n)
    # kNN: identical lists, except swaps among candidates whose oracle distances tie within 1e-6
    same = np.all(knn == idx_o, axis=1)
    bad = np.nonzero(~same)[0]
    P = pts.astype(np.float64)
    for i in bad:
        gi = knn[i, :kk]
        assert np.all(gi >= 0) and len(set(gi.tolist())) == kk
        dg = np.sort(np.sum((P[gi] - P[i]) ** 2, axis=1))
        kth = d2_o[i, kk - 1]
        assert np.all(dg <= kth * (1 + KNN_TIE_REL) + 1e-30), (i, dg, kth)
        assert np.allclose(dg, d2_o[i, :kk], rtol=KNN_TIE_REL, atol=1e-30)
    if k > n:
        assert np.all(knn[:, n:] == -1)
    # covariances: relative Frobenius, excluding ill-posed normals under PLANE and tie-swapped sets
    keep = same.copy()
    if mode == orc.PLANE and gap_exclude:
        keep &= ref["gap"] >= PLANE_GAP_EXCLUDE
    if mode != orc.NONE:  # the line-like test (middle/largest eigenvalue <= 1e-5) is a threshold: skip its edge
        w = np.linalg.eigvalsh(sym(ref["raw"]))
        ratio = w[:, 1] / np.maximum(w[:, 2], 1e-300)
        keep &= ~((ratio > 0.5e-5) & (ratio < 2e-5))
    err = cov_rel_err(covs, ref["covs"])
    worst = float(err[keep].max()) if keep.any() else 0.0
    assert worst <= COV_REL_TOL, (worst, np.argmax(np.where(keep, err, 0)))
    return dict(n=n, knn_mismatch=len(bad), excluded=int((~keep).sum()), worst=worst)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 19, 20, 21, 33, 100, 1000, 4097])
def test_source_covariances_small_and_ragged(g, ctx, n):
    rng = np.random.default_rng(n)
    pts = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    if n > 10:
        pts[rng.integers(0, n, n // 10)] = pts[rng.integers(0, n, n // 10)]  # exact duplicates
    for mode in (orc.PLANE, orc.ELLIPSE, orc.NONE):
        _check_knn_and_covs(pts, None, mode, 0.0, 20, g, ctx)


@pytest.mark.parametrize("k", [1, 5, 8, 16, 20, 32])
def test_source_covariances_k(g, ctx, k):
    src, _, _ = __import__("synth").pair_config1(3, 0, n=3000)
    _check_knn_and_covs(src, None, orc.ELLIPSE, 0.0, k, g, ctx)


@pytest.mark.parametrize("mode", [orc.PLANE, orc.ELLIPSE, orc.NONE])
def test_source_covariances_config1(g, ctx, mode):
    src, _, _ = __import__("synth").pair_config1(0, 0, n=10_000)
    r = _check_knn_and_covs(src, None, mode, 0.0, 20, g, ctx)
    assert r["excluded"] < 0.01 * r["n"]


@pytest.mark.parametrize("p", [1.0, 1.5])
def test_source_covariances_frame_with_scale_aligning(g, ctx, p):
    f = frame_config2(0, n_views=0)
    pts, z = oracle_frame_points(f["depth"])
    r = _check_knn_and_covs(pts, z, orc.PLANE, p, 20, g, ctx)
    assert r["excluded"] < 0.01 * r["n"]


def test_source_covariances_collinear_and_coincident(g, ctx):
    t = np.linspace(0, 1, 50, dtype=np.float32)
    line = np.stack([t, 2 * t, -t], 1)
    same = np.ones((25, 3), dtype=np.float32)
    for pts in (line, same):
        for mode in (orc.PLANE, orc.ELLIPSE):
            ref = orc.source_covariances(pts, k=20, reg_mode=mode)["covs"]
            covs = g.gsicp_source_covariances(ctx, cu(pts), None, g.CovParams(20, 1e-3, mode, 0.0)).cpu().numpy()
            np.testing.assert_allclose(covs, ref, atol=1e-6)


# ----------------------------------------------------------------------------- a4 index structure

def _morton30(p, lo, ext, cell):
    """Reference 30-bit Morton key (10 bits per axis) on cells of size `cell`, or of 1/1024 of the
    bounding cube when 1024 cells do not cover it; integer bit interleaving."""
    scale = np.float32(1024.0) / np.float32(ext) if ext > 0 else np.float32(0)
    if cell > 0 and not (np.float32(ext) > np.float32(1024.0) * np.float32(cell)):
        scale = np.float32(1.0) / np.float32(cell)
    q = np.clip(((p - lo).astype(np.float32) * scale).astype(np.int64), 0, 1023)
    key = np.zeros(len(p), dtype=np.int64)
    for b in range(10):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            key |= ((q[:, a] >> b) & 1) << (3 * b + sh)
    return key


@pytest.mark.parametrize("m,bucket,cell", [(1, 16, 0.008), (33, 8, 0.008), (5000, 16, 0.008), (100_000, 32, 0.002),
                                          (100_000, 16, 0.05)])
def test_map_index_is_morton_sorted_with_tight_boxes(g, ctx, m, bucket, cell):
    rng = np.random.default_rng(m)
    means = rng.uniform([-1, 0, 2], [3, 2, 2.5], size=(m, 3)).astype(np.float32)
    covs = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (m, 1))
    mp = g.gsicp_build_map_index(ctx, cu(means), cu(covs), bucket=bucket, cell=cell)
    ins = g.gsicp_map_inspect(mp)
    pts = ins["pts"].cpu().numpy()
    order = pts[:, 3].copy().view(np.int32)
    assert sorted(order.tolist()) == list(range(m))  # a permutation
    np.testing.assert_array_equal(pts[:, :3], means[order])
    lo = means.min(0)
    ext = float((means.max(0) - lo).max())
    key = _morton30(means[order], lo, ext, cell)
    assert np.all(np.diff(key) >= 0)  # Morton order
    # stable: equal keys keep input order
    same = np.diff(key) == 0
    assert np.all(np.diff(order)[same] > 0)
    L, B = ins["L"], ins["B"]
    assert B == bucket and L >= (m + B - 1) // B and (L & (L - 1)) == 0
    boxes = ins["boxes"].cpu().numpy()
    for leaf in range(L):
        seg = pts[leaf * B:min((leaf + 1) * B, m), :3]
        blo, bhi = boxes[L + leaf, :3], boxes[L + leaf, 4:7]
        if len(seg):
            np.testing.assert_array_equal(blo, seg.min(0))
            np.testing.assert_array_equal(bhi, seg.max(0))
        else:
            assert np.all(np.isinf(blo)) and np.all(blo > 0) and np.all(bhi < 0)
    for node in range(1, L):
        c0, c1 = boxes[2 * node], boxes[2 * node + 1]
        np.testing.assert_array_equal(boxes[node, :3], np.minimum(c0[:3], c1[:3]))
        np.testing.assert_array_equal(boxes[node, 4:7], np.maximum(c0[4:7], c1[4:7]))
    mp.close()


# ----------------------------------------------------------------------------- a4 + a5 nearest neighbours

def _check_nearest(map_pts, queries, max_dist, g, ctx, bucket=0, cell=0.0):
    covs = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (len(map_pts), 1))
    m = g.gsicp_build_map_index(ctx, cu(map_pts), cu(covs), bucket=bucket, cell=cell)
    idx, d2 = g.gsicp_map_nearest(ctx, m, cu(queries), max_dist)
    idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
    io, do = orc.KDTree(map_pts).nn(queries, float(np.float32(max_dist)))
    r2 = float(np.float32(max_dist)) ** 2
    diff = np.nonzero(idx != io)[0]
    P, Q = map_pts.astype(np.float64), queries.astype(np.float64)
    for i in diff:
        if idx[i] < 0 or io[i] < 0:  # inlier decision differs only at the radius boundary
            dd = do[i] if io[i] >= 0 else np.sum((P[idx[i]] - Q[i]) ** 2)
            assert abs(dd - r2) <= 1e-6 * r2
        else:
            dg = np.sum((P[idx[i]] - Q[i]) ** 2)
            assert dg <= do[i] * (1 + 1e-6)
    fin = idx >= 0
    np.testing.assert_allclose(d2[fin], np.sum((P[idx[fin]] - Q[fin]) ** 2, axis=1), rtol=1e-6, atol=1e-12)
    m.close()
    return len(diff)


@pytest.mark.parametrize("bucket,cell", [(8, 0.0), (16, 0.0), (32, 0.0), (16, 0.02), (16, 0.1), (16, 0.5)])
def test_map_nearest_small(g, ctx, bucket, cell):
    rng = np.random.default_rng(bucket)
    for m_n in (1, 7, 100, 5000):
        mp = rng.uniform(-1, 1, size=(m_n, 3)).astype(np.float32)
        q = np.concatenate([rng.uniform(-1.2, 1.2, size=(3000, 3)), mp[: min(m_n, 500)],
                            mp[: min(m_n, 500)] + rng.normal(0, 0.01, size=(min(m_n, 500), 3))]).astype(np.float32)
        assert _check_nearest(mp, q, 0.1, g, ctx, bucket, cell) <= 2


def test_map_nearest_ties(g, ctx):
    mp = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 0, 0]], np.float32)
    q = np.zeros((1, 3), np.float32)
    m = g.gsicp_build_map_index(ctx, cu(mp), cu(np.tile([1, 0, 0, 1, 0, 1], (6, 1)).astype(np.float32)))
    idx, _ = g.gsicp_map_nearest(ctx, m, cu(q), 2.0)
    assert idx.item() == 0
    idx, _ = g.gsicp_map_nearest(ctx, m, cu(q), 1.0)  # boundary inclusive
    assert idx.item() == 0
    idx, _ = g.gsicp_map_nearest(ctx, m, cu(q), 0.999)
    assert idx.item() == -1


def test_map_nearest_config2_full_size(g, ctx):
    """2M-Gaussian map, 200k queries: every answer checked against the oracle."""
    f, means, _ = _cfg2()
    pts, _ = oracle_frame_points(f["depth"])
    q = transform_points(f["T0"], pts.astype(np.float64)).astype(np.float32)
    nd = _check_nearest(means, q, 0.1, g, ctx)
    assert nd < 1e-4 * len(q)


# ----------------------------------------------------------------------------- a5 + a6 linearisation

def test_linearise_matches_oracle(g, ctx):
    src, cs, tgt, ct, T_gt = config1_inputs(0, 0)
    m = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    om = orc.Map(tgt, ct)
    for T in (np.eye(4), T_gt, T_gt @ random_offset(np.random.default_rng(1), 1.0, 0.01)):
        lg = g.gsicp_linearise(ctx, cu(src), cu(cs), m, T, 0.1)
        lo = orc.linearise(src, cs, om, T, 0.1)
        corr = lg["corr"].cpu().numpy()
        bad = np.nonzero(corr != lo["corr"])[0]
        mism = len(bad)
        assert mism <= 1e-3 * len(src)
        # a differing correspondence is a near-tie under the float transform (|y| * 1e-6 m)
        y = transform_points(T, src.astype(np.float64))
        for i in bad:
            dg = np.linalg.norm(tgt[corr[i]] - y[i]) if corr[i] >= 0 else 0.1
            do = np.linalg.norm(tgt[lo["corr"][i]] - y[i]) if lo["corr"][i] >= 0 else 0.1
            assert abs(dg - do) <= 1e-6 * (1 + np.linalg.norm(y[i])), (i, dg, do)
        assert abs(lg["inliers"] - lo["inliers"]) <= mism
        herr = np.linalg.norm(lg["H"] - lo["H"]) / np.linalg.norm(lo["H"])
        berr = np.linalg.norm(lg["b"] - lo["b"]) / max(np.linalg.norm(lo["b"]), 1e-12)
        cerr = abs(lg["cost"] - lo["cost"]) / max(lo["cost"], 1e-12)
        assert herr < 1e-3 and cerr < 1e-3 and (berr < 1e-2 or np.linalg.norm(lo["b"]) < 1e-3 * np.linalg.norm(lo["H"])), \
            (herr, berr, cerr, mism)
        # the squared Euclidean residuals of the inliers (the tracker's fallback residual), against
        # the sum over the oracle's own correspondences (near-ties differ by ~1e-6 m each)
        sq, ninl = g.gsicp_ctx_last_residual(ctx)
        sel = lo["corr"] >= 0
        sq_o = float(np.sum((tgt[lo["corr"][sel]].astype(np.float64) - y[sel]) ** 2))
        assert ninl == lg["inliers"] and abs(sq - sq_o) <= 1e-5 * sq_o + mism * 1e-3 * 0.01, (sq, sq_o)
    m.close()


# ----------------------------------------------------------------------------- a5-a7 registration

@pytest.mark.parametrize("scene_seed,pose_seed", [(0, 0), (1, 1), (2, 2), (3, 0), (4, 1)])
def test_register_config1_matches_oracle(g, ctx, scene_seed, pose_seed):
    src, cs, tgt, ct, T_gt = config1_inputs(scene_seed, pose_seed)
    rg_ = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    m = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    rg = g.gsicp_register(ctx, cu(src), cu(cs), m, np.eye(4), rg_)
    ro = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4), 0.1, 30, 1e-6, 1e-6, 6)
    assert rg["status"] == g.OK and ro["status"] == orc.OK
    dr, dt = pose_diff(rg["T"], ro["T"])
    assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (dr, dt, rg["iters"], ro["iters"])
    # and the oracle itself recovers the ground truth to the sampling-noise level
    gr, gt = pose_diff(ro["T"], T_gt)
    assert gr < np.deg2rad(0.5) and gt < 0.01
    m.close()


def test_register_end_to_end_gpu_covariances(g, ctx):
    """GPU covariances -> GPU registration vs oracle covariances -> oracle registration."""
    import synth
    src, tgt, T_gt = synth.pair_config1(5, 0, n=10_000)
    p = g.CovParams(20, 1e-3, g.PLANE, 0.0)
    cs_g = g.gsicp_source_covariances(ctx, cu(src), None, p)
    ct_g = g.gsicp_source_covariances(ctx, cu(tgt), None, p)
    m = g.gsicp_build_map_index(ctx, cu(tgt), ct_g)
    rg = g.gsicp_register(ctx, cu(src), cs_g, m, np.eye(4), g.RegParams())
    cs = orc.source_covariances(src, k=20, reg_mode=orc.PLANE)["covs"]
    ct = orc.source_covariances(tgt, k=20, reg_mode=orc.PLANE)["covs"]
    ro = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4))
    dr, dt = pose_diff(rg["T"], ro["T"])
    assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (dr, dt)


def test_register_degenerate_and_edge_cases(g, ctx):
    src, cs, tgt, ct, _ = config1_inputs(0, 0, n=2000)
    m = g.gsicp_build_map_index(ctx, cu(tgt + 10.0), cu(ct))  # far away: no correspondences
    r = g.gsicp_register(ctx, cu(src), cu(cs), m, np.eye(4), g.RegParams())
    assert r["status"] == g.ERR_DEGENERATE and r["inliers"] == 0 and r["iters"] == 1
    np.testing.assert_array_equal(r["T"], np.eye(4))
    # empty source
    m2 = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    r = g.gsicp_register(ctx, cu(src[:0]), cu(cs[:0]), m2, np.eye(4), g.RegParams())
    assert r["status"] == g.ERR_DEGENERATE
    # empty map
    m3 = g.gsicp_build_map_index(ctx, cu(tgt[:0]), cu(ct[:0]))
    r = g.gsicp_register(ctx, cu(src), cu(cs), m3, np.eye(4), g.RegParams())
    assert r["status"] == g.ERR_DEGENERATE
    # a single iteration equals the oracle's single iteration
    r = g.gsicp_register(ctx, cu(src), cu(cs), m2, np.eye(4), g.RegParams(max_iters=1))
    ro = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4), max_iters=1)
    assert r["iters"] == 1 and ro["iters"] == 1
    dr, dt = pose_diff(r["T"], ro["T"])
    assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL
    # invalid arguments are rejected without touching the device
    with pytest.raises(g.GsicpError) as e:
        g.gsicp_register(ctx, cu(src), cu(cs), m2, np.eye(4), g.RegParams(max_iters=0))
    assert e.value.status == g.ERR_INVALID_ARG
    for mm in (m, m2, m3):
        mm.close()


def test_map_append_equals_full_build(g, ctx):
    src, cs, tgt, ct, _ = config1_inputs(1, 0, n=4000)
    a = g.gsicp_build_map_index(ctx, cu(tgt[:1500]), cu(ct[:1500]))
    g.gsicp_map_append(ctx, a, cu(tgt[1500:]), cu(ct[1500:]))
    b = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    assert a.size == b.size == 4000
    ra = g.gsicp_register(ctx, cu(src), cu(cs), a, np.eye(4), g.RegParams())
    rb = g.gsicp_register(ctx, cu(src), cu(cs), b, np.eye(4), g.RegParams())
    np.testing.assert_array_equal(ra["T"], rb["T"])


def test_transform_gaussians(g, ctx):
    rng = np.random.default_rng(0)
    pts = rng.normal(size=(1000, 3)).astype(np.float32)
    covs = rng.normal(size=(1000, 6)).astype(np.float32)
    T = random_offset(rng, 30, 1.0)
    po, co = g.gsicp_transform_gaussians(T, cu(pts), cu(covs))
    ro, rc = orc.transform_gaussians(T, pts, covs)
    np.testing.assert_allclose(po.cpu().numpy(), ro, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(co.cpu().numpy(), rc, rtol=1e-5, atol=1e-5)


# ----------------------------------------------------------------------------- whole frame (config 2, full size)

_CFG2 = {}


def _cfg2():
    if not _CFG2:
        _CFG2["v"] = config2_inputs(0)
    return _CFG2["v"]


def test_track_frame_config2_matches_oracle(g, ctx):
    """1200x680 frame (~204k points) against a 2M-Gaussian map, in the launch
    configuration the benchmark times."""
    f, means, covs = _cfg2()
    m = g.gsicp_build_map_index(ctx, cu(means), cu(covs))
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    r = g.gsicp_track_frame(ctx, cu(f["depth"]), REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp, m, f["T0"], rp)
    pts, z = oracle_frame_points(f["depth"])
    cs = orc.source_covariances(pts, z, k=20, eps=1e-3, reg_mode=orc.PLANE, p=1.5)["covs"]
    ro = orc.register(pts, cs, orc.Map(means, covs), f["T0"], 0.1, 30, 1e-6, 1e-6, 6)
    assert r["status"] == g.OK and ro["status"] == orc.OK
    assert r["n_points"] == len(pts)
    dr, dt = pose_diff(r["T"], ro["T"])
    assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (dr, dt, r["iters"], ro["iters"])
    # host-buffer entry point gives the same answer
    rh = g.gsicp_track_frame_host(ctx, f["depth"], REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp, m, f["T0"], rp)
    np.testing.assert_array_equal(rh["T"], r["T"])
    m.close()


@pytest.mark.parametrize("stride", [1, 2, 3])
def test_track_frame_host_uploads_sampled_rows(g, ctx, stride):
    """The host-buffer frame call uploads only the rows a1 samples (every stride-th, a 2D copy);
    its points and pose equal gsicp_track_frame's on the whole device image bit for bit, with a
    height that is not a multiple of the stride, from a pinned tensor and from a numpy array."""
    intr, d = _depth_case(203, 157, 11)
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    pts, z = orc.depth_to_points(d, intr.as_array(), 1, 0.1, 10.0)
    cs = orc.source_covariances(pts, z, k=20, reg_mode=orc.PLANE)["covs"].astype(np.float32)
    m = g.gsicp_build_map_index(ctx, cu(pts.astype(np.float32)), cu(cs))
    T0 = random_offset(np.random.default_rng(3), 1.0, 0.01)
    r = g.gsicp_track_frame(ctx, cu(d), intr.as_array(), stride, 0.1, 10.0, cp, m, T0, rp)
    pinned = torch.from_numpy(np.ascontiguousarray(d)).pin_memory()
    for host in (pinned, d):
        rh = g.gsicp_track_frame_host(ctx, host, intr.as_array(), stride, 0.1, 10.0, cp, m, T0, rp)
        assert rh["n_points"] == r["n_points"] > 0
        for key in ("T", "H"):
            np.testing.assert_array_equal(rh[key], r[key])
        assert (rh["iters"], rh["inliers"], rh["cost"]) == (r["iters"], r["inliers"], r["cost"])
    m.close()


def test_coop_walks_do_not_change_results(g, ctx):
    """The cooperative tree walk (a whole warp per query), the packet walk (a warp for all of its
    points' nearest points) and the per-point walk are all exact: the full-size frame and a
    config-1 registration give bit-identical poses, systems, iteration counts and refresh counts
    whichever is used (threshold 0 = never together, 32 = always; packet walks in none, the first,
    or every iteration)."""
    f, means, covs = _cfg2()
    m = g.gsicp_build_map_index(ctx, cu(means), cu(covs))
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    src, cs, tgt, ct, _ = config1_inputs(1, 2)
    m1 = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    T1 = random_offset(np.random.default_rng(7), 5.0, 0.05)
    out = {}
    settings = ((0, 0), (4, 0), (32, 0), (4, 1), (0, 30))  # (cooperative-walk threshold, packet iterations)
    try:
        for c, pk in settings:
            g.gsicp_ctx_set_coop_walks(ctx, c)
            g.gsicp_ctx_set_packet_iters(ctx, pk)
            r = g.gsicp_track_frame(ctx, cu(f["depth"]), REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp, m, f["T0"], rp)
            st = g.gsicp_ctx_reg_stats(ctx, r["iters"])
            r1 = g.gsicp_register(ctx, cu(src), cu(cs), m1, T1, rp)
            out[(c, pk)] = (r, st["refreshes"], r1)
    finally:
        g.gsicp_ctx_set_coop_walks(ctx, 4)
        g.gsicp_ctx_set_packet_iters(ctx, 1)
    r0, ref0, r10 = out[(0, 0)]
    assert r0["status"] == g.OK and r10["status"] == g.OK
    for key in settings[1:]:
        r, ref, r1 = out[key]
        for key in ("T", "H"):
            np.testing.assert_array_equal(r[key], r0[key])
            np.testing.assert_array_equal(r1[key], r10[key])
        assert (r["iters"], r["cost"], r["inliers"]) == (r0["iters"], r0["cost"], r0["inliers"])
        assert (r1["iters"], r1["cost"], r1["inliers"]) == (r10["iters"], r10["cost"], r10["inliers"])
        assert list(ref) == list(ref0)
    with pytest.raises(RuntimeError):
        g.gsicp_ctx_set_coop_walks(ctx, 33)
    m.close()
    m1.close()


@pytest.mark.parametrize("d", [0.003, 0.04])
def test_near_ties_follow_the_exact_query_on_every_search_path(g, ctx, d):
    """Pairs of map points equidistant from y = T x to within the float rounding of y, where the
    rounded query (hi alone) orders the two the other way round: every search path -- the grid
    block (d = 3 mm, certified), and beyond it (d = 40 mm) per-point, cooperative and packet walks
    -- returns the nearest by the hi + lo query, i.e. the oracle's FP64 correspondence, bit for bit."""
    from ._util import near_tie_pairs
    src, cs, means, covs, T, nearest, flipped = near_tie_pairs(5, d)
    assert flipped.mean() > 0.9
    lo = orc.linearise(src, cs, orc.Map(means, covs), T, 0.1)
    np.testing.assert_array_equal(lo["corr"], nearest)
    m = g.gsicp_build_map_index(ctx, cu(means), cu(covs))
    try:
        for coop, pk in ((0, 0), (32, 0), (2, 1), (0, 1)):
            g.gsicp_ctx_set_coop_walks(ctx, coop)
            g.gsicp_ctx_set_packet_iters(ctx, pk)
            lg = g.gsicp_linearise(ctx, cu(src), cu(cs), m, T, 0.1)
            np.testing.assert_array_equal(lg["corr"].cpu().numpy(), nearest, err_msg=f"coop {coop} packet {pk}")
            assert lg["inliers"] == len(src)
    finally:
        g.gsicp_ctx_set_coop_walks(ctx, 4)
        g.gsicp_ctx_set_packet_iters(ctx, 1)
        m.close()


def test_cache_step_does_not_change_results(g, ctx):
    """Every search (grid block, per-point, packet and cooperative walks, a cache check) returns the
    nearest map point by the same hi + lo distance, so the cache step, which only decides when a
    point builds a cache instead of searching alone, leaves poses, systems, iteration counts and
    inliers bit-identical: the full-size frame and a config-1 registration; 0 = never cache."""
    f, means, covs = _cfg2()
    m = g.gsicp_build_map_index(ctx, cu(means), cu(covs))
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    src, cs, tgt, ct, _ = config1_inputs(1, 2)
    m1 = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    T1 = random_offset(np.random.default_rng(7), 5.0, 0.05)
    out = {}
    steps = (0.0005, 0.0, 0.0003, 0.001, 0.002, 0.005)
    try:
        for step in steps:
            g.gsicp_ctx_set_cache_step(ctx, step)
            r = g.gsicp_track_frame(ctx, cu(f["depth"]), REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp, m, f["T0"], rp)
            refreshes = sum(g.gsicp_ctx_reg_stats(ctx, r["iters"])["refreshes"])
            r1 = g.gsicp_register(ctx, cu(src), cu(cs), m1, T1, rp)
            out[step] = (r, r1, refreshes)
    finally:
        g.gsicp_ctx_set_cache_step(ctx, 0.0005)  # the library default
    r0, r10, _ = out[steps[0]]
    assert r0["status"] == g.OK and r10["status"] == g.OK
    for step in steps[1:]:
        r, r1, _ = out[step]
        for key in ("T", "H"):
            np.testing.assert_array_equal(r[key], r0[key])
            np.testing.assert_array_equal(r1[key], r10[key])
        assert (r["iters"], r["cost"], r["inliers"]) == (r0["iters"], r0["cost"], r0["inliers"])
        assert (r1["iters"], r1["cost"], r1["inliers"]) == (r10["iters"], r10["cost"], r10["inliers"])
    assert out[0.0][2] > out[0.0005][2]  # with no caches every point searches in every iteration
    for bad in (-1e-3, float("nan"), float("inf")):
        with pytest.raises(RuntimeError):
            g.gsicp_ctx_set_cache_step(ctx, bad)
    m.close()
    m1.close()


def test_gn_launch_modes_give_identical_results(g, ctx):
    """The Gauss-Newton iterations as one conditional graph (default) and as plain launches give
    bit-identical results: a config-1 registration and the full-size frame."""
    f, means, covs = _cfg2()
    m = g.gsicp_build_map_index(ctx, cu(means), cu(covs))
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    src, cs, tgt, ct, _ = config1_inputs(2, 1)
    m1 = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    out = {}
    try:
        for mode in (g.GN_GRAPH, g.GN_PLAIN):
            g.gsicp_ctx_set_gn_launch_mode(ctx, mode)
            r = g.gsicp_track_frame(ctx, cu(f["depth"]), REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp, m, f["T0"], rp)
            r1 = g.gsicp_register(ctx, cu(src), cu(cs), m1, np.eye(4), rp)
            out[mode] = (r, r1)
    finally:
        g.gsicp_ctx_set_gn_launch_mode(ctx, g.GN_GRAPH)
    for a, b in zip(out[g.GN_GRAPH], out[g.GN_PLAIN]):
        assert a["status"] == b["status"] == g.OK
        np.testing.assert_array_equal(a["T"], b["T"])
        np.testing.assert_array_equal(a["H"], b["H"])
        assert (a["iters"], a["cost"], a["inliers"]) == (b["iters"], b["cost"], b["inliers"])
    with pytest.raises(g.GsicpError):
        g.gsicp_ctx_set_gn_launch_mode(ctx, 2)
    m.close()
    m1.close()


def test_gn_block_sizes_meet_the_oracle(g, ctx):
    """128, 256 and 384 source points per Gauss-Newton block: the rows of the reduction change with
    the block, so the sums' order does, but every size lands on the oracle's pose within the bar (the
    full-size frame and a config-1 pair); 256 stays the batched kernel's bits (checked by the batch
    tests)."""
    f, means, covs = _cfg2()
    m = g.gsicp_build_map_index(ctx, cu(means), cu(covs))
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    src, cs, tgt, ct, _ = config1_inputs(0, 0)
    m1 = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    pts, z = oracle_frame_points(f["depth"])
    cso = orc.source_covariances(pts, z, k=20, eps=1e-3, reg_mode=orc.PLANE, p=1.5)["covs"]
    ro = orc.register(pts, cso, orc.Map(means, covs), f["T0"], 0.1, 30, 1e-6, 1e-6, 6)
    ro1 = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4), 0.1, 30, 1e-6, 1e-6, 6)
    try:
        for bs in (128, 384, 256):
            g.gsicp_ctx_set_gn_block(ctx, bs)
            r = g.gsicp_track_frame(ctx, cu(f["depth"]), REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp, m, f["T0"], rp)
            r1 = g.gsicp_register(ctx, cu(src), cu(cs), m1, np.eye(4), rp)
            for a, b in ((r, ro), (r1, ro1)):
                assert a["status"] == g.OK
                dr, dt = pose_diff(a["T"], b["T"])
                assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (bs, dr, dt, a["iters"], b["iters"])
    finally:
        g.gsicp_ctx_set_gn_block(ctx, 256)
    with pytest.raises(g.GsicpError):
        g.gsicp_ctx_set_gn_block(ctx, 64)
    m.close()
    m1.close()


def test_track_frame_empty_depth(g, ctx):
    src, cs, tgt, ct, _ = config1_inputs(0, 0, n=2000)
    m = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    d = np.zeros((68, 120), np.float32)
    r = g.gsicp_track_frame(ctx, cu(d), [60, 60, 59.5, 33.5], 2, 0.1, 10.0, g.CovParams(), m, np.eye(4),
                            g.RegParams())
    assert r["status"] == g.ERR_DEGENERATE and r["n_points"] == 0


# ----------------------------------------------------------------------------- batched registration

def test_register_batch_equals_single_and_oracle(g, ctx):
    """Pairs of uneven sizes (incl. an empty source and one below a chunk) in one persistent
    launch: each pair's result equals gsicp_register on it alone, bit for bit, and the oracle's
    within the pose bar."""
    sizes = [6000, 0, 150, 23000, 1200, 9000, 40]
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    pairs, maps = [], []
    for b, n in enumerate(sizes):
        src, cs, tgt, ct, T_gt = config1_inputs(b % 5, b % 3, n=max(n, 300))
        src, cs = src[:n], cs[:n]
        pairs.append((src, cs, tgt, ct))
        maps.append(g.gsicp_build_map_index(ctx, cu(tgt), cu(ct)))
    T0s = np.stack([random_offset(np.random.default_rng(50 + b), 1.0, 0.01) for b in range(len(sizes))])
    rb = g.gsicp_register_batch(ctx, [cu(p[0]).reshape(-1, 3) for p in pairs], [cu(p[1]).reshape(-1, 6) for p in pairs],
                                maps, T0s, rp)
    for b, (src, cs, tgt, ct) in enumerate(pairs):
        if len(src) == 0:
            assert rb["status"][b] == g.ERR_DEGENERATE and rb["iters"][b] == 0
            np.testing.assert_array_equal(rb["T"][b], T0s[b])
            continue
        rs = g.gsicp_register(ctx, cu(src), cu(cs), maps[b], T0s[b], rp)
        assert rb["status"][b] == rs["status"], b
        np.testing.assert_array_equal(rb["T"][b], rs["T"])
        assert rb["iters"][b] == rs["iters"] and rb["inliers"][b] == rs["inliers"] and rb["cost"][b] == rs["cost"]
        if rs["status"] == g.OK and len(src) >= 1000:
            ro = orc.register(src, cs, orc.Map(tgt, ct), T0s[b], 0.1, 30, 1e-6, 1e-6, 6)
            dr, dt = pose_diff(rb["T"][b], ro["T"])
            assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (b, dr, dt)
    # a second batch on the same context reuses its buffers and gives the same answer
    rb2 = g.gsicp_register_batch(ctx, [cu(p[0]).reshape(-1, 3) for p in pairs], [cu(p[1]).reshape(-1, 6) for p in pairs],
                                 maps, T0s, rp)
    np.testing.assert_array_equal(rb2["T"], rb["T"])
    for m in maps:
        m.close()


def test_register_batch_config4_sizes_equal_single_and_oracle(g, ctx):
    """Pairs of the batched workload itself (64 config-1-style rooms, 5k-300k points): the four
    largest-class pairs drawn (133k-276k points) and two that stop at max_iters = 30 in a
    re-association limit cycle, in one persistent launch.  Each pair equals gsicp_register on it
    alone bit for bit (pose, cost, inliers, iterations) and the oracle within the pose bar;
    the limit-cycle pairs run the full 30 iterations on every side."""
    from synth import batch_config4
    pick = [5, 55, 27, 8, 11, 49]
    allp = batch_config4(0, n_pairs=64)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    srcs, scovs, maps, ins = [], [], [], []
    for b in pick:
        p = allp[b]
        cs = orc.source_covariances(p["src"], k=20, eps=1e-3, reg_mode=orc.PLANE)["covs"].astype(np.float32)
        ct = orc.source_covariances(p["tgt"], k=20, eps=1e-3, reg_mode=orc.PLANE)["covs"].astype(np.float32)
        srcs.append(cu(p["src"]))
        scovs.append(cu(cs))
        maps.append(g.gsicp_build_map_index(ctx, cu(p["tgt"]), cu(ct)))
        ins.append((p["src"], cs, p["tgt"], ct))
    T0s = np.stack([np.eye(4)] * len(pick))
    rb = g.gsicp_register_batch(ctx, srcs, scovs, maps, T0s, rp)
    assert max(len(s_[0]) for s_ in ins) > 250_000
    for j, b in enumerate(pick):
        src, cs, tgt, ct = ins[j]
        rs = g.gsicp_register(ctx, srcs[j], scovs[j], maps[j], T0s[j], rp)
        assert rb["status"][j] == rs["status"] == g.OK, (b, rb["status"][j], rs["status"])
        np.testing.assert_array_equal(rb["T"][j], rs["T"])
        assert (rb["iters"][j], rb["inliers"][j], rb["cost"][j]) == (rs["iters"], rs["inliers"], rs["cost"]), b
        ro = orc.register(src, cs, orc.Map(tgt, ct), T0s[j], 0.1, 30, 1e-6, 1e-6, 6)
        assert ro["status"] == orc.OK
        dr, dt = pose_diff(rb["T"][j], ro["T"])
        assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (b, dr, dt, rb["iters"][j], ro["iters"])
        if b in (11, 49):
            assert rb["iters"][j] == ro["iters"] == 30, (b, rb["iters"][j], ro["iters"])
    for m in maps:
        m.close()


def test_register_batch_queue_wait_is_bounded(g, ctx):
    """A queue that claims a running pair but never gets an item: every wait runs out (about a
    second), the call reports TIMEOUT, and the context keeps working."""
    import time
    t0 = time.time()
    assert g.gsicp_selftest_batch_timeout(ctx) == g.ERR_TIMEOUT
    assert time.time() - t0 < 30
    src, cs, tgt, ct, _ = config1_inputs(0, 0, n=3000)
    m = g.gsicp_build_map_index(ctx, cu(tgt), cu(ct))
    r = g.gsicp_register_batch(ctx, [cu(src)], [cu(cs)], [m], np.eye(4)[None], g.RegParams(0.1, 30, 1e-6, 1e-6, 6))
    rs = g.gsicp_register(ctx, cu(src), cu(cs), m, np.eye(4), g.RegParams(0.1, 30, 1e-6, 1e-6, 6))
    np.testing.assert_array_equal(r["T"][0], rs["T"])
    m.close()


def test_register_batch_empty(g, ctx):
    r = g.gsicp_register_batch(ctx, [], [], [], np.zeros((0, 4, 4)), g.RegParams())
    assert r["T"].shape == (0, 4, 4)


# ----------------------------------------------------------------------------- a1+a2+a3 of a depth frame

def _frame_cases():
    scene = make_room(3)
    rng = np.random.default_rng(55)
    P = circle_poses(rng, scene, 1)[0]
    vga = Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5)
    small = Intrinsics(40, 30, 30.0, 30.0, 19.5, 14.5)
    tiny = Intrinsics(7, 5, 6.0, 6.0, 3.0, 2.0)
    return [(REPLICA_INTR, 2, 0.0), (vga, 1, 0.0), (vga, 2, 0.3), (vga, 3, 0.0), (small, 1, 0.1), (tiny, 1, 0.0)], \
        scene, P


_FRAME_DEPTHS = {}


def _frame_depth(case):
    """Depth image of frame case `case` (rendered once per module)."""
    if case not in _FRAME_DEPTHS:
        cases, scene, P = _frame_cases()
        intr, stride, dropout = cases[case]
        rng = np.random.default_rng(100 + case)
        _FRAME_DEPTHS[case] = (intr, stride, add_depth_noise(raycast_depth(scene, P, intr), rng, 1e-3,
                                                             dropout=dropout))
    return _FRAME_DEPTHS[case]


@pytest.mark.parametrize("k", [5, 8, 12, 16, 20, 32])
@pytest.mark.parametrize("mode", [orc.PLANE, orc.ELLIPSE, orc.NONE])
def test_frame_covariances_equal_tree_path(g, ctx, mode, k):
    """The image-window k-NN (certified by the camera geometry, tree search for the rest) gives
    bit-for-bit the points of gsicp_depth_to_points and the covariances of
    gsicp_source_covariances on them: both are the exact float k-NN with the same ties.  Every
    regularisation (Sec. 3.1: plane, ellipse, none) and every neighbour-list width the window
    kernels are built for (8, 16, 20, 32; k = 5 and 12 run inside the 8- and 16-wide lists), with
    and without scale aligning (Sec. 3.2), on six frames from 1200 x 680 at stride 2 down to 7 x 5."""
    for case in range(6):
        intr, stride, depth = _frame_depth(case)
        for p in (1.5, 0.0):
            cp = g.CovParams(k, 1e-3, mode, p)
            pf, zf, cf = g.gsicp_frame_covariances(ctx, cu(depth), intr.as_array(), stride, 0.1, 10.0, cp)
            fs = g.gsicp_ctx_frame_stats(ctx)
            pts, z = g.gsicp_depth_to_points(ctx, cu(depth), intr.as_array(), stride, 0.1, 10.0)
            pts, z = pts.clone(), z.clone()
            ct = g.gsicp_source_covariances(ctx, pts, z, cp)
            assert torch.equal(pf, pts) and torch.equal(zf, z)
            assert 0 <= fs["tree_queries"] <= fs["wide_window_queries"] <= len(pts)
            bad = (cf != ct).any(dim=1).nonzero().flatten().cpu().numpy()
            assert len(bad) == 0, (case, mode, k, p, len(bad), fs, len(pts))


@pytest.mark.parametrize("mode", [orc.PLANE, orc.ELLIPSE, orc.NONE])
def test_frame_covariances_full_bench_frame_match_oracle(g, ctx, mode):
    """The 1200 x 680 frame the benchmark tracks (stride 2, 204,000 points), through the image-window
    path the tracker runs, against the oracle directly: the neighbour lists (exported by the tree
    path, which the window path equals bit for bit) identical up to distance ties, covariances
    within the relative Frobenius bar with the exclusions counted, for each regularisation."""
    f, _, _ = _cfg2()
    cp = g.CovParams(20, 1e-3, mode, 1.5)
    pf, zf, cf = g.gsicp_frame_covariances(ctx, cu(f["depth"]), REPLICA_INTR.as_array(), 2, 0.1, 10.0, cp)
    pts, z = oracle_frame_points(f["depth"])
    np.testing.assert_array_equal(pf.cpu().numpy(), pts)
    np.testing.assert_array_equal(zf.cpu().numpy(), z)
    ct = g.gsicp_source_covariances(ctx, pf.clone(), zf.clone(), cp)
    assert torch.equal(cf, ct)
    r = _check_knn_and_covs(pts, z, mode, 1.5, 20, g, ctx)
    assert r["n"] == 204_000 and r["excluded"] < 0.01 * r["n"], r
    assert r["knn_mismatch"] < 1e-3 * r["n"], r
    # cf equals the tree path's covariances bit for bit, so the bar just checked holds for it


def test_frame_covariances_match_oracle(g, ctx):
    cases, scene, P = _frame_cases()
    intr, stride, dropout = cases[2]
    depth = add_depth_noise(raycast_depth(scene, P, intr), np.random.default_rng(7), 1e-3, dropout=dropout)
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    pf, zf, cf = g.gsicp_frame_covariances(ctx, cu(depth), intr.as_array(), stride, 0.1, 10.0, cp)
    pts, z = oracle_frame_points(depth, intr, stride)
    np.testing.assert_array_equal(pf.cpu().numpy(), pts)
    ro = orc.source_covariances(pts, z, k=20, eps=1e-3, reg_mode=orc.PLANE, p=1.5)
    keep = ro["gap"] >= PLANE_GAP_EXCLUDE
    err = cov_rel_err(cf.cpu().numpy().astype(np.float64), ro["covs"])
    assert np.all(err[keep] <= COV_REL_TOL), (err[keep].max(), int((~keep).sum()))
    assert (~keep).mean() < 0.01


def test_frame_covariances_capacity_and_empty(g, ctx):
    intr = Intrinsics(16, 12, 12.0, 12.0, 7.5, 5.5)
    d = np.full((12, 16), 2.0, np.float32)
    cap = 10
    pts = torch.empty((cap, 3), device="cuda")
    z = torch.empty((cap,), device="cuda")
    covs = torch.empty((cap, 6), device="cuda")
    import ctypes as C
    n = C.c_int64(0)
    fi = (C.c_float * 4)(*intr.as_array().tolist())
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    st = g.lib.gsicp_frame_covariances(ctx.ptr, cu(d).data_ptr(), 16, 12, fi, 1, 0.1, 10.0, C.byref(cp),
                                       pts.data_ptr(), z.data_ptr(), covs.data_ptr(), cap, C.byref(n), None)
    torch.cuda.synchronize()
    assert st == g.ERR_CAPACITY and n.value == cap
    pf, zf, cf = g.gsicp_frame_covariances(ctx, cu(np.zeros((12, 16), np.float32)), intr.as_array(), 1, 0.1, 10.0,
                                           cp)
    assert len(pf) == 0 and len(cf) == 0


# ----------------------------------------------------------------------------- tracking loop with keyframes

def test_tracker_policy_static_camera(g, ctx):
    """The library's tracker follows the keyframe schedule and the non-overlap filter exactly as
    the oracle's on a static camera (small frames)."""
    from oracle.tracker import Tracker as OTracker
    from synth import look_pose
    intr = Intrinsics(48, 36, 40.0, 40.0, 23.5, 17.5)
    scene = make_room(2)
    P = look_pose(scene.centre + np.array([0.3, -0.2, 0.0]), 0.7, 0.2)
    depth = raycast_depth(scene, P, intr)
    trk = g.Tracker(ctx, 1, 0.1, 10.0, g.CovParams(20, 1e-3, g.PLANE, 0.0), g.RegParams(0.1, 30, 1e-6, 1e-6, 6))
    otrk = OTracker(intr.as_array(), stride=1, p=0.0)
    d = cu(depth)
    for f in range(41):
        T, info = trk.frame(d, intr.as_array(), P if f == 0 else None)
        To, io = otrk.frame(depth, P if f == 0 else None)
        assert info["kind"] == io["kind"], f
        assert (info["added_tracking"], info["added_mapping"]) == (io["added_tracking"], io["added_mapping"]), f
        dr, dt = pose_diff(T, To)
        assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL
    assert trk.map_sizes() == (len(otrk.track_means), len(otrk.map_means))
    trk.close()


def test_tracker_mapping_only_keyframe_matches_oracle(g, ctx):
    """A mapping-only keyframe that sees new geometry (Sec. 3, Additional Keyframe Selection for
    Mapping) extends the mapping map only, in the library's tracker as in the oracle's."""
    from oracle.tracker import Tracker as OTracker
    from synth import look_pose
    intr = Intrinsics(48, 36, 40.0, 40.0, 23.5, 17.5)
    scene = make_room(2)
    P = look_pose(scene.centre + np.array([0.3, -0.2, 0.0]), 0.7, 0.2)
    depth = raycast_depth(scene, P, intr)
    d2 = depth.copy()
    d2[:, 44:] += 0.5  # new geometry in the last 4 columns, under 15 % of the points
    trk = g.Tracker(ctx, 1, 0.1, 10.0, g.CovParams(20, 1e-3, g.PLANE, 0.0), g.RegParams(0.1, 30, 1e-6, 1e-6, 6))
    otrk = OTracker(intr.as_array(), stride=1, p=0.0)
    for f in range(11):
        dep = d2 if f == 10 else depth
        T, info = trk.frame(cu(dep), intr.as_array(), P if f == 0 else None)
        To, io = otrk.frame(dep, P if f == 0 else None)
        assert info["kind"] == io["kind"], f
        assert (info["added_tracking"], info["added_mapping"]) == (io["added_tracking"], io["added_mapping"]), f
        dr, dt = pose_diff(T, To)
        assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL
    assert info["kind"] == 2 and info["added_tracking"] == 0 and info["added_mapping"] > 0
    assert trk.map_sizes() == (len(otrk.track_means), len(otrk.map_means))
    trk.close()


def test_tracker_sequence_matches_oracle(g, ctx):
    """TUM-shaped sequence, 45 frames: the library's tracker and the oracle's take the same
    keyframe decisions, grow maps of the same size (up to points at the overlap radius) and track
    with the same ATE."""
    from oracle.tracker import Tracker as OTracker
    F = 45
    seq = sequence_config3(1, n_frames=F)
    io_ = seq["intr"]
    trk = g.Tracker(ctx, 2, 0.1, 10.0, g.CovParams(20, 1e-3, g.PLANE, 1.5), g.RegParams(0.1, 30, 1e-6, 1e-6, 6))
    otrk = OTracker(io_.as_array(), stride=2, p=1.5)
    est_g, est_o, kinds_g, kinds_o = [], [], [], []
    for f in range(F):
        depth = seq["depth"](f)
        T, info = trk.frame(cu(depth), io_.as_array(), seq["poses"][0] if f == 0 else None)
        To, io = otrk.frame(depth, seq["poses"][0] if f == 0 else None)
        est_g.append(T)
        est_o.append(To)
        kinds_g.append(info["kind"])
        kinds_o.append(io["kind"])
    assert kinds_g == kinds_o, (kinds_g, kinds_o)
    assert 1 in kinds_g[1:] and 2 in kinds_g  # the sequence exercises both kinds
    sg, so = trk.map_sizes(), (len(otrk.track_means), len(otrk.map_means))
    assert all(abs(a - b) <= 1e-3 * b for a, b in zip(sg, so)), (sg, so)

    def ate(est):
        return float(np.sqrt(np.mean([np.sum((est[f][:3, 3] - seq["poses"][f][:3, 3]) ** 2) for f in range(F)])))
    assert ate(est_o) < 0.01 and abs(ate(est_g) - ate(est_o)) < 1e-4, (ate(est_g), ate(est_o))
    trk.close()


# ----------------------------------------------------------------------------- TUM-shaped sequence

def test_sequence_config3_matches_oracle(g, ctx):
    """640x480 sequence at 30 Hz (stride 2, ~77k points per frame), keyframes every 10th frame
    appended to the map.  Per frame, the GPU registers against a map holding the oracle's
    Gaussians from the oracle's start pose and must land on the oracle's pose; an independent
    GPU run (its own keyframes, its own constant-velocity starts) must track as well as the
    oracle's run (ATE against the ground truth)."""
    F = 21
    seq = sequence_config3(0, n_frames=F)
    io = seq["intr"]
    intr = io.as_array()
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    depths = [seq["depth"](f) for f in range(F)]

    def ate(est):
        return float(np.sqrt(np.mean([np.sum((est[f][:3, 3] - seq["poses"][f][:3, 3]) ** 2) for f in range(F)])))

    # oracle run; the GPU is checked frame by frame against it
    om_means, om_covs, omap, gm = [], [], None, None
    est_o, worst = [], (0.0, 0.0)
    for f in range(F):
        pts, z = oracle_frame_points(depths[f], io)
        cs = orc.source_covariances(pts, z, k=20, eps=1e-3, reg_mode=orc.PLANE, p=1.5)["covs"]
        if f == 0:
            To = seq["poses"][0].copy()
        else:
            T0 = const_velocity(est_o[-1], est_o[-2] if f >= 2 else None)
            ro = orc.register(pts, cs, omap, T0, 0.1, 30, 1e-6, 1e-6, 6)
            r = g.gsicp_track_frame(ctx, cu(depths[f]), intr, 2, 0.1, 10.0, cp, gm, T0, rp)
            assert ro["status"] == orc.OK and r["status"] == g.OK, (f, ro["status"], r["status"])
            assert r["n_points"] == len(pts)
            dr, dt = pose_diff(r["T"], ro["T"])
            worst = (max(worst[0], dr), max(worst[1], dt))
            assert dr < POSE_ROT_TOL and dt < POSE_TRANS_TOL, (f, dr, dt, r["iters"], ro["iters"])
            To = ro["T"]
        est_o.append(To)
        if f % 10 == 0:
            mw, cw = orc.transform_gaussians(To, pts, cs)
            mw, cw = mw.astype(np.float32), cw.astype(np.float32)
            om_means.append(mw)
            om_covs.append(cw)
            omap = orc.Map(np.concatenate(om_means), np.concatenate(om_covs))
            if gm is None:
                gm = g.gsicp_build_map_index(ctx, cu(mw), cu(cw))
            else:
                g.gsicp_map_append(ctx, gm, cu(mw), cu(cw))
    assert gm.size == sum(len(a) for a in om_means)
    gm.close()

    # independent GPU run
    est_g, m = [], None
    for f in range(F):
        d = cu(depths[f])
        if f == 0:
            T = seq["poses"][0].copy()
        else:
            T0 = const_velocity(est_g[-1], est_g[-2] if f >= 2 else None)
            r = g.gsicp_track_frame(ctx, d, intr, 2, 0.1, 10.0, cp, m, T0, rp)
            assert r["status"] == g.OK
            T = r["T"]
        est_g.append(T)
        if f % 10 == 0:
            pts, z = g.gsicp_depth_to_points(ctx, d, intr, 2, 0.1, 10.0)
            pts, z = pts.clone(), z.clone()
            c = g.gsicp_source_covariances(ctx, pts, z, cp)
            mw, cw = g.gsicp_transform_gaussians(T, pts, c)
            if m is None:
                m = g.gsicp_build_map_index(ctx, mw, cw)
            else:
                g.gsicp_map_append(ctx, m, mw, cw)
    m.close()
    ate_o, ate_g = ate(est_o), ate(est_g)
    assert ate_o < 0.01 and ate_g < 0.01, (ate_o, ate_g)
    assert abs(ate_g - ate_o) < 10 * POSE_TRANS_TOL, (ate_g, ate_o, worst)
