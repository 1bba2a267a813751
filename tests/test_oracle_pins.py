"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute force
on tiny inputs, closed forms, textbook special cases (Kabsch), library
routines it does not call (LAPACK eigh, scipy expm, cKDTree, numpy cov), and
invariants.  No GPU is needed.
"""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial import cKDTree

import oracle as orc
from synth import (Intrinsics, Scene, inv_pose, make_pose, pair_config1, random_offset, raycast_depth,
                   rot_axis_angle, transform_points)


def _cloud(rng, n, dup=0):
    p = rng.uniform(-1, 1, size=(n, 3))
    if dup:
        p[rng.integers(0, n, dup)] = p[rng.integers(0, n, dup)]  # exact duplicates -> distance ties
    return p.astype(np.float32).astype(np.float64)


def _sym(c6):
    a, b, c, d, e, f = c6
    return np.array([[a, b, c], [b, d, e], [c, e, f]])


# ----------------------------------------------------------------------------- neighbour search

@pytest.mark.parametrize("n,k,dup", [(1, 5, 0), (7, 20, 0), (300, 20, 40), (2000, 20, 200), (2000, 1, 100)])
def test_knn_tree_equals_brute_force(n, k, dup):
    rng = np.random.default_rng(n + k)
    p = _cloud(rng, n, dup)
    # a lattice adds many exact distance ties
    lat = np.stack(np.meshgrid(*[np.arange(4.0)] * 3), -1).reshape(-1, 3) * 0.25
    p = np.concatenate([p, lat]) if n > 100 else p
    t = orc.KDTree(p)
    i1, d1 = t.knn(p, k)
    i2, d2 = orc.knn_brute(p, p, k)
    assert np.array_equal(i1, i2)
    assert np.array_equal(d1, d2)
    kk = min(k, len(p))
    # self is the first neighbour unless a duplicate with a smaller index exists
    assert np.all(d1[:, 0] == 0.0)
    # distances agree with scipy's cKDTree (a library routine the oracle does not use)
    dref, _ = cKDTree(p).query(p, k=kk)
    dref = dref.reshape(len(p), kk)
    np.testing.assert_allclose(np.sqrt(d1[:, :kk]), dref, rtol=1e-12, atol=1e-15)
    if kk < k:
        assert np.all(i1[:, kk:] == -1)


def test_knn_ties_break_to_smaller_index():
    # four points at the same distance from the origin query
    p = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 2.0]])
    idx, d2 = orc.KDTree(p).knn(np.zeros((1, 3)), 3)
    assert idx.tolist() == [[0, 1, 2]]
    p2 = p[[3, 2, 1, 0, 4]]
    idx2, _ = orc.KDTree(p2).knn(np.zeros((1, 3)), 3)
    assert idx2.tolist() == [[0, 1, 2]]


@pytest.mark.parametrize("d", [0.003, 0.04])
def test_correspondences_resolve_near_ties_by_the_fp64_query(d):
    """Sec. 3 (Eq. MLE_for_T): each transformed source point y = T x takes its nearest map mean.
    On pairs of map points equidistant from y to within the float rounding of y, where the rounded
    query orders the two the other way round, the oracle's correspondences are the brute-force
    nearest by the FP64 query (and the construction has teeth: the rounded query disagrees on
    nearly every pair)."""
    from tests._util import near_tie_pairs
    src, cs, means, covs, T, nearest, flipped = near_tie_pairs(5, d, n_side=8)
    assert flipped.mean() > 0.9
    y = src.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    d2 = ((means.astype(np.float64)[None, :, :] - y[:, None, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(np.argmin(d2, axis=1), nearest)  # brute force over the whole map
    yh = y.astype(np.float32).astype(np.float64)
    d2h = ((means.astype(np.float64)[None, :, :] - yh[:, None, :]) ** 2).sum(-1)
    assert (np.argmin(d2h, axis=1) != nearest).mean() > 0.9
    lo = orc.linearise(src, cs, orc.Map(means, covs), T, 0.1)
    np.testing.assert_array_equal(lo["corr"], nearest)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_radius_nn_tree_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    p = _cloud(rng, 3000, 300)
    q = np.concatenate([_cloud(rng, 500) * 1.2, p[:100]])
    r = 0.07
    t = orc.KDTree(p)
    i1, d1 = t.nn(q, r)
    i2, d2 = orc.nn_brute(p, q, r)
    assert np.array_equal(i1, i2)
    assert np.array_equal(d1, d2)
    dref, iref = cKDTree(p).query(q, k=1)
    inl = dref <= r * (1 - 1e-12)
    assert np.all(i1[inl] >= 0) and np.all(i1[dref > r * (1 + 1e-12)] == -1)
    np.testing.assert_allclose(np.sqrt(d1[inl]), dref[inl], rtol=1e-12)


def test_radius_nn_bound_is_inclusive():
    p = np.array([[0.5, 0, 0], [0, 0, 0.75]])
    i, d = orc.KDTree(p).nn(np.zeros((1, 3)), 0.5)
    assert i[0] == 0 and d[0] == 0.25


# ----------------------------------------------------------------------------- eigen / covariance

def test_eigh3_matches_lapack():
    rng = np.random.default_rng(3)
    for _ in range(200):
        A = rng.normal(size=(3, 3))
        A = A @ A.T * rng.uniform(1e-6, 1e2)
        c6 = [A[0, 0], A[0, 1], A[0, 2], A[1, 1], A[1, 2], A[2, 2]]
        w, V = orc.eigh3(c6)
        wr, Vr = np.linalg.eigh(A)
        np.testing.assert_allclose(w, wr, rtol=1e-12, atol=1e-14 * np.abs(wr).max())
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-13)
        np.testing.assert_allclose(V @ np.diag(w) @ V.T, A, atol=1e-12 * np.abs(A).max())
        gaps = np.diff(wr) / wr.max()
        if gaps.min() > 1e-6:
            np.testing.assert_allclose(np.abs(np.sum(V * Vr, axis=0)), 1.0, atol=1e-9)


def test_planar_patch_normal_and_spectrum():
    # noise-free points on z = a x + b y + c: smallest eigenvector is the plane normal
    rng = np.random.default_rng(4)
    a, b, c = 0.3, -0.7, 1.5
    xy = rng.uniform(-0.05, 0.05, size=(40, 2))
    p = np.column_stack([xy, a * xy[:, 0] + b * xy[:, 1] + c])
    out = orc.source_covariances(p, k=20, reg_mode=orc.NONE)
    n = np.array([a, b, -1.0]) / np.linalg.norm([a, b, -1.0])
    for i in range(len(p)):
        w, V = orc.eigh3(out["raw"][i])
        assert abs(w[0]) <= 1e-14 * w[2]
        assert abs(abs(V[:, 0] @ n) - 1) < 1e-12
    reg = orc.source_covariances(p, k=20, eps=1e-3, reg_mode=orc.PLANE)["covs"]
    for i in range(len(p)):
        M = _sym(reg[i])
        np.testing.assert_allclose(np.linalg.eigvalsh(M), [1e-3, 1, 1], rtol=1e-6, atol=1e-12)
        # eigenvalue eps along the normal (eps is widened from float32 in the shim)
        assert abs(n @ M @ n - np.float32(1e-3)) < 1e-12


def test_raw_covariance_equals_numpy_cov_of_brute_force_neighbours():
    rng = np.random.default_rng(5)
    p = _cloud(rng, 400, 10)
    out = orc.source_covariances(p, k=20, reg_mode=orc.NONE)
    idx, _ = orc.knn_brute(p, p, 20)
    for i in range(0, 400, 7):
        Cref = np.cov(p[idx[i]].T, bias=True)
        np.testing.assert_allclose(_sym(out["raw"][i]), Cref, atol=1e-14, rtol=1e-10)
        np.testing.assert_allclose(_sym(out["covs"][i]), Cref, atol=1e-14, rtol=1e-10)


def test_covariance_equivariance():
    rng = np.random.default_rng(6)
    p = _cloud(rng, 300)
    R = rot_axis_angle([0.2, -0.5, 0.8], 0.9)
    t = np.array([0.3, -2.0, 5.0])
    a = orc.source_covariances(p, k=20, reg_mode=orc.NONE)["raw"]
    b = orc.source_covariances(p @ R.T + t, k=20, reg_mode=orc.NONE)["raw"]
    for i in range(0, 300, 11):
        np.testing.assert_allclose(_sym(b[i]), R @ _sym(a[i]) @ R.T, atol=1e-12)


def test_regularisation_closed_forms():
    rng = np.random.default_rng(7)
    eps = 1e-3
    for _ in range(100):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = np.sort(rng.uniform(0.01, 1, 3)) * rng.uniform(1e-6, 1)
        C = Q @ np.diag(lam) @ Q.T
        c6 = [C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]]
        plane, gap, fl = orc.regularise(c6, orc.PLANE, eps)
        P = _sym(plane)
        np.testing.assert_allclose(P, np.eye(3) - (1 - eps) * np.outer(Q[:, 0], Q[:, 0]), atol=1e-12)
        assert abs(gap - (lam[1] - lam[0]) / lam[1]) < 1e-9
        ell, _, fl2 = orc.regularise(c6, orc.ELLIPSE, eps)
        E = _sym(ell)
        # Lambda' = Lambda / median(S): covariance / middle eigenvalue, middle eigenvalue exactly 1
        np.testing.assert_allclose(E, C / lam[1], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(np.linalg.eigvalsh(E)[1], 1.0, rtol=1e-12)
        none, _, _ = orc.regularise(c6, orc.NONE, eps)
        np.testing.assert_allclose(none, c6, rtol=0, atol=0)


def test_ellipse_floor_and_rank_deficient():
    eps = 1e-3
    C = np.diag([1e-9, 1.0, 4.0])
    e, _, fl = orc.regularise([C[0, 0], 0, 0, C[1, 1], 0, C[2, 2]], orc.ELLIPSE, eps)
    assert fl & orc.FLAG_FLOORED
    np.testing.assert_allclose(e, [eps, 0, 0, 1, 0, 4], atol=1e-15)
    line = np.diag([0.0, 0.0, 2.0])
    for mode in (orc.PLANE, orc.ELLIPSE):
        e, _, fl = orc.regularise([0, 0, 0, 0, 0, 2.0], mode, eps)
        assert fl & orc.FLAG_RANK_DEFICIENT
        np.testing.assert_allclose(e, [1, 0, 0, 1, 0, 1])
    # collinear neighbourhood through the whole pipeline
    p = np.column_stack([np.linspace(0, 1, 30), 2 * np.linspace(0, 1, 30), np.zeros(30)])
    out = orc.source_covariances(p, k=20, reg_mode=orc.PLANE)
    assert np.all(out["flags"] & orc.FLAG_RANK_DEFICIENT)
    # fewer than three points
    out = orc.source_covariances(p[:2], k=20, reg_mode=orc.PLANE)
    assert np.all(out["flags"] & orc.FLAG_FEW_POINTS)
    np.testing.assert_allclose(out["covs"], [[1, 0, 0, 1, 0, 1]] * 2)
    del line


def test_scale_aligning_is_z_power():
    rng = np.random.default_rng(8)
    p = _cloud(rng, 200) + np.array([0, 0, 3.0])
    z = p[:, 2].copy()
    base = orc.source_covariances(p, z, k=20, reg_mode=orc.PLANE, p=0.0)["covs"]
    for pp in (1.0, 1.5):
        al = orc.source_covariances(p, z, k=20, reg_mode=orc.PLANE, p=pp)["covs"]
        pf = float(np.float32(pp))
        np.testing.assert_allclose(al, base * z[:, None] ** (-2 * pf), rtol=1e-13)


# ----------------------------------------------------------------------------- SE(3), Jacobian, GN system

def _hat(xi):
    w, v = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def test_transform_gaussians_is_a_rigid_motion():
    # moving Gaussians by T keeps pairwise distances and each covariance's spectrum, moves the
    # camera-frame origin to T's translation, and two moves compose as their product T2 T1
    rng = np.random.default_rng(15)
    p = rng.normal(size=(40, 3))
    c6 = np.array([(lambda A: (A @ A.T)[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]])(rng.normal(size=(3, 3)))
                   for _ in range(40)])
    T1, T2 = random_offset(rng, 50.0, 1.0), random_offset(rng, 120.0, 2.0)
    q, d = orc.transform_gaussians(T1, p, c6)
    iu = np.triu_indices(40, 1)
    dist = lambda a: np.linalg.norm(a[:, None] - a[None], axis=-1)[iu]
    np.testing.assert_allclose(dist(q), dist(p), rtol=1e-12)
    for a, b in zip(c6, d):
        np.testing.assert_allclose(np.linalg.eigvalsh(_sym(b)), np.linalg.eigvalsh(_sym(a)), rtol=1e-10, atol=1e-12)
    o, _ = orc.transform_gaussians(T1, np.zeros((1, 3)))
    np.testing.assert_allclose(o[0], T1[:3, 3], atol=1e-15)
    q2, d2 = orc.transform_gaussians(T2, q, d)
    q12, d12 = orc.transform_gaussians(T2 @ T1, p, c6)
    np.testing.assert_allclose(q2, q12, atol=1e-12)
    np.testing.assert_allclose(d2, d12, atol=1e-12 * np.abs(d12).max())
    # a handedness check: the x and y axes move to vectors whose cross product is the moved z axis
    ax, _ = orc.transform_gaussians(T1, np.eye(3))
    e = ax - T1[:3, 3]
    np.testing.assert_allclose(np.cross(e[0], e[1]), e[2], atol=1e-12)
    np.testing.assert_allclose(e, T1[:3, :3].T, atol=1e-12)


@pytest.mark.parametrize("scale", [0.0, 1e-12, 1e-7, 1e-4, 1e-3, 0.1, 1.0, 3.0])
def test_se3_exp_matches_expm(scale):
    rng = np.random.default_rng(int(scale * 1e6) % 1000)
    for _ in range(20):
        xi = rng.normal(size=6)
        xi[:3] *= scale / max(np.linalg.norm(xi[:3]), 1e-300)
        np.testing.assert_allclose(orc.se3_exp(xi), expm(_hat(xi)), atol=1e-14, rtol=1e-13)


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(9)
    T = random_offset(rng, 30, 0.5)
    for _ in range(20):
        x, mu = rng.normal(size=3), rng.normal(size=3)
        d, J = orc.residual_jacobian(T, x, mu)
        Jn = np.empty((3, 6))
        h = 1e-6
        for a in range(6):
            e = np.zeros(6)
            e[a] = h
            dp, _ = orc.residual_jacobian(orc.se3_exp(e) @ T, x, mu)
            dm, _ = orc.residual_jacobian(orc.se3_exp(-e) @ T, x, mu)
            Jn[:, a] = (dp - dm) / (2 * h)
        np.testing.assert_allclose(J, Jn, rtol=1e-7, atol=1e-8)


def _sparse_pair(rng, n=60, noise=0.0):
    # well separated points: nearest neighbours are the index partners
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4)), -1).reshape(-1, 3)[:n] * 0.5
    tgt = g + rng.uniform(-0.05, 0.05, size=g.shape)
    T_gt = random_offset(rng, 3, 0.02)
    src = transform_points(inv_pose(T_gt), tgt + noise * rng.normal(size=tgt.shape))
    return src, tgt, T_gt


def test_gradient_and_hessian_match_finite_differences():
    # isotropic source covariances make W independent of the pose, so the
    # cost sum d^T W d has gradient 2 b and (at zero residual) Hessian 2 H
    rng = np.random.default_rng(10)
    src, tgt, T_gt = _sparse_pair(rng)
    cs = np.tile([0.01, 0, 0, 0.01, 0, 0.01], (len(src), 1))
    ct = np.array([[0.02 + 0.01 * i % 3, 0.001, 0, 0.03, -0.002, 0.05] for i in range(len(tgt))])
    m = orc.Map(tgt, ct)
    T = T_gt @ random_offset(rng, 1.0, 0.01)
    lin = orc.linearise(src, cs, m, T, 0.2)
    assert lin["inliers"] == len(src)
    h = 1e-6
    g = np.empty(6)
    for a in range(6):
        e = np.zeros(6)
        e[a] = h
        cp = orc.linearise(src, cs, m, orc.se3_exp(e) @ T, 0.2)["cost"]
        cm = orc.linearise(src, cs, m, orc.se3_exp(-e) @ T, 0.2)["cost"]
        g[a] = (cp - cm) / (2 * h)
    np.testing.assert_allclose(g, 2 * lin["b"], rtol=1e-6, atol=1e-6 * np.abs(lin["b"]).max())
    H = lin["H"]
    np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0
    lin0 = orc.linearise(src, cs, m, T_gt, 0.2)
    assert lin0["cost"] < 1e-20
    hh = 1e-4
    Hn = np.empty((6, 6))
    for a in range(6):
        for c in range(6):
            ea, ec = np.zeros(6), np.zeros(6)
            ea[a], ec[c] = hh, hh
            f = lambda s, t: orc.linearise(src, cs, m, orc.se3_exp(s * ea + t * ec) @ T_gt, 0.2)["cost"]
            Hn[a, c] = (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * hh * hh)
    np.testing.assert_allclose(Hn, 2 * lin0["H"], rtol=1e-4, atol=1e-4 * np.abs(lin0["H"]).max())


def test_one_gauss_newton_step_solves_the_normal_equations():
    # one iteration from T0 moves to exp(delta^) T0 with H delta = -b for the H, b of the
    # linearisation at T0: the step recovered by the matrix logarithm (scipy) solves the system
    from scipy.linalg import logm
    src32, tgt32, T_gt = pair_config1(2, 1, n=1500)
    s, t = src32.astype(np.float64), tgt32.astype(np.float64)
    cs = orc.source_covariances(s, k=20, reg_mode=orc.PLANE)["covs"]
    ct = orc.source_covariances(t, k=20, reg_mode=orc.PLANE)["covs"]
    m = orc.Map(t, ct)
    T0 = T_gt @ random_offset(np.random.default_rng(16), 2.0, 0.02)
    lin = orc.linearise(s, cs, m, T0, 0.1)
    r = orc.register(s, cs, m, T0, 0.1, 1)
    assert r["iters"] == 1 and np.allclose(r["H"], lin["H"], rtol=1e-12) and np.allclose(r["b"], lin["b"], rtol=1e-12)
    L = np.real(logm(r["T"] @ np.linalg.inv(T0)))
    delta = np.array([L[2, 1], L[0, 2], L[1, 0], L[0, 3], L[1, 3], L[2, 3]])
    np.testing.assert_allclose(lin["H"] @ delta, -lin["b"], rtol=1e-7, atol=1e-8 * np.abs(lin["b"]).max())
    # the exported update (the split registration's step) is the same step: from the same H, b and
    # T0 it lands on the same pose, its matrix logarithm solving the same system
    Tu, conv = orc.gn_update(lin["H"], lin["b"], T0)
    assert conv == 0
    np.testing.assert_array_equal(Tu, r["T"])
    Lu = np.real(logm(Tu @ np.linalg.inv(T0)))
    du = np.array([Lu[2, 1], Lu[0, 2], Lu[1, 0], Lu[0, 3], Lu[1, 3], Lu[2, 3]])
    np.testing.assert_allclose(lin["H"] @ du, -lin["b"], rtol=1e-7, atol=1e-8 * np.abs(lin["b"]).max())
    # a zero system is not positive definite: no step, pose unchanged
    Tz, cz = orc.gn_update(np.zeros((6, 6)), np.zeros(6), T0)
    assert cz == -1 and np.array_equal(Tz, T0)


def _kabsch(P, Q):
    """Least-squares rigid transform mapping P onto Q (Umeyama/Kabsch, via SVD)."""
    mp, mq = P.mean(0), Q.mean(0)
    U, _, Vt = np.linalg.svd((P - mp).T @ (Q - mq))
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return make_pose(R, mq - R @ mp)


def test_point_to_point_special_case_is_kabsch():
    # NONE regularisation with every covariance 1/2 I gives W = I: the MLE is
    # the least-squares rigid fit, whose closed form is the Kabsch SVD solution
    rng = np.random.default_rng(11)
    src, tgt, _ = _sparse_pair(rng, noise=0.01)
    half = np.tile([0.5, 0, 0, 0.5, 0, 0.5], (len(src), 1))
    ref = _kabsch(src, tgt)
    r = orc.register_fixed(src, half, tgt, half, np.eye(4))
    assert r["status"] == orc.OK
    np.testing.assert_allclose(r["T"], ref, atol=1e-10)
    # with nearest-neighbour association on well separated points: same answer
    rr = orc.register(src, half, orc.Map(tgt, half), np.eye(4), max_corr_dist=0.2, tol_rot=1e-12, tol_trans=1e-12)
    assert rr["status"] == orc.OK and rr["inliers"] == len(src)
    np.testing.assert_allclose(rr["T"], ref, atol=1e-10)


def test_exact_recovery_on_noise_free_room():
    # source = T_gt^-1 applied to the very map points, covariances carried along
    src32, tgt32, _ = pair_config1(0, 0, n=3000, noise=0.0)
    tgt = tgt32.astype(np.float64)
    ct = orc.source_covariances(tgt, k=20, reg_mode=orc.PLANE)["covs"]
    rng = np.random.default_rng(12)
    T_gt = random_offset(rng, 5.0, 0.05)
    src = transform_points(inv_pose(T_gt), tgt)
    R = T_gt[:3, :3]
    cs = np.array([(R.T @ _sym(c) @ R)[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]] for c in ct])
    r = orc.register(src, cs, orc.Map(tgt, ct), np.eye(4), max_corr_dist=0.1, max_iters=50,
                     tol_rot=1e-12, tol_trans=1e-12)
    assert r["status"] == orc.OK
    np.testing.assert_allclose(r["T"], T_gt, atol=1e-9)
    assert r["cost"] < 1e-12
    del src32


def test_registration_invariants():
    src32, tgt32, T_gt = pair_config1(1, 0, n=2000)
    s, t = src32.astype(np.float64), tgt32.astype(np.float64)
    cs = orc.source_covariances(s, k=20, reg_mode=orc.PLANE)["covs"]
    ct = orc.source_covariances(t, k=20, reg_mode=orc.PLANE)["covs"]
    m = orc.Map(t, ct)
    r = orc.register(s, cs, m, np.eye(4))
    assert r["status"] == orc.OK
    H = r["H"]
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0
    # recovers the ground truth to within the sampling noise
    dT = np.linalg.inv(T_gt) @ r["T"]
    assert np.linalg.norm(dT[:3, 3]) < 5e-3
    assert np.arccos(np.clip((np.trace(dT[:3, :3]) - 1) / 2, -1, 1)) < np.deg2rad(0.3)
    # invariant to the order of the source points
    perm = np.random.default_rng(0).permutation(len(s))
    r2 = orc.register(s[perm], cs[perm], m, np.eye(4))
    np.testing.assert_allclose(r2["T"], r["T"], atol=1e-12)
    assert r2["iters"] == r["iters"]


def _rotate6(Q, c6):
    return np.array([(Q @ _sym(c) @ Q.T)[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]] for c in c6])


def test_linearisation_is_invariant_to_the_source_and_map_frames():
    # Moving the source cloud by a rigid motion G = (Q, u) -- points G x, covariances Q C Q^T --
    # and the pose to T G^-1 leaves every world-frame residual, combined covariance and Jacobian of
    # the left update as it was: cost, H and b are unchanged.  Moving the map instead (means G mu,
    # covariances Q C Q^T, pose G T) rotates every residual and combined covariance together, so
    # the cost d^T Sigma^-1 d is unchanged.  Both need Sigma = C^t + R C^s R^T with anisotropic
    # covariances on both sides.
    src32, tgt32, T_gt = pair_config1(3, 1, n=1500)
    s, t = src32.astype(np.float64), tgt32.astype(np.float64)
    cs = orc.source_covariances(s, k=20, reg_mode=orc.PLANE)["covs"]
    ct = orc.source_covariances(t, k=20, reg_mode=orc.ELLIPSE)["covs"]
    m = orc.Map(t, ct)
    T = T_gt @ random_offset(np.random.default_rng(13), 1.0, 0.01)
    ref = orc.linearise(s, cs, m, T, 0.1)
    assert ref["inliers"] > 500
    G = make_pose(rot_axis_angle([0.3, -0.8, 0.5], 0.7), [0.4, -1.1, 2.0])
    Q = G[:3, :3]
    mv = orc.linearise(transform_points(G, s), _rotate6(Q, cs), m, T @ inv_pose(G), 0.1)
    np.testing.assert_array_equal(mv["corr"], ref["corr"])
    assert mv["cost"] == pytest.approx(ref["cost"], rel=1e-10)
    np.testing.assert_allclose(mv["H"], ref["H"], rtol=1e-9, atol=1e-10 * np.abs(ref["H"]).max())
    np.testing.assert_allclose(mv["b"], ref["b"], rtol=1e-9, atol=1e-9 * np.abs(ref["b"]).max())
    mm = orc.linearise(s, cs, orc.Map(transform_points(G, t), _rotate6(Q, ct)), G @ T, 0.1)
    np.testing.assert_array_equal(mm["corr"], ref["corr"])
    assert mm["cost"] == pytest.approx(ref["cost"], rel=1e-10)


def test_cost_tends_to_point_to_plane_error_in_the_flat_limit():
    # G-ICP generalises point-to-plane ICP: with source covariances 0 and each target a plane,
    # C^t = I - (1 - eps) n n^T, a residual d costs |d|^2 + (1/eps - 1)(n.d)^2, so eps * cost tends
    # to the point-to-plane error sum (n.d)^2 as eps -> 0, and the cost is never below sum |d|^2.
    rng = np.random.default_rng(14)
    tgt = np.stack(np.meshgrid(np.arange(5), np.arange(5), np.arange(4)), -1).reshape(-1, 3) * 0.5
    n = rng.normal(size=tgt.shape)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    delta = rng.uniform(-0.02, 0.02, size=tgt.shape)
    src = tgt - delta   # at T = I the residual of pair i is mu - x = delta_i
    p2p = float(np.sum(np.sum(n * delta, axis=1) ** 2))
    d2 = float(np.sum(delta * delta))
    for eps in (1e-3, 1e-6):
        ct = np.array([(np.eye(3) - (1 - eps) * np.outer(v, v))[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]] for v in n])
        lin = orc.linearise(src, np.zeros((len(src), 6)), orc.Map(tgt, ct), np.eye(4), 0.1)
        assert lin["inliers"] == len(src) and np.array_equal(lin["corr"], np.arange(len(src)))
        assert lin["cost"] >= d2 * (1 - 1e-12)
        assert abs(eps * lin["cost"] - p2p) <= 2 * eps * d2 + 1e-12 * p2p


def test_degenerate_when_too_few_inliers():
    src32, tgt32, _ = pair_config1(2, 0, n=500)
    s, t = src32.astype(np.float64), tgt32.astype(np.float64) + 10.0  # far apart: no correspondences
    c = np.tile([1, 0, 0, 1, 0, 1.0], (500, 1))
    r = orc.register(s, c, orc.Map(t, c), np.eye(4))
    assert r["status"] == orc.ERR_DEGENERATE and r["inliers"] == 0
    np.testing.assert_allclose(r["T"], np.eye(4))


# ----------------------------------------------------------------------------- depth -> points

def test_depth_to_points_on_analytic_plane():
    intr = Intrinsics(64, 48, 50.0, 55.0, 31.5, 23.5)
    # a single tilted wall in front of the camera: the room's far wall
    scene = Scene(np.array([-5.0, -5.0, -5.0]), np.array([5.0, 5.0, 2.0]))
    T = make_pose(rot_axis_angle([1, 0.3, 0], 0.3), [0.0, 0.0, 0.0])
    depth = raycast_depth(scene, T, intr)
    depth[3, 5] = np.nan
    depth[10, 10] = 0.0
    depth[20, 40] = 100.0
    pts, z = orc.depth_to_points(depth, intr.as_array(), 2, 0.1, 10.0)
    # every sampled finite pixel in range survives, in row-major order
    sub = depth[::2, ::2]
    keep = np.isfinite(sub) & (sub >= np.float32(0.1)) & (sub <= np.float32(10.0))
    assert len(pts) == keep.sum()
    vv, uu = np.nonzero(keep)
    # round trip: projecting each point returns its pixel
    u = intr.fx * pts[:, 0] / pts[:, 2] + intr.cx
    v = intr.fy * pts[:, 1] / pts[:, 2] + intr.cy
    np.testing.assert_allclose(u, 2 * uu, atol=1e-9)
    np.testing.assert_allclose(v, 2 * vv, atol=1e-9)
    np.testing.assert_array_equal(z, pts[:, 2])
    # the points lie on the plane z_world = 2 (float32 depth rounding only)
    w = transform_points(T, pts)
    np.testing.assert_allclose(w[:, 2], 2.0, atol=2e-6)
