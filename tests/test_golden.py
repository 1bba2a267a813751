"""The hand-worked examples under tests/golden/ (regularisation and scale aligning of Sec. 3.1 and
Sec. 3.2 on six-point stars; the SE(3) exponential of the pose update) against the oracle and,
for the covariances, against the CUDA path through the C ABI."""
import configparser
import os

import numpy as np
import pytest

import oracle as orc

from ._util import COV_REL_TOL, cov_rel_err

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MODES = (("plane", orc.PLANE), ("ellipse", orc.ELLIPSE), ("none", orc.NONE))


def _read(name):
    cp = configparser.ConfigParser(inline_comment_prefixes=None)
    cp.optionxform = str  # keys are case-sensitive (R, t)
    with open(os.path.join(GOLDEN, name)) as fh:
        cp.read_file(fh)
    return {s: {k: np.array([float(x) for x in v.split()]) for k, v in cp[s].items()} for s in cp.sections()}


STARS = _read("regularisation_star.ini")
SE3 = _read("se3_exp.ini")
LIN = _read("linearise_single.ini")
D2P = _read("depth_to_points_small.ini")


def star_points(c):
    """Centre plus and minus a*u, b*v, w_len*w (the six points every case is built from)."""
    pts = []
    for axis, length in (("u", "a"), ("v", "b"), ("w", "w_len")):
        for sign in (1.0, -1.0):
            pts.append(c["centre"] + sign * c[length][0] * c[axis])
    return np.array(pts)


def test_fixtures_are_well_formed():
    assert set(STARS) == {"star_345", "star_axes_yxz"} and set(SE3) == {"translation_only", "quarter_turn_z",
                                                                      "half_turn_x"}
    assert set(LIN) == {"identity_pose", "quarter_turn_z"}
    for c in LIN.values():
        assert c["T"].shape == (16,) and c["H"].shape == (36,) and c["b"].shape == (6,)
        np.testing.assert_array_equal(c["H"].reshape(6, 6), c["H"].reshape(6, 6).T)
    for c in STARS.values():
        F = np.stack([c["u"], c["v"], c["w"]])
        np.testing.assert_allclose(F @ F.T, np.eye(3), atol=1e-15)
        assert c["a"][0] < c["b"][0] < c["w_len"][0]
        for key, _ in MODES:
            assert c[key].shape == (6,)


@pytest.mark.parametrize("case", sorted(STARS))
def test_oracle_regularise_on_the_worked_raw_covariances(case):
    c = STARS[case]
    eps = c["eps"][0]
    for key, mode in MODES[:2]:
        out, _gap, flags = orc.regularise(c["none"], mode, eps)
        assert flags == 0
        np.testing.assert_allclose(out, c[key], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("case", sorted(STARS))
@pytest.mark.parametrize("p", [0.0, 1.5])
def test_oracle_source_covariances_on_the_star(case, p):
    c = STARS[case]
    pts = star_points(c)
    z = pts[:, 2].copy()
    for key, mode in MODES:
        out = orc.source_covariances(pts, z, k=20, eps=c["eps"][0], reg_mode=mode, p=p)
        np.testing.assert_allclose(out["raw"], np.tile(c["none"], (6, 1)), rtol=1e-12, atol=1e-15)
        # eps reaches the oracle as a float32 (as the C ABI passes it), which moves each entry of the
        # plane and ellipse forms by at most that rounding of eps (about 5e-11 for 1e-3)
        deps = abs(float(np.float32(c["eps"][0])) - c["eps"][0])
        expect = c[key][None] * z[:, None] ** (-2.0 * p)
        np.testing.assert_allclose(out["covs"], expect, rtol=1e-12, atol=deps * z.min() ** (-2.0 * p) + 1e-14)


@pytest.mark.parametrize("case", sorted(SE3))
def test_oracle_se3_exp(case):
    c = SE3[case]
    T = orc.se3_exp(c["xi"])
    np.testing.assert_allclose(T[:3, :3], c["R"].reshape(3, 3), atol=1e-15)
    np.testing.assert_allclose(T[:3, 3], c["t"], atol=1e-15)
    np.testing.assert_array_equal(T[3], [0, 0, 0, 1])


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(STARS))
@pytest.mark.parametrize("p", [0.0, 1.5])
def test_cuda_source_covariances_on_the_star(case, p):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12550_b300 as g
    c = STARS[case]
    pts = star_points(c).astype(np.float32)
    z = pts[:, 2].copy()
    ctx = g.Context()
    try:
        for key, mode in MODES:
            covs = g.gsicp_source_covariances(ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(z).cuda(),
                                              g.CovParams(20, float(c["eps"][0]), mode, p))
            covs = covs.cpu().numpy().astype(np.float64)
            expect = c[key][None] * z.astype(np.float64)[:, None] ** (-2.0 * p)
            err = cov_rel_err(covs, expect)
            assert err.max() <= COV_REL_TOL, (key, err)
    finally:
        ctx.close()


def test_fixture_values_follow_from_their_derivation():
    # the stored numbers are the closed forms written in the fixtures, evaluated exactly (rational
    # arithmetic for the stars, sympy's symbolic matrix exponential for SE(3)), independent of
    # the oracle: a typo in a fixture fails here
    from fractions import Fraction as F

    import sympy as sp

    def exact(v):
        return [F(str(x)) for x in v]

    def outer(a, b):
        return [[a[i] * b[j] for j in range(3)] for i in range(3)]

    def six(M):
        return [M[0][0], M[0][1], M[0][2], M[1][1], M[1][2], M[2][2]]

    for c in STARS.values():
        u, v, w = exact(c["u"]), exact(c["v"]), exact(c["w"])
        a, b, wl, eps = F(str(c["a"][0])), F(str(c["b"][0])), F(str(c["w_len"][0])), F(str(c["eps"][0]))
        uu, vv, ww = outer(u, u), outer(v, v), outer(w, w)
        S = [[a * a * uu[i][j] + b * b * vv[i][j] + wl * wl * ww[i][j] for j in range(3)] for i in range(3)]
        raw = [[S[i][j] / 3 for j in range(3)] for i in range(3)]
        plane = [[(1 if i == j else 0) - (1 - eps) * uu[i][j] for j in range(3)] for i in range(3)]
        ellipse = [[S[i][j] / (b * b) for j in range(3)] for i in range(3)]
        for key, M in (("none", raw), ("plane", plane), ("ellipse", ellipse)):
            np.testing.assert_allclose(c[key], [float(x) for x in six(M)], rtol=1e-15, atol=1e-15)

    for c in LIN.values():
        T = sp.Matrix(4, 4, [sp.nsimplify(v) for v in c["T"]])
        R, t = T[:3, :3], T[:3, 3]
        x = sp.Matrix([sp.nsimplify(v) for v in c["x"]])
        mu = sp.Matrix([sp.nsimplify(v) for v in c["mu"]])

        def sym3(v):
            a, b_, c_, d_, e_, f_ = (sp.nsimplify(q) for q in v)
            return sp.Matrix([[a, b_, c_], [b_, d_, e_], [c_, e_, f_]])
        y = R * x + t
        d = mu - y
        W = (sym3(c["ct"]) + R * sym3(c["cs"]) * R.T).inv()
        Y = sp.Matrix([[0, -y[2], y[1]], [y[2], 0, -y[0]], [-y[1], y[0], 0]])
        J = Y.row_join(-sp.eye(3))
        np.testing.assert_allclose(float((d.T * W * d)[0]), c["cost"][0], rtol=1e-15)
        np.testing.assert_allclose(np.array((J.T * W * d).evalf(), dtype=float).ravel(), c["b"], atol=1e-15)
        np.testing.assert_allclose(np.array((J.T * W * J).evalf(), dtype=float).ravel(), c["H"], atol=1e-15)

    for c in SE3.values():
        wx, wy, wz, vx, vy, vz = (sp.nsimplify(x, [sp.pi]) for x in c["xi"])
        X = sp.Matrix([[0, -wz, wy, vx], [wz, 0, -wx, vy], [-wy, wx, 0, vz], [0, 0, 0, 0]])
        E = sp.simplify(X.exp())
        np.testing.assert_allclose(np.array(E[:3, :3].evalf(), dtype=float).ravel(), c["R"], atol=1e-15)
        np.testing.assert_allclose(np.array(E[:3, 3].evalf(), dtype=float).ravel(), c["t"], atol=1e-15)


@pytest.mark.parametrize("case", sorted(LIN))
def test_oracle_linearise_one_correspondence(case):
    c = LIN[case]
    m = orc.Map(c["mu"][None], c["ct"][None])
    lin = orc.linearise(c["x"][None], c["cs"][None], m, c["T"].reshape(4, 4), 0.5)
    assert lin["inliers"] == 1
    assert lin["cost"] == pytest.approx(c["cost"][0], rel=1e-12)
    np.testing.assert_allclose(lin["b"], c["b"], atol=1e-15)
    np.testing.assert_allclose(lin["H"], c["H"].reshape(6, 6), atol=1e-15)


@pytest.mark.parametrize("stride", [1, 2])
def test_oracle_depth_to_points_small_image(stride):
    img = D2P["image"]
    depth = img["depth"].reshape(3, 4).astype(np.float32)
    pts, z = orc.depth_to_points(depth, img["intr"], stride, *img["range"])
    expect = D2P[f"stride_{stride}"]["points"].reshape(-1, 3)
    np.testing.assert_array_equal(pts, expect)
    np.testing.assert_array_equal(z, expect[:, 2])


@pytest.mark.gpu
@pytest.mark.parametrize("stride", [1, 2])
def test_cuda_depth_to_points_small_image(stride):
    """Both CUDA a1 entry points (the allocating one and the allocation-free one) on the hand-worked
    4 x 3 image: the missing sample, the samples below z_min and above z_max are dropped and the
    rest equal the worked points exactly (the a1 bar is bit-exact)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12550_b300 as g
    img = D2P["image"]
    depth = torch.from_numpy(img["depth"].reshape(3, 4).astype(np.float32)).cuda()
    expect = D2P[f"stride_{stride}"]["points"].reshape(-1, 3).astype(np.float32)
    ctx = g.Context()
    try:
        pts, z = g.gsicp_depth_to_points(ctx, depth, img["intr"], stride, *img["range"])
        np.testing.assert_array_equal(pts.cpu().numpy(), expect)
        np.testing.assert_array_equal(z.cpu().numpy(), expect[:, 2])
    finally:
        ctx.close()
    cap = 12
    pts = torch.full((cap, 3), np.nan, device="cuda", dtype=torch.float32)
    z = torch.full((cap,), np.nan, device="cuda", dtype=torch.float32)
    n = torch.zeros((1,), device="cuda", dtype=torch.int32)
    total = torch.zeros((1,), device="cuda", dtype=torch.int32)
    g.gsicp_depth_to_points_noalloc(depth, img["intr"], stride, *img["range"], pts, z, n, total)
    torch.cuda.synchronize()
    k = int(n.item())
    assert k == int(total.item()) == len(expect)
    np.testing.assert_array_equal(pts[:k].cpu().numpy(), expect)
    np.testing.assert_array_equal(z[:k].cpu().numpy(), expect[:, 2])
