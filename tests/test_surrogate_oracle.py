"""Pins of the surrogate oracle (oracle/surrogate.py) to things other than itself: the C oracle's
a1 and plane regularisation, brute-force convolution loops, the bfloat16 format's rounding rule
on float32 bit patterns, the network's translation and scale invariances, finite differences of
the loss, and Adam's closed-form first step."""
import numpy as np
import pytest

import oracle as orc
from oracle import surrogate as sg


def _smooth_depth(h=48, w=64, seed=0):
    rng = np.random.default_rng(seed)
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    d = 2.0 + 0.3 * np.sin(u / 9.0) + 0.2 * np.cos(v / 7.0) + 0.004 * u
    d += rng.normal(size=d.shape) * 1e-3
    d[5, 7] = 0.0          # missing sample
    d[20:23, 30:33] = 50.0  # out of range
    return d.astype(np.float32)


def test_point_grid_equals_c_oracle_points():
    depth = _smooth_depth()
    intr = [40.0, 41.0, 31.5, 23.5]
    for stride in (1, 2, 3):
        P, M = sg.point_grid(depth, intr, stride, 0.1, 10.0)
        pts, z = orc.depth_to_points(depth, intr, stride, 0.1, 10.0)
        np.testing.assert_array_equal(P[M], pts)
        assert M.sum() == len(pts)


def _bf16_bits(x32):
    """Round-to-nearest-even of float32 bit patterns to their top 16 bits (the bfloat16 format)."""
    b = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (r << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding():
    assert sg.bf16(1.0) == 1.0
    assert sg.bf16(1.0 + 2.0 ** -8) == 1.0                       # tie -> even
    assert sg.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie -> even (upwards)
    assert sg.bf16(-(1.0 + 2.0 ** -7)) == -(1.0 + 2.0 ** -7)     # representable
    assert sg.bf16(255.9) == 256.0                                # carry into the next binade
    assert sg.bf16(0.0) == 0.0
    rng = np.random.default_rng(1)
    x = (rng.normal(size=20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    np.testing.assert_array_equal(sg.bf16(x.astype(np.float64)), _bf16_bits(x))


def _brute_conv(x, W):
    h, w, _ = x.shape
    y = np.zeros((h, w, W.shape[0]))
    for i in range(h):
        for j in range(w):
            for o in range(W.shape[0]):
                s = 0.0
                for c in range(W.shape[1]):
                    for dy in range(5):
                        for dx in range(5):
                            ii, jj = i + dy - 2, j + dx - 2
                            if 0 <= ii < h and 0 <= jj < w:
                                s += W[o, c, dy, dx] * x[ii, jj, c]
                y[i, j, o] = s
    return y


def test_conv_equals_brute_force():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(6, 7, 4))
    W = rng.normal(size=(3, 4, 5, 5))
    np.testing.assert_allclose(sg._conv(x, W), _brute_conv(x, W), rtol=1e-12, atol=1e-12)


def test_layer1_equals_brute_force():
    rng = np.random.default_rng(3)
    P = rng.normal(size=(6, 7, 3))
    M = rng.random((6, 7)) > 0.2
    W = rng.normal(size=(5, 3, 5, 5))
    ref = np.zeros((6, 7, 5))
    for i in range(6):
        for j in range(7):
            for o in range(5):
                s = 0.0
                for c in range(3):
                    for dy in range(5):
                        for dx in range(5):
                            ii, jj = i + dy - 2, j + dx - 2
                            if 0 <= ii < 6 and 0 <= jj < 7 and M[ii, jj]:
                                s += W[o, c, dy, dx] * (P[ii, jj, c] - P[i, j, c])
                ref[i, j, o] = s
    np.testing.assert_allclose(sg._layer1(P, M, W), ref, rtol=1e-12, atol=1e-12)


def _grid(seed=0, h=14, w=18):
    depth = _smooth_depth(h, w, seed)
    return sg.point_grid(depth, [20.0, 20.0, w / 2 - 0.5, h / 2 - 0.5], 1, 0.1, 10.0)


def test_translation_and_scale_invariance():
    P, M = _grid(4)
    w = sg.init_weights(5)
    v = sg.forward(P, M, w, round_bf16=False)["v"]
    vt = sg.forward(P + np.array([0.7, -1.3, 2.1]), M, w, round_bf16=False)["v"]
    np.testing.assert_allclose(vt, v, rtol=1e-9, atol=1e-12 * np.abs(v).max())
    vs = sg.forward(2.5 * P, M, w, round_bf16=False)["v"]
    np.testing.assert_allclose(vs, 2.5 * v, rtol=1e-9, atol=1e-12 * np.abs(v).max())
    assert np.all(v[~M] == 0) and np.abs(v[M]).max() > 0


def test_plane_covariance_equals_c_oracle_regularisation():
    rng = np.random.default_rng(6)
    for _ in range(20):
        U, _r = np.linalg.qr(rng.normal(size=(3, 3)))
        C = U @ np.diag([0.01, 1.0, 2.5]) @ U.T   # smallest-eigenvalue direction U[:, 0]
        C6 = np.array([C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]])
        ref, _gap, flags = orc.regularise(C6, orc.PLANE, 1e-3)
        assert flags == 0
        z = rng.uniform(0.5, 4.0)
        got = sg.plane_covariance(U[:, 0] * rng.choice([-1, 1]), z, 1e-3, 1.5)
        np.testing.assert_allclose(got, ref * z ** -3.0, rtol=1e-10, atol=1e-12)
        T = sg.knn_projector(got[None], np.array([z]), 1e-3, 1.5)[0]
        np.testing.assert_allclose(T, np.outer(U[:, 0], U[:, 0]), atol=1e-10)


def test_loss_values():
    M = np.ones((1, 3), bool)
    n = np.array([0.0, 0.6, 0.8])
    T = np.repeat(np.outer(n, n)[None], 3, axis=0)
    v = np.stack([3 * n, -0.5 * n, np.array([1.0, 0.0, 0.0])])[None]
    # parallel (either sign): 0; perpendicular: 1
    assert sg.loss(v, M, T) == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert sg.loss(v, M, T, mask_t=[True, True, False]) == pytest.approx(0.0, abs=1e-15)


def test_gradient_matches_finite_differences():
    P, M = _grid(7, 9, 11)
    w = sg.init_weights(8).astype(np.float64)
    rng = np.random.default_rng(9)
    nvalid = int(M.sum())
    nn = rng.normal(size=(nvalid, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    T = np.einsum("ni,nj->nij", nn, nn)
    sel = rng.random(nvalid) > 0.1
    L, g = sg.loss_and_grad(P, M, w, T, sel, round_bf16=False)
    assert L == pytest.approx(sg.loss(sg.forward(P, M, w, False)["v"], M, T, sel), abs=1e-14)
    idx = np.concatenate([rng.choice(sg.SIZES[0], 15, replace=False),
                          sg.SIZES[0] + rng.choice(sg.SIZES[1], 15, replace=False),
                          sg.SIZES[0] + sg.SIZES[1] + rng.choice(sg.SIZES[2], 15, replace=False)])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        Lp = sg.loss(sg.forward(P, M, wp, False)["v"], M, T, sel)
        Lm = sg.loss(sg.forward(P, M, wm, False)["v"], M, T, sel)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)), (i, fd, g[i])


def test_adam_first_step_and_convergence():
    rng = np.random.default_rng(10)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, s = sg.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 1e-2)
    # first step: bias-corrected moments are g and g^2, so each weight moves by lr g / (|g| + eps)
    np.testing.assert_allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(s, 0.001 * g * g, rtol=1e-12)
    # minimising 0.5 |w|^2 drives w towards 0
    w = np.full(4, 3.0)
    m = s = np.zeros(4)
    for t in range(1, 3001):
        w, m, s = sg.adam_step(w, w.copy(), m, s, t, 0.05)
    assert np.abs(w).max() < 0.05


def test_zero_prediction_gives_isotropic_covariance_and_full_loss():
    # where the network predicts v = 0 the normal is undefined: the covariance is z^(-2p) I (the
    # plane form has no direction to use) and the pixel counts as loss 1
    M = np.ones((1, 2), bool)
    P = np.array([[[0.0, 0.0, 2.0], [0.1, 0.0, 4.0]]])
    v = np.array([[[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]]])
    C, ok = sg.covariances(v, M, P, 1e-3, 1.5)
    assert ok.tolist() == [False, True]
    np.testing.assert_allclose(C[0], np.array([1, 0, 0, 1, 0, 1]) * 2.0 ** -3, rtol=1e-15)
    np.testing.assert_allclose(C[1], sg.plane_covariance(np.array([0.0, 0.0, 1.0]), 4.0, 1e-3, 1.5), rtol=1e-15)
    T = np.repeat(np.diag([0.0, 0.0, 1.0])[None], 2, axis=0)
    assert sg.loss(v, M, T) == pytest.approx(0.5, abs=1e-15)
