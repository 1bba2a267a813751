"""The covariance surrogate's CUDA kernels vs its FP64 oracle (oracle/surrogate.py), through the
C ABI: forward outputs and covariances, loss and gradients of one training step, the Adam update,
and that training lowers the loss.

Tolerances.  The kernels sum in float where the oracle sums in float64, and both round the
hidden activations to bfloat16: where the two sums straddle a bfloat16 rounding boundary the
two sides' activation differs by one bfloat16 step (2^-8 relative).  Such flips are rare
(most pixels agree to ~1e-7), but v = sum of 800 terms W3 h2 can be much smaller than the terms
(they cancel), so one flipped h2 can move v by 2^-8 of a term.  The bound per pixel and output
is therefore 2^-7 S with S = sum |W3| |h2| (the absolute sum of v's terms, from the oracle),
with the median relative error required below 1e-5; covariances get the same bound carried
through n = v / |v|.  The inputs of both sides are the same float32 points (a1's output widened)."""
import numpy as np
import pytest

import oracle as orc
from oracle import surrogate as sgo
from synth import HALF_TUM_INTR, surrogate_train_config5

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


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frame(f=0, crop=None):
    cfg = surrogate_train_config5(0, n_frames=8, n_scenes=4)
    d = cfg["depth"](f)
    if crop:
        d = np.ascontiguousarray(d[:crop[0], :crop[1]])
    intr = HALF_TUM_INTR.as_array()
    return d, intr


def _oracle_grid(d, intr, stride):
    P, M = sgo.point_grid(d, intr, stride, 0.1, 10.0)
    return P.astype(np.float32).astype(np.float64), M  # the float32 points a1 writes


def _weights(seed, scale=1.0):
    return (sgo.init_weights(seed) * scale).astype(np.float32)


@pytest.mark.parametrize("shape,stride", [((90, 121), 1), ((240, 320), 2), ((37, 50), 1), ("full", 2)])
def test_forward_matches_oracle(g, ctx, shape, stride):
    if shape == "full":  # the benchmark's frame: 640 x 480 at stride 2 (a 320 x 240 grid, 600 tiles)
        from synth import TUM_INTR, sequence_config5
        d, intr = sequence_config5(0, n_frames=3)["depth"](1), TUM_INTR.as_array()
    else:
        d, intr = _frame(1, crop=shape)
    w = _weights(3)
    sg = g.Surrogate(w)
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    pts, z, covs, v = g.gsicp_surrogate_covariances(ctx, sg, cu(d), intr, stride, 0.1, 10.0, cp, want_v=True)
    P, M = _oracle_grid(d, intr, stride)
    f = sgo.forward(P, M, w)
    vo, vg = f["v"], v.cpu().numpy().astype(np.float64)
    assert vg.shape == vo.shape
    assert np.all(vg[~M] == 0)
    # S[o](u) = sum_{c, t} |W3[o, c, t]| |h2[c](u + d_t)|
    W3 = np.abs(sgo.bf16(sgo.split_weights(w)[2]))
    S = sgo._conv(np.abs(f["h2"]), W3)
    dv = np.abs(vg - vo)
    assert np.all(dv <= 2.0 ** -7 * S + 1e-7 * np.abs(vo).max()), np.max(dv / (S + 1e-30))
    nv = np.linalg.norm(vo, axis=-1)[M]
    rel = np.linalg.norm(vg - vo, axis=-1)[M] / np.maximum(nv, 1e-6 * nv.max())
    assert np.median(rel) < 1e-5, np.median(rel)
    # covariances: plane covariance on the oracle's normal, within the bound carried through n
    Co, ok = sgo.covariances(vo, M, P, 1e-3, 1.5)
    Cg = covs.cpu().numpy().astype(np.float64)
    assert len(Cg) == len(Co) == int(M.sum())
    bound_n = 2.0 ** -7 * np.linalg.norm(S, axis=-1)[M] / np.maximum(nv, 1e-30)

    def full(C):
        return np.stack([C[:, 0], C[:, 1], C[:, 2], C[:, 1], C[:, 3], C[:, 4], C[:, 2], C[:, 4], C[:, 5]], 1)
    relc = np.linalg.norm(full(Cg) - full(Co), axis=1) / np.linalg.norm(full(Co), axis=1)
    assert np.all(relc <= 2.0 * bound_n + 1e-5), np.max(relc / (2.0 * bound_n + 1e-5))
    assert np.median(relc) < 1e-5
    np.testing.assert_array_equal(pts.cpu().numpy().astype(np.float64), P[M])
    sg.close()


def _targets(P, M):
    """Oracle k-NN plane covariances of the grid's points (a1 order), float32 as the GPU reads them."""
    pts = P[M]
    return orc.source_covariances(pts, pts[:, 2], k=20, eps=1e-3, reg_mode=orc.PLANE, p=1.5)["covs"].astype(np.float32)


def _mask(Ct, P, M):
    T = sgo.knn_projector(Ct.astype(np.float64), P[M][:, 2], 1e-3, 1.5)
    return T, np.abs(np.trace(T, axis1=1, axis2=2) - 1.0) < 0.01


def test_gradients_match_oracle(g, ctx):
    d, intr = _frame(2, crop=(70, 90))
    w = _weights(4)
    sg = g.Surrogate(w)
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    P, M = _oracle_grid(d, intr, 1)
    Ct = _targets(P, M)
    r = g.gsicp_surrogate_train_step(ctx, sg, cu(d), intr, 1, 0.1, 10.0, cp, target_covs=cu(Ct), apply=False,
                                     want_grad=True)
    T, sel = _mask(Ct, P, M)
    Lo, go = sgo.loss_and_grad(P, M, w, T, sel)
    assert r["count"] == int(sel.sum())
    assert abs(r["loss"] - Lo) < 1e-4 * max(Lo, 1e-3), (r["loss"], Lo)
    gg = r["grad"].astype(np.float64)
    a, b = sgo.SIZES[0], sgo.SIZES[0] + sgo.SIZES[1]
    for lo, hi in ((0, a), (a, b), (b, sgo.N_WEIGHTS)):
        e = np.linalg.norm(gg[lo:hi] - go[lo:hi]) / np.linalg.norm(go[lo:hi])
        assert e < 1e-3, (lo, e)
    # apply = False leaves the weights alone
    np.testing.assert_array_equal(sg.weights(), w)
    sg.close()


def test_adam_step_matches_oracle(g, ctx):
    d, intr = _frame(3, crop=(64, 80))
    w = _weights(5)
    sg = g.Surrogate(w)
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    P, M = _oracle_grid(d, intr, 1)
    Ct = _targets(P, M)
    T, sel = _mask(Ct, P, M)
    lr = 1e-3
    g.gsicp_surrogate_train_step(ctx, sg, cu(d), intr, 1, 0.1, 10.0, cp, target_covs=cu(Ct), lr=lr, apply=True)
    w1 = sg.weights().astype(np.float64)
    _, go = sgo.loss_and_grad(P, M, w, T, sel)
    wo, m, s = sgo.adam_step(w.astype(np.float64), go, 0.0 * go, 0.0 * go, 1, lr)
    # the first step moves each weight by lr g / (|g| + 1e-8): compare where |g| is well above
    # both 1e-8 and the float-vs-float64 gradient difference
    big = np.abs(go) > 1e-4 * np.abs(go).max()
    np.testing.assert_allclose(w1[big], wo[big], rtol=0, atol=2e-3 * lr)
    assert np.all(np.abs(w1 - w) <= lr * 1.001 + 1e-7)
    # second step on another frame: moments carry over
    d2, _ = _frame(5, crop=(64, 80))
    P2, M2 = _oracle_grid(d2, intr, 1)
    Ct2 = _targets(P2, M2)
    T2, sel2 = _mask(Ct2, P2, M2)
    g.gsicp_surrogate_train_step(ctx, sg, cu(d2), intr, 1, 0.1, 10.0, cp, target_covs=cu(Ct2), lr=lr, apply=True)
    w2 = sg.weights().astype(np.float64)
    # the oracle's own second step, from its own first-step weights (a wrong bias correction or
    # moment carry-over moves these steps by 10-40 %)
    _, go2 = sgo.loss_and_grad(P2, M2, wo, T2, sel2)
    wo2, _, _ = sgo.adam_step(wo, go2, m, s, 2, lr)
    big2 = (np.abs(go) > 1e-3 * np.abs(go).max()) & (np.abs(go2) > 1e-3 * np.abs(go2).max())
    np.testing.assert_allclose(w2[big2], wo2[big2], rtol=0, atol=2e-2 * lr)
    sg.close()


def test_training_lowers_the_loss(g, ctx):
    cfg = surrogate_train_config5(1, n_frames=12, n_scenes=4)
    intr = HALF_TUM_INTR.as_array()
    frames = [cu(cfg["depth"](f)) for f in range(12)]
    sg = g.Surrogate(_weights(6))
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    first = np.mean([g.gsicp_surrogate_train_step(ctx, sg, fr, intr, 1, 0.1, 10.0, cp, apply=False)["loss"]
                     for fr in frames])
    for epoch in range(6):
        for fr in frames:
            g.gsicp_surrogate_train_step(ctx, sg, fr, intr, 1, 0.1, 10.0, cp, lr=2e-3, apply=True)
    last = np.mean([g.gsicp_surrogate_train_step(ctx, sg, fr, intr, 1, 0.1, 10.0, cp, apply=False)["loss"]
                    for fr in frames])
    assert last < 0.7 * first, (first, last)
    sg.close()


def test_surrogate_entry_points_reject_bad_input(g, ctx):
    d, intr = _frame(0, crop=(32, 32))
    sg = g.Surrogate(_weights(7))
    with pytest.raises(RuntimeError):
        g.gsicp_surrogate_covariances(ctx, sg, cu(d), intr, 1, 0.1, 10.0, g.CovParams(20, 0.0, g.PLANE, 1.5))
    with pytest.raises(RuntimeError):
        g.gsicp_surrogate_train_step(ctx, sg, cu(d), intr, 1, 0.1, 10.0, g.CovParams(20, 1e-3, g.ELLIPSE, 1.5))
    with pytest.raises(ValueError):
        g.Surrogate(np.zeros(10, np.float32))
    sg.close()


def test_tracker_fallback_policy(g, ctx):
    """A tracker with a surrogate and fallback ratio 0 rejects every surrogate registration and
    re-tracks with k-NN covariances: poses bit-identical to the k-NN tracker's.  With an infinite
    ratio every non-calibration frame keeps the surrogate's registration."""
    from synth import TUM_INTR, sequence_config5
    seq = sequence_config5(0, n_frames=12)
    intr = TUM_INTR.as_array()
    frames = [cu(seq["depth"](f)) for f in range(12)]
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    sg = g.Surrogate(_weights(9))

    def run(ratio, calib, use):
        tr = g.Tracker(ctx, 2, 0.1, 10.0, cp, rp)
        if use:
            tr.set_surrogate(sg, ratio, calib)
        out = [tr.frame(fr, intr, seq["poses"][0] if i == 0 else None) for i, fr in enumerate(frames)]
        tr.close()
        return out

    plain = run(0.0, 30, False)
    never = run(0.0, 30, True)
    for (Tp, ip), (Tn, inn) in zip(plain, never):
        np.testing.assert_array_equal(Tn, Tp)
        assert inn["cov_source"] == 0 and ip["cov_source"] == 0
    assert sum(i["fell_back"] for _, i in never) == 12 - 2  # all but the keyframe and the calibration frame
    always = run(float("inf"), 5, True)
    kinds = [(i["cov_source"], i["fell_back"]) for _, i in always]
    # frame 0: keyframe (k-NN); frame 1 and every 5th after it: calibration (k-NN); the rest surrogate
    assert kinds[0] == (0, 0) and kinds[1] == (0, 0)
    assert all(fb == 0 for _, fb in kinds)
    assert [src for src, _ in kinds[2:]] == [1, 1, 1, 1, 0, 1, 1, 1, 1, 0]
    sg.close()


def test_track_frame_surrogate_equals_register_on_its_covariances(g, ctx):
    """gsicp_track_frame_surrogate is a1 + the network + the registration: the same pose, system and
    counts (to the rounding of the sums' order) as gsicp_register on the points and covariances
    gsicp_surrogate_covariances returns."""
    from paper_2403_12550_b300 import surrogate as S
    from synth import TUM_INTR, sequence_config5
    seq = sequence_config5(0, n_frames=500)  # frames 0 and 3 of the held-out sequence (~4 cm apart)
    intr = TUM_INTR.as_array()
    cp = g.CovParams(20, 1e-3, g.PLANE, 1.5)
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    # map: frame 0's k-NN Gaussians in the world frame
    d0 = cu(seq["depth"](0))
    p0, z0, c0 = g.gsicp_frame_covariances(ctx, d0, intr, 2, 0.1, 10.0, cp)
    T = seq["poses"][0]
    R = torch.from_numpy(T[:3, :3]).float().cuda()
    pw = (p0 @ R.T + torch.from_numpy(T[:3, 3]).float().cuda()).contiguous()
    C = torch.stack([c0[:, 0], c0[:, 1], c0[:, 2], c0[:, 1], c0[:, 3], c0[:, 4], c0[:, 2], c0[:, 4], c0[:, 5]],
                    1).reshape(-1, 3, 3)
    Cw = R @ C @ R.T
    cw = torch.stack([Cw[:, 0, 0], Cw[:, 0, 1], Cw[:, 0, 2], Cw[:, 1, 1], Cw[:, 1, 2], Cw[:, 2, 2]], 1).contiguous()
    m = g.gsicp_build_map_index(ctx, pw, cw)
    sg = g.Surrogate(S.load_weights())
    d = cu(seq["depth"](3))
    rt = g.gsicp_track_frame_surrogate(ctx, sg, d, intr, 2, 0.1, 10.0, cp, m, T, rp)
    pts, z, covs = g.gsicp_surrogate_covariances(ctx, sg, d, intr, 2, 0.1, 10.0, cp)
    rr = g.gsicp_register(ctx, pts.contiguous(), covs.contiguous(), m, T, rp)
    assert rt["status"] == rr["status"] == g.OK and rt["n_points"] == len(pts)
    # the frame entry point orders a frame's points by their samples (2D Morton order) and
    # gsicp_register an arbitrary cloud by its points (3D Morton order): the same terms summed in
    # another order, so the results agree to rounding
    np.testing.assert_allclose(rt["T"], rr["T"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(rt["H"], rr["H"], rtol=1e-6, atol=1e-6 * np.abs(rr["H"]).max())
    assert (rt["iters"], rt["inliers"]) == (rr["iters"], rr["inliers"])
    assert abs(rt["cost"] - rr["cost"]) <= 1e-6 * abs(rr["cost"])
    # and the result is a sensible pose: within 5 mm of the ground truth (started 4 cm away)
    Tg = seq["poses"][3]
    assert np.linalg.norm(rt["T"][:3, 3] - Tg[:3, 3]) < 0.005
    sg.close()
    m.close()
