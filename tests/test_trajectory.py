"""Trajectory error: the rigid alignment against a known motion, and the aligned error against
the tracked one (CPU)."""
import numpy as np

from paper_2403_12550_b300.trajectory import align_rigid, ate_rmse, ate_rmse_aligned
from synth import make_pose, random_offset, rot_axis_angle


def _trajectory(rng, n=40):
    out = []
    for f in range(n):
        out.append(make_pose(rot_axis_angle([0.1, 1.0, 0.2], 0.02 * f), [0.05 * f, 0.3 * np.sin(0.2 * f), 0.01 * f * f]))
    return out


def test_alignment_recovers_a_known_rigid_motion():
    rng = np.random.default_rng(0)
    P = rng.normal(size=(50, 3))
    G = random_offset(rng, 40.0, 2.0)
    R, t = align_rigid(P, P @ G[:3, :3].T + G[:3, 3])
    np.testing.assert_allclose(R, G[:3, :3], atol=1e-12)
    np.testing.assert_allclose(t, G[:3, 3], atol=1e-12)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_alignment_is_a_rotation_for_mirrored_points():
    # a mirror image is best matched by a reflection; the closed form must still return a rotation
    rng = np.random.default_rng(1)
    P = rng.normal(size=(30, 3))
    R, _ = align_rigid(P, P * np.array([1.0, 1.0, -1.0]))
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_rigidly_moved_estimate_has_zero_aligned_error():
    rng = np.random.default_rng(2)
    gt = _trajectory(rng)
    G = random_offset(rng, 10.0, 0.5)
    est = [G @ T for T in gt]
    assert ate_rmse(est, gt) > 0.1
    assert ate_rmse_aligned(est, gt) < 1e-12
    assert ate_rmse(gt, gt) == 0.0


def test_aligned_error_never_exceeds_the_tracked_one():
    rng = np.random.default_rng(3)
    gt = _trajectory(rng)
    for s in (1e-3, 1e-2):
        est = [T @ random_offset(rng, 0.5, s) for T in gt]
        a, u = ate_rmse_aligned(est, gt), ate_rmse(est, gt)
        assert 0 < a <= u + 1e-15
    # a single translation offset: the tracked error is its length, the aligned error 0
    est = [make_pose(T[:3, :3], T[:3, 3] + [0.03, 0, -0.04]) for T in gt]
    assert abs(ate_rmse(est, gt) - 0.05) < 1e-12 and ate_rmse_aligned(est, gt) < 1e-12
