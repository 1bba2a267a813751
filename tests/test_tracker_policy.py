"""The keyframe policy of the tracking loop on the oracle (CPU): forced and mapping-only
keyframes on schedule, and the non-overlap filter, on a small static scene."""
import numpy as np

from oracle.tracker import Tracker
from synth import Intrinsics, look_pose, make_room, raycast_depth

SMALL = Intrinsics(48, 36, 40.0, 40.0, 23.5, 17.5)


def _static_frames():
    scene = make_room(2)
    P = look_pose(scene.centre + np.array([0.3, -0.2, 0.0]), 0.7, 0.2)
    return raycast_depth(scene, P, SMALL), P


def test_schedule_and_overlap_on_a_static_camera():
    depth, P = _static_frames()
    trk = Tracker(SMALL.as_array(), stride=1, p=0.0, force_every=30, mapping_every=10)
    kinds, added = [], []
    for f in range(41):
        T, info = trk.frame(depth, P if f == 0 else None)
        kinds.append(info["kind"])
        added.append((info["added_tracking"], info["added_mapping"]))
        if f > 0:
            assert info["inlier_ratio"] == 1.0  # every point sees its own copy in the map
            assert np.abs(T - P).max() < 1e-6  # the map holds the points rounded to float
    expect = [1 if f in (0, 30) else (2 if f in (10, 20, 40) else 0) for f in range(41)]
    assert kinds == expect
    # the first keyframe adds every point; later ones add nothing (everything overlaps)
    assert added[0][0] == added[0][1] == int(np.isfinite(depth).sum())
    assert all(a == (0, 0) for f, a in enumerate(added) if f > 0)


def test_low_inlier_ratio_makes_a_keyframe():
    depth, P = _static_frames()
    trk = Tracker(SMALL.as_array(), stride=1, p=0.0, min_inlier_ratio=0.85)
    trk.frame(depth, P)
    # a frame whose right third sees nothing the map holds (pushed 0.5 m back): under 85 % inliers
    d2 = depth.copy()
    d2[:, 32:] += 0.5
    _, info = trk.frame(d2, P)
    assert info["inlier_ratio"] < 0.85 and info["kind"] == 1
    assert 0 < info["added_tracking"] <= (d2[:, 32:] > 0).sum()


def test_mapping_only_keyframe_extends_only_the_mapping_map():
    # Sec. 3, Additional Keyframe Selection for Mapping: a mapping-only keyframe's new Gaussians go
    # to the mapping map; tracking goes on against the keyframes' map alone
    depth, P = _static_frames()
    trk = Tracker(SMALL.as_array(), stride=1, p=0.0, force_every=30, mapping_every=10, min_inlier_ratio=0.85)
    trk.frame(depth, P)
    n_track, n_map = len(trk.track_means), len(trk.map_means)
    d2 = depth.copy()
    d2[:, 44:] += 0.5  # the last 4 of 48 columns move 0.5 m back: new geometry, under 15 % of the points
    for f in range(1, 11):
        _, info = trk.frame(d2 if f == 10 else depth)
    assert info["kind"] == 2 and info["inlier_ratio"] >= 0.85
    assert info["added_tracking"] == 0 and len(trk.track_means) == n_track
    assert info["added_mapping"] > 0 and len(trk.map_means) == n_map + info["added_mapping"]


def test_constant_velocity_prediction_on_a_screw_trajectory():
    # the motion model (a reading: constant velocity) predicts T_k exactly on T_k = T_0 D^k, and
    # returns a proper rotation for a slightly non-orthonormal input
    from oracle.tracker import _predict
    from synth import make_pose, rot_axis_angle
    T0 = make_pose(rot_axis_angle([0.3, -0.2, 0.9], 0.4), [1.0, -2.0, 0.5])
    D = make_pose(rot_axis_angle([0.5, 1.0, -0.3], 0.05), [0.02, -0.01, 0.03])
    traj = [T0]
    for _ in range(6):
        traj.append(traj[-1] @ D)
    for k in range(2, 7):
        np.testing.assert_allclose(_predict(traj[k - 1], traj[k - 2]), traj[k], atol=1e-12)
    np.testing.assert_array_equal(_predict(traj[3], None), traj[3])
    bent = traj[4].copy()
    bent[:3, :3] *= 1.0 + 1e-4
    R = _predict(bent, traj[3])[:3, :3]
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12
