"""The seeded input generators: shapes and the motion limits the sequences promise."""
import numpy as np

from synth import TUM_INTR, const_velocity, inv_pose, make_pose, rot_axis_angle, sequence_config3


def test_sequence_config3_shape_and_motion_limits():
    seq = sequence_config3(0, n_frames=40)
    assert len(seq["poses"]) == 40 and seq["intr"] == TUM_INTR
    d = seq["depth"](3)
    assert d.shape == (480, 640) and d.dtype == np.float32
    np.testing.assert_array_equal(d, seq["depth"](3))  # noise seeded per frame
    dt = 1.0 / 30.0
    for a, b in zip(seq["poses"][:-1], seq["poses"][1:]):
        rel = inv_pose(a) @ b
        ang = np.arccos(np.clip((np.trace(rel[:3, :3]) - 1) / 2, -1, 1))
        assert np.linalg.norm(b[:3, 3] - a[:3, 3]) <= 1.0 * dt * 1.02
        # the heading rate is capped at 60 deg/s; pitch changes add a little
        assert ang <= np.deg2rad(60.0) * dt * 1.5


def test_const_velocity_repeats_the_last_motion():
    step = make_pose(rot_axis_angle(np.array([0.3, -0.5, 0.8]), 0.02), [0.01, -0.02, 0.005])
    T1 = make_pose(rot_axis_angle(np.array([1.0, 0.0, 0.0]), 0.4), [1.0, 2.0, 0.5])
    T2 = T1 @ step
    np.testing.assert_allclose(const_velocity(T2, T1), T2 @ step, atol=1e-12)
    np.testing.assert_array_equal(const_velocity(T2, None), T2)


def test_rot_angle_reads_angles_and_ignores_scale():
    from tests._util import rot_angle
    for a in (0.0, 1e-7, 1e-4, 0.3, 2.0, 3.1):
        R = rot_axis_angle(np.array([0.2, -0.7, 0.4]), a)
        assert abs(rot_angle(R) - a) < 1e-12
        assert abs(rot_angle(R * (1 - 3e-9)) - a) < 1e-8  # not sqrt(6 * 3e-9) = 1.3e-4


def test_config5_half_res_grid_and_held_out_rooms():
    """A HALF_TUM_INTR render is the stride-2 sample grid of the TUM_INTR render from the same
    pose; the training rooms exclude the held-out sequence's room; frames are deterministic."""
    from synth import HALF_TUM_INTR, TUM_INTR, raycast_depth, sequence_config5, surrogate_train_config5
    tr = surrogate_train_config5(0, n_frames=6, n_scenes=3)
    full = raycast_depth(tr["scenes"][1], tr["poses"][1], TUM_INTR)
    half = raycast_depth(tr["scenes"][1], tr["poses"][1], HALF_TUM_INTR)
    np.testing.assert_allclose(half, full[::2, ::2], rtol=1e-6)
    np.testing.assert_array_equal(tr["depth"](4), tr["depth"](4))
    seq = sequence_config5(0, n_frames=10)
    held = seq["scene"]
    for sc in tr["scenes"]:
        assert not (np.array_equal(sc.box_center, held.box_center) and np.array_equal(sc.sph_center, held.sph_center))
    assert seq["depth"](3).shape == (480, 640)


def test_parallel_rendering_equals_in_order_rendering():
    from synth import render_sequence_frames, sequence_config3, sequence_config5
    for kind, make in (("config3", sequence_config3), ("config5", sequence_config5)):
        got = render_sequence_frames(kind, 2, 3, workers=2)
        cfg = make(2, n_frames=3)
        assert got.shape[0] == 3
        for f in range(3):
            np.testing.assert_array_equal(got[f], cfg["depth"](f))
