"""The pins catch plausible mistakes: each case plants one mistake in a copy of an oracle
(a dropped term, a wrong sign, index or power, a transposed operand) -- the C oracle, built with
gcc, or the surrogate's or the tracking loop's Python oracle, loaded as a module of its own -- and
checks that the pins named for it fail on the copy while they pass on the real oracle.  CPU only."""
import importlib.util
import os
import shutil

import numpy as np
import pytest

import oracle as orc
from oracle.build import compile_shared

from . import test_golden as golden
from . import test_oracle_pins as pins
from . import test_surrogate_oracle as spins
from . import test_tracker_policy as tpins

HERE = os.path.dirname(os.path.abspath(orc.__file__))

# (name, text in gsicp_oracle.c, planted text, pins that must catch it)
MUTANTS = [
    ("combined covariance without the rotation of C^s",
     "Sig[a] = Ct[a] + RCs[a];", "Sig[a] = Ct[a] + Cs[a];",
     [pins.test_linearisation_is_invariant_to_the_source_and_map_frames,
      lambda: golden.test_oracle_linearise_one_correspondence("quarter_turn_z")]),
    ("weight Sigma instead of Sigma^-1",
     "if (inv_sym3(Sig, W6) != 0) return;", "memcpy(W6, Sig, sizeof(W6));",
     [pins.test_cost_tends_to_point_to_plane_error_in_the_flat_limit]),
    ("R C R instead of R C R^T",
     "s += RS[3 * r + j] * R[3 * c + j];", "s += RS[3 * r + j] * R[3 * j + c];",
     [pins.test_linearisation_is_invariant_to_the_source_and_map_frames]),
    ("plane eps on the largest axis",
     "double lam[3] = {eps, 1.0, 1.0};", "double lam[3] = {1.0, 1.0, eps};",
     [pins.test_regularisation_closed_forms, lambda: golden.test_oracle_regularise_on_the_worked_raw_covariances("star_345")]),
    ("ellipse scaled by the largest scale, not the median",
     "double lam[3] = {r0, 1.0, w[2] / w[1]};", "double lam[3] = {r0 * w[1] / w[2], w[1] / w[2], 1.0};",
     [pins.test_regularisation_closed_forms]),
    ("spectrum rebuilt as V^T diag V",
     "s += V[3 * r + j] * lam[j] * V[3 * c + j];", "s += V[3 * j + r] * lam[j] * V[3 * j + c];",
     [pins.test_regularisation_closed_forms]),
    ("scale aligning by z^-p instead of z^-2p",
     "pow(z[i], -2.0 * p)", "pow(z[i], -p)",
     [pins.test_scale_aligning_is_z_power, lambda: golden.test_oracle_source_covariances_on_the_star("star_345", 1.5)]),
    ("covariance divided by k - 1",
     "for (int a = 0; a < 6; ++a) C[a] /= kk;", "for (int a = 0; a < 6; ++a) C[a] /= (kk - 1);",
     [pins.test_raw_covariance_equals_numpy_cov_of_brute_force_neighbours]),
    ("Jacobi rotation of the eigenvectors with a wrong sign",
     "Q[r][q] = s * qrp + c * qrq;", "Q[r][q] = -s * qrp + c * qrq;",
     [pins.test_eigh3_matches_lapack]),
    ("eigenvalues sorted in descending order",
     "if (d[order[j]] < d[order[i]])", "if (d[order[j]] > d[order[i]])",
     [pins.test_eigh3_matches_lapack, pins.test_regularisation_closed_forms]),
    ("SE(3) exp: translation factor with sin(th)/th",
     "Vm[i] = id + B * K[i] + Cc * K2[i];", "Vm[i] = id + A * K[i] + Cc * K2[i];",
     [lambda: pins.test_se3_exp_matches_expm(1.0), lambda: golden.test_oracle_se3_exp("quarter_turn_z")]),
    ("Jacobian d d / d v = +I",
     "J[6 * r + 3 + c] = (r == c) ? -1.0 : 0.0;", "J[6 * r + 3 + c] = (r == c) ? 1.0 : 0.0;",
     [pins.test_jacobian_matches_finite_differences]),
    ("Gauss-Newton step +H^-1 b",
     "nb[a] = -b[a];", "nb[a] = b[a];",
     [pins.test_exact_recovery_on_noise_free_room]),
    ("back substitution with L for L^T",
     "for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];", "for (int k = i + 1; k < 6; ++k) s -= L[6 * i + k] * x[k];",
     [pins.test_one_gauss_newton_step_solves_the_normal_equations]),
    ("pose update on the right",
     "    pose_mul(E, T, T);", "    pose_mul(T, E, T);",
     [pins.test_one_gauss_newton_step_solves_the_normal_equations]),
    ("distance ties to the larger index",
     "(d == e && i < j)", "(d == e && i > j)",
     [pins.test_knn_ties_break_to_smaller_index]),
    ("k-d tree prunes the far side too early",
     "if (diff * diff <= L->d[L->k - 1])", "if (diff * diff <= 0.25 * L->d[L->k - 1])",
     [lambda: pins.test_knn_tree_equals_brute_force(2000, 20, 200), lambda: pins.test_radius_nn_tree_equals_brute_force(0)]),
    ("Gaussians moved by R^T instead of R",
     "pts_out[3 * i + r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + t[r];",
     "pts_out[3 * i + r] = R[r] * x[0] + R[3 + r] * x[1] + R[6 + r] * x[2] + t[r];",
     [pins.test_transform_gaussians_is_a_rigid_motion]),
    ("back-projection with cx in place of cy",
     "((double)v - cy) * d / fy", "((double)v - cx) * d / fy",
     [pins.test_depth_to_points_on_analytic_plane, lambda: golden.test_oracle_depth_to_points_small_image(1)]),
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("case", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(case, workdir):
    name, old, new, catchers = MUTANTS[case]
    with open(os.path.join(HERE, "gsicp_oracle.c")) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
    d = workdir / f"m{case}"
    d.mkdir()
    shutil.copy(os.path.join(HERE, "gsicp_oracle.h"), d / "gsicp_oracle.h")
    (d / "gsicp_oracle.c").write_text(src.replace(old, new))
    lib = compile_shared(str(d / "gsicp_oracle.c"), str(d / "liboracle.so"))
    for pin in catchers:
        pin()  # passes on the real oracle
        with orc.library(lib):
            with pytest.raises(AssertionError):
                pin()
    # the real oracle is back in place afterwards
    np.testing.assert_allclose(orc.se3_exp(np.zeros(6)), np.eye(4))


# (name, text in oracle/surrogate.py, planted text, names of the surrogate pins that must catch it)
SURROGATE_MUTANTS = [
    ("layer 1 not centred",
     "a += (Ps - Ms * P) @ W1[:, :, dy, dx].T", "a += Ps @ W1[:, :, dy, dx].T",
     ["test_layer1_equals_brute_force", "test_translation_and_scale_invariance"]),
    ("convolution with the kernel flipped",
     "y += _shift(x, dy - R, dx - R) @ W[:, :, dy, dx].T", "y += _shift(x, R - dy, R - dx) @ W[:, :, dy, dx].T",
     ["test_conv_equals_brute_force"]),
    ("bfloat16 by truncation",
     "np.rint(m * 256.0)", "np.trunc(m * 256.0)",
     ["test_bf16_rounding"]),
    ("plane covariance with 1 + eps",
     "k = 1.0 - eps", "k = 1.0 + eps",
     ["test_plane_covariance_equals_c_oracle_regularisation"]),
    ("scale aligning by z^-p",
     "s = np.asarray(z, dtype=np.float64) ** (-2.0 * p)", "s = np.asarray(z, dtype=np.float64) ** (-p)",
     ["test_plane_covariance_equals_c_oracle_regularisation"]),
    ("isotropic fallback without scale aligning's square",
     "        s = z[~ok] ** (-2.0 * p)", "        s = z[~ok] ** (-p)",
     ["test_zero_prediction_gives_isotropic_covariance_and_full_loss"]),
    ("loss 1 + n^T T n",
     "return float(np.mean(1.0 - q))", "return float(np.mean(1.0 + q))",
     ["test_loss_values"]),
    ("gradient without the ReLU gate of layer 2",
     'da2 = dh2 * (f["a2"] > 0) * Mf', "da2 = dh2 * Mf",
     ["test_gradient_matches_finite_differences"]),
    ("gradient without the normalisation's projection",
     "dv_valid[ok] = (dLdn - n * np.sum(n * dLdn, axis=1, keepdims=True)) / nrm[ok][:, None]",
     "dv_valid[ok] = dLdn / nrm[ok][:, None]",
     ["test_gradient_matches_finite_differences"]),
    ("layer-3 back-propagation shifted the wrong way",
     "dh2 += _shift(dv @ W3r[:, :, dy, dx], R - dy, R - dx)", "dh2 += _shift(dv @ W3r[:, :, dy, dx], dy - R, dx - R)",
     ["test_gradient_matches_finite_differences"]),
    ("grid back-projection with cx in place of cy",
     "P = np.stack([(u - cx) * dz / fx, (v - cy) * dz / fy, dz], axis=-1)",
     "P = np.stack([(u - cx) * dz / fx, (v - cx) * dz / fy, dz], axis=-1)",
     ["test_point_grid_equals_c_oracle_points"]),
    ("k-NN projector with the wrong sign",
     "return (np.eye(3)[None] - full * s[:, None, None]) / (1.0 - eps)",
     "return (np.eye(3)[None] + full * s[:, None, None]) / (1.0 - eps)",
     ["test_plane_covariance_equals_c_oracle_regularisation"]),
    ("Adam without bias correction",
     "mh = m / (1 - b1 ** t)", "mh = m",
     ["test_adam_first_step_and_convergence"]),
]


# (name, text in oracle/tracker.py, planted text, names of the tracking-loop pins that must catch it)
TRACKER_MUTANTS = [
    ("non-overlap filter inverted",
     "keep = idx < 0", "keep = idx >= 0",
     ["test_schedule_and_overlap_on_a_static_camera"]),
    ("forced keyframe one frame late",
     "self.since_kf >= self.kf[1]", "self.since_kf > self.kf[1]",
     ["test_schedule_and_overlap_on_a_static_camera"]),
    ("mapping-only keyframes extend the tracking map",
     'if info["kind"] == 1:\n                info["added_tracking"]', 'if info["kind"] >= 1:\n                info["added_tracking"]',
     ["test_mapping_only_keyframe_extends_only_the_mapping_map"]),
    ("inlier-ratio test reversed",
     'info["inlier_ratio"] < self.kf[0]', 'info["inlier_ratio"] > self.kf[0]',
     ["test_low_inlier_ratio_makes_a_keyframe"]),
    ("motion model composed in the wrong order",
     "T = T1 @ (inv2 @ T1)", "T = T1 @ (T1 @ inv2)",
     ["test_constant_velocity_prediction_on_a_screw_trajectory"]),
]


def _planted_module(file_name, old, new, name):
    path = os.path.join(HERE, file_name)
    with open(path) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
    spec = importlib.util.spec_from_loader("oracle._planted_" + file_name[:-3], loader=None)
    mutant = importlib.util.module_from_spec(spec)
    mutant.__package__ = "oracle"  # relative imports resolve to the real oracle package
    exec(compile(src.replace(old, new), path, "exec"), mutant.__dict__)
    return mutant


@pytest.mark.parametrize("case", range(len(SURROGATE_MUTANTS)), ids=[m[0] for m in SURROGATE_MUTANTS])
def test_surrogate_pins_catch_planted_mistake(case, monkeypatch):
    name, old, new, catchers = SURROGATE_MUTANTS[case]
    mutant = _planted_module("surrogate.py", old, new, name)
    for pin_name in catchers:
        pin = getattr(spins, pin_name)
        pin()  # passes on the real oracle
        with monkeypatch.context() as mp:
            mp.setattr(spins, "sg", mutant)
            with pytest.raises(AssertionError):
                pin()


@pytest.mark.parametrize("case", range(len(TRACKER_MUTANTS)), ids=[m[0] for m in TRACKER_MUTANTS])
def test_tracker_pins_catch_planted_mistake(case, monkeypatch):
    name, old, new, catchers = TRACKER_MUTANTS[case]
    mutant = _planted_module("tracker.py", old, new, name)
    for pin_name in catchers:
        pin = getattr(tpins, pin_name)
        pin()  # passes on the real oracle
        with monkeypatch.context() as mp:
            mp.setattr(tpins, "Tracker", mutant.Tracker)
            mp.setattr("oracle.tracker._predict", mutant._predict)
            with pytest.raises(AssertionError):
                pin()
