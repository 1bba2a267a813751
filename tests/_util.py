"""Shared helpers for the parity tests: input preparation through the oracle only,
and pose / covariance comparisons."""
from __future__ import annotations

import numpy as np

import oracle as orc
from synth import REPLICA_INTR, frame_config2, pair_config1, transform_points

# Tolerances: poses within 1e-4 rad and 1e-5 m and covariances within 1e-4 relative Frobenius of
# the FP64 oracle; k-NN sets identical except swaps among candidates whose distances tie within 1e-6.
POSE_ROT_TOL = 1e-4      # rad
POSE_TRANS_TOL = 1e-5    # m
COV_REL_TOL = 1e-4       # relative Frobenius
KNN_TIE_REL = 1e-6       # kNN set swaps allowed between oracle distances this close
PLANE_GAP_EXCLUDE = 1e-3


def rot_angle(R: np.ndarray) -> float:
    """Rotation angle of R from both its antisymmetric part (sin) and its trace (cos): unlike
    arccos of the trace alone, a common scale error of nearly orthonormal inputs (1 + e) does not
    read as an angle of sqrt(6 e)."""
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    return float(np.arctan2(0.5 * np.linalg.norm(w), 0.5 * (np.trace(R) - 1.0)))


def pose_diff(Ta: np.ndarray, Tb: np.ndarray):
    """(rotation angle of Ra^T Rb, |ta - tb|)."""
    return rot_angle(Ta[:3, :3].T @ Tb[:3, :3]), float(np.linalg.norm(Ta[:3, 3] - Tb[:3, 3]))


def sym(c6):
    c6 = np.asarray(c6)
    return np.stack([np.stack([c6[..., 0], c6[..., 1], c6[..., 2]], -1),
                     np.stack([c6[..., 1], c6[..., 3], c6[..., 4]], -1),
                     np.stack([c6[..., 2], c6[..., 4], c6[..., 5]], -1)], -2)


def cov_rel_err(a6, b6):
    """Relative Frobenius error of symmetric 3x3 matrices given as 6-vectors (per row)."""
    A, B = sym(a6), sym(b6)
    return np.linalg.norm((A - B).reshape(len(A), -1), axis=1) / np.maximum(np.linalg.norm(B.reshape(len(B), -1), axis=1), 1e-300)


def config1_inputs(scene_seed: int, pose_seed: int, n: int = 10_000, reg_mode: int = orc.PLANE):
    """Config-1 pair with oracle-made covariances, everything float32 as the GPU reads it."""
    src, tgt, T_gt = pair_config1(scene_seed, pose_seed, n=n)
    cs = orc.source_covariances(src, k=20, eps=1e-3, reg_mode=reg_mode)["covs"].astype(np.float32)
    ct = orc.source_covariances(tgt, k=20, eps=1e-3, reg_mode=reg_mode)["covs"].astype(np.float32)
    return src, cs, tgt, ct, T_gt


def oracle_frame_points(depth, intr=REPLICA_INTR, stride=2, z_min=0.1, z_max=10.0):
    pts, z = orc.depth_to_points(depth, intr.as_array(), stride, z_min, z_max)
    return pts.astype(np.float32), z.astype(np.float32)


def oracle_map_from_views(view_depths, view_poses, intr=REPLICA_INTR, stride=2, p=1.5, reg_mode=orc.PLANE):
    """Map Gaussians built by the oracle: each prior view back-projected, its
    covariances computed and scale-aligned, then moved into the world frame."""
    means, covs = [], []
    for d, P in zip(view_depths, view_poses):
        pts, z = oracle_frame_points(d, intr, stride)
        c = orc.source_covariances(pts, z, k=20, eps=1e-3, reg_mode=reg_mode, p=p)["covs"]
        mw, cw = orc.transform_gaussians(P, pts, c)
        means.append(mw)
        covs.append(cw)
    return np.concatenate(means).astype(np.float32), np.concatenate(covs).astype(np.float32)


def config2_inputs(seed: int = 0):
    f = frame_config2(seed)
    means, covs = oracle_map_from_views(f["view_depths"], f["view_poses"])
    return f, means, covs


__all__ = ["POSE_ROT_TOL", "POSE_TRANS_TOL", "COV_REL_TOL", "KNN_TIE_REL", "PLANE_GAP_EXCLUDE", "rot_angle",
           "pose_diff", "sym", "cov_rel_err", "config1_inputs", "oracle_frame_points", "oracle_map_from_views",
           "config2_inputs", "transform_points"]


def near_tie_pairs(seed: int, d: float, n_side: int = 16, spacing: float = 0.4):
    """Source points whose two nearest map points are equidistant to within the float rounding of
    the transformed query, arranged so that the rounded query (hi alone) and the exact query
    disagree on which is nearer.

    A grid of n_side^3 float32 source points near (5, 5, 5) m (where an ulp of a coordinate is
    4.8e-7 m) and a pose with a rotation, so that y = R x + t is not a float.  For each point, two
    float32 map points at distance ~d from y in FP64: a at a random direction, b chosen among random
    directions at the same radius so that the FP64 distances differ by more than `gap` (well above
    what the distances' own float rounding can flip) while the distances from float32(y) order the
    two the other way round by more than `gap`, when a direction doing so is found (else the first
    candidate).  Returns src, covs_s, means, covs (map: point i's pair at 2i, 2i + 1), T,
    nearest (FP64 nearest map index per point), flipped (bool: the rounded query picks the other)."""
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) - (n_side - 1) / 2) * spacing
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    src = (np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + np.array([5.3, 4.9, 5.7])).astype(np.float32)
    ax = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    ang = 0.21
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = [0.37, -0.21, 0.13]
    y = src.astype(np.float64) @ R.T + T[:3, 3]
    yh = y.astype(np.float32).astype(np.float64)
    gap = 2e-9 if d < 0.01 else 2e-8
    n = len(src)
    means = np.empty((2 * n, 3), np.float32)
    flipped = np.zeros(n, bool)
    for i in range(n):
        u = rng.normal(size=3)
        a = (y[i] + d * u / np.linalg.norm(u)).astype(np.float32)
        da = np.linalg.norm(a - y[i])
        V = rng.normal(size=(256, 3))
        B = (y[i] + da * V / np.linalg.norm(V, axis=1, keepdims=True)).astype(np.float32)
        db = np.linalg.norm(B - y[i], axis=1)
        ha, hb = np.linalg.norm(a - yh[i]), np.linalg.norm(B - yh[i], axis=1)
        ok = (np.abs(da - db) > gap) & (np.abs(ha - hb) > gap) & (np.sign(da - db) != np.sign(ha - hb))
        j = int(np.argmax(ok)) if ok.any() else 0
        flipped[i] = bool(ok[j])
        means[2 * i], means[2 * i + 1] = a, B[j]
    d2 = ((means.astype(np.float64).reshape(n, 2, 3) - y[:, None, :]) ** 2).sum(-1)
    nearest = 2 * np.arange(n) + np.argmin(d2, axis=1)
    covs_s = np.tile(np.array([1e-4, 0, 0, 1e-4, 0, 1e-4], np.float32), (n, 1))
    covs = np.tile(np.array([1e-4, 0, 0, 1e-4, 0, 1e-4], np.float32), (2 * n, 1))
    return src, covs_s, means, covs, T, nearest.astype(np.int32), flipped
