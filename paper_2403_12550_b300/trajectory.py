"""Absolute trajectory error (ATE) of estimated camera poses against the ground truth: the RMSE of
the camera positions, both as tracked (the tracker starts from the ground-truth first pose, so the
two trajectories share their origin) and after the rigid alignment (rotation and translation, no
scale) of the estimated positions onto the ground-truth ones that the TUM RGB-D benchmark's
evaluation applies before it takes the RMSE.  The alignment is the least-squares closed form of
Horn (1987) and Umeyama (1991) with the scale fixed at 1."""
from __future__ import annotations

import numpy as np


def _positions(poses) -> np.ndarray:
    return np.array([np.asarray(T, dtype=np.float64)[:3, 3] for T in poses]).reshape(-1, 3)


def ate_rmse(est, gt) -> float:
    """RMSE of the camera positions as tracked (no alignment)."""
    d = _positions(est) - _positions(gt)
    return float(np.sqrt(np.mean(np.sum(d * d, axis=1)))) if len(d) else 0.0


def align_rigid(P: np.ndarray, Q: np.ndarray):
    """(R, t) minimising sum_i |R P_i + t - Q_i|^2 over rotations R (det +1): the SVD of the
    cross-covariance of the centred point sets, with the sign of the last singular direction
    flipped where needed to exclude a reflection."""
    P, Q = np.asarray(P, dtype=np.float64), np.asarray(Q, dtype=np.float64)
    mp, mq = P.mean(axis=0), Q.mean(axis=0)
    U, _, Vt = np.linalg.svd((Q - mq).T @ (P - mp))
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt)) or 1.0])
    R = U @ D @ Vt
    return R, mq - R @ mp


def ate_rmse_aligned(est, gt) -> float:
    """RMSE of the camera positions after the rigid alignment of the estimate onto the ground truth."""
    P, Q = _positions(est), _positions(gt)
    if len(P) < 3:
        return ate_rmse(est, gt)
    R, t = align_rigid(P, Q)
    d = P @ R.T + t - Q
    return float(np.sqrt(np.mean(np.sum(d * d, axis=1))))
