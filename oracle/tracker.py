"""Oracle of the tracking loop with the paper's keyframe policy (TEST INFRASTRUCTURE ONLY).

Sec. 3 Keyframe Selection: a frame whose proportion of correspondences with the map falls below
a threshold becomes a keyframe, and only its Gaussians that do not overlap the existing map are
added.  Sec. 3 Additional Keyframe Selection for Mapping: if no keyframe was selected up to the
`force_every`-th frame after the last one, that frame becomes one; every `mapping_every`-th frame
after a keyframe is a mapping-only keyframe (its Gaussians go to the mapping map only).  The
threshold and the overlap radius are not given by the paper; the values here are the readings
the CUDA library uses (0.85, 1 cm).  Motion model between frames: constant velocity (a reading
too), T_{f-1} (T_{f-2}^-1 T_{f-1}) with its rotation replaced by the nearest rotation.

Every step is the FP64 oracle's (depth_to_points, source_covariances, register,
transform_gaussians, the k-d tree's nearest neighbour), in the order the policy states.
"""
from __future__ import annotations

import numpy as np

from . import Map, OK, depth_to_points, register, source_covariances, transform_gaussians


def _predict(T1: np.ndarray, T2: np.ndarray | None) -> np.ndarray:
    if T2 is None:
        return T1.copy()
    inv2 = np.eye(4)
    inv2[:3, :3] = T2[:3, :3].T
    inv2[:3, 3] = -T2[:3, :3].T @ T2[:3, 3]
    T = T1 @ (inv2 @ T1)
    U, _, Vt = np.linalg.svd(T[:3, :3])
    T[:3, :3] = U @ Vt
    return T


class Tracker:
    def __init__(self, intr, stride=2, z_min=0.1, z_max=10.0, k=20, eps=1e-3, reg_mode=0, p=1.5, max_dist=0.1,
                 max_iters=30, tol_rot=1e-6, tol_trans=1e-6, min_inliers=6, min_inlier_ratio=0.85, force_every=30,
                 mapping_every=10, overlap_radius=0.01):
        self.intr = np.asarray(intr, dtype=np.float32)
        self.a1 = (stride, z_min, z_max)
        self.cov = dict(k=k, eps=eps, reg_mode=reg_mode, p=p)
        self.reg = (max_dist, max_iters, tol_rot, tol_trans, min_inliers)
        self.kf = (min_inlier_ratio, force_every, mapping_every, overlap_radius)
        self.track_means, self.track_covs = np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32)
        self.map_means, self.map_covs = np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32)
        self.track_map = None
        self.poses = []
        self.since_kf = 0

    def _add(self, means, covs, which: str) -> int:
        """Appends the Gaussians that have no map mean within the overlap radius; returns how many."""
        cur_m = getattr(self, which + "_means")
        cur_c = getattr(self, which + "_covs")
        if len(cur_m):
            idx, _ = Map(cur_m, cur_c).tree.nn(means, self.kf[3])
            keep = idx < 0
            means, covs = means[keep], covs[keep]
        setattr(self, which + "_means", np.concatenate([cur_m, means]))
        setattr(self, which + "_covs", np.concatenate([cur_c, covs]))
        return len(means)

    def frame(self, depth, T_start=None):
        pts, z = depth_to_points(depth, self.intr, *self.a1)
        pts, z = pts.astype(np.float32), z.astype(np.float32)
        covs = source_covariances(pts, z, **self.cov)["covs"].astype(np.float32)
        info = dict(kind=0, status=OK, iters=0, n_points=len(pts), inliers=0, inlier_ratio=0.0, added_tracking=0,
                    added_mapping=0)
        if not self.poses:
            T = np.asarray(T_start, dtype=np.float64).copy()
            info["kind"] = 1
        else:
            T0 = np.asarray(T_start, dtype=np.float64) if T_start is not None else \
                _predict(self.poses[-1], self.poses[-2] if len(self.poses) >= 2 else None)
            r = register(pts, covs, self.track_map, T0, *self.reg)
            T = r["T"]
            info.update(status=r["status"], iters=r["iters"], inliers=r["inliers"],
                        inlier_ratio=r["inliers"] / len(pts) if len(pts) else 0.0)
            self.since_kf += 1
            ok = r["status"] == OK
            if ok and (info["inlier_ratio"] < self.kf[0] or self.since_kf >= self.kf[1]):
                info["kind"] = 1
            elif ok and self.kf[2] > 0 and self.since_kf % self.kf[2] == 0:
                info["kind"] = 2
        if info["kind"] and len(pts):
            wm, wc = transform_gaussians(T, pts, covs)
            wm, wc = wm.astype(np.float32), wc.astype(np.float32)
            if info["kind"] == 1:
                info["added_tracking"] = self._add(wm, wc, "track")
                self.track_map = Map(self.track_means, self.track_covs)
            info["added_mapping"] = self._add(wm, wc, "map")
        if info["kind"] == 1:
            self.since_kf = 0
        self.poses.append(T)
        return T, info
