"""B300-native G-ICP tracking hot path of "RGBD GS-ICP SLAM" (arXiv 2403.12550).

Thin Python binding over the C ABI of ``libgsicp.so`` (``include/gsicp.h``):
the functions below carry the C entry points' names and only marshal
arguments (torch CUDA tensors -> device pointers, the current torch stream ->
``cudaStream_t``).  Every step of the path runs in the library's CUDA kernels;
there is no fallback.  Importing this package raises if the library has not
been built (``python paper_2403_12550_b300/build.py``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

__all__ = [
    "GsicpError", "CovParams", "RegParams", "IndexParams", "Context", "MapHandle",
    "PLANE", "ELLIPSE", "NONE", "LIB_PATH", "lib",
    "gsicp_ctx_create", "gsicp_ctx_destroy", "gsicp_ctx_set_timing", "gsicp_ctx_last_residual", "gsicp_ctx_set_coop_walks", "gsicp_ctx_set_gn_launch_mode", "gsicp_ctx_set_gn_block", "gsicp_ctx_set_packet_iters", "gsicp_ctx_set_cache_step", "GN_GRAPH", "GN_PLAIN", "gsicp_ctx_phase_times", "gsicp_ctx_reg_stats", "gsicp_ctx_frame_stats", "gsicp_status_string", "gsicp_last_error", "gsicp_version",
    "gsicp_depth_to_points", "gsicp_depth_to_points_noalloc", "gsicp_source_covariances", "gsicp_frame_covariances",
    "gsicp_build_map_index", "gsicp_map_append", "gsicp_shard_begin", "gsicp_shard_linearise", "gsicp_shard_update",
    "SHARD_SUMS", "SHARD_RUNNING", "SHARD_CONVERGED", "SHARD_MAXITER", "SHARD_DEGENERATE",
    "gsicp_map_rebuild", "gsicp_map_inspect", "gsicp_map_size", "gsicp_map_destroy", "gsicp_transform_gaussians", "gsicp_register", "gsicp_register_batch", "gsicp_selftest_batch_timeout", "gsicp_linearise",
    "gsicp_map_nearest", "gsicp_track_frame", "gsicp_track_frame_host",
    "KeyframeParams", "FrameInfo", "Tracker", "FRAME", "KEYFRAME", "MAPPING_KEYFRAME",
    "Surrogate", "SURROGATE_WEIGHTS", "gsicp_surrogate_covariances", "gsicp_surrogate_train_step",
    "gsicp_track_frame_surrogate",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgsicp.so")

PLANE, ELLIPSE, NONE = 0, 1, 2
GN_GRAPH, GN_PLAIN = 0, 1
SHARD_SUMS = 30
SHARD_RUNNING, SHARD_CONVERGED, SHARD_MAXITER, SHARD_DEGENERATE = range(4)
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_DEGENERATE, ERR_TIMEOUT, ERR_NOT_IMPLEMENTED, ERR_CAPACITY = range(8)


class GsicpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {gsicp_status_string(status)}"
        detail = gsicp_last_error()
        if status == ERR_CUDA and detail:
            msg += f" ({detail})"
        super().__init__(msg)


class CovParams(C.Structure):
    _fields_ = [("k", C.c_int), ("eps", C.c_float), ("reg_mode", C.c_int), ("p", C.c_float)]

    def __init__(self, k: int = 20, eps: float = 1e-3, reg_mode: int = PLANE, p: float = 0.0):
        super().__init__(k, eps, reg_mode, p)


class RegParams(C.Structure):
    _fields_ = [("max_corr_dist", C.c_float), ("max_iters", C.c_int), ("tol_rot", C.c_double),
                ("tol_trans", C.c_double), ("min_inliers", C.c_int)]

    def __init__(self, max_corr_dist: float = 0.1, max_iters: int = 30, tol_rot: float = 1e-6,
                 tol_trans: float = 1e-6, min_inliers: int = 6):
        super().__init__(max_corr_dist, max_iters, tol_rot, tol_trans, min_inliers)


class IndexParams(C.Structure):
    _fields_ = [("bucket", C.c_int), ("cell", C.c_float)]


class KeyframeParams(C.Structure):
    _fields_ = [("min_inlier_ratio", C.c_float), ("force_every", C.c_int), ("mapping_every", C.c_int),
                ("overlap_radius", C.c_float)]

    def __init__(self, min_inlier_ratio: float = 0.85, force_every: int = 30, mapping_every: int = 10,
                 overlap_radius: float = 0.01):
        super().__init__(min_inlier_ratio, force_every, mapping_every, overlap_radius)


class FrameInfo(C.Structure):
    _fields_ = [("kind", C.c_int), ("status", C.c_int), ("iters", C.c_int), ("n_points", C.c_int64),
                ("inliers", C.c_int64), ("inlier_ratio", C.c_double), ("added_tracking", C.c_int64),
                ("added_mapping", C.c_int64), ("cov_source", C.c_int), ("fell_back", C.c_int),
                ("residual", C.c_double)]


FRAME, KEYFRAME, MAPPING_KEYFRAME = 0, 1, 2


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2403_12550_b300/build.py` "
                      "(there is no non-CUDA fallback)")

lib = C.CDLL(LIB_PATH)

_vp, _i32p, _i64p, _fp, _dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_float), \
    C.POINTER(C.c_double)


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("gsicp_ctx_create", C.c_int, [C.POINTER(C.c_void_p)])
_sig("gsicp_ctx_destroy", None, [_vp])
_sig("gsicp_status_string", C.c_char_p, [C.c_int])
_sig("gsicp_last_error", C.c_char_p, [])
_sig("gsicp_version", C.c_char_p, [])
_sig("gsicp_ctx_set_timing", C.c_int, [_vp, C.c_int])
_sig("gsicp_ctx_last_residual", C.c_int, [_vp, _dp, _i64p])
_sig("gsicp_ctx_set_coop_walks", C.c_int, [_vp, C.c_int])
_sig("gsicp_ctx_set_gn_launch_mode", C.c_int, [_vp, C.c_int])
_sig("gsicp_ctx_set_gn_block", C.c_int, [_vp, C.c_int])
_sig("gsicp_ctx_set_packet_iters", C.c_int, [_vp, C.c_int])
_sig("gsicp_ctx_set_cache_step", C.c_int, [_vp, C.c_float])
_sig("gsicp_ctx_phase_times", C.c_int, [_vp, _dp])
_sig("gsicp_ctx_reg_stats", C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp])
_sig("gsicp_ctx_frame_stats", C.c_int, [_vp, _i64p])
_sig("gsicp_depth_to_points", C.c_int, [_vp, _vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float, _vp, _vp,
                                        C.c_int64, _vp, _i64p, _vp])
_sig("gsicp_depth_to_points_noalloc", C.c_int, [_vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float, _vp,
                                                _vp, C.c_int64, _vp, _vp, _vp])
_sig("gsicp_source_covariances", C.c_int, [_vp, _vp, _vp, C.c_int64, C.POINTER(CovParams), _vp, _vp, _vp])
_sig("gsicp_frame_covariances", C.c_int, [_vp, _vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float,
                                          C.POINTER(CovParams), _vp, _vp, _vp, C.c_int64, _i64p, _vp])
_sig("gsicp_build_map_index", C.c_int, [_vp, _vp, _vp, C.c_int64, C.POINTER(IndexParams), _vp,
                                        C.POINTER(C.c_void_p)])
_sig("gsicp_map_append", C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, _vp])
_sig("gsicp_map_size", C.c_int64, [_vp])
_sig("gsicp_map_rebuild", C.c_int, [_vp, _vp, _vp])
_sig("gsicp_map_inspect", C.c_int, [_vp, _vp, _vp, _i64p, C.POINTER(C.c_int), _vp])
_sig("gsicp_map_destroy", None, [_vp])
_sig("gsicp_transform_gaussians", C.c_int, [_dp, _vp, _vp, C.c_int64, _vp, _vp, _vp])
_sig("gsicp_register", C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _dp, C.POINTER(RegParams), _dp, _dp, _dp,
                                 C.POINTER(C.c_int), _dp, _i64p, _vp])
_sig("gsicp_shard_begin", C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _dp, C.POINTER(RegParams), _vp])
_sig("gsicp_shard_linearise", C.c_int, [_vp, _vp, _vp])
_sig("gsicp_shard_update", C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_int), _dp, _dp, C.POINTER(C.c_int), _dp,
                                     _i64p, _vp])
_sig("gsicp_register_batch", C.c_int, [_vp, C.c_int, _vp, _vp, _i64p, _vp, _dp, C.POINTER(RegParams), _dp,
                                       C.POINTER(C.c_int), _dp, _i64p, C.POINTER(C.c_int), _vp])
_sig("gsicp_selftest_batch_timeout", C.c_int, [_vp, _vp])
_sig("gsicp_tracker_create", C.c_int, [_vp, C.c_int, C.c_float, C.c_float, C.POINTER(CovParams),
                                       C.POINTER(RegParams), C.POINTER(KeyframeParams), C.POINTER(C.c_void_p)])
_sig("gsicp_tracker_destroy", None, [_vp])
_sig("gsicp_tracker_frame", C.c_int, [_vp, _vp, C.c_int, C.c_int, _fp, _dp, _dp, C.POINTER(FrameInfo), _vp])
_sig("gsicp_tracker_maps", C.c_int, [_vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)])
_sig("gsicp_tracker_set_surrogate", C.c_int, [_vp, _vp, C.c_float, C.c_int, C.c_int])
_sig("gsicp_linearise", C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _dp, C.c_float, _dp, _dp, _dp, _i64p, _vp, _vp])
_sig("gsicp_map_nearest", C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_float, _vp, _vp, _vp])
for _n in ("gsicp_track_frame", "gsicp_track_frame_host"):
    _sig(_n, C.c_int, [_vp, _vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float, C.POINTER(CovParams), _vp,
                       _dp, C.POINTER(RegParams), _dp, _dp, C.POINTER(C.c_int), _dp, _i64p, _i64p, _vp])
_sig("gsicp_track_frame_surrogate", C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float,
                                              C.POINTER(CovParams), _vp, _dp, C.POINTER(RegParams), _dp, _dp,
                                              C.POINTER(C.c_int), _dp, _i64p, _i64p, _vp])
_sig("gsicp_surrogate_create", C.c_int, [_fp, C.POINTER(C.c_void_p)])
_sig("gsicp_surrogate_destroy", None, [_vp])
_sig("gsicp_surrogate_get_weights", C.c_int, [_vp, _fp])
_sig("gsicp_surrogate_set_weights", C.c_int, [_vp, _fp])
_sig("gsicp_surrogate_set_timing", C.c_int, [_vp, C.c_int])
_sig("gsicp_surrogate_layer_times", C.c_int, [_vp, _dp])
_sig("gsicp_surrogate_covariances", C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float,
                                              C.POINTER(CovParams), _vp, _vp, _vp, _vp, C.c_int64, _i64p, _vp])
_sig("gsicp_surrogate_train_step", C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _fp, C.c_int, C.c_float, C.c_float,
                                             C.POINTER(CovParams), _vp, C.c_float, C.c_int, _dp, _i64p, _fp, _vp])
SURROGATE_WEIGHTS = 30400


# ----------------------------------------------------------------------------- helpers

def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor | None, dtype=torch.float32, cols: int | None = None) -> C.c_void_p | None:
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"expected shape (n, {cols}), got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _pose(T) -> C.Array:
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return (C.c_double * 16)(*a)


def _check(st: int, where: str, allow=()):
    if st != OK and st not in allow:
        raise GsicpError(st, where)
    return st


def gsicp_status_string(st: int) -> str:
    return lib.gsicp_status_string(st).decode()


def gsicp_last_error() -> str:
    return lib.gsicp_last_error().decode()


def gsicp_version() -> str:
    return lib.gsicp_version().decode()


class Context:
    """Owns a ``gsicp_ctx`` (device scratch + the Gauss-Newton CUDA graph)."""

    def __init__(self):
        h = C.c_void_p()
        _check(lib.gsicp_ctx_create(C.byref(h)), "gsicp_ctx_create")
        self.ptr = h

    def close(self):
        if self.ptr:
            lib.gsicp_ctx_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MapHandle:
    """Owns a ``gsicp_map`` (the map index and its packed copy of the Gaussians)."""

    def __init__(self, ptr):
        self.ptr = ptr

    @property
    def size(self) -> int:
        return int(lib.gsicp_map_size(self.ptr))

    def close(self):
        if self.ptr:
            lib.gsicp_map_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gsicp_ctx_create() -> Context:
    return Context()


def gsicp_ctx_destroy(ctx: Context):
    ctx.close()


# ----------------------------------------------------------------------------- entry points

def gsicp_ctx_set_timing(ctx: Context, enable: bool):
    _check(lib.gsicp_ctx_set_timing(ctx.ptr, int(bool(enable))), "gsicp_ctx_set_timing")


def gsicp_ctx_set_coop_walks(ctx: Context, max_per_warp: int):
    """Warps with at most max_per_warp tree walks in an iteration walk together (0..32; results
    do not depend on it)."""
    _check(lib.gsicp_ctx_set_coop_walks(ctx.ptr, int(max_per_warp)), "gsicp_ctx_set_coop_walks")


def gsicp_ctx_set_gn_launch_mode(ctx: Context, mode: int):
    """GN_GRAPH (default): the iterations run as one conditional CUDA graph; GN_PLAIN: one plain
    launch per iteration (same results; visible to launch-listing profilers)."""
    _check(lib.gsicp_ctx_set_gn_launch_mode(ctx.ptr, int(mode)), "gsicp_ctx_set_gn_launch_mode")


def gsicp_ctx_set_gn_block(ctx: Context, points_per_block: int):
    """Source points per block of the Gauss-Newton iterations: 128, 256 (default) or 384."""
    _check(lib.gsicp_ctx_set_gn_block(ctx.ptr, int(points_per_block)), "gsicp_ctx_set_gn_block")


def gsicp_ctx_set_packet_iters(ctx: Context, iters: int):
    """Iterations (from the first) whose busy warps walk for their nearest points together."""
    _check(lib.gsicp_ctx_set_packet_iters(ctx.ptr, int(iters)), "gsicp_ctx_set_packet_iters")


def gsicp_ctx_set_cache_step(ctx: Context, meters: float):
    """Motion (m) since a point's last search above which it searches without building a cache."""
    _check(lib.gsicp_ctx_set_cache_step(ctx.ptr, float(meters)), "gsicp_ctx_set_cache_step")


def gsicp_ctx_last_residual(ctx: Context) -> tuple:
    """(sum of squared Euclidean residuals over the inliers, inlier count) of the last registration's
    final linearisation."""
    sq = C.c_double(0.0)
    n = C.c_int64(0)
    _check(lib.gsicp_ctx_last_residual(ctx.ptr, C.byref(sq), C.byref(n)), "gsicp_ctx_last_residual")
    return sq.value, n.value


def gsicp_ctx_phase_times(ctx: Context) -> dict:
    """Device times (ms) of the last timed frame's phases and its iteration count."""
    out = (C.c_double * 6)()
    _check(lib.gsicp_ctx_phase_times(ctx.ptr, out), "gsicp_ctx_phase_times")
    keys = ("depth_to_points", "source_index", "knn_cov", "gauss_newton", "frame", "iters")
    return dict(zip(keys, list(out)))


def gsicp_ctx_reg_stats(ctx: Context, n: int = 64) -> dict:
    """Per-iteration telemetry of the last registration: cache refreshes and tail time (ns)."""
    rf, tl, sv, mn = ((C.c_int32 * n)() for _ in range(4))
    _check(lib.gsicp_ctx_reg_stats(ctx.ptr, n, rf, tl, sv, mn), "gsicp_ctx_reg_stats")
    return dict(refreshes=list(rf), tail_ns=list(tl), solve_ns=list(sv), main_ns=list(mn))


def gsicp_ctx_frame_stats(ctx: Context) -> dict:
    """Telemetry of the last frame's covariances: points the 9 x 9 window left to the 25 x 25 one,
    and those left to the tree search."""
    v = (C.c_int64 * 2)()
    _check(lib.gsicp_ctx_frame_stats(ctx.ptr, v), "gsicp_ctx_frame_stats")
    return dict(wide_window_queries=v[0], tree_queries=v[1])


def gsicp_depth_to_points(ctx: Context, depth: torch.Tensor, intr, stride: int, z_min: float, z_max: float,
                          pts_out: torch.Tensor | None = None, z_out: torch.Tensor | None = None):
    """a1.  Returns ``(pts[:n], z[:n])`` (views of the output buffers)."""
    H, W = depth.shape
    cap = ((W + stride - 1) // stride) * ((H + stride - 1) // stride)
    if pts_out is None:
        pts_out = torch.empty((cap, 3), device=depth.device, dtype=torch.float32)
    if z_out is None:
        z_out = torch.empty((cap,), device=depth.device, dtype=torch.float32)
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    n = C.c_int64(0)
    _check(lib.gsicp_depth_to_points(ctx.ptr, _dev(depth), W, H, fi, stride, z_min, z_max, _dev(pts_out, cols=3),
                                     _dev(z_out), pts_out.shape[0], None, C.byref(n), _stream()),
           "gsicp_depth_to_points")
    return pts_out[:n.value], z_out[:n.value]


def gsicp_depth_to_points_noalloc(depth: torch.Tensor, intr, stride: int, z_min: float, z_max: float,
                                  pts_out: torch.Tensor, z_out: torch.Tensor | None, n_out: torch.Tensor,
                                  total_out: torch.Tensor | None = None):
    """a1 without any allocation by the library (its scratch is a fixed array inside it): for
    callers that cannot allocate device memory when they run this step.  Results go to the
    caller's buffers; n_out / total_out are one-element int32 device tensors.  No synchronisation."""
    H, W = depth.shape
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    _check(lib.gsicp_depth_to_points_noalloc(_dev(depth), W, H, fi, stride, z_min, z_max, _dev(pts_out, cols=3),
                                             _dev(z_out), pts_out.shape[0], _dev(n_out, torch.int32),
                                             _dev(total_out, torch.int32), _stream()),
           "gsicp_depth_to_points_noalloc")


def gsicp_source_covariances(ctx: Context, pts: torch.Tensor, z: torch.Tensor | None, params: CovParams,
                             covs_out: torch.Tensor | None = None, want_knn: bool = False):
    """a2+a3.  Returns covs (n x 6), or (covs, knn n x k int32) with ``want_knn``."""
    n = pts.shape[0]
    if covs_out is None:
        covs_out = torch.empty((n, 6), device=pts.device, dtype=torch.float32)
    knn = torch.empty((n, params.k), device=pts.device, dtype=torch.int32) if want_knn else None
    _check(lib.gsicp_source_covariances(ctx.ptr, _dev(pts, cols=3), _dev(z), n, C.byref(params),
                                        _dev(covs_out, cols=6), _dev(knn, torch.int32), _stream()),
           "gsicp_source_covariances")
    return (covs_out, knn) if want_knn else covs_out


def gsicp_frame_covariances(ctx: Context, depth: torch.Tensor, intr, stride: int, z_min: float, z_max: float,
                            params: CovParams):
    """a1 + a2 + a3 of one depth frame.  Returns ``(pts[:n], z[:n], covs[:n])``."""
    H, W = depth.shape
    cap = ((W + stride - 1) // stride) * ((H + stride - 1) // stride)
    pts = torch.empty((cap, 3), device=depth.device, dtype=torch.float32)
    z = torch.empty((cap,), device=depth.device, dtype=torch.float32)
    covs = torch.empty((cap, 6), device=depth.device, dtype=torch.float32)
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    n = C.c_int64(0)
    _check(lib.gsicp_frame_covariances(ctx.ptr, _dev(depth), W, H, fi, stride, z_min, z_max, C.byref(params),
                                       _dev(pts, cols=3), _dev(z), _dev(covs, cols=6), cap, C.byref(n), _stream()),
           "gsicp_frame_covariances")
    return pts[:n.value], z[:n.value], covs[:n.value]


def gsicp_build_map_index(ctx: Context, means: torch.Tensor, covs: torch.Tensor, bucket: int = 0,
                          cell: float = 0.0) -> MapHandle:
    """a4.  Returns a MapHandle (the library keeps its own copy of the Gaussians)."""
    h = C.c_void_p()
    ip = IndexParams(bucket, cell)
    _check(lib.gsicp_build_map_index(ctx.ptr, _dev(means, cols=3), _dev(covs, cols=6), means.shape[0],
                                     C.byref(ip), _stream(), C.byref(h)), "gsicp_build_map_index")
    return MapHandle(h)


def gsicp_map_append(ctx: Context, map_: MapHandle, means: torch.Tensor, covs: torch.Tensor):
    _check(lib.gsicp_map_append(ctx.ptr, map_.ptr, _dev(means, cols=3), _dev(covs, cols=6), means.shape[0],
                                _stream()), "gsicp_map_append")


def gsicp_map_rebuild(ctx: Context, map_: MapHandle):
    """a4 alone: rebuild the map's index over the Gaussians it holds."""
    _check(lib.gsicp_map_rebuild(ctx.ptr, map_.ptr, _stream()), "gsicp_map_rebuild")


def gsicp_map_inspect(map_: MapHandle) -> dict:
    """The map index's Morton-ordered means (m x 4: x, y, z, original index bits) and node boxes
    (2L x 8: lo.xyz, 0, hi.xyz, 0), with L and the bucket size."""
    L = C.c_int64(0)
    B = C.c_int(0)
    _check(lib.gsicp_map_inspect(map_.ptr, None, None, C.byref(L), C.byref(B), _stream()), "gsicp_map_inspect")
    pts = torch.empty((map_.size, 4), device="cuda", dtype=torch.float32)
    boxes = torch.empty((2 * L.value, 8), device="cuda", dtype=torch.float32)
    _check(lib.gsicp_map_inspect(map_.ptr, _dev(pts), _dev(boxes), None, None, _stream()), "gsicp_map_inspect")
    return dict(pts=pts, boxes=boxes, L=L.value, B=B.value)


def gsicp_map_size(map_: MapHandle) -> int:
    return map_.size


def gsicp_map_destroy(map_: MapHandle):
    map_.close()


def gsicp_transform_gaussians(T, pts: torch.Tensor, covs: torch.Tensor | None = None):
    po = torch.empty_like(pts)
    co = None if covs is None else torch.empty_like(covs)
    _check(lib.gsicp_transform_gaussians(_pose(T), _dev(pts, cols=3), _dev(covs, cols=6), pts.shape[0],
                                         _dev(po, cols=3), _dev(co, cols=6), _stream()), "gsicp_transform_gaussians")
    return po, co


def _reg_outputs():
    return (C.c_double * 16)(), (C.c_double * 36)(), (C.c_double * 6)(), C.c_int(0), C.c_double(0.0), C.c_int64(0)


def gsicp_register(ctx: Context, src: torch.Tensor, covs: torch.Tensor, map_: MapHandle, T0,
                   params: RegParams) -> dict:
    """a5-a7.  Returns dict(T, H, b, iters, cost, inliers, status); raises on errors other
    than a degenerate system (status ERR_DEGENERATE, T = last valid pose)."""
    T, H, b, it, cost, cnt = _reg_outputs()
    st = lib.gsicp_register(ctx.ptr, _dev(src, cols=3), _dev(covs, cols=6), src.shape[0], map_.ptr, _pose(T0),
                            C.byref(params), T, H, b, C.byref(it), C.byref(cost), C.byref(cnt), _stream())
    _check(st, "gsicp_register", allow=(ERR_DEGENERATE,))
    return dict(T=np.array(T).reshape(4, 4), H=np.array(H).reshape(6, 6), b=np.array(b), iters=it.value,
                cost=cost.value, inliers=cnt.value, status=st)


def gsicp_shard_begin(ctx: Context, src: torch.Tensor, covs: torch.Tensor, map_: MapHandle, T0, params: RegParams):
    """Set up this context's registration of its share of a split registration's source points."""
    _check(lib.gsicp_shard_begin(ctx.ptr, _dev(src, cols=3), _dev(covs, cols=6), src.shape[0], map_.ptr, _pose(T0),
                                 C.byref(params), _stream()), "gsicp_shard_begin")


def gsicp_shard_linearise(ctx: Context, partial_out: torch.Tensor):
    """Linearise the share at the current pose: its SHARD_SUMS float64 sums go to partial_out (device,
    stream-ordered, no synchronisation)."""
    if partial_out.numel() != SHARD_SUMS:
        raise ValueError(f"partial_out must hold {SHARD_SUMS} values")
    _check(lib.gsicp_shard_linearise(ctx.ptr, _dev(partial_out, torch.float64), _stream()), "gsicp_shard_linearise")


def gsicp_shard_update(ctx: Context, sums: torch.Tensor) -> dict:
    """Solve and update from every share's sums (sums: nparts x SHARD_SUMS float64 device rows, summed
    in row order).  Returns dict(status (SHARD_*), T, H, iters, cost, inliers); synchronises."""
    if sums.dim() != 2 or sums.shape[1] != SHARD_SUMS:
        raise ValueError(f"sums must be (nparts, {SHARD_SUMS})")
    T, H, b, it, cost, cnt = _reg_outputs()
    status = C.c_int(-1)
    st = lib.gsicp_shard_update(ctx.ptr, _dev(sums, torch.float64), sums.shape[0], C.byref(status), T, H,
                                C.byref(it), C.byref(cost), C.byref(cnt), _stream())
    _check(st, "gsicp_shard_update", allow=(ERR_DEGENERATE,))
    return dict(status=status.value, T=np.array(T).reshape(4, 4), H=np.array(H).reshape(6, 6), iters=it.value,
                cost=cost.value, inliers=cnt.value)


def gsicp_register_batch(ctx: Context, srcs: list, covs: list, maps: list, T0s, params: RegParams) -> dict:
    """Batched a5-a7: pair b registers srcs[b] (n_b x 3) with covs[b] (n_b x 6) against maps[b]
    from T0s[b].  Returns dict(T (B,4,4), iters, cost, inliers, status) as numpy arrays."""
    B = len(srcs)
    assert len(covs) == B and len(maps) == B
    T0s = np.ascontiguousarray(np.asarray(T0s, dtype=np.float64).reshape(B, 16))
    P = (C.c_void_p * max(B, 1))(*[_dev(t, cols=3).value if t.shape[0] else None for t in srcs])
    Q = (C.c_void_p * max(B, 1))(*[_dev(t, cols=6).value if t.shape[0] else None for t in covs])
    nn = (C.c_int64 * max(B, 1))(*[t.shape[0] for t in srcs])
    M = (C.c_void_p * max(B, 1))(*[m.ptr for m in maps])
    T = np.zeros((max(B, 1), 16))
    it = (C.c_int * max(B, 1))()
    cost = np.zeros(max(B, 1))
    inl = (C.c_int64 * max(B, 1))()
    stt = (C.c_int * max(B, 1))()
    dp = C.POINTER(C.c_double)
    _check(lib.gsicp_register_batch(ctx.ptr, B, P, Q, nn, M, T0s.ctypes.data_as(dp), C.byref(params),
                                    T.ctypes.data_as(dp), it, cost.ctypes.data_as(dp), inl, stt, _stream()),
           "gsicp_register_batch")
    return dict(T=T[:B].reshape(B, 4, 4), iters=np.array(it[:B]), cost=cost[:B], inliers=np.array(inl[:B]),
                status=np.array(stt[:B]))


def gsicp_selftest_batch_timeout(ctx: Context) -> int:
    """Status of the batch queue's bounded-wait self-test (ERR_TIMEOUT when the bound works)."""
    return lib.gsicp_selftest_batch_timeout(ctx.ptr, _stream())


class Tracker:
    """The tracking loop with the paper's keyframe policy (gsicp_tracker_*)."""

    def __init__(self, ctx: Context, stride: int, z_min: float, z_max: float, cov: CovParams, reg: RegParams,
                 kf: KeyframeParams | None = None):
        self.ctx = ctx  # kept alive: the tracker uses it
        self.ptr = C.c_void_p()
        self.kf = kf if kf is not None else KeyframeParams()
        _check(lib.gsicp_tracker_create(ctx.ptr, stride, z_min, z_max, C.byref(cov), C.byref(reg), C.byref(self.kf),
                                        C.byref(self.ptr)), "gsicp_tracker_create")

    def frame(self, depth: torch.Tensor, intr, T_start=None):
        """Tracks one depth frame; returns (T 4x4, info dict)."""
        H, W = depth.shape
        fi = (C.c_float * 4)(*[float(v) for v in intr])
        T = (C.c_double * 16)()
        info = FrameInfo()
        ts = _pose(T_start) if T_start is not None else None
        st = lib.gsicp_tracker_frame(self.ptr, _dev(depth), W, H, fi, ts, T, C.byref(info), _stream())
        _check(st, "gsicp_tracker_frame", allow=(ERR_DEGENERATE,))
        d = {name: getattr(info, name) for name, _ in FrameInfo._fields_}
        return np.array(T).reshape(4, 4), d

    def set_surrogate(self, sg, fallback_ratio: float = 1.1, calib_every: int = 30, keyframe_knn: bool = True):
        """Track with the surrogate's covariances (None: k-NN only), falling back to k-NN per frame
        when the residual (RMS correspondence distance) exceeds fallback_ratio times the last k-NN
        frame's; keyframe_knn: the maps receive k-NN covariances only."""
        self.sg = sg  # kept alive: the tracker uses it
        _check(lib.gsicp_tracker_set_surrogate(self.ptr, sg.ptr if sg is not None else None, float(fallback_ratio),
                                               int(calib_every), int(bool(keyframe_knn))),
               "gsicp_tracker_set_surrogate")

    def map_sizes(self) -> tuple:
        """(tracking map size, mapping map size)."""
        a, b = C.c_void_p(), C.c_void_p()
        _check(lib.gsicp_tracker_maps(self.ptr, C.byref(a), C.byref(b)), "gsicp_tracker_maps")
        return (lib.gsicp_map_size(a) if a.value else 0), (lib.gsicp_map_size(b) if b.value else 0)

    def close(self):
        if self.ptr:
            lib.gsicp_tracker_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gsicp_linearise(ctx: Context, src: torch.Tensor, covs: torch.Tensor, map_: MapHandle, T,
                    max_corr_dist: float, want_corr: bool = True) -> dict:
    _, H, b, _, cost, cnt = _reg_outputs()
    corr = torch.empty((src.shape[0],), device=src.device, dtype=torch.int32) if want_corr else None
    _check(lib.gsicp_linearise(ctx.ptr, _dev(src, cols=3), _dev(covs, cols=6), src.shape[0], map_.ptr, _pose(T),
                               max_corr_dist, H, b, C.byref(cost), C.byref(cnt), _dev(corr, torch.int32), _stream()),
           "gsicp_linearise")
    return dict(H=np.array(H).reshape(6, 6), b=np.array(b), cost=cost.value, inliers=cnt.value, corr=corr)


def gsicp_map_nearest(ctx: Context, map_: MapHandle, queries: torch.Tensor, max_dist: float):
    q = queries.shape[0]
    idx = torch.empty((q,), device=queries.device, dtype=torch.int32)
    d2 = torch.empty((q,), device=queries.device, dtype=torch.float32)
    _check(lib.gsicp_map_nearest(ctx.ptr, map_.ptr, _dev(queries, cols=3), q, max_dist, _dev(idx, torch.int32),
                                 _dev(d2), _stream()), "gsicp_map_nearest")
    return idx, d2


def _frame(fn, ctx, depth_ptr, W, H, intr, stride, z_min, z_max, cov_params, map_, T0, reg_params):
    T, Hm, _, it, cost, cnt = _reg_outputs()
    npts = C.c_int64(0)
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    st = fn(ctx.ptr, depth_ptr, W, H, fi, stride, z_min, z_max, C.byref(cov_params), map_.ptr, _pose(T0),
            C.byref(reg_params), T, Hm, C.byref(it), C.byref(cost), C.byref(cnt), C.byref(npts), _stream())
    _check(st, fn.__name__, allow=(ERR_DEGENERATE,))
    return dict(T=np.array(T).reshape(4, 4), H=np.array(Hm).reshape(6, 6), iters=it.value, cost=cost.value,
                inliers=cnt.value, n_points=npts.value, status=st)


def gsicp_track_frame(ctx: Context, depth: torch.Tensor, intr, stride: int, z_min: float, z_max: float,
                      cov_params: CovParams, map_: MapHandle, T0, reg_params: RegParams) -> dict:
    """One whole frame (a1 -> a2+a3 -> a5-a7) from a device depth image."""
    H, W = depth.shape
    return _frame(lib.gsicp_track_frame, ctx, _dev(depth), W, H, intr, stride, z_min, z_max, cov_params, map_, T0,
                  reg_params)


def gsicp_track_frame_surrogate(ctx: Context, sg: "Surrogate", depth: torch.Tensor, intr, stride: int, z_min: float,
                                z_max: float, cov_params: CovParams, map_: MapHandle, T0, reg_params: RegParams) -> dict:
    """gsicp_track_frame with the surrogate's covariances (cov_params gives eps and p)."""
    H, W = depth.shape
    fn = lib.gsicp_track_frame_surrogate
    T, Hm, _, it, cost, cnt = _reg_outputs()
    npts = C.c_int64(0)
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    st = fn(ctx.ptr, sg.ptr, _dev(depth), W, H, fi, stride, z_min, z_max, C.byref(cov_params), map_.ptr, _pose(T0),
            C.byref(reg_params), T, Hm, C.byref(it), C.byref(cost), C.byref(cnt), C.byref(npts), _stream())
    _check(st, "gsicp_track_frame_surrogate", allow=(ERR_DEGENERATE,))
    return dict(T=np.array(T).reshape(4, 4), H=np.array(Hm).reshape(6, 6), iters=it.value, cost=cost.value,
                inliers=cnt.value, n_points=npts.value, status=st)


class Surrogate:
    """Owns a ``gsicp_surrogate``: the covariance network's weights (float master copy, bfloat16
    kernel copies) and its Adam state on the current device."""

    def __init__(self, weights):
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        if w.size != SURROGATE_WEIGHTS:
            raise ValueError(f"expected {SURROGATE_WEIGHTS} weights")
        h = C.c_void_p()
        _check(lib.gsicp_surrogate_create(w.ctypes.data_as(_fp), C.byref(h)), "gsicp_surrogate_create")
        self.ptr = h

    def weights(self) -> np.ndarray:
        out = np.empty(SURROGATE_WEIGHTS, np.float32)
        _check(lib.gsicp_surrogate_get_weights(self.ptr, out.ctypes.data_as(_fp)), "gsicp_surrogate_get_weights")
        return out

    def set_weights(self, weights):
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        if w.size != SURROGATE_WEIGHTS:
            raise ValueError(f"expected {SURROGATE_WEIGHTS} weights")
        _check(lib.gsicp_surrogate_set_weights(self.ptr, w.ctypes.data_as(_fp)), "gsicp_surrogate_set_weights")

    def set_timing(self, enable: bool):
        _check(lib.gsicp_surrogate_set_timing(self.ptr, int(bool(enable))), "gsicp_surrogate_set_timing")

    def layer_times(self) -> tuple:
        """Device ms of the last forward: (grid + layer 1, layer 2, layer 3 + covariances)."""
        out = (C.c_double * 3)()
        _check(lib.gsicp_surrogate_layer_times(self.ptr, out), "gsicp_surrogate_layer_times")
        return tuple(out)

    def close(self):
        if self.ptr:
            lib.gsicp_surrogate_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gsicp_surrogate_covariances(ctx: Context, sg: Surrogate, depth: torch.Tensor, intr, stride: int, z_min: float,
                                z_max: float, params: CovParams, want_v: bool = False):
    """a1 + surrogate covariances of one device depth frame.  Returns (pts[:n], z[:n], covs[:n])
    and, with want_v, the raw network output per sample (h, w, 3)."""
    H, W = depth.shape
    hs, ws = (H + stride - 1) // stride, (W + stride - 1) // stride
    cap = hs * ws
    pts = torch.empty((cap, 3), device=depth.device, dtype=torch.float32)
    z = torch.empty((cap,), device=depth.device, dtype=torch.float32)
    covs = torch.empty((cap, 6), device=depth.device, dtype=torch.float32)
    v = torch.empty((hs, ws, 3), device=depth.device, dtype=torch.float32) if want_v else None
    fi = (C.c_float * 4)(*[float(a) for a in intr])
    n = C.c_int64(0)
    _check(lib.gsicp_surrogate_covariances(ctx.ptr, sg.ptr, _dev(depth), W, H, fi, stride, z_min, z_max,
                                           C.byref(params), _dev(pts, cols=3), _dev(z), _dev(covs, cols=6),
                                           _dev(v) if v is not None else None, cap, C.byref(n), _stream()),
           "gsicp_surrogate_covariances")
    m = n.value
    out = (pts[:m], z[:m], covs[:m])
    return out + (v,) if want_v else out


def gsicp_surrogate_train_step(ctx: Context, sg: Surrogate, depth: torch.Tensor, intr, stride: int, z_min: float,
                               z_max: float, params: CovParams, target_covs: torch.Tensor | None = None,
                               lr: float = 1e-3, apply: bool = True, want_grad: bool = False) -> dict:
    """One training step (targets: target_covs in a1 order, or the frame's own k-NN covariances).
    Returns dict(loss, count[, grad])."""
    H, W = depth.shape
    fi = (C.c_float * 4)(*[float(a) for a in intr])
    loss = C.c_double(0.0)
    cnt = C.c_int64(0)
    grad = np.empty(SURROGATE_WEIGHTS, np.float32) if want_grad else None
    _check(lib.gsicp_surrogate_train_step(ctx.ptr, sg.ptr, _dev(depth), W, H, fi, stride, z_min, z_max,
                                          C.byref(params), _dev(target_covs, cols=6) if target_covs is not None else None,
                                          float(lr), int(bool(apply)), C.byref(loss), C.byref(cnt),
                                          grad.ctypes.data_as(_fp) if grad is not None else None, _stream()),
           "gsicp_surrogate_train_step")
    out = dict(loss=loss.value, count=cnt.value)
    if want_grad:
        out["grad"] = grad
    return out


def gsicp_track_frame_host(ctx: Context, depth_host, intr, stride: int, z_min: float, z_max: float,
                           cov_params: CovParams, map_: MapHandle, T0, reg_params: RegParams) -> dict:
    """One whole frame from a host depth image (a CPU torch tensor, pinned for async copies,
    or a numpy array); the host-to-device copy happens inside the call."""
    if isinstance(depth_host, torch.Tensor):
        if depth_host.is_cuda or depth_host.dtype != torch.float32 or not depth_host.is_contiguous():
            raise TypeError("expected a contiguous CPU float32 tensor")
        H, W = depth_host.shape
        ptr = C.c_void_p(depth_host.data_ptr())
    else:
        arr = np.ascontiguousarray(depth_host, dtype=np.float32)
        H, W = arr.shape
        ptr = C.c_void_p(arr.ctypes.data)
    return _frame(lib.gsicp_track_frame_host, ctx, ptr, W, H, intr, stride, z_min, z_max, cov_params, map_, T0,
                  reg_params)
