"""FP64 CPU oracle for the G-ICP tracking path (ctypes shim over ``liboracle.so``).

TEST INFRASTRUCTURE ONLY.  This is the plain reference the CUDA library is
checked against; only the tests, the smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA library and never
consumes anything the CUDA library produced.

Every function takes numpy arrays; float32 data is widened exactly to
float64 before the call, so the oracle sees the very values the GPU reads.
Citations (sections / equations of the paper, arXiv 2403.12550) sit in
``gsicp_oracle.c`` beside each routine.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os

import numpy as np

from .build import build, lib_path

PLANE, ELLIPSE, NONE = 0, 1, 2
OK, ERR_ARG, ERR_DEGENERATE = 0, 1, 4
FLAG_FEW_POINTS, FLAG_RANK_DEFICIENT, FLAG_FLOORED = 1, 2, 4

_lib = None

_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I32 = C.POINTER(C.c_int32)


class RegParams(C.Structure):
    _fields_ = [("max_corr_dist", C.c_double), ("max_iters", C.c_int), ("tol_rot", C.c_double),
                ("tol_trans", C.c_double), ("min_inliers", C.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        build()
    _lib = _bind(C.CDLL(path))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Route every call of this module to another build of the C oracle while the block runs: the
    tests that plant a mistake in a copy of ``gsicp_oracle.c`` use it to show that a pin catches it."""
    global _lib
    saved = _lib
    _lib = _bind(C.CDLL(os.path.abspath(path)))
    try:
        yield
    finally:
        _lib = saved


def _bind(lib):
    lib.orc_depth_to_points.restype = C.c_long
    lib.orc_depth_to_points.argtypes = [_F, C.c_int, C.c_int, _D, C.c_int, C.c_double, C.c_double, _D, _D, C.c_long]
    lib.orc_kdtree_build.restype = C.c_void_p
    lib.orc_kdtree_build.argtypes = [_D, C.c_long]
    lib.orc_kdtree_free.argtypes = [C.c_void_p]
    lib.orc_knn.argtypes = [C.c_void_p, _D, C.c_long, C.c_int, _I32, _D]
    lib.orc_knn_brute.argtypes = [_D, C.c_long, _D, C.c_long, C.c_int, _I32, _D]
    lib.orc_nn.argtypes = [C.c_void_p, _D, C.c_long, C.c_double, _I32, _D]
    lib.orc_nn_brute.argtypes = [_D, C.c_long, _D, C.c_long, C.c_double, _I32, _D]
    lib.orc_eigh3.argtypes = [_D, _D, _D]
    lib.orc_source_covariances.argtypes = [_D, _D, C.c_long, C.c_int, C.c_double, C.c_int, C.c_double,
                                           _D, _D, _D, _I32]
    lib.orc_regularise.argtypes = [_D, C.c_int, C.c_double, _D, _D]
    lib.orc_transform_gaussians.argtypes = [_D, _D, _D, C.c_long, _D, _D]
    lib.orc_se3_exp.argtypes = [_D, _D]
    lib.orc_linearise.argtypes = [_D, _D, C.c_long, C.c_void_p, _D, _D, _D, C.c_double, _D, _D, _D,
                                  C.POINTER(C.c_long), _I32]
    lib.orc_residual_jacobian.argtypes = [_D, _D, _D, _D, _D]
    lib.orc_register.argtypes = [_D, _D, C.c_long, C.c_void_p, _D, _D, _D, C.POINTER(RegParams), _D, _D, _D,
                                 C.POINTER(C.c_int), _D, C.POINTER(C.c_long)]
    lib.orc_gn_update.argtypes = [_D, _D, _D, C.POINTER(RegParams)]
    lib.orc_register_fixed.argtypes = [_D, _D, C.c_long, _D, _D, _D, C.POINTER(RegParams), _D,
                                       C.POINTER(C.c_int), _D]
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_threads.restype = C.c_int
    return lib


def set_threads(n: int) -> None:
    """OpenMP threads for the oracle's per-point loops from now on (n <= 0: all processors)."""
    _load().orc_set_threads(int(n))


def threads() -> int:
    return int(_load().orc_threads())


def _d(a, shape_last=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape_last is not None:
        a = a.reshape(-1, shape_last)
    return a


def _p(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.float32:
        return a.ctypes.data_as(_F)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I32)
    raise TypeError(a.dtype)


# ----------------------------------------------------------------------------- API

def depth_to_points(depth, intr, stride: int, z_min: float, z_max: float):
    """Back-project every ``stride``-th pixel of a float32 depth image
    (row-major scan order, invalid pixels dropped).  Returns (pts n x 3, z n)."""
    lib = _load()
    depth = np.ascontiguousarray(depth, dtype=np.float32)
    H, W = depth.shape
    cap = ((H + stride - 1) // stride) * ((W + stride - 1) // stride)
    pts = np.empty((max(cap, 1), 3))
    z = np.empty(max(cap, 1))
    # the bounds are float32 values in the C ABI; widen the same values here
    n = lib.orc_depth_to_points(_p(depth), W, H, _p(_d(np.float32(intr).astype(np.float64))), stride,
                                float(np.float32(z_min)), float(np.float32(z_max)), _p(pts), _p(z), cap)
    if n < 0:
        raise ValueError("bad arguments")
    return pts[:n], z[:n]


class KDTree:
    """Exact k-d tree over an n x 3 array (kept alive by this object)."""

    def __init__(self, pts):
        self._lib = _load()
        self.pts = _d(pts, 3)
        self.n = len(self.pts)
        self.handle = self._lib.orc_kdtree_build(_p(self.pts), self.n)

    def __del__(self):
        if getattr(self, "handle", None):
            self._lib.orc_kdtree_free(self.handle)
            self.handle = None

    def knn(self, queries, k: int):
        q = _d(queries, 3)
        idx = np.empty((len(q), k), dtype=np.int32)
        d2 = np.empty((len(q), k))
        self._lib.orc_knn(self.handle, _p(q), len(q), k, _p(idx), _p(d2))
        return idx, d2

    def nn(self, queries, max_dist: float):
        q = _d(queries, 3)
        idx = np.empty(len(q), dtype=np.int32)
        d2 = np.empty(len(q))
        self._lib.orc_nn(self.handle, _p(q), len(q), float(max_dist) ** 2, _p(idx), _p(d2))
        return idx, d2


def knn_brute(pts, queries, k: int):
    lib = _load()
    p, q = _d(pts, 3), _d(queries, 3)
    idx = np.empty((len(q), k), dtype=np.int32)
    d2 = np.empty((len(q), k))
    lib.orc_knn_brute(_p(p), len(p), _p(q), len(q), k, _p(idx), _p(d2))
    return idx, d2


def nn_brute(pts, queries, max_dist: float):
    lib = _load()
    p, q = _d(pts, 3), _d(queries, 3)
    idx = np.empty(len(q), dtype=np.int32)
    d2 = np.empty(len(q))
    lib.orc_nn_brute(_p(p), len(p), _p(q), len(q), float(max_dist) ** 2, _p(idx), _p(d2))
    return idx, d2


def eigh3(A6):
    lib = _load()
    A = _d(A6).reshape(6)
    w = np.empty(3)
    V = np.empty((3, 3))
    lib.orc_eigh3(_p(A), _p(w), _p(V))
    return w, V


def regularise(C6, reg_mode: int, eps: float):
    lib = _load()
    C6 = _d(C6).reshape(6)
    out = np.empty(6)
    gap = np.empty(1)
    flags = lib.orc_regularise(_p(C6), reg_mode, eps, _p(out), _p(gap))
    return out, float(gap[0]), flags


def source_covariances(pts, z=None, k: int = 20, eps: float = 1e-3, reg_mode: int = PLANE, p: float = 0.0):
    """Per-point regularised, scale-aligned covariances.  Returns a dict with
    ``covs`` (n x 6), ``raw`` (n x 6 unregularised), ``gap`` ((l1-l0)/l1) and ``flags``."""
    lib = _load()
    P = _d(pts, 3)
    n = len(P)
    Z = None if z is None else _d(z).reshape(-1)
    covs = np.empty((n, 6))
    raw = np.empty((n, 6))
    gap = np.empty(n)
    flags = np.empty(n, dtype=np.int32)
    st = lib.orc_source_covariances(_p(P), _p(Z), n, k, float(np.float32(eps)), reg_mode,
                                    float(np.float32(p)), _p(covs), _p(raw), _p(gap), _p(flags))
    if st != OK:
        raise ValueError(f"orc_source_covariances status {st}")
    return dict(covs=covs, raw=raw, gap=gap, flags=flags)


def transform_gaussians(T, pts, covs=None):
    lib = _load()
    P = _d(pts, 3)
    Cv = None if covs is None else _d(covs, 6)
    po = np.empty_like(P)
    co = None if Cv is None else np.empty_like(Cv)
    lib.orc_transform_gaussians(_p(_d(T).reshape(16)), _p(P), _p(Cv), len(P), _p(po), _p(co))
    return po, co


def se3_exp(xi):
    lib = _load()
    T = np.empty((4, 4))
    lib.orc_se3_exp(_p(_d(xi).reshape(6)), _p(T))
    return T


def residual_jacobian(T, x, mu):
    lib = _load()
    d = np.empty(3)
    J = np.empty((3, 6))
    lib.orc_residual_jacobian(_p(_d(T).reshape(16)), _p(_d(x).reshape(3)), _p(_d(mu).reshape(3)), _p(d), _p(J))
    return d, J


class Map:
    """Target Gaussians with their k-d tree."""

    def __init__(self, means, covs):
        self.means = _d(means, 3)
        self.covs = _d(covs, 6)
        self.tree = KDTree(self.means)


def linearise(src, covs_s, map_: Map, T, max_dist: float):
    lib = _load()
    S, Cs = _d(src, 3), _d(covs_s, 6)
    H = np.empty((6, 6))
    b = np.empty(6)
    cost = np.empty(1)
    cnt = C.c_long(0)
    corr = np.empty(len(S), dtype=np.int32)
    lib.orc_linearise(_p(S), _p(Cs), len(S), map_.tree.handle, _p(map_.means), _p(map_.covs),
                      _p(_d(T).reshape(16)), float(np.float32(max_dist)), _p(H), _p(b), _p(cost),
                      C.byref(cnt), _p(corr))
    return dict(H=H, b=b, cost=float(cost[0]), inliers=int(cnt.value), corr=corr)


def register(src, covs_s, map_: Map, T0, max_corr_dist: float = 0.1, max_iters: int = 30,
             tol_rot: float = 1e-6, tol_trans: float = 1e-6, min_inliers: int = 6):
    """Gauss-Newton G-ICP registration.  Returns a dict with T, H, b, iters,
    cost, inliers, status."""
    lib = _load()
    S, Cs = _d(src, 3), _d(covs_s, 6)
    prm = RegParams(float(np.float32(max_corr_dist)), max_iters, tol_rot, tol_trans, min_inliers)
    T = np.empty((4, 4))
    H = np.empty((6, 6))
    b = np.empty(6)
    cost = np.empty(1)
    it = C.c_int(0)
    cnt = C.c_long(0)
    st = lib.orc_register(_p(S), _p(Cs), len(S), map_.tree.handle, _p(map_.means), _p(map_.covs),
                          _p(_d(T0).reshape(16)), C.byref(prm), _p(T), _p(H), _p(b), C.byref(it),
                          _p(cost), C.byref(cnt))
    return dict(T=T, H=H, b=b, iters=int(it.value), cost=float(cost[0]), inliers=int(cnt.value), status=int(st))


def gn_update(H, b, T, tol_rot: float = 1e-6, tol_trans: float = 1e-6):
    """One Gauss-Newton update of the registration loop (Sec. 3): delta = -H^-1 b (Cholesky),
    T <- exp(delta^) T.  Returns (T_new, r): r = 1 converged (|delta_omega| < tol_rot and
    |delta_v| < tol_trans), 0 not yet, -1 H not positive definite (T unchanged)."""
    lib = _load()
    prm = RegParams(0.0, 1, tol_rot, tol_trans, 0)
    Tn = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16)).copy()
    r = lib.orc_gn_update(_p(_d(np.asarray(H).reshape(36))), _p(_d(np.asarray(b).reshape(6))), _p(Tn), C.byref(prm))
    return Tn.reshape(4, 4), int(r)


def register_fixed(src, covs_s, tgt, covs_t, T0, max_iters: int = 50, tol_rot: float = 1e-12,
                   tol_trans: float = 1e-12):
    """Gauss-Newton with correspondences fixed by index (source i <-> target i)."""
    lib = _load()
    S, Cs, Tg, Ct = _d(src, 3), _d(covs_s, 6), _d(tgt, 3), _d(covs_t, 6)
    prm = RegParams(0.0, max_iters, tol_rot, tol_trans, 0)
    T = np.empty((4, 4))
    cost = np.empty(1)
    it = C.c_int(0)
    st = lib.orc_register_fixed(_p(S), _p(Cs), len(S), _p(Tg), _p(Ct), _p(_d(T0).reshape(16)), C.byref(prm),
                                _p(T), C.byref(it), _p(cost))
    return dict(T=T, iters=int(it.value), cost=float(cost[0]), status=int(st))
