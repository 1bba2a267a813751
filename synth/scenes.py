"""Seeded synthetic inputs shaped like the paper's RGB-D tracking workloads.

This module only *makes inputs*: analytic rooms (walls, yawed boxes, spheres),
area-uniform surface samples, pinhole ray-cast depth images, camera poses and
noise.  It holds none of the tracking method's arithmetic (no neighbour
search, no covariance, no registration), so that both the CUDA path and the
CPU oracle can be fed from it without sharing any of the computation under
test.

The paper evaluates on Replica (1200x680 synthetic renders) and TUM RGB-D
(640x480 sensor captures), Sec. 4.1.  Neither dataset is used; these scenes
stand in for them with the same image sizes and intrinsics shapes.

Conventions
-----------
* World frame: z up, metres.
* Camera frame: x right, y down, z forward (depth = camera-frame z).
* A pose ``T_wc`` (4x4 float64, row-major) maps camera coordinates into world
  coordinates: ``p_w = R_wc p_c + t_wc``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "make_room", "sample_surface", "raycast_depth", "add_depth_noise",
    "look_pose", "circle_poses", "random_offset", "rot_axis_angle", "inv_pose", "make_pose",
    "transform_points", "Intrinsics", "REPLICA_INTR", "TUM_INTR",
    "pair_config1", "frame_config2", "spline_trajectory", "sequence_config3", "const_velocity",
    "batch_config4", "HALF_TUM_INTR", "surrogate_train_config5", "sequence_config5", "orbit_trajectory",
    "render_sequence_frames",
]


# --------------------------------------------------------------------------- poses

def rot_axis_angle(axis, angle: float) -> np.ndarray:
    """Rotation matrix for ``angle`` radians about the unit ``axis`` (Rodrigues)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]], dtype=np.float64)
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def make_pose(R: np.ndarray, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = np.asarray(t, dtype=np.float64)
    return T


def inv_pose(T: np.ndarray) -> np.ndarray:
    R = T[:3, :3]
    t = T[:3, 3]
    return make_pose(R.T, -R.T @ t)


def transform_points(T: np.ndarray, pts: np.ndarray) -> np.ndarray:
    return pts @ T[:3, :3].T + T[:3, 3]


def _unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def random_offset(rng: np.random.Generator, angle_deg: float, trans_m: float) -> np.ndarray:
    """A rigid offset: ``angle_deg`` about a uniform random axis, ``trans_m``
    along a uniform random direction."""
    R = rot_axis_angle(_unit(rng), np.deg2rad(angle_deg))
    return make_pose(R, trans_m * _unit(rng))


def look_pose(position, yaw: float, pitch: float = 0.0) -> np.ndarray:
    """Camera-to-world pose at ``position`` looking along heading ``yaw``
    (radians about world z) tilted down by ``pitch`` radians."""
    cp, sp = np.cos(pitch), np.sin(pitch)
    f = np.array([cp * np.cos(yaw), cp * np.sin(yaw), -sp])
    r = np.array([np.sin(yaw), -np.cos(yaw), 0.0])
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=1)  # columns: camera x, y, z in world
    return make_pose(R, position)


# --------------------------------------------------------------------------- scene

@dataclass
class Scene:
    room_lo: np.ndarray
    room_hi: np.ndarray
    box_center: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    box_half: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    box_yaw: np.ndarray = field(default_factory=lambda: np.zeros((0,)))
    sph_center: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    sph_radius: np.ndarray = field(default_factory=lambda: np.zeros((0,)))

    @property
    def centre(self) -> np.ndarray:
        return 0.5 * (self.room_lo + self.room_hi)


def make_room(seed: int, size=(4.0, 3.0, 2.5), n_boxes: int = 8, n_spheres: int = 4,
              box_side=(0.2, 1.0), sph_radius=(0.1, 0.4), keep_clear: float = 0.5) -> Scene:
    """A closed room of inward-facing walls with ``n_boxes`` yawed boxes
    standing on the floor and ``n_spheres`` spheres.

    Boxes are at most 1 m tall; spheres are kept out of a vertical cylinder of
    radius ``keep_clear`` + 0.3 m around the room centre between heights 0.9
    and 1.9 m, where cameras are placed."""
    rng = np.random.default_rng(seed)
    lo = np.zeros(3)
    hi = np.asarray(size, dtype=np.float64)
    c = 0.5 * (lo + hi)
    bc, bh, by = [], [], []
    for _ in range(n_boxes):
        side = rng.uniform(box_side[0], box_side[1], size=3)
        half = 0.5 * side
        rad = np.hypot(half[0], half[1])
        for _try in range(100):
            xy = rng.uniform(lo[:2] + rad + 0.05, hi[:2] - rad - 0.05)
            if np.hypot(*(xy - c[:2])) > keep_clear + rad + 0.1:
                break
        bc.append([xy[0], xy[1], half[2]])
        bh.append(half)
        by.append(rng.uniform(0, np.pi))
    sc, sr = [], []
    for _ in range(n_spheres):
        r = rng.uniform(sph_radius[0], sph_radius[1])
        for _try in range(1000):
            p = rng.uniform(lo + r + 0.05, hi - r - 0.05)
            horiz = np.hypot(*(p[:2] - c[:2]))
            if horiz > keep_clear + r + 0.3 or p[2] + r < 0.9 or p[2] - r > 1.9:
                break
        sc.append(p)
        sr.append(r)
    return Scene(lo, hi, np.array(bc).reshape(-1, 3), np.array(bh).reshape(-1, 3),
                 np.array(by), np.array(sc).reshape(-1, 3), np.array(sr))


def _rz(yaw: float) -> np.ndarray:
    c, s = np.cos(yaw), np.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


# --------------------------------------------------------------------------- surface sampling

def sample_surface(scene: Scene, n: int, rng: np.random.Generator, noise_sigma: float = 0.0,
                   include_box_bottoms: bool = False) -> np.ndarray:
    """``n`` points sampled uniformly by area over every surface of ``scene``
    (walls, box faces, spheres), including surfaces hidden from any given
    viewpoint.  With ``noise_sigma`` > 0 each point is displaced by
    N(0, sigma) along the ray from the room centre."""
    patches = []  # (area, sampler)
    lo, hi = scene.room_lo, scene.room_hi
    ext = hi - lo
    # 6 walls: axis a fixed at lo[a] or hi[a]
    for a in range(3):
        b, c2 = [i for i in range(3) if i != a]
        area = ext[b] * ext[c2]
        for val in (lo[a], hi[a]):
            def samp(k, a=a, b=b, c2=c2, val=val):
                p = np.empty((k, 3))
                p[:, a] = val
                p[:, b] = rng.uniform(lo[b], hi[b], k)
                p[:, c2] = rng.uniform(lo[c2], hi[c2], k)
                return p
            patches.append((area, samp))
    for bi in range(len(scene.box_yaw)):
        cen, half, R = scene.box_center[bi], scene.box_half[bi], _rz(scene.box_yaw[bi])
        for a in range(3):
            b, c2 = [i for i in range(3) if i != a]
            area = 4.0 * half[b] * half[c2]
            for sgn in (-1.0, 1.0):
                if a == 2 and sgn < 0 and not include_box_bottoms:
                    continue
                def samp(k, a=a, b=b, c2=c2, sgn=sgn, cen=cen, half=half, R=R):
                    q = np.empty((k, 3))
                    q[:, a] = sgn * half[a]
                    q[:, b] = rng.uniform(-half[b], half[b], k)
                    q[:, c2] = rng.uniform(-half[c2], half[c2], k)
                    return q @ R.T + cen
                patches.append((area, samp))
    for si in range(len(scene.sph_radius)):
        cen, r = scene.sph_center[si], scene.sph_radius[si]
        def samp(k, cen=cen, r=r):
            v = rng.normal(size=(k, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            return cen + r * v
        patches.append((4.0 * np.pi * r * r, samp))
    areas = np.array([p[0] for p in patches])
    counts = rng.multinomial(n, areas / areas.sum())
    pts = np.concatenate([patches[i][1](int(k)) for i, k in enumerate(counts) if k > 0], axis=0)
    pts = pts[rng.permutation(len(pts))]
    if noise_sigma > 0:
        ray = pts - scene.centre
        ray /= np.maximum(np.linalg.norm(ray, axis=1, keepdims=True), 1e-12)
        pts = pts + rng.normal(0.0, noise_sigma, size=(len(pts), 1)) * ray
    return pts


# --------------------------------------------------------------------------- ray casting

@dataclass(frozen=True)
class Intrinsics:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float

    def as_array(self) -> np.ndarray:
        return np.array([self.fx, self.fy, self.cx, self.cy], dtype=np.float32)


REPLICA_INTR = Intrinsics(1200, 680, 600.0, 600.0, 599.5, 339.5)
# Generic VGA intrinsics for the TUM-shaped sequence (the exact TUM calibration is not used).
TUM_INTR = Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5)


def raycast_depth(scene: Scene, T_wc: np.ndarray, intr: Intrinsics) -> np.ndarray:
    """Noise-free depth image (H x W, float32 metres, camera-frame z) of the
    scene seen from ``T_wc`` by an ideal pinhole camera; pixel (u, v) looks
    along ((u - cx)/fx, (v - cy)/fy, 1) in the camera frame."""
    u, v = np.meshgrid(np.arange(intr.W, dtype=np.float64), np.arange(intr.H, dtype=np.float64))
    dc = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, np.ones_like(u)], axis=-1).reshape(-1, 3)
    R, o = T_wc[:3, :3], T_wc[:3, 3]
    d = dc @ R.T  # world direction; the ray parameter equals camera depth
    tbest = np.full(len(d), np.inf)
    # room interior: exit distance through the nearest wall
    with np.errstate(divide="ignore", invalid="ignore"):
        tw = np.where(d > 0, (scene.room_hi - o) / d, np.where(d < 0, (scene.room_lo - o) / d, np.inf))
    tbest = np.minimum(tbest, tw.min(axis=1))
    for bi in range(len(scene.box_yaw)):
        Rb = _rz(scene.box_yaw[bi])
        ob = (o - scene.box_center[bi]) @ Rb
        db = d @ Rb
        h = scene.box_half[bi]
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (-h - ob) / db
            t2 = (h - ob) / db
        tn = np.nanmax(np.minimum(t1, t2), axis=1)
        tf = np.nanmin(np.maximum(t1, t2), axis=1)
        hit = (tn <= tf) & (tn > 1e-9)
        tbest = np.where(hit & (tn < tbest), tn, tbest)
    for si in range(len(scene.sph_radius)):
        oc = o - scene.sph_center[si]
        a = np.einsum("ij,ij->i", d, d)
        b = 2.0 * d @ oc
        c = oc @ oc - scene.sph_radius[si] ** 2
        disc = b * b - 4 * a * c
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t = (-b - sq) / (2 * a)
        hit = ok & (t > 1e-9)
        tbest = np.where(hit & (t < tbest), t, tbest)
    return tbest.reshape(intr.H, intr.W).astype(np.float32)


def add_depth_noise(depth: np.ndarray, rng: np.random.Generator, coeff: float = 1e-3,
                    dropout: float = 0.0) -> np.ndarray:
    """Depth noise N(0, (coeff * z^2)^2) per pixel (coeff in 1/m), plus an
    optional fraction of pixels set to 0 (missing depth)."""
    z = depth.astype(np.float64)
    out = z + rng.normal(size=z.shape) * coeff * z * z
    if dropout > 0:
        out[rng.random(z.shape) < dropout] = 0.0
    return out.astype(np.float32)


def circle_poses(rng: np.random.Generator, scene: Scene, n: int, radius: float = 0.5,
                 height=(1.2, 1.6), pitch_deg=(5.0, 25.0)) -> list:
    """``n`` camera poses on a horizontal circle of ``radius`` around the room
    centre, heights uniform in ``height``, headings spread over 0-360 degrees
    (evenly, with jitter) and a small downward pitch."""
    c = scene.centre
    poses = []
    base = rng.uniform(0, 2 * np.pi)
    for i in range(n):
        phi = base + 2 * np.pi * i / n + rng.uniform(-0.2, 0.2)
        pos = np.array([c[0] + radius * np.cos(phi), c[1] + radius * np.sin(phi), rng.uniform(*height)])
        yaw = base + 2 * np.pi * i / n + rng.uniform(-0.3, 0.3)
        pitch = np.deg2rad(rng.uniform(*pitch_deg))
        poses.append(look_pose(pos, yaw, pitch))
    return poses


# --------------------------------------------------------------------------- configurations

def pair_config1(scene_seed: int, pose_seed: int, n: int = 10_000, noise: float = 2e-3,
                 angle_deg: float = 5.0, trans_m: float = 0.05):
    """Single-registration inputs: a source and an independently resampled
    target cloud of the same room, the source expressed in the frame
    ``T_gt^-1`` (so that ``T_gt`` maps source into target coordinates).

    Returns ``(src float32 n x 3, tgt float32 n x 3, T_gt float64 4 x 4)``."""
    scene = make_room(scene_seed)
    rng = np.random.default_rng(1_000_003 * scene_seed + 7919 * pose_seed + 17)
    src_w = sample_surface(scene, n, rng, noise)
    tgt = sample_surface(scene, n, rng, noise)
    T_gt = random_offset(rng, angle_deg, trans_m)
    src = transform_points(inv_pose(T_gt), src_w)
    return src.astype(np.float32), tgt.astype(np.float32), T_gt


def frame_config2(seed: int, n_views: int = 10, intr: Intrinsics = REPLICA_INTR,
                  offset_deg: float = 2.0, offset_m: float = 0.02, noise_coeff: float = 1e-3):
    """Replica-shaped single-frame inputs: ``n_views`` noisy prior depth images
    with their camera poses (to build a map from), the current noisy depth
    image, its ground-truth pose and an initial guess ``T0 = T_gt @ offset``.

    Returns a dict with keys ``scene, intr, view_depths, view_poses, depth,
    T_gt, T0``."""
    scene = make_room(seed)
    rng = np.random.default_rng(9176 + 31 * seed)
    poses = circle_poses(rng, scene, n_views + 1)
    cur = poses.pop(int(rng.integers(0, n_views + 1)))
    # move the current camera off the prior circle a little
    cur = cur.copy()
    cur[:3, 3] += np.array([rng.uniform(-0.15, 0.15), rng.uniform(-0.15, 0.15), 0.0])
    view_depths = [add_depth_noise(raycast_depth(scene, P, intr), rng, noise_coeff) for P in poses]
    depth = add_depth_noise(raycast_depth(scene, cur, intr), rng, noise_coeff)
    T0 = cur @ random_offset(rng, offset_deg, offset_m)
    return dict(scene=scene, intr=intr, view_depths=view_depths, view_poses=poses, depth=depth,
                T_gt=cur, T0=T0)


def spline_trajectory(seed: int, scene: Scene, n_frames: int = 500, fps: float = 30.0,
                      vmax: float = 1.0, wmax_deg: float = 60.0, n_knots: int = 12,
                      clearance: float = 0.6) -> list:
    """A smooth camera trajectory: positions and headings follow clamped
    natural cubic splines through seeded knots near the room centre, sampled
    at ``fps``; speeds are capped at ``vmax`` m/s and ``wmax_deg`` deg/s by
    slowing the time parameterisation.  The camera keeps ``clearance`` from
    the walls, the ceiling and every sphere, and stays above the boxes (the
    knots are drawn again, from the same seeded stream, until it does)."""
    from scipy.interpolate import CubicSpline

    rng = np.random.default_rng(4242 + seed)
    c = scene.centre
    span = 0.35 * (scene.room_hi - scene.room_lo)
    box_top = float(np.max(2.0 * scene.box_half[:, 2])) if len(scene.box_half) else 0.0
    dt = 1.0 / fps

    def clear(pos) -> bool:
        if np.any(pos - scene.room_lo < clearance) or np.any(scene.room_hi - pos < clearance):
            return False
        if pos[2] < box_top + 0.2:
            return False
        return all(np.linalg.norm(pos - sc) > r + clearance for sc, r in zip(scene.sph_center, scene.sph_radius))

    for _attempt in range(200):
        knots_p = c + rng.uniform(-1, 1, size=(n_knots, 3)) * np.array([span[0], span[1], 0.0])
        knots_p[:, 2] = rng.uniform(1.2, 1.8, n_knots)
        knots_yaw = np.cumsum(rng.uniform(-1.2, 1.2, n_knots))
        knots_pitch = np.deg2rad(rng.uniform(5, 25, n_knots))
        s = np.arange(n_knots, dtype=np.float64)
        sp_p = CubicSpline(s, knots_p, bc_type="clamped")
        sp_y = CubicSpline(s, knots_yaw, bc_type="clamped")
        sp_pt = CubicSpline(s, knots_pitch, bc_type="clamped")
        # dense arc-parameter march with speed caps
        poses, u, ok = [], 0.0, True
        for _ in range(n_frames):
            pos = sp_p(u)
            if not clear(pos):
                ok = False
                break
            poses.append(look_pose(pos, float(sp_y(u)), float(sp_pt(u))))
            v = np.linalg.norm(sp_p(u, 1))
            w = abs(float(sp_y(u, 1)))
            du = min(vmax * dt / max(v, 1e-9), np.deg2rad(wmax_deg) * dt / max(w, 1e-9), 0.05)
            # the rates change along the step: shrink it until the step itself keeps both caps
            while du > 1e-9 and (np.linalg.norm(sp_p(min(u + du, n_knots - 1.0)) - sp_p(u)) > vmax * dt or
                                 abs(float(sp_y(min(u + du, n_knots - 1.0)) - sp_y(u))) > np.deg2rad(wmax_deg) * dt):
                du *= 0.9
            u = min(u + du, n_knots - 1.0)
        if ok:
            return poses
    raise RuntimeError("no clear trajectory in this scene")


def sequence_config3(seed: int, n_frames: int = 500, intr: Intrinsics = TUM_INTR, noise_coeff: float = 1e-3):
    """TUM-shaped tracking sequence: a 6 x 5 x 3 m room with 24 boxes and 12 spheres,
    ``n_frames`` poses at 30 Hz along :func:`spline_trajectory` (<= 1 m/s,
    <= 60 deg/s), and ``depth(f)``, the noisy 640x480 depth image of frame f
    (ray-cast on demand; its noise is seeded by (seed, f)).

    Returns a dict with keys ``scene, intr, poses, depth``."""
    # a 6 x 5 m room needs more furniture than the 4 x 3 m one for most views to constrain all six
    # degrees of freedom (a view of bare wall and floor leaves a translation along them free)
    scene = make_room(seed + 100, size=(6.0, 5.0, 3.0), n_boxes=24, n_spheres=12)
    poses = spline_trajectory(seed, scene, n_frames=n_frames)

    def depth(f: int) -> np.ndarray:
        rng = np.random.default_rng(7_000_001 * (seed + 1) + f)
        return add_depth_noise(raycast_depth(scene, poses[f], intr), rng, noise_coeff)

    return dict(scene=scene, intr=intr, poses=poses, depth=depth)


def const_velocity(T_prev: np.ndarray, T_prev2: np.ndarray | None) -> np.ndarray:
    """Constant-velocity prediction of the next pose from the last two: the
    relative motion T_prev2^-1 T_prev applied once more (T_prev alone when
    there is no earlier pose)."""
    if T_prev2 is None:
        return T_prev.copy()
    T = T_prev @ (inv_pose(T_prev2) @ T_prev)
    # nearest rotation (polar factor): products of estimated poses drift off orthonormal
    U, _, Vt = np.linalg.svd(T[:3, :3])
    T[:3, :3] = U @ Vt
    return T


def batch_config4(seed: int, n_pairs: int = 64, n_min: int = 5_000, n_max: int = 300_000,
                  max_deg: float = 5.0, max_m: float = 0.05, noise: float = 2e-3) -> list:
    """Independent config-1-style registration pairs with point counts log-uniform in
    [n_min, n_max] and offsets of uniform angle <= max_deg about a uniform axis and uniform
    length <= max_m.  Each entry: dict(src, tgt float32 n x 3, T_gt), the source in the frame
    T_gt^-1 (start from the identity)."""
    rng = np.random.default_rng(31337 + seed)
    out = []
    for b in range(n_pairs):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        scene = make_room(int(rng.integers(0, 1 << 30)))
        prng = np.random.default_rng(int(rng.integers(0, 1 << 62)))
        src_w = sample_surface(scene, n, prng, noise)
        tgt = sample_surface(scene, n, prng, noise)
        T_gt = random_offset(prng, prng.uniform(0.0, max_deg), prng.uniform(0.0, max_m))
        out.append(dict(src=transform_points(inv_pose(T_gt), src_w).astype(np.float32), tgt=tgt.astype(np.float32),
                        T_gt=T_gt))
    return out


# --------------------------------------------------------------------------- learned-covariance configuration

# TUM_INTR's stride-2 sample grid as an image of its own: pixel (j, i) here looks along the same ray
# as pixel (2j, 2i) of a 640 x 480 TUM_INTR image, so a 320 x 240 render at stride 1 yields the
# points a 640 x 480 render yields at stride 2, at a quarter of the ray-casting cost.
HALF_TUM_INTR = Intrinsics(320, 240, 262.5, 262.5, 159.75, 119.75)


def surrogate_train_config5(seed: int = 0, n_frames: int = 2000, n_scenes: int = 20,
                            intr: Intrinsics = HALF_TUM_INTR, noise_coeff: float = 1e-3):
    """Training frames of the covariance surrogate: ``n_scenes`` config-2-style rooms (4 x 3 x 2.5 m,
    8 boxes, 4 spheres; room seeds 1000 (seed + 1) + s, disjoint from :func:`sequence_config5`'s)
    seen from ``n_frames`` random poses (frame f in room f mod n_scenes): positions within 0.45 m
    of the room centre (horizontally) at heights 1.0-1.8 m, any heading, 0-40 degrees down.
    ``depth(f)`` ray-casts frame f on demand with noise N(0, (noise_coeff z^2)^2) seeded by
    (seed, f).  Returns a dict with keys ``scenes, intr, poses, depth``."""
    scenes = [make_room(1000 * (seed + 1) + s) for s in range(n_scenes)]
    rng = np.random.default_rng(555_001 + seed)
    poses = []
    for f in range(n_frames):
        sc = scenes[f % n_scenes]
        r, phi = 0.45 * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
        pos = np.array([sc.centre[0] + r * np.cos(phi), sc.centre[1] + r * np.sin(phi), rng.uniform(1.0, 1.8)])
        poses.append(look_pose(pos, rng.uniform(0, 2 * np.pi), np.deg2rad(rng.uniform(0.0, 40.0))))

    def depth(f: int) -> np.ndarray:
        frng = np.random.default_rng(3_000_017 * (seed + 1) + f)
        return add_depth_noise(raycast_depth(scenes[f % n_scenes], poses[f], intr), frng, noise_coeff)

    return dict(scenes=scenes, intr=intr, poses=poses, depth=depth)


def orbit_trajectory(seed: int, scene: Scene, n_frames: int = 500, fps: float = 30.0, turns: float = 1.0) -> list:
    """A camera orbiting the room centre while looking inwards: position on an ellipse with semi-axes
    0.3 of the room's length and width (radius and height wobbling smoothly), heading towards the
    centre plus a smooth swing of up to 25 degrees, 15-30 degrees down; ``turns`` orbits over the
    sequence.  Views keep the middle of the room (the furniture) in sight, where a free-roaming
    camera in a small room keeps facing bare walls and floor, which leave translations along them
    unconstrained."""
    rng = np.random.default_rng(6161 + seed)
    c = scene.centre
    ax, ay = 0.3 * (scene.room_hi - scene.room_lo)[:2]
    ph = rng.uniform(0, 2 * np.pi, size=4)
    phi0 = rng.uniform(0, 2 * np.pi)
    poses = []
    for f in range(n_frames):
        s = f / max(1, n_frames - 1)
        phi = phi0 + 2 * np.pi * turns * s
        rad = 1.0 + 0.12 * np.sin(2 * np.pi * 2 * s + ph[0])
        pos = np.array([c[0] + ax * rad * np.cos(phi), c[1] + ay * rad * np.sin(phi),
                        1.5 + 0.2 * np.sin(2 * np.pi * 1.5 * s + ph[1])])
        to_c = c[:2] - pos[:2]
        yaw = np.arctan2(to_c[1], to_c[0]) + np.deg2rad(25.0) * np.sin(2 * np.pi * 2.5 * s + ph[2])
        pitch = np.deg2rad(22.5 + 7.5 * np.sin(2 * np.pi * 1.7 * s + ph[3]))
        poses.append(look_pose(pos, yaw, pitch))
    return poses


def sequence_config5(seed: int = 0, n_frames: int = 500, intr: Intrinsics = TUM_INTR, noise_coeff: float = 1e-3):
    """Held-out sequence of the covariance surrogate: a config-2-style room (4 x 3 x 2.5 m, 8 boxes,
    4 spheres; seed 500 + seed, none of the training rooms) seen along :func:`orbit_trajectory` at
    30 Hz (one orbit in ``n_frames`` frames: ~0.4 m/s, ~25 deg/s), 640 x 480 depth frames
    ``depth(f)`` with noise seeded by (seed, f).  Returns a dict with keys ``scene, intr, poses,
    depth``."""
    scene = make_room(500 + seed)
    poses = orbit_trajectory(seed, scene, n_frames=n_frames)

    def depth(f: int) -> np.ndarray:
        rng = np.random.default_rng(8_000_009 * (seed + 1) + f)
        return add_depth_noise(raycast_depth(scene, poses[f], intr), rng, noise_coeff)

    return dict(scene=scene, intr=intr, poses=poses, depth=depth)


# --------------------------------------------------------------------------- parallel rendering

_SEQUENCES = {"config3": "sequence_config3", "config5": "sequence_config5"}


def _render_frames_job(args):
    kind, seed, n_frames, frames = args
    cfg = globals()[_SEQUENCES[kind]](seed, n_frames=n_frames)
    return [cfg["depth"](f) for f in frames]


def render_sequence_frames(kind: str, seed: int, n_frames: int, workers: int) -> np.ndarray:
    """Depth images 0 .. n_frames-1 of ``sequence_config3`` (kind "config3") or ``sequence_config5``
    ("config5") with that seed and length, ray-cast by ``workers`` processes (started by spawn, so a
    parent that holds a CUDA context is safe); the same images as calling ``depth(f)`` in order."""
    if kind not in _SEQUENCES:
        raise ValueError(f"unknown sequence {kind!r}")
    step = max(1, -(-n_frames // (max(1, workers) * 4)))
    jobs = [(kind, seed, n_frames, list(range(a, min(n_frames, a + step)))) for a in range(0, n_frames, step)]
    if workers <= 1 or len(jobs) <= 1:
        parts = [_render_frames_job(j) for j in jobs]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            parts = pool.map(_render_frames_job, jobs)
    return np.stack([d for part in parts for d in part]) if n_frames > 0 else np.zeros((0, 0, 0), np.float32)
