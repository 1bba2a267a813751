"""FP64 oracle of the learned covariance surrogate (a small depth-patch CNN).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module.  It shares no code with the CUDA library and
never consumes anything the CUDA library produced.

What the surrogate computes (not in the paper; it stands in for the k-NN
covariance step of Sec. 3 and is trained on that step's outputs):

* Input: the point map of a depth frame on its sampled grid (every
  ``stride``-th pixel, back-projected as in a1), with a validity mask.
* Layer 1, 3 -> 32 channels, 5 x 5 taps, on centred differences: channel o at
  pixel u is sum over taps d and coordinates c of W1[o, c, d] * M(u + d) *
  (P_c(u + d) - P_c(u)).  Centring makes the layer blind to where the patch
  sits; the missing bias terms make every layer positively homogeneous, so the
  output scales with the patch and its direction does not depend on distance.
* ReLU, rounded to bfloat16, zero at invalid pixels.
* Layer 2, 32 -> 32, 5 x 5 taps (zero outside the image), ReLU, bfloat16,
  zero at invalid pixels.
* Layer 3, 32 -> 3, 5 x 5 taps: an unnormalised normal v.
* The point's covariance is the plane-regularised one of Sec. 3 built on the
  predicted normal n = v / |v|: C = (I - (1 - eps) n n^T) z^(-2p), the
  covariance with unit spread in the tangent plane and eps along n, scaled by
  the scale aligning of Sec. 3 (z = the point's depth).

Weights are bfloat16 values (the caller's float weights rounded to nearest
even); arithmetic here is float64.  Training minimises, over the valid pixels
with a k-NN covariance C_knn, the mean of 1 - n^T T n, T = n_knn n_knn^T the
projector on the k-NN normal, recovered from the plane-regularised k-NN
covariance as T = (I - C_knn z^(2p)) / (1 - eps).  Gradients treat the
bfloat16 roundings as the identity (the usual mixed-precision convention).

Taps: output pixel (i, j) reads input pixel (i + dy - 2, j + dx - 2) for tap
(dy, dx), 0 <= dy, dx < 5 (cross-correlation).  Weight layout, flattened in
this order: W1[32][3][5][5], W2[32][32][5][5], W3[3][32][5][5].
"""
from __future__ import annotations

import numpy as np

C_IN, C_HID, C_OUT, KS = 3, 32, 3, 5
R = KS // 2
SIZES = (C_HID * C_IN * KS * KS, C_HID * C_HID * KS * KS, C_OUT * C_HID * KS * KS)
N_WEIGHTS = sum(SIZES)


def split_weights(w):
    """Flat weight vector -> (W1, W2, W3) arrays (float64 copies)."""
    w = np.asarray(w, dtype=np.float64).ravel()
    if w.size != N_WEIGHTS:
        raise ValueError(f"expected {N_WEIGHTS} weights, got {w.size}")
    a, b = SIZES[0], SIZES[0] + SIZES[1]
    return (w[:a].reshape(C_HID, C_IN, KS, KS), w[a:b].reshape(C_HID, C_HID, KS, KS),
            w[b:].reshape(C_OUT, C_HID, KS, KS))


def bf16(x):
    """Round to the nearest bfloat16 value (8 significant bits, ties to even); float64 result.
    Values are assumed inside bfloat16's normal range or zero."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                      # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def point_grid(depth, intr, stride: int, z_min: float, z_max: float):
    """a1 on the sampled grid: (P (h, w, 3), M (h, w) bool) for every stride-th pixel; pixel
    (u, v) with depth d in [z_min, z_max] is ((u - cx) d / fx, (v - cy) d / fy, d)."""
    depth = np.asarray(depth, dtype=np.float32)
    d = depth[::stride, ::stride].astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in intr)
    z_lo, z_hi = float(np.float32(z_min)), float(np.float32(z_max))
    M = np.isfinite(d) & (d >= z_lo) & (d <= z_hi)
    H, W = depth.shape
    v, u = np.meshgrid(np.arange(0, H, stride, dtype=np.float64), np.arange(0, W, stride, dtype=np.float64),
                       indexing="ij")
    dz = np.where(M, d, 0.0)
    P = np.stack([(u - cx) * dz / fx, (v - cy) * dz / fy, dz], axis=-1)
    return P, M


def _shift(x, dy: int, dx: int):
    """y[i, j] = x[i + dy, j + dx] (zero outside); x is (h, w, ...)."""
    h, w = x.shape[:2]
    y = np.zeros_like(x)
    i0, i1 = max(0, -dy), min(h, h - dy)
    j0, j1 = max(0, -dx), min(w, w - dx)
    if i0 < i1 and j0 < j1:
        y[i0:i1, j0:j1] = x[i0 + dy:i1 + dy, j0 + dx:j1 + dx]
    return y


def _conv(x, W):
    """Cross-correlation with zero padding: y[i, j, o] = sum_{c, dy, dx} W[o, c, dy, dx] x[i+dy-2, j+dx-2, c]."""
    y = np.zeros(x.shape[:2] + (W.shape[0],))
    for dy in range(KS):
        for dx in range(KS):
            y += _shift(x, dy - R, dx - R) @ W[:, :, dy, dx].T
    return y


def _layer1(P, M, W1):
    """Centred first layer: a1[i, j, o] = sum W1[o, c, d] M(u+d) (P_c(u+d) - P_c(u))."""
    Pm = P * M[..., None]
    Mf = M.astype(np.float64)[..., None]
    a = np.zeros(P.shape[:2] + (W1.shape[0],))
    for dy in range(KS):
        for dx in range(KS):
            Ps = _shift(Pm, dy - R, dx - R)
            Ms = _shift(Mf, dy - R, dx - R)
            a += (Ps - Ms * P) @ W1[:, :, dy, dx].T
    return a


def forward(P, M, weights, round_bf16: bool = True):
    """The network on one point grid.  Returns a dict with a1, h1, a2, h2 (hidden layers) and
    v (h, w, 3), the unnormalised normal at every pixel (zero where M is false)."""
    W1, W2, W3 = split_weights(weights)
    rnd = bf16 if round_bf16 else (lambda t: np.asarray(t, dtype=np.float64))
    W1, W2, W3 = rnd(W1), rnd(W2), rnd(W3)
    Mf = M.astype(np.float64)[..., None]
    a1 = _layer1(P, M, W1) * Mf
    h1 = rnd(np.maximum(a1, 0.0)) * Mf
    a2 = _conv(h1, W2) * Mf
    h2 = rnd(np.maximum(a2, 0.0)) * Mf
    v = _conv(h2, W3) * Mf
    return dict(a1=a1, h1=h1, a2=a2, h2=h2, v=v)


def plane_covariance(n, z, eps: float, p: float):
    """Plane-regularised covariance on unit normals n (..., 3) with the scale aligning factor
    z^(-2p): (I - (1 - eps) n n^T) z^(-2p).  Returns (..., 6) as (xx, xy, xz, yy, yz, zz)."""
    n = np.asarray(n, dtype=np.float64)
    s = np.asarray(z, dtype=np.float64) ** (-2.0 * p)
    k = 1.0 - eps
    xx = (1 - k * n[..., 0] * n[..., 0]) * s
    xy = (-k * n[..., 0] * n[..., 1]) * s
    xz = (-k * n[..., 0] * n[..., 2]) * s
    yy = (1 - k * n[..., 1] * n[..., 1]) * s
    yz = (-k * n[..., 1] * n[..., 2]) * s
    zz = (1 - k * n[..., 2] * n[..., 2]) * s
    return np.stack([xx, xy, xz, yy, yz, zz], axis=-1)


def covariances(v, M, P, eps: float, p: float):
    """Per valid pixel, in raster order (the order of a1's points): the covariance built on
    n = v / |v|, and whether |v| > 0 (where it is 0 the direction is undefined and the
    covariance is the isotropic z^(-2p) I)."""
    vv = v[M]
    z = P[M][:, 2]
    nrm = np.linalg.norm(vv, axis=1)
    ok = nrm > 0
    n = np.where(ok[:, None], vv / np.where(ok, nrm, 1.0)[:, None], 0.0)
    C = plane_covariance(n, z, eps, p)
    if not ok.all():
        s = z[~ok] ** (-2.0 * p)
        C[~ok] = np.stack([s, 0 * s, 0 * s, s, 0 * s, s], axis=-1)
    return C, ok


def knn_projector(C_knn, z, eps: float, p: float):
    """T = (I - C_knn z^(2p)) / (1 - eps) from plane-regularised covariances (n, 6): the projector
    n_knn n_knn^T on the k-NN normal.  Returns (n, 3, 3)."""
    C = np.asarray(C_knn, dtype=np.float64)
    s = np.asarray(z, dtype=np.float64) ** (2.0 * p)
    full = np.stack([C[:, 0], C[:, 1], C[:, 2], C[:, 1], C[:, 3], C[:, 4], C[:, 2], C[:, 4], C[:, 5]],
                    axis=-1).reshape(-1, 3, 3)
    return (np.eye(3)[None] - full * s[:, None, None]) / (1.0 - eps)


def loss(v, M, T, mask_t=None):
    """Mean over valid pixels (and mask_t, if given, in raster order of the valid pixels) of
    1 - n^T T n, n = v / |v|; pixels with |v| = 0 count as loss 1."""
    vv = v[M]
    sel = np.ones(len(vv), bool) if mask_t is None else np.asarray(mask_t, bool)
    vv, Ts = vv[sel], T[sel]
    nrm = np.linalg.norm(vv, axis=1)
    ok = nrm > 0
    n = np.where(ok[:, None], vv / np.where(ok, nrm, 1.0)[:, None], 0.0)
    q = np.einsum("ni,nij,nj->n", n, Ts, n)
    return float(np.mean(1.0 - q)) if len(q) else 0.0


def loss_and_grad(P, M, weights, T, mask_t=None, round_bf16: bool = True):
    """The training loss and its gradient with respect to the flat weight vector (back-propagation
    through the three layers; bfloat16 roundings pass gradients unchanged)."""
    W1, W2, W3 = split_weights(weights)
    rnd = bf16 if round_bf16 else (lambda t: np.asarray(t, dtype=np.float64))
    W1r, W2r, W3r = rnd(W1), rnd(W2), rnd(W3)
    f = forward(P, M, weights, round_bf16)
    v = f["v"]
    h, w = M.shape
    sel = np.ones(int(M.sum()), bool) if mask_t is None else np.asarray(mask_t, bool)
    N = int(sel.sum())
    # dL/dv at the selected valid pixels
    vv = v[M]
    nrm = np.linalg.norm(vv, axis=1)
    dv_valid = np.zeros_like(vv)
    ok = (nrm > 0) & sel
    n = vv[ok] / nrm[ok][:, None]
    Tn = np.einsum("nij,nj->ni", T[ok], n)
    dLdn = -2.0 * Tn / max(N, 1)
    # through n = v / |v|: (I - n n^T) dL/dn / |v|
    dv_valid[ok] = (dLdn - n * np.sum(n * dLdn, axis=1, keepdims=True)) / nrm[ok][:, None]
    dv = np.zeros((h, w, C_OUT))
    dv[M] = dv_valid
    Mf = M.astype(np.float64)[..., None]
    # layer 3: v = conv(h2, W3)
    gW3 = np.zeros_like(W3)
    dh2 = np.zeros((h, w, C_HID))
    for dy in range(KS):
        for dx in range(KS):
            hs = _shift(f["h2"], dy - R, dx - R)
            gW3[:, :, dy, dx] = dv.reshape(-1, C_OUT).T @ hs.reshape(-1, C_HID)
            dh2 += _shift(dv @ W3r[:, :, dy, dx], R - dy, R - dx)
    da2 = dh2 * (f["a2"] > 0) * Mf
    gW2 = np.zeros_like(W2)
    dh1 = np.zeros((h, w, C_HID))
    for dy in range(KS):
        for dx in range(KS):
            hs = _shift(f["h1"], dy - R, dx - R)
            gW2[:, :, dy, dx] = da2.reshape(-1, C_HID).T @ hs.reshape(-1, C_HID)
            dh1 += _shift(da2 @ W2r[:, :, dy, dx], R - dy, R - dx)
    da1 = dh1 * (f["a1"] > 0) * Mf
    gW1 = np.zeros_like(W1)
    Pm = P * Mf
    for dy in range(KS):
        for dx in range(KS):
            Ps = _shift(Pm, dy - R, dx - R)
            Ms = _shift(Mf, dy - R, dx - R)
            D = Ps - Ms * P
            gW1[:, :, dy, dx] = da1.reshape(-1, C_HID).T @ D.reshape(-1, C_IN)
    L = loss(v, M, T, mask_t)
    return L, np.concatenate([gW1.ravel(), gW2.ravel(), gW3.ravel()])


def adam_step(w, g, m, s, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1) at step t >= 1: m <- b1 m + (1-b1) g,
    s <- b2 s + (1-b2) g^2, w <- w - lr m_hat / (sqrt(s_hat) + eps) with the bias-corrected
    moments m_hat = m / (1 - b1^t), s_hat = s / (1 - b2^t).  Returns (w, m, s)."""
    m = b1 * m + (1 - b1) * g
    s = b2 * s + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    sh = s / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(sh) + eps), m, s


def init_weights(seed: int):
    """He-normal initial weights (std sqrt(2 / fan_in)), seeded; float32 flat vector."""
    rng = np.random.default_rng(seed)
    out = []
    for size, fan_in in zip(SIZES, (C_IN * KS * KS, C_HID * KS * KS, C_HID * KS * KS)):
        out.append(rng.normal(size=size) * np.sqrt(2.0 / fan_in))
    return np.concatenate(out).astype(np.float32)
