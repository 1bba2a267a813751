"""Training and evaluation of the learned covariance surrogate (the k-NN covariance step replaced by a
small convolutional network; gsicp_surrogate_* in the C ABI).

Training (``python -m paper_2403_12550_b300.surrogate train``): the config-5 training frames
(synthetic config-2-style rooms, seeded, ray-cast in worker processes), each frame's own k-NN
plane covariances from the plain GPU path as targets, one Adam step per frame
(gsicp_surrogate_train_step), 20 epochs in a seeded shuffled order, the learning rate 2e-3
decaying by 0.85 per epoch.  The trained weights are
written to ``data/cov_surrogate.npy`` beside this file, which :func:`load_weights` reads.

Evaluation (``... evaluate``): the held-out config-5 sequence (640 x 480 frames of a room none of
the training frames show) tracked twice by the native tracker, once with k-NN covariances and
once with the surrogate's (per-frame fallback to k-NN when the frame's residual, the RMS distance of
its correspondences, exceeds 1.1 times the last k-NN frame's), reporting frames/s, the absolute
trajectory error (RMSE of camera positions against the ground truth) of both, and how many frames
fell back.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

from .trajectory import ate_rmse, ate_rmse_aligned

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS_PATH = os.path.join(HERE, "data", "cov_surrogate.npy")
N_WEIGHTS = 30400
LAYERS = ((32, 3), (32, 32), (3, 32))  # (out, in) channels, 5 x 5 taps each

# the covariance and registration settings of the tracking configurations
COV = dict(k=20, eps=1e-3, p=1.5)


def init_weights(seed: int) -> np.ndarray:
    """He-normal initial weights (std sqrt(2 / fan_in), fan_in = in channels x 25), seeded."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(size=o * i * 25) * np.sqrt(2.0 / (i * 25)) for o, i in LAYERS]
    return np.concatenate(parts).astype(np.float32)


def load_weights(path: str = WEIGHTS_PATH) -> np.ndarray:
    w = np.load(path).astype(np.float32).ravel()
    if w.size != N_WEIGHTS:
        raise ValueError(f"{path}: expected {N_WEIGHTS} weights")
    return w


# ----------------------------------------------------------------------------- frames

def _render_train(args):
    seed, n_frames, n_scenes, frames = args
    from synth import surrogate_train_config5
    cfg = surrogate_train_config5(seed, n_frames=n_frames, n_scenes=n_scenes)
    return [cfg["depth"](f) for f in frames]


def _render_seq(args):
    seed, n_frames, frames = args
    from synth import sequence_config5
    cfg = sequence_config5(seed, n_frames=n_frames)
    return [cfg["depth"](f) for f in frames]


def _parallel(fn, jobs, workers: int):
    if workers <= 1:
        return [x for j in jobs for x in fn(j)]
    # spawn: the parent may already hold a CUDA context, which a forked child must not inherit
    with mp.get_context("spawn").Pool(workers) as pool:
        return [x for part in pool.map(fn, jobs) for x in part]


def _chunks(n: int, k: int):
    step = (n + k - 1) // k
    return [list(range(a, min(n, a + step))) for a in range(0, n, step)]


def render_train_frames(seed: int, n_frames: int, n_scenes: int, workers: int) -> np.ndarray:
    jobs = [(seed, n_frames, n_scenes, c) for c in _chunks(n_frames, max(1, workers) * 4)]
    return np.stack(_parallel(_render_train, jobs, workers))


def render_sequence(seed: int, n_frames: int, workers: int) -> np.ndarray:
    jobs = [(seed, n_frames, c) for c in _chunks(n_frames, max(1, workers) * 4)]
    return np.stack(_parallel(_render_seq, jobs, workers))


# ----------------------------------------------------------------------------- training

def train(seed: int = 0, n_frames: int = 2000, n_scenes: int = 20, epochs: int = 20, lr: float = 2e-3,
          decay: float = 0.85, workers: int | None = None, out: str = WEIGHTS_PATH, log=print, frames=None) -> dict:
    import torch
    import paper_2403_12550_b300 as g
    from synth import HALF_TUM_INTR

    workers = workers or max(1, min(32, os.cpu_count() or 1))
    t0 = time.time()
    if frames is None:
        frames = render_train_frames(seed, n_frames, n_scenes, workers)
    t_render = time.time() - t0
    dev = torch.from_numpy(frames).cuda()
    intr = HALF_TUM_INTR.as_array()
    ctx = g.Context()
    sg = g.Surrogate(init_weights(seed))
    cp = g.CovParams(COV["k"], COV["eps"], g.PLANE, COV["p"])
    rng = np.random.default_rng(seed + 77)
    hist = []
    t1 = time.time()
    for ep in range(epochs):
        lr_ep = lr * (decay ** ep)
        losses = []
        for f in rng.permutation(n_frames):
            r = g.gsicp_surrogate_train_step(ctx, sg, dev[f], intr, 1, 0.1, 10.0, cp, lr=lr_ep, apply=True)
            losses.append(r["loss"])
        hist.append(float(np.mean(losses)))
        log(f"epoch {ep}: lr {lr_ep:.2e} mean loss {hist[-1]:.5f}")
    t_train = time.time() - t1
    w = sg.weights()
    if out:
        os.makedirs(os.path.dirname(out), exist_ok=True)
        np.save(out, w)
    sg.close()
    ctx.close()
    return dict(epochs=epochs, frames=n_frames, loss=hist, render_s=t_render, train_s=t_train,
                steps_per_s=epochs * n_frames / t_train)


# ----------------------------------------------------------------------------- evaluation

def evaluate(weights=None, seed: int = 0, n_frames: int = 500, fallback_ratio: float = 1.1, calib_every: int = 30,
             keyframe_knn: bool = True, workers: int | None = None, frames=None, log=print, modes=("knn", "surrogate")) -> dict:
    import torch
    import paper_2403_12550_b300 as g
    from synth import TUM_INTR, sequence_config5

    workers = workers or max(1, min(32, os.cpu_count() or 1))
    seq = sequence_config5(seed, n_frames=n_frames)
    if frames is None:
        frames = render_sequence(seed, n_frames, workers)
    dev = [torch.from_numpy(f).cuda() for f in frames]
    intr = TUM_INTR.as_array()
    gt = seq["poses"]
    w = load_weights() if weights is None else weights
    ctx = g.Context()
    sg = g.Surrogate(w)
    cp = g.CovParams(COV["k"], COV["eps"], g.PLANE, COV["p"])
    rp = g.RegParams(0.1, 30, 1e-6, 1e-6, 6)
    out = {}
    for name in modes:
        tr = g.Tracker(ctx, 2, 0.1, 10.0, cp, rp)
        if name == "surrogate":
            tr.set_surrogate(sg, fallback_ratio, calib_every, keyframe_knn)
        # warm-up on the first frames of the sequence (kernels, buffers), not counted
        warm = g.Tracker(ctx, 2, 0.1, 10.0, cp, rp)
        if name == "surrogate":
            warm.set_surrogate(sg, fallback_ratio, calib_every, keyframe_knn)
        for f in range(min(5, n_frames)):
            warm.frame(dev[f], intr, gt[0] if f == 0 else None)
        warm.close()
        est, infos, lat = [], [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in range(n_frames):
            a = time.perf_counter()
            T, info = tr.frame(dev[f], intr, gt[0] if f == 0 else None)
            lat.append(time.perf_counter() - a)
            est.append(T)
            infos.append(info)
        wall = time.perf_counter() - t0
        res = dict(frames_per_s=n_frames / wall, ate_m=ate_rmse(est, gt), ate_aligned_m=ate_rmse_aligned(est, gt),
                   p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                   keyframes=int(sum(i["kind"] == g.KEYFRAME for i in infos)),
                   surrogate_frames=int(sum(i["cov_source"] == 1 for i in infos)),
                   fell_back=int(sum(i["fell_back"] for i in infos)),
                   degenerate=int(sum(i["status"] != g.OK for i in infos)))
        out[name] = res
        log(f"{name}: {json.dumps(res)}")
        tr.close()
    sg.close()
    ctx.close()
    if "knn" in out and "surrogate" in out:
        out["ate_gap_m"] = out["surrogate"]["ate_m"] - out["knn"]["ate_m"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=("train", "evaluate"))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--weights", default=None)
    args = ap.parse_args(argv)
    if args.cmd == "train":
        r = train(args.seed, n_frames=args.frames or 2000, epochs=args.epochs, lr=args.lr, out=args.out)
    else:
        w = load_weights(args.weights) if args.weights else None
        r = evaluate(w, args.seed, n_frames=args.frames or 500)
    print(json.dumps(r))


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(HERE))
    main()
