"""Ablations of the covariance regularisation and the scale-alignment exponent on synthetic
sequences (analogues of the paper's Tables 5 and 6, ATE only): the library's tracker runs one
TUM-shaped sequence per setting and the RMSE of the translation error against the ground truth
is reported.

    python -m paper_2403_12550_b300.ablation [--frames 150] [--seed 0]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import paper_2403_12550_b300 as g
from paper_2403_12550_b300.trajectory import ate_rmse, ate_rmse_aligned


def run(depths, poses, intr, reg_mode: int, p: float, ctx) -> dict:
    trk = g.Tracker(ctx, 2, 0.1, 10.0, g.CovParams(20, 1e-3, reg_mode, p), g.RegParams(0.1, 30, 1e-6, 1e-6, 6))
    est, kinds = [], []
    t0 = time.perf_counter()
    for f, d in enumerate(depths):
        T, info = trk.frame(d, intr, poses[0] if f == 0 else None)
        est.append(T)
        kinds.append(info["kind"])
    dt = time.perf_counter() - t0
    sizes = trk.map_sizes()
    trk.close()
    return dict(ate_m=ate_rmse(est, poses), ate_aligned_m=ate_rmse_aligned(est, poses), keyframes=kinds.count(g.KEYFRAME),
                mapping_keyframes=kinds.count(g.MAPPING_KEYFRAME), map_size=sizes[0], seconds=dt)


def main():
    from synth import sequence_config3
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=150)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    seq = sequence_config3(a.seed, n_frames=a.frames)
    depths = [torch.from_numpy(seq["depth"](f)).cuda() for f in range(a.frames)]
    intr = seq["intr"].as_array()
    ctx = g.Context()
    out = {}
    for name, mode in (("plane", g.PLANE), ("ellipse", g.ELLIPSE), ("none", g.NONE)):
        for p in (0.0, 1.0, 1.5):
            out[f"{name}/p={p}"] = run(depths, seq["poses"], intr, mode, p, ctx)
    ctx.close()
    print(json.dumps({"frames": a.frames, "seed": a.seed, "results": out}))


if __name__ == "__main__":
    main()
