"""Write tests/golden/tiny_render.json: the FP64 oracle's render and adjoint of
a small scene given explicitly below (no random draws), for the two marching
modes of Algorithm 1 (uniform steps without skipping; Eq. 5 adaptive steps with
empty-space skipping).  Only the oracle computes the stored values.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2509_07782_b300 import synth  # noqa: E402  (input containers only)


def tiny_scene() -> synth.Scene:
    means = np.array([[0.00, 0.00, 0.00], [0.25, -0.10, 0.30], [-0.30, 0.20, -0.20],
                      [0.10, 0.35, 0.15], [-0.15, -0.30, 0.25]], np.float32)
    scales = np.array([[0.12, 0.08, 0.10], [0.06, 0.15, 0.07], [0.10, 0.10, 0.10],
                       [0.20, 0.05, 0.09], [0.07, 0.07, 0.16]], np.float32)
    quats = np.array([[1.0, 0.0, 0.0, 0.0], [0.9, 0.3, -0.2, 0.1], [0.7, 0.0, 0.7, 0.0],
                      [0.5, 0.5, 0.5, 0.5], [0.8, -0.4, 0.1, 0.3]], np.float32)
    densities = np.array([4.0, 9.0, 2.5, 6.0, 12.0], np.float32)
    k = np.arange(16, dtype=np.float32)[None, :, None]
    l = np.arange(5, dtype=np.float32)[:, None, None]
    c = np.arange(3, dtype=np.float32)[None, None, :]
    sh = (0.3 * np.cos(0.7 * k + 1.3 * l + 2.1 * c) / (1.0 + k)).astype(np.float32)
    return synth.Scene(means, scales, quats, densities, sh, 3)


def tiny_camera() -> synth.Camera:
    # at (0.05, -0.03, 2) looking down -z at the origin (camera x = world x, camera y = world -y)
    c2w = np.array([[1.0, 0.0, 0.0, 0.05], [0.0, -1.0, 0.0, -0.03], [0.0, 0.0, -1.0, 2.0]], np.float32)
    return synth.Camera(c2w=c2w, fx=9.0, fy=9.0, cx=3.0, cy=2.5, width=6, height=5)


def modes():
    return {"uniform": synth.Options(dt=0.01, n_s=16),
            "adaptive_skip": synth.Options(skip=True, adaptive=True, dt_min=0.005, dt_max=0.02, beta=1024.0,
                                           n_s=8)}


def upstream(n_rays: int) -> np.ndarray:
    p = np.arange(n_rays)[:, None]
    ch = np.arange(4)[None, :]
    return (((7 * p + 3 * ch) % 5) - 2) / 2.0


def main() -> None:
    sc, cam = tiny_scene(), tiny_camera()
    W = upstream(cam.n_rays)
    out = {"_about": "FP64 oracle render and adjoint of tests/golden/make_golden.py's scene (regression "
                     "fixture for the oracle; parity fixture for the CUDA path)", "modes": {}}
    for name, o in modes().items():
        r = oracle.render(sc, cam, o)
        g = oracle.backward(sc, cam, o, W)
        out["modes"][name] = {"rgba": r["rgba"].tolist(),
                              "grad": {k: np.asarray(g[k]).tolist() for k in
                                       ("means", "scales", "quats", "densities", "sh")}}
    with open(os.path.join(HERE, "tiny_render.json"), "w") as f:
        json.dump(out, f)
    print("wrote", os.path.join(HERE, "tiny_render.json"))


if __name__ == "__main__":
    main()
