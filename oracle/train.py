"""Optimiser and adaptive density control of the training step -- oracle side (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Adam (Kingma & Ba 2015), one step on a tensor: m = b1 m + (1 - b1) g,
v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
With the exponential parameterisation the variable p is log(value) and the
gradient given is d/d value, so g = grad * exp(p).

Densification (Sec. 3.5, Eq. 11 criterion stat / count > tau; the clone/split rule
the paper keeps from the methods it builds on): over the threshold, a Gaussian whose
largest scale is at most size_threshold is kept and copied (clone); otherwise it is
replaced by two children at mu + R(q) (s * z_k) with scales s / 1.6 (split).
Outputs are written in input order: kept -> 1, clone -> 2, split -> 2.
"""
from __future__ import annotations

import numpy as np

SPLIT_SCALE = 1.6


def adam_step(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15, exp_param=False):
    """Returns (p, m, v, activated) after one step (inputs unchanged)."""
    p = np.asarray(p, np.float64).copy()
    g = np.asarray(g, np.float64)
    if exp_param:
        g = g * np.exp(p)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v, (np.exp(p) if exp_param else p)


def rotation(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify_plan(stat, count, scales, tau, size_threshold):
    """(action [n], offset [n], n_out): 0 keep, 1 clone, 2 split.  The decisions turn
    floats into an integer, so they are taken in float32 (the kernel's precision):
    stat / count > tau and max scale <= size_threshold, each operation rounded."""
    stat = np.asarray(stat, np.float32)
    count = np.asarray(count)
    smax = np.asarray(scales, np.float32).reshape(-1, 3).max(1)
    ratio = (stat / np.maximum(count, 1).astype(np.float32)).astype(np.float32)
    over = (count > 0) & (ratio > np.float32(tau))
    action = np.where(over, np.where(smax <= np.float32(size_threshold), 1, 2), 0).astype(np.int32)
    nout = np.where(action == 0, 1, 2)
    offset = (np.cumsum(nout) - nout).astype(np.int32)
    return action, offset, int(nout.sum())


def densify_apply(action, normals, means, scales, quats, dens, sh, sg=None):
    """New parameter arrays and the source index of every output."""
    out = {k: [] for k in ("means", "scales", "quats", "densities", "sh", "sg", "src")}
    for l, a in enumerate(action):
        kids = [(means[l], scales[l])] if a == 0 else [(means[l], scales[l])] * 2
        if a == 2:
            R = rotation(quats[l])
            kids = [(means[l] + R @ (scales[l] * normals[l, k]), scales[l] / SPLIT_SCALE) for k in range(2)]
        for mu, s in kids:
            out["means"].append(mu)
            out["scales"].append(s)
            out["quats"].append(quats[l])
            out["densities"].append(dens[l])
            out["sh"].append(sh[l])
            if sg is not None:
                out["sg"].append(sg[l])
            out["src"].append(l)
    return {k: np.asarray(v) for k, v in out.items() if len(v) or k != "sg"}
