"""Pins of the oracle's image loss (Sec. 3.4: (1 - lambda) L1 + lambda DSSIM),
against definitions written out independently here:

* SSIM by a direct double loop over the 11 x 11 window with zero padding (no
  separable filtering), on small images;
* SSIM(x, x) = 1 and L(x, x) = 0; lambda = 0 gives the plain mean absolute error;
* the analytic gradient against FP64 central differences of the loss.
"""
import math

import numpy as np

from oracle import losses


def _ssim_direct(x, y):
    H, W, C = x.shape
    g = np.array([math.exp(-((i - 5) ** 2) / (2 * 1.5 ** 2)) for i in range(11)])
    g /= g.sum()
    out = np.zeros_like(x)
    for i in range(H):
        for j in range(W):
            for c in range(C):
                sx = sy = sxx = syy = sxy = 0.0
                for di in range(-5, 6):
                    for dj in range(-5, 6):
                        ii, jj = i + di, j + dj
                        if 0 <= ii < H and 0 <= jj < W:
                            w = g[di + 5] * g[dj + 5]
                            a, b = x[ii, jj, c], y[ii, jj, c]
                            sx += w * a; sy += w * b; sxx += w * a * a; syy += w * b * b; sxy += w * a * b
                vx, vy, cv = sxx - sx * sx, syy - sy * sy, sxy - sx * sy
                out[i, j, c] = ((2 * sx * sy + 1e-4) * (2 * cv + 9e-4)) / ((sx * sx + sy * sy + 1e-4) * (vx + vy + 9e-4))
    return out


def test_ssim_map_equals_the_direct_window_sum():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(size=(9, 13, 3)), rng.uniform(size=(9, 13, 3))
    S = losses.ssim_terms(x, y)[0]
    np.testing.assert_allclose(S, _ssim_direct(x, y), rtol=1e-12, atol=1e-13)


def test_identical_images_and_pure_l1():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(7, 8, 3))
    L, g = losses.image_loss(x, x)
    assert abs(L) < 1e-12 and np.abs(losses.ssim_terms(x, x)[0] - 1.0).max() < 1e-12
    y = rng.uniform(size=(7, 8, 3))
    L0, g0 = losses.image_loss(x, y, lam=0.0)
    assert np.isclose(L0, np.abs(x - y).mean())
    np.testing.assert_allclose(g0, np.sign(x - y) / x.size)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0.1, 0.9, size=(10, 12, 3)), rng.uniform(0.1, 0.9, size=(10, 12, 3))
    L, g = losses.image_loss(x, y, lam=0.2)
    h = 1e-6
    worst = 0.0
    for idx in [(0, 0, 0), (3, 4, 1), (9, 11, 2), (5, 0, 0), (0, 7, 2), (6, 6, 1), (2, 10, 0), (8, 3, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (losses.image_loss(xp, y)[0] - losses.image_loss(xm, y)[0]) / (2 * h)
        worst = max(worst, abs(fd - g[idx]) / np.abs(g).max())
    assert worst < 1e-6
