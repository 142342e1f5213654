"""Per-Gaussian training terms of RayGaussX -- oracle side (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Isotropic loss (Sec. 3.4, Eqs. 6-8): with
    r_max,l = 2 / (pi sqrt 3) * (s1^2 + s2^2 + s3^2)^(3/2) / (s1 s2 s3)
(the rotation-independent upper bound of the AABB / ellipsoid volume ratio,
Supp. Sec. 2.3),
    L_s = 1/N sum_l (max(r_max,l, r0) - r0)
and, where r_max,l > r0,  d r_max / d s_j = r_max (3 s_j / |s|^2 - 1 / s_j).

Densification statistic (Sec. 3.5, Eq. 11): for a view i with camera centre
o_i and focal length f_i, every Gaussian observed in the view (non-zero mean
gradient) accumulates alpha_i |grad_mu L_i| with alpha_i = |mu_l - o_i| / f_i,
and its view count I_l increments; the criterion is the ratio of the two.
"""
from __future__ import annotations

import math

import numpy as np

K_BOUND = 2.0 / (math.pi * math.sqrt(3.0))


def r_max(scales) -> np.ndarray:
    s = np.asarray(scales, dtype=np.float64).reshape(-1, 3)
    ss = (s * s).sum(1)
    return K_BOUND * ss ** 1.5 / np.prod(s, axis=1)


def isotropic_loss(scales, r0: float = 10.0):
    """(L_s, dL_s/ds [N,3]) of Eqs. 6-8."""
    s = np.asarray(scales, dtype=np.float64).reshape(-1, 3)
    n = s.shape[0]
    if n == 0:
        return 0.0, np.zeros((0, 3))
    r = r_max(s)
    over = r > r0
    loss = float(np.where(over, r - r0, 0.0).sum() / n)
    ss = (s * s).sum(1, keepdims=True)
    dr = r[:, None] * (3.0 * s / ss - 1.0 / s)
    grad = np.where(over[:, None], dr, 0.0) / n
    return loss, grad


def densify_update(means, d_means, cam_origin, focal, stat, count):
    """Add one view's contribution to (stat, count) in place (Eq. 11)."""
    mu = np.asarray(means, dtype=np.float64).reshape(-1, 3)
    g = np.asarray(d_means, dtype=np.float64).reshape(-1, 3)
    gn = np.linalg.norm(g, axis=1)
    alpha = np.linalg.norm(mu - np.asarray(cam_origin, dtype=np.float64)[None, :], axis=1) / float(focal)
    seen = gn > 0
    stat += np.where(seen, alpha * gn, 0.0)
    count += seen.astype(count.dtype)


# ---------------------------------------------------------------------------
# Image loss of the training step (Sec. 3.4): L = (1 - lambda) L1 + lambda DSSIM
# (+ lambda_s L_s, above).  The paper writes the total loss without fixing the
# image terms' constants; the readings taken here: DSSIM = 1 - SSIM, SSIM with
# an 11 x 11 Gaussian window of standard deviation 1.5, C1 = 0.01^2,
# C2 = 0.03^2, zero padding outside the image ("same" size), averaged over
# pixels and channels; L1 averaged the same way; lambda = 0.2.  Both terms
# act on the composited RGB (C + T bg); opacity is not part of the loss.
# ---------------------------------------------------------------------------
SSIM_WIN, SSIM_SIGMA, SSIM_C1, SSIM_C2 = 11, 1.5, 0.01 ** 2, 0.03 ** 2


def ssim_window(size: int = SSIM_WIN, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """Normalised 1-D Gaussian taps; the 2-D window is their outer product."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(img: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """Window-weighted local sum with zero padding, separable: rows then columns.
    img [H, W, C]."""
    H, W = img.shape[:2]
    r = len(w1) // 2
    pad = np.zeros((H + 2 * r, W + 2 * r) + img.shape[2:])
    pad[r:r + H, r:r + W] = img
    tmp = sum(w1[k] * pad[:, k:k + W] for k in range(len(w1)))
    return sum(w1[k] * tmp[k:k + H] for k in range(len(w1)))


def ssim_terms(x: np.ndarray, y: np.ndarray):
    """SSIM map of images x, y [H, W, C] (FP64) and its partial derivatives with
    respect to the local statistics of x: mean mu_x, E[x^2] and E[xy]."""
    w1 = ssim_window()
    mx, my = _blur(x, w1), _blur(y, w1)
    exx, eyy, exy = _blur(x * x, w1), _blur(y * y, w1), _blur(x * y, w1)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + SSIM_C1, 2 * cxy + SSIM_C2
    B1, B2 = mx * mx + my * my + SSIM_C1, vx + vy + SSIM_C2
    S = A1 * A2 / (B1 * B2)
    dS_dmx = S * (2 * my / A1 - 2 * my / A2 - 2 * mx / B1 + 2 * mx / B2)
    dS_dexx = -S / B2
    dS_dexy = 2 * S / A2
    return S, dS_dmx, dS_dexx, dS_dexy


def image_loss(pred: np.ndarray, target: np.ndarray, lam: float = 0.2):
    """(L, dL/dpred) of one view: L = (1 - lam) mean|pred - target| + lam (1 - mean SSIM),
    pred and target [H, W, 3]."""
    x = np.asarray(pred, dtype=np.float64)
    y = np.asarray(target, dtype=np.float64)
    n = x.size
    S, a, b, c = ssim_terms(x, y)
    w1 = ssim_window()
    # d mean(S) / dx_p = (1/n) sum_q w(q - p) [a_q + 2 x_p b_q + y_p c_q]  (w symmetric)
    dS = (_blur(a, w1) + 2.0 * x * _blur(b, w1) + y * _blur(c, w1)) / n
    L = (1.0 - lam) * np.abs(x - y).mean() + lam * (1.0 - S.mean())
    g = (1.0 - lam) * np.sign(x - y) / n - lam * dS
    return float(L), g
