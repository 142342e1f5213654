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
