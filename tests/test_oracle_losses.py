"""Pins of the oracle's isotropic loss (Eqs. 6-8) and densification statistic
(Eq. 11) against independent mathematics.

* r_max bounds the true AABB/ellipsoid volume ratio for every rotation (Monte
  Carlo over rotations, exact AABB from the rotated axes) and is approached
  by the worst rotation; it equals 6/pi for isotropic Gaussians;
* the loss vanishes below r0 and its gradient matches central differences;
* the densification weight alpha |grad mu| equals the norm of the loss's
  derivative by the image of the mean on a radius-f sphere centred at the
  camera (Supp. Sec. 3), when the gradient is tangential -- checked by
  differentiating through that central projection numerically.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import losses


def true_ratio(s, R):
    # AABB half-lengths of the ellipsoid with semi-axes s rotated by R: |R| s
    L = np.sqrt((R ** 2) @ (s ** 2))
    return np.prod(2 * L) / (4 * math.pi / 3 * np.prod(s))


def test_r_max_bounds_every_rotation_and_is_reached():
    rng = np.random.default_rng(0)
    for _ in range(20):
        s = np.exp(rng.normal(-3, 1, size=3))
        Rs = Rotation.random(4000, random_state=rng.integers(1 << 31)).as_matrix()
        ratios = np.array([true_ratio(s, R) for R in Rs])
        bound = losses.r_max(s[None])[0]
        assert ratios.max() <= bound * (1 + 1e-12)
        assert ratios.max() >= 0.85 * bound
    iso = np.full((5, 3), 0.37)
    np.testing.assert_allclose(losses.r_max(iso), 6 / math.pi, rtol=1e-14)


def test_isotropic_loss_values_and_gradient():
    rng = np.random.default_rng(1)
    s = np.exp(rng.normal(-3, 1.2, size=(64, 3)))
    s[:8] = 0.2  # isotropic: below the threshold
    loss, grad = losses.isotropic_loss(s, r0=10.0)
    r = losses.r_max(s)
    assert loss == pytest.approx(np.maximum(r - 10.0, 0).mean(), rel=1e-14)
    assert np.all(grad[:8] == 0)
    fd = np.zeros_like(s)
    for i in range(s.shape[0]):
        for j in range(3):
            h = 1e-7 * s[i, j]
            sp, sm = s.copy(), s.copy()
            sp[i, j] += h
            sm[i, j] -= h
            fd[i, j] = (losses.isotropic_loss(sp)[0] - losses.isotropic_loss(sm)[0]) / (2 * h)
    active = r > 10.0 * (1 + 1e-6)
    np.testing.assert_allclose(grad[active], fd[active], rtol=1e-5, atol=1e-9 * np.abs(grad).max())
    assert active.sum() > 10


def test_densification_weight_is_projected_gradient_norm():
    rng = np.random.default_rng(2)
    o = np.array([0.3, -1.0, 2.0])
    f = 700.0
    for _ in range(20):
        mu = rng.normal(size=3) * 2.0
        u = (mu - o) / np.linalg.norm(mu - o)
        g = rng.normal(size=3)
        g -= (g @ u) * u  # tangential gradient (Supp. Sec. 3's assumption)
        r = np.linalg.norm(mu - o)

        # L(mu) = g . mu locally; mu = F(mu_P, r) = o + r/f (mu_P - o); differentiate along
        # an orthonormal basis of the tangent plane at mu_P = o + f u
        def L_of_muP(muP):
            return g @ (o + r / f * (muP - o))
        muP = o + f * u
        e1 = np.cross(u, [1.0, 0.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(u, e1)
        h = 1e-3
        dP = [(L_of_muP(muP + h * e) - L_of_muP(muP - h * e)) / (2 * h) for e in (e1, e2)]
        proj_norm = math.hypot(*dP)
        stat, cnt = np.zeros(1), np.zeros(1, dtype=np.int64)
        losses.densify_update(mu[None], g[None], o, f, stat, cnt)
        assert stat[0] == pytest.approx(proj_norm, rel=1e-9)
        assert cnt[0] == 1
    # unobserved Gaussians (zero gradient) are not counted
    stat, cnt = np.zeros(2), np.zeros(2, dtype=np.int64)
    losses.densify_update(np.zeros((2, 3)), np.array([[0, 0, 0], [1e-3, 0, 0]]), o, f, stat, cnt)
    assert cnt.tolist() == [0, 1] and stat[0] == 0
