"""Pins of the oracle's real spherical harmonics (the c_l(d) of Eq. 1).

The oracle builds Y_k from the normalisation formula and associated Legendre
recurrences.  These tests tie it to scipy's complex spherical harmonics and
to orthonormality on the sphere, so a wrong constant, sign or index fails.
"""
import math

import numpy as np
from scipy.special import sph_harm_y

import oracle


def real_sh_scipy(l, m, d):
    x, y, z = d / np.linalg.norm(d)
    theta, phi = math.acos(max(-1.0, min(1.0, z))), math.atan2(y, x)
    if m > 0:
        return math.sqrt(2) * sph_harm_y(l, m, theta, phi).real
    if m < 0:
        return math.sqrt(2) * sph_harm_y(l, -m, theta, phi).imag
    return sph_harm_y(l, 0, theta, phi).real


def test_sh_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(200):
        d = rng.normal(size=3)
        Y = oracle.sh_basis(d, 3)
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - real_sh_scipy(l, m, d)) < 1e-12


def test_sh_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            Y = oracle.sh_basis([st * math.cos(ph), st * math.sin(ph), ct], 3)
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_low_order_closed_forms():
    # textbook polynomials for l <= 1 with the Condon-Shortley phase
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    for d in ([0.3, -0.5, 0.81], [1, 0, 0], [0, 0, -1]):
        d = np.asarray(d, float) / np.linalg.norm(d)
        Y = oracle.sh_basis(d, 1)
        np.testing.assert_allclose(Y, [c0, -c1 * d[1], c1 * d[2], -c1 * d[0]], atol=1e-15)
