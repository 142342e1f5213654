"""Pins of the oracle's per-Gaussian geometry against independent mathematics.

* rotation of a quaternion vs scipy's Rotation;
* the Q_eps quadratic form vs scipy's multivariate normal with
  Sigma = R S S^T R^T (Supp. Sec. 2.1);
* minimal AABB half-lengths (Supp. Sec. 2.2) vs dense sampling of the
  ellipsoid surface;
* AABB/ellipsoid volume ratio and its rotation-invariant bound (Sec. 3.4,
  Supp. Sec. 2.1 and 2.3), with equality for isotropic Gaussians;
* ellipsoid volume (Supp. Sec. 2.1) vs Monte Carlo;
* ray chords vs root bracketing of q(t) - Q_eps.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.spatial.transform import Rotation
from scipy.stats import multivariate_normal

import oracle
from paper_2509_07782_b300 import synth

SIG_EPS = 1e-3


def small_scene(n=16, seed=3, log_s=-2.0):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.5, 0.5, size=(n, 3))
    scales = np.exp(rng.normal(log_s, 0.6, size=(n, 3)))
    quats = rng.normal(size=(n, 4))  # unnormalised on purpose
    dens = np.exp(rng.normal(1.0, 0.5, size=n))
    sh = rng.normal(0, 0.2, size=(n, 16, 3))
    return synth.Scene(means, scales, quats, dens, sh, 3)


def test_quat_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.normal(size=4) * rng.uniform(0.1, 5.0)
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: scalar last
        np.testing.assert_allclose(R, ref, atol=1e-13)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1) < 1e-13


def test_quadratic_form_matches_multivariate_normal():
    sc = small_scene()
    R, M, Qe, _ = oracle.prim_geometry(sc, SIG_EPS)
    rng = np.random.default_rng(1)
    for l in range(sc.n):
        Rs = Rotation.from_quat(np.r_[sc.quats[l, 1:], sc.quats[l, 0]]).as_matrix()
        Sigma = Rs @ np.diag(sc.scales[l] ** 2) @ Rs.T
        mvn = multivariate_normal(mean=sc.means[l], cov=Sigma)
        norm = (2 * math.pi) ** 1.5 * math.sqrt(np.linalg.det(Sigma))
        x = sc.means[l] + rng.normal(size=(20, 3)) * sc.scales[l].max()
        y = (x - sc.means[l]) @ M[l].T
        q = (y * y).sum(1)
        np.testing.assert_allclose(np.exp(-0.5 * q), mvn.pdf(x) * norm, rtol=1e-9)
        assert Qe[l] == pytest.approx(2 * math.log(sc.densities[l] / SIG_EPS), rel=1e-14)


def test_aabb_half_lengths_vs_surface_sampling():
    sc = small_scene(n=8)
    R, M, Qe, half = oracle.prim_geometry(sc, SIG_EPS)
    rng = np.random.default_rng(2)
    z = rng.normal(size=(400_000, 3))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    for l in range(sc.n):
        # surface points x = mu + R diag(s~) z, |z| = 1  (s~ = sqrt(Q_eps) s)
        pts = (z * (math.sqrt(Qe[l]) * sc.scales[l])) @ R[l].T
        ext = np.abs(pts).max(0)
        assert np.all(ext <= half[l] * (1 + 1e-12))
        np.testing.assert_allclose(ext, half[l], rtol=2e-3)


def test_volume_ratio_and_bound():
    rng = np.random.default_rng(4)
    sc = small_scene(n=64)
    R, M, Qe, half = oracle.prim_geometry(sc, SIG_EPS)
    for l in range(sc.n):
        s = sc.scales[l]
        vol_box = np.prod(2 * half[l])
        vol_ell = 4 * math.pi / 3 * Qe[l] ** 1.5 * np.prod(s)
        r = vol_box / vol_ell
        # closed form of the ratio (independent of sigma~ and sigma_eps)
        li = (R[l] ** 2 * s[None, :] ** 2).sum(1)
        r_cf = 6 / math.pi * math.sqrt(np.prod(li)) / np.prod(s)
        assert r == pytest.approx(r_cf, rel=1e-10)
        bound = 2 / (math.pi * math.sqrt(3)) * (s @ s) ** 1.5 / np.prod(s)
        assert r <= bound * (1 + 1e-12)
    # isotropic scales reach the bound for every rotation
    iso = small_scene(n=10)
    iso.scales = np.repeat(rng.uniform(0.01, 0.1, size=(10, 1)), 3, axis=1)
    R, M, Qe, half = oracle.prim_geometry(iso, SIG_EPS)
    for l in range(iso.n):
        s = iso.scales[l]
        r = np.prod(2 * half[l]) / (4 * math.pi / 3 * Qe[l] ** 1.5 * np.prod(s))
        bound = 2 / (math.pi * math.sqrt(3)) * (s @ s) ** 1.5 / np.prod(s)
        assert r == pytest.approx(bound, rel=1e-10)
        assert r == pytest.approx(6 / math.pi, rel=1e-10)


def test_ellipsoid_volume_monte_carlo():
    sc = small_scene(n=4, seed=9)
    R, M, Qe, half = oracle.prim_geometry(sc, SIG_EPS)
    rng = np.random.default_rng(5)
    for l in range(sc.n):
        pts = rng.uniform(-1, 1, size=(400_000, 3)) * half[l]
        y = pts @ M[l].T
        inside = ((y * y).sum(1) <= Qe[l]).mean()
        vol_mc = inside * np.prod(2 * half[l])
        vol = 4 * math.pi / 3 * Qe[l] ** 1.5 * np.prod(sc.scales[l])
        assert vol_mc == pytest.approx(vol, rel=0.01)


def test_chords_vs_root_bracketing():
    sc = small_scene(n=12, seed=11, log_s=-1.5)
    R, M, Qe, _ = oracle.prim_geometry(sc, SIG_EPS)
    rng = np.random.default_rng(6)
    nfound = 0
    for trial in range(40):
        o = rng.normal(size=3) * 2.0
        tgt = sc.means[rng.integers(sc.n)] + rng.normal(size=3) * 0.05
        d = tgt - o
        d /= np.linalg.norm(d)
        tin, tout = oracle.chords(sc, SIG_EPS, o, d)
        ts = np.linspace(-10, 10, 400_001)  # grid step 5e-5
        for l in range(sc.n):
            def f(t):
                y = M[l] @ (o + t * d - sc.means[l])
                return y @ y - Qe[l]
            Y = (o[None, :] + ts[:, None] * d[None, :] - sc.means[l]) @ M[l].T
            neg = (Y * Y).sum(1) - Qe[l] < 0
            if not neg.any():
                # no sampled point inside: either no chord or one shorter than the grid step
                assert np.isnan(tin[l]) or (tout[l] - tin[l]) < 1e-4
                continue
            idx = np.nonzero(neg)[0]
            r0 = brentq(f, ts[idx[0] - 1], ts[idx[0]], xtol=1e-14)
            r1 = brentq(f, ts[idx[-1]], ts[idx[-1] + 1], xtol=1e-14)
            assert tin[l] == pytest.approx(r0, abs=1e-9)
            assert tout[l] == pytest.approx(r1, abs=1e-9)
            nfound += 1
    assert nfound > 20
