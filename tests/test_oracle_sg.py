"""Pins of the oracle's spherical-Gaussian appearance term (Eq. 1's c_l "with
SH/SG"; Supp. Sec. 6.1 uses nine SH and seven SG per primitive).

Reading: c_l(d) = max(0, 1/2 + sum_k Y_k(d) K_lk + sum_j a_lj exp(lambda_lj
(mu_lj . d - 1))), mu_lj = u_lj / |u_lj| from a raw axis u, d the ray direction.

* closed form: a single Gaussian has one colour along a ray, so the render is
  c(d) (1 - T) + T bg exactly; c(d) is computed here from the lobe formula with
  the ray direction built independently from the pinhole model;
* special values: along the axis a lobe gives a, perpendicular a e^-lambda,
  against it a e^-2 lambda;
* the adjoint of the lobe parameters against FP64 central differences on the
  frozen schedule (with the SH, geometry and density gradients unchanged).
"""
import numpy as np
import pytest

import oracle
from paper_2509_07782_b300 import synth


def _dirs(cam):
    """Unit ray directions of every pixel, built from the pinhole model here."""
    u, v = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    dc = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u)], -1).reshape(-1, 3)
    R = np.asarray(cam.c2w, np.float64)[:, :3]
    d = dc @ R.T
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _one_gaussian(sg, sh0=(0.1, -0.2, 0.05)):
    n_sg = sg.shape[0]
    sh = np.zeros((1, 1, 3))
    sh[0, 0] = sh0
    return synth.Scene(np.zeros((1, 3)), np.full((1, 3), 0.3), np.array([[1.0, 0, 0, 0]]), np.array([4.0]),
                       sh, 0, sg.reshape(1, n_sg, 7))


def test_single_gaussian_render_is_the_lobe_closed_form():
    sg = np.array([[0.3, -1.2, 0.8, 6.0, 0.4, -0.1, 0.25],
                   [-2.0, 0.5, 1.0, 1.5, -0.2, 0.3, 0.1]])
    scene = _one_gaussian(sg)
    cam = synth.look_at(np.array([0.4, -0.3, 2.2]), np.zeros(3), 40.0, 16, 16)
    o = synth.Options(dt=0.002, n_s=8, t_eps=0.0, bg=(0.2, 0.3, 0.1))
    r = oracle.render(scene, cam, o)
    d = _dirs(cam)
    Y0 = 0.5 / np.sqrt(np.pi)
    pre = 0.5 + Y0 * np.asarray(scene.sh[0, 0])[None, :]
    for u, lam, a in ((sg[j, :3], sg[j, 3], sg[j, 4:]) for j in range(len(sg))):
        mu = u / np.linalg.norm(u)
        pre = pre + a[None, :] * np.exp(lam * (d @ mu - 1.0))[:, None]
    c = np.maximum(pre, 0.0)
    A = r["rgba"][:, 3]
    assert A.max() > 0.5 and A.min() < 0.05
    expect = c * A[:, None] + (1.0 - A[:, None]) * np.asarray(o.bg)[None, :]
    np.testing.assert_allclose(r["rgba"][:, :3], expect, rtol=0, atol=1e-12)
    # the lobes really change the colour across the image
    assert np.ptp(c[A > 0.5], axis=0).max() > 0.01


@pytest.mark.parametrize("where,factor", [("along", 0.0), ("perpendicular", -1.0), ("against", -2.0)])
def test_lobe_special_values(where, factor):
    cam = synth.look_at(np.array([0.0, 0.0, 3.0]), np.zeros(3), 10.0, 1, 1)
    d = _dirs(cam)[0]                     # (0, 0, -1) up to rounding
    axis = {"along": d, "perpendicular": np.cross(d, [1.0, 0.0, 0.0]), "against": -d}[where]
    lam, a = 3.0, np.array([0.3, 0.2, -0.1])
    sg = np.concatenate([2.5 * axis, [lam], a])[None, :]   # raw axis of length 2.5
    scene = _one_gaussian(sg, sh0=(0.0, 0.0, 0.0))
    o = synth.Options(dt=0.002, n_s=8, t_eps=0.0)
    r = oracle.render(scene, cam, o)
    A = r["rgba"][0, 3]
    assert A > 0.5
    np.testing.assert_allclose(r["rgba"][0, :3] / A, 0.5 + a * np.exp(lam * factor), rtol=1e-10)


def _loss(scene, cam, o_, W, sched, sched_n):
    r = oracle.render(scene, cam, o_, sched=sched, sched_n=sched_n)
    return float((W * r["rgba"]).sum()), r["active"]


def test_lobe_adjoint_matches_central_differences():
    rng = np.random.default_rng(5)
    n = 5
    base = synth.Scene(rng.normal(0, 0.12, size=(n, 3)), np.exp(rng.normal(-2.3, 0.3, size=(n, 3))),
                       rng.normal(size=(n, 4)), np.exp(rng.normal(1.5, 0.4, size=n)),
                       rng.normal(0, 0.2, size=(n, 16, 3)), 3)
    sc = synth.with_sg_appearance(base, seed=9, n_sg=3)
    sc = synth.Scene(*(np.asarray(a, np.float64) for a in (sc.means, sc.scales, sc.quats, sc.densities, sc.sh)),
                     sc.sh_degree, np.asarray(sc.sg, np.float64))
    cam = synth.look_at(np.array([0.2, -0.4, 1.6]), np.zeros(3), 22.0, 6, 6)
    o_ = synth.Options(dt=0.004, n_s=8, t_eps=0.0, sigma_eps=1e-3, bg=(0.3, 0.1, 0.6))
    W = np.random.default_rng(7).normal(size=(cam.n_rays, 4))
    ref = oracle.render(sc, cam, o_, sched_cap=512)
    assert ref["rgba"][:, 3].max() > 0.3
    g = oracle.backward(sc, cam, o_, W)
    an = g["sg"].reshape(-1)
    flat = sc.sg.reshape(-1)
    fd = np.full_like(an, np.nan)
    for i in range(flat.size):
        h = 1e-6 * max(abs(flat[i]), 1e-2)
        vals, ok = [], True
        for sgn in (1, -1):
            p = sc.sg.copy()
            p.reshape(-1)[i] += sgn * h
            L, act = _loss(synth.Scene(sc.means, sc.scales, sc.quats, sc.densities, sc.sh, sc.sh_degree, p),
                           cam, o_, W, ref["sched"], ref["sched_n"])
            ok &= bool(np.array_equal(act, ref["active"]))
            vals.append(L)
        if ok:
            fd[i] = (vals[0] - vals[1]) / (2 * h)
    m = ~np.isnan(fd)
    assert m.mean() > 0.9
    scale = np.abs(an[m]).max()
    assert scale > 1e-4
    assert np.abs(fd[m] - an[m]).max() / scale < 2e-6
    # the axis gradient is orthogonal to the axis (the length of u does not matter)
    u = sc.sg[:, :, :3]
    gu = g["sg"][:, :, :3]
    assert np.abs((u * gu).sum(-1)).max() <= 1e-12 * max(np.abs(gu).max(), 1e-30) * 10


def test_clamped_channel_gets_no_lobe_gradient():
    """Where a colour channel is clamped at 0 no lobe parameter moves it: the
    adjoint gives that channel's amplitudes exactly zero, and the sharpness and
    axis gradients agree with central differences (which see only the other
    channels)."""
    rng = np.random.default_rng(3)
    n = 4
    sh = rng.normal(0, 0.2, size=(n, 16, 3))
    sh[:, 0, 1] = -6.0  # green DC far below the offset: green clamped in every direction
    base = synth.Scene(rng.normal(0, 0.12, size=(n, 3)), np.exp(rng.normal(-2.3, 0.3, size=(n, 3))),
                       rng.normal(size=(n, 4)), np.exp(rng.normal(1.5, 0.4, size=n)), sh, 3)
    sc = synth.with_sg_appearance(base, seed=4, n_sg=2, sh_degree=3)
    sg = np.asarray(sc.sg, np.float64)
    sg[:, :, 5] = np.clip(sg[:, :, 5], -0.1, 0.1)  # green lobes cannot lift it above 0
    sc = synth.Scene(base.means, base.scales, base.quats, base.densities, sh, 3, sg)
    cam = synth.look_at(np.array([0.2, -0.4, 1.6]), np.zeros(3), 22.0, 5, 5)
    o_ = synth.Options(dt=0.004, n_s=8, t_eps=0.0, sigma_eps=1e-3)
    W = np.random.default_rng(8).normal(size=(cam.n_rays, 4))
    base_r = oracle.render(sc, cam, o_, sched_cap=512)
    assert np.all(base_r["rgba"][:, 1] == 0.0) and base_r["rgba"][:, 0].max() > 0.05
    g = oracle.backward(sc, cam, o_, W)["sg"]
    np.testing.assert_array_equal(g[:, :, 5], 0.0)
    assert np.abs(g[:, :, 4]).max() > 1e-5
    for (l, j, c) in ((0, 0, 3), (1, 1, 0), (2, 0, 2), (3, 1, 3), (0, 1, 1)):
        h = 1e-6 * max(abs(sg[l, j, c]), 1e-2)
        vals = []
        for sgn in (1, -1):
            p = sg.copy()
            p[l, j, c] += sgn * h
            L, _ = _loss(synth.Scene(base.means, base.scales, base.quats, base.densities, sh, 3, p), cam, o_, W,
                         base_r["sched"], base_r["sched_n"])
            vals.append(L)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[l, j, c]) <= 1e-6 * max(1.0, np.abs(g).max())
