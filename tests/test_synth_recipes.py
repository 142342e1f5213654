"""The seeded workload generators follow their stated recipes.

The synthetic scenes stand in for the paper's datasets, so their recipe (the
distributions of means, scales, densities and SH coefficients, the camera
placement and resolutions, the seeds) is part of what the measurements mean.
These checks hold the generators to it on samples large enough that the
sample moments are tight; they need no GPU.
"""
import math

import numpy as np
import pytest

from paper_2509_07782_b300 import synth


def _moments(x):
    x = np.asarray(x, np.float64).ravel()
    return x.mean(), x.std()


def test_generators_are_deterministic():
    for name, n in (("plain_2k", None), ("torus_100k", 5000), ("outdoor_3m", 5000), ("sweep_6m", 1000)):
        a, b = synth.workload(name, n=n), synth.workload(name, n=n)
        for f in ("means", "scales", "quats", "densities", "sh"):
            np.testing.assert_array_equal(getattr(a.scene, f), getattr(b.scene, f))
        for ca, cb in zip(a.cameras, b.cameras):
            np.testing.assert_array_equal(ca.c2w, cb.c2w)
            assert (ca.width, ca.height, ca.fx) == (cb.width, cb.height, cb.fx)


def test_cube_recipe():
    w = synth.workload("plain_2k")
    sc = w.scene
    assert sc.n == 2000 and sc.means.dtype == np.float32
    assert np.all(np.abs(sc.means) <= 1.0)
    m, s = _moments(np.log(sc.scales))
    assert abs(m + 3.0) < 0.03 and abs(s - 0.5) < 0.02
    m, s = _moments(np.log(sc.densities))
    assert abs(m - 1.0) < 0.05 and abs(s - 0.5) < 0.03
    cam = w.cameras[0]
    assert (cam.width, cam.height) == (64, 64)
    assert np.linalg.norm(cam.c2w[:, 3]) == pytest.approx(3.0, rel=1e-6)
    assert cam.fx == pytest.approx(32 / math.tan(math.radians(25.0)), rel=1e-6)
    assert not w.options.skip and not w.options.adaptive and w.options.dt == 0.01 and w.options.n_s == 16


def test_torus_recipe():
    w = synth.workload("torus_100k", n=40000)
    sc = w.scene
    x, y, z = sc.means.astype(np.float64).T
    tube = np.sqrt((np.hypot(x, y) - 1.0) ** 2 + z ** 2)  # distance from the major circle
    m, s = _moments(tube)
    assert abs(m - 0.35) < 0.002 and 0.009 < s < 0.02
    assert np.all(np.abs(tube - 0.35) < 0.03 + 6 * 0.01)
    m, s = _moments(np.log(sc.scales))
    assert abs(m + 4.5) < 0.01 and abs(s - 0.4) < 0.01
    m, s = _moments(np.log(sc.densities))
    assert abs(m - 2.0) < 0.02 and abs(s - 0.7) < 0.02
    m, s = _moments(sc.sh)
    assert abs(m) < 0.003 and abs(s - 0.2) < 0.003
    np.testing.assert_allclose(np.linalg.norm(sc.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    cam = w.cameras[0]
    pos = cam.c2w[:, 3].astype(np.float64)
    assert (cam.width, cam.height) == (800, 800)
    assert np.linalg.norm(pos) == pytest.approx(4.0, rel=1e-6)
    assert -30.0 <= math.degrees(math.asin(pos[2] / 4.0)) <= 60.0
    # the camera looks at the origin: its forward axis points there
    np.testing.assert_allclose(cam.c2w[:, 2], -pos / 4.0, atol=1e-6)
    o = w.options
    assert o.skip and o.adaptive and o.morton and o.ztiles and not o.morton63
    assert (o.dt_min, o.dt_max, o.beta) == (0.005, 0.02, 1024.0)
    assert w.cameras[0].n_rays == 640_000


def test_outdoor_recipe():
    w = synth.workload("outdoor_3m", n=60000)
    r = np.linalg.norm(w.scene.means.astype(np.float64), axis=1)
    fg, bg = r[:36000], r[36000:]
    assert np.all(fg < 1.0 + 6 * 0.15)  # blob centres in the unit ball, blob sd <= 0.15
    assert bg.min() >= 1.0 * (1 - 1e-6) and bg.max() <= 100.0 * (1 + 1e-6)
    m, s = _moments(np.log(bg))  # log-uniform radius on [1, 100]
    assert abs(m - math.log(100.0) / 2) < 0.03 and abs(s - math.log(100.0) / math.sqrt(12)) < 0.03
    resid = np.log(w.scene.scales.astype(np.float64)) - (-4.5 + np.log(np.maximum(r, 1.0)))[:, None]
    m, s = _moments(resid)
    assert abs(m) < 0.01 and abs(s - 0.4) < 0.01
    m, s = _moments(np.log(w.scene.densities))
    assert abs(m - 1.0) < 0.03 and abs(s - 1.0) < 0.03
    cam = w.cameras[0]
    assert (cam.width, cam.height) == (1237, 822) and cam.n_rays == 1_016_814
    assert np.linalg.norm(cam.c2w[:, 3]) <= 0.3 + 1e-6
    assert w.options.morton63


def test_multi_view_recipes():
    b = synth.workload("batch_1m", n=1000)
    assert [(c.width, c.height) for c in b.cameras] == synth.BATCH_RES
    assert sum(c.n_rays for c in b.cameras) == 7_082_990
    s = synth.workload("sweep_6m", n=1000)
    assert len(s.cameras) == 64
    assert all(256 <= c.width <= 1920 and 256 <= c.height <= 1080 for c in s.cameras)
    for c in b.cameras + s.cameras:
        assert np.linalg.norm(c.c2w[:, 3]) == pytest.approx(4.0, rel=1e-6)
        assert c.fx == pytest.approx(0.5 * c.height / math.tan(math.radians(25.0)), rel=1e-6)
    assert not s.backward and b.backward
