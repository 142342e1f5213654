"""Pin of the oracle's analytic adjoint against FP64 central finite differences.

The loss is L = sum_p <W_p, RGBA_p> with seeded W.  Finite differences replay
the schedule recorded at the unperturbed parameters (segment starts and steps
frozen, as the adjoint treats them as piecewise constant) and are rejected
per parameter if the set of (sample, Gaussian) pairs inside the truncation
changes under the perturbation.  A dropped term, a wrong sign or a transposed
factor anywhere in the adjoint fails this test.
"""
import numpy as np
import pytest

import oracle
from paper_2509_07782_b300 import synth

SIG_EPS = 1e-3


def cluster_scene(n=6, seed=0):
    rng = np.random.default_rng(seed)
    means = rng.normal(0, 0.12, size=(n, 3))
    scales = np.exp(rng.normal(-2.3, 0.3, size=(n, 3)))
    quats = rng.normal(size=(n, 4))
    dens = np.exp(rng.normal(1.5, 0.4, size=n))
    sh = rng.normal(0, 0.2, size=(n, 16, 3))
    return synth.Scene(means.astype(np.float64), scales, quats, dens, sh, 3)


def _loss(scene, cam, o_, W, sched, sched_n):
    r = oracle.render(scene, cam, o_, sched=sched, sched_n=sched_n)
    return float((W * r["rgba"]).sum()), r["active"]


@pytest.mark.parametrize("mode", ["uniform", "adaptive_skip"])
def test_adjoint_matches_central_differences(mode):
    sc = cluster_scene()
    cam = synth.look_at(np.array([0.2, -0.4, 1.6]), np.zeros(3), 22.0, 6, 6)
    if mode == "uniform":
        o_ = synth.Options(dt=0.004, n_s=8, t_eps=0.0, sigma_eps=SIG_EPS, bg=(0.3, 0.1, 0.6))
    else:
        o_ = synth.Options(adaptive=True, skip=True, dt_min=0.003, dt_max=0.012, beta=200.0, n_s=8,
                           t_eps=1e-3, sigma_eps=SIG_EPS, bg=(0.3, 0.1, 0.6))
    W = np.random.default_rng(7).normal(size=(cam.n_rays, 4))
    base = oracle.render(sc, cam, o_, sched_cap=512)
    assert base["rgba"][:, 3].max() > 0.3
    sched, sched_n = base["sched"], base["sched_n"]
    g = oracle.backward(sc, cam, o_, W)

    names = ["means", "scales", "quats", "densities", "sh"]
    arrays = [sc.means, sc.scales, sc.quats, sc.densities, sc.sh]
    checked = 0
    for name, arr in zip(names, arrays):
        an = g[name].reshape(-1)
        fd = np.full_like(an, np.nan)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(abs(flat[i]), 1e-2)
            vals = []
            ok = True
            for sgn in (+1, -1):
                pert = [a.copy() for a in arrays]
                pert[names.index(name)].reshape(-1)[i] += sgn * h
                ps = synth.Scene(*pert, 3)
                L, act = _loss(ps, cam, o_, W, sched, sched_n)
                if not np.array_equal(act, base["active"]):
                    ok = False
                vals.append(L)
            if ok:
                fd[i] = (vals[0] - vals[1]) / (2 * h)
        m = ~np.isnan(fd)
        assert m.mean() > 0.9, f"{name}: too many rejected perturbations"
        scale = np.abs(an[m]).max() + 1e-12
        err = np.abs(fd[m] - an[m]).max() / scale
        assert err < 2e-6, f"{name}: max rel err {err:.3g}"
        rel_l2 = np.linalg.norm(fd[m] - an[m]) / (np.linalg.norm(an[m]) + 1e-30)
        assert rel_l2 < 1e-6, f"{name}: rel L2 {rel_l2:.3g}"
        checked += int(m.sum())
    assert checked > 300


def test_clamped_colour_channels_get_no_sh_gradient():
    """c_l = max(0, 1/2 + sum_k Y_k K_lk) per channel: where a channel is clamped
    to 0 its SH coefficients do not move the render, so central differences and
    the adjoint both give exactly zero for them, while the unclamped channels
    still match central differences."""
    sc = cluster_scene(n=4, seed=3)
    sh = sc.sh.copy()
    sh[:, 0, 1] = -6.0  # green DC far below the offset: green clamped in every direction
    sc = synth.Scene(sc.means, sc.scales, sc.quats, sc.densities, sh, 3)
    cam = synth.look_at(np.array([0.2, -0.4, 1.6]), np.zeros(3), 22.0, 5, 5)
    o_ = synth.Options(dt=0.004, n_s=8, t_eps=0.0, sigma_eps=SIG_EPS)
    W = np.random.default_rng(8).normal(size=(cam.n_rays, 4))
    base = oracle.render(sc, cam, o_, sched_cap=512)
    assert np.all(base["rgba"][:, 1] == 0.0) and base["rgba"][:, 0].max() > 0.05
    g = oracle.backward(sc, cam, o_, W)["sh"]
    np.testing.assert_array_equal(g[:, :, 1], 0.0)
    assert np.abs(g[:, :, 0]).max() > 1e-4
    rng = np.random.default_rng(0)
    for _ in range(12):
        l, k, c = int(rng.integers(4)), int(rng.integers(16)), int(rng.integers(2))
        h = 1e-6
        vals = []
        for sgn in (1, -1):
            pert = sh.copy()
            pert[l, k, c] += sgn * h
            L, _ = _loss(synth.Scene(sc.means, sc.scales, sc.quats, sc.densities, pert, 3), cam, o_, W,
                         base["sched"], base["sched_n"])
            vals.append(L)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[l, k, c]) <= 1e-6 * max(1.0, abs(g[:, :, 0]).max())
