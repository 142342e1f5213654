"""Parity at the full sizes of the large workloads, through the paths a user
calls, against the FP64 oracle (max-abs 1e-4 on RGBA, relative L2 1e-3 per
gradient tensor):

* the 3M-Gaussian outdoor view at full size (63-bit codes) with a 128-entry
  hit list, so most segments overflow the list: chunked segments and the
  adjoint's per-warp chunk scratch are both exercised;
* the 1M-Gaussian batch of 8 uneven views in ONE persistent forward and ONE
  adjoint launch, against the sum over views of the oracle's gradients;
* the torch.autograd.Function (render() + loss.backward()) against the
  oracle's analytic gradient, and on a tiny scene against FP64 central
  differences of the oracle on the frozen schedule;
* the autotuner with N_S tuning on: parity at the N_S it picked (N_S changes
  the result in adaptive mode, so the oracle runs at that N_S).

The loss is L = sum_p <W_p, RGBA_p> over seeded pixels (W ~ N(0,1), zero
elsewhere).  In adaptive mode only pixels whose GPU schedule agrees with the
oracle's carry weight (a schedule that differs by rounding is another,
equally valid, piecewise-constant branch, reading R14); at least 99 % must.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2509_07782_b300 import autograd, rgx, synth
from helpers import (TOL_GRAD, TOL_RGBA, compare_rgba, gpu_backward, gpu_render, rel_l2, schedules_agree,
                     record_divergence, record_parity)

pytestmark = pytest.mark.gpu

NAMES = ["means", "scales", "quats", "densities", "sh"]


def _weights(rng, n, agree):
    W = rng.normal(size=(n, 4))
    W[~agree] = 0.0
    return W


def test_outdoor_3m_full_size_chunked_gradients():
    w = synth.workload("outdoor_3m")
    cam = w.cameras[0]
    o = dataclasses.replace(w.options, hit_cap=128)
    r = gpu_render(w.scene, [cam], o, sched_cap=96)
    assert r["status"] == 0
    pix = synth.pixel_subset(cam, 320, seed=21)
    params = oracle.Params(w.scene)
    err, ndiv = compare_rgba(r["rgba"], cam, w.scene, o, pix=pix, gpu_sched=r["sched"],
                             gpu_sched_n=r["sched_n"], params=params)
    record_divergence("outdoor_3m full, hit_cap 128, forward", ndiv, len(pix))
    assert err <= TOL_RGBA
    ref = oracle.render(w.scene, cam, o, pix=pix, sched_cap=96, params=params)
    agree = schedules_agree(r["sched"], r["sched_n"], ref["sched"], ref["sched_n"], pix)
    assert agree.mean() >= 0.99, f"only {agree.mean():.4f} of schedules agree"
    W = _weights(np.random.default_rng(22), len(pix), agree)
    d = np.zeros((cam.n_rays, 4))
    d[pix] = W
    cnt = r["scene"].counters()
    g = gpu_backward(r, d)
    assert g["status"] == 0
    gr = oracle.backward(w.scene, cam, o, W, pix=pix, params=params)
    errs = {k: rel_l2(g[k], gr[k]) for k in NAMES}
    record_parity("outdoor_3m full, hit_cap 128, 320 px", "max-abs RGBA", err)
    record_parity("outdoor_3m full, hit_cap 128, 320 px", "worst gradient rel L2", max(errs.values()))
    for k in NAMES:
        assert np.linalg.norm(gr[k]) > 0, k
        assert errs[k] <= TOL_GRAD, f"{k}: rel L2 {errs[k]:.3g} ({errs})"
    # the dense regime really ran: segments with more hits than the list holds
    assert cnt["hits"] > 128 * cnt["segments"] * 0.5


def test_batch_1m_one_launch_adjoint_matches_oracle_sum_over_views():
    w = synth.workload("batch_1m")
    r = gpu_render(w.scene, w.cameras, w.options, sched_cap=48)
    assert r["status"] == 0
    offs = np.concatenate([[0], np.cumsum([c.n_rays for c in w.cameras])])
    params = oracle.Params(w.scene)
    rng = np.random.default_rng(31)
    d = np.zeros((int(offs[-1]), 4))
    per_view = []
    for ci, cam in enumerate(w.cameras):
        pix = synth.pixel_subset(cam, 24, seed=300 + ci)
        sl = slice(offs[ci], offs[ci + 1])
        ref = oracle.render(w.scene, cam, w.options, pix=pix, sched_cap=48, params=params)
        agree = schedules_agree(r["sched"][sl], r["sched_n"][sl], ref["sched"], ref["sched_n"], pix)
        assert agree.mean() >= 0.95, f"view {ci}: {agree.mean():.3f} of schedules agree"
        W = _weights(rng, len(pix), agree)
        d[offs[ci] + pix] = W
        per_view.append((cam, pix, W))
    g = gpu_backward(r, d)
    assert g["status"] == 0
    total = {k: 0.0 for k in NAMES}
    for cam, pix, W in per_view:
        gv = oracle.backward(w.scene, cam, w.options, W, pix=pix, params=params)
        for k in NAMES:
            total[k] = total[k] + gv[k]
    errs = {k: rel_l2(g[k], total[k]) for k in NAMES}
    record_parity("batch_1m one-launch adjoint, 8 views x 24 px", "worst gradient rel L2", max(errs.values()))
    for k in NAMES:
        assert np.linalg.norm(total[k]) > 0, k
        assert errs[k] <= TOL_GRAD, f"{k}: rel L2 {errs[k]:.3g} ({errs})"


def _leaf_tensors(scene):
    return [t.clone().requires_grad_(True) for t in rgx.scene_tensors(scene)]


def test_autograd_function_matches_oracle_gradient():
    w = synth.workload("torus_100k", n=40_000, scale_res=0.3)
    cam = w.cameras[0]
    opts = rgx.make_opts(w.options)
    cams = rgx.Cameras([cam])
    leaves = _leaf_tensors(w.scene)
    sc = rgx.Scene()
    rgba = autograd.render(sc, cams, opts, *leaves)
    assert rgba.shape == (cam.n_rays, 4) and rgba.requires_grad
    pix = synth.pixel_subset(cam, 1024, seed=41)
    params = oracle.Params(w.scene)
    ref = oracle.render(w.scene, cam, w.options, pix=pix, sched_cap=64, params=params)
    assert np.abs(rgba.detach().cpu().numpy()[pix] - ref["rgba"]).max() <= TOL_RGBA
    # schedules of the same render, recorded on a scene of its own (the autograd scene keeps
    # its tape for the adjoint)
    rs = gpu_render(w.scene, [cam], w.options, sched_cap=64)
    assert np.array_equal(rs["rgba"], rgba.detach().cpu().numpy().astype(np.float64))
    agree = schedules_agree(rs["sched"], rs["sched_n"], ref["sched"], ref["sched_n"], pix)
    assert agree.mean() >= 0.99
    W = _weights(np.random.default_rng(42), len(pix), agree)
    Wd = torch.zeros(cam.n_rays, 4, device="cuda")
    Wd[torch.as_tensor(pix, device="cuda")] = torch.as_tensor(W, dtype=torch.float32, device="cuda")
    loss = (rgba * Wd).sum()
    loss.backward()
    assert sc.status() == 0
    gr = oracle.backward(w.scene, cam, w.options, W, pix=pix, params=params)
    for k, leaf in zip(NAMES, leaves):
        assert leaf.grad is not None, k
        e = rel_l2(leaf.grad.cpu().numpy(), gr[k])
        assert e <= TOL_GRAD, f"{k}: rel L2 {e:.3g}"


def test_autograd_function_matches_central_differences_on_tiny_scene():
    rng = np.random.default_rng(0)
    n = 6
    scene = synth.Scene(rng.normal(0, 0.12, size=(n, 3)), np.exp(rng.normal(-2.3, 0.3, size=(n, 3))),
                        rng.normal(size=(n, 4)), np.exp(rng.normal(1.5, 0.4, size=n)),
                        rng.normal(0, 0.2, size=(n, 16, 3)), 3)
    # float32 parameters on both sides: the oracle promotes the same float32 values
    scene = synth.Scene(*(np.asarray(a, np.float32) for a in (scene.means, scene.scales, scene.quats,
                                                              scene.densities, scene.sh)), 3)
    cam = synth.look_at(np.array([0.2, -0.4, 1.6]), np.zeros(3), 22.0, 6, 6)
    o = synth.Options(dt=0.004, n_s=8, t_eps=0.0, sigma_eps=1e-3, bg=(0.3, 0.1, 0.6))
    leaves = _leaf_tensors(scene)
    sc = rgx.Scene()
    rgba = autograd.render(sc, rgx.Cameras([cam]), rgx.make_opts(o), *leaves)
    W = np.random.default_rng(7).normal(size=(cam.n_rays, 4))
    (rgba * torch.as_tensor(W, dtype=torch.float32, device="cuda")).sum().backward()
    assert sc.status() == 0
    base = oracle.render(scene, cam, o, sched_cap=512)
    assert np.abs(rgba.detach().cpu().numpy() - base["rgba"]).max() <= TOL_RGBA
    arrays = [np.asarray(a, np.float64) for a in (scene.means, scene.scales, scene.quats, scene.densities,
                                                  scene.sh)]
    for k, leaf, arr in zip(NAMES, leaves, arrays):
        flat = arr.reshape(-1)
        fd = np.full(flat.size, np.nan)
        for i in range(flat.size):
            h = 1e-6 * max(abs(flat[i]), 1e-2)
            vals, ok = [], True
            for sgn in (1, -1):
                pert = [a.copy() for a in arrays]
                pert[NAMES.index(k)].reshape(-1)[i] += sgn * h
                rr = oracle.render(synth.Scene(*pert, 3), cam, o, sched=base["sched"], sched_n=base["sched_n"])
                ok &= bool(np.array_equal(rr["active"], base["active"]))
                vals.append(float((W * rr["rgba"]).sum()))
            if ok:
                fd[i] = (vals[0] - vals[1]) / (2 * h)
        m = ~np.isnan(fd)
        assert m.mean() > 0.9, k
        g = leaf.grad.cpu().numpy().astype(np.float64).reshape(-1)
        e = np.linalg.norm(g[m] - fd[m]) / max(np.linalg.norm(fd[m]), 1e-30)
        assert e <= TOL_GRAD, f"{k}: rel L2 vs central differences {e:.3g}"


def test_tuned_segment_length_parity():
    """rgx_autotune with N_S tuning, then oracle parity (forward and adjoint) of the
    torus view at the N_S it picked."""
    w = synth.workload("torus_100k")
    cam = w.cameras[0]
    sc = rgx.Scene()
    t = rgx.scene_tensors(w.scene)
    base = rgx.make_opts(w.options)
    sc.build(*t, base)
    best, ms = sc.autotune(rgx.Cameras([cam]), base, tune_ns=True, with_backward=True)
    assert ms > 0 and best.n_s in (4, 8, 16, 32)
    o = dataclasses.replace(w.options, n_s=int(best.n_s), hit_cap=int(best.hit_cap), tile_w=int(best.tile_w),
                            tile_h=int(best.tile_h), lower_first=bool(best.flags & rgx.RGX_LOWER_FIRST))
    r = gpu_render(w.scene, [cam], o, sched_cap=128)
    assert r["status"] == 0
    params = oracle.Params(w.scene)
    pix = synth.pixel_subset(cam, 2048, seed=51)
    err, ndiv = compare_rgba(r["rgba"], cam, w.scene, o, pix=pix, gpu_sched=r["sched"],
                             gpu_sched_n=r["sched_n"], params=params)
    record_divergence(f"torus_100k at tuned N_S={best.n_s}, forward", ndiv, len(pix))
    assert err <= TOL_RGBA
    pix = pix[:768]
    ref = oracle.render(w.scene, cam, o, pix=pix, sched_cap=128, params=params)
    agree = schedules_agree(r["sched"], r["sched_n"], ref["sched"], ref["sched_n"], pix)
    assert agree.mean() >= 0.99
    W = _weights(np.random.default_rng(52), len(pix), agree)
    d = np.zeros((cam.n_rays, 4))
    d[pix] = W
    g = gpu_backward(r, d)
    assert g["status"] == 0
    gr = oracle.backward(w.scene, cam, o, W, pix=pix, params=params)
    for k in NAMES:
        e = rel_l2(g[k], gr[k])
        assert e <= TOL_GRAD, f"{k}: rel L2 {e:.3g}"


def test_batch_1m_at_the_bench_knobs():
    """The 8-view batch at the knobs its benchmark line tunes to (N_S = 32, hit_cap 32,
    32x1 tiles; short lists, so the 168-register kernels run and almost every segment is
    chunked and taken from the forward's sums records in the adjoint): forward and adjoint
    against the oracle run at the same N_S."""
    w = synth.workload("batch_1m")
    o = dataclasses.replace(w.options, n_s=32, hit_cap=32, tile_w=32, tile_h=1)
    r = gpu_render(w.scene, w.cameras, o, sched_cap=32)
    assert r["status"] == 0
    offs = np.concatenate([[0], np.cumsum([c.n_rays for c in w.cameras])])
    params = oracle.Params(w.scene)
    rng = np.random.default_rng(81)
    d = np.zeros((int(offs[-1]), 4))
    per_view = []
    ndiv_all, n_all, worst = 0, 0, 0.0
    for ci, cam in enumerate(w.cameras):
        pix = synth.pixel_subset(cam, 24, seed=800 + ci)
        sl = slice(offs[ci], offs[ci + 1])
        err, ndiv = compare_rgba(r["rgba"][sl], cam, w.scene, o, pix=pix, gpu_sched=r["sched"][sl],
                                 gpu_sched_n=r["sched_n"][sl], params=params)
        assert err <= TOL_RGBA
        ndiv_all += ndiv
        n_all += len(pix)
        worst = max(worst, err)
        ref = oracle.render(w.scene, cam, o, pix=pix, sched_cap=32, params=params)
        agree = schedules_agree(r["sched"][sl], r["sched_n"][sl], ref["sched"], ref["sched_n"], pix)
        assert agree.mean() >= 0.95
        W = _weights(rng, len(pix), agree)
        d[offs[ci] + pix] = W
        per_view.append((cam, pix, W))
    record_divergence("batch_1m at N_S=32, hit_cap 32", ndiv_all, n_all)
    g = gpu_backward(r, d)
    assert g["status"] == 0
    total = {k: 0.0 for k in NAMES}
    for cam, pix, W in per_view:
        gv = oracle.backward(w.scene, cam, o, W, pix=pix, params=params)
        for k in NAMES:
            total[k] = total[k] + gv[k]
    errs = {k: rel_l2(g[k], total[k]) for k in NAMES}
    record_parity("batch_1m at the bench knobs (N_S 32, hit_cap 32)", "max-abs RGBA", worst)
    record_parity("batch_1m at the bench knobs (N_S 32, hit_cap 32)", "worst gradient rel L2", max(errs.values()))
    for k in NAMES:
        assert errs[k] <= TOL_GRAD, f"{k}: rel L2 {errs[k]:.3g}"
