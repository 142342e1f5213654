"""Adjoint parity of the CUDA backward march with the oracle's analytic
gradient (itself pinned to FP64 central differences): relative L2 <= 1e-3
per parameter tensor, through the C-ABI.

The loss is L = sum_p <W_p, RGBA_p> over a seeded pixel set (W ~ N(0,1),
zero elsewhere), so the GPU and the oracle differentiate the same function.
In adaptive mode only pixels whose GPU schedule agrees with the oracle's
carry weight (a schedule that differs by rounding is a different, equally
valid, piecewise-constant branch).
"""
import numpy as np
import pytest

import oracle
from paper_2509_07782_b300 import synth
from helpers import TOL_GRAD, gpu_backward, gpu_render, record_parity, rel_l2, schedules_agree

pytestmark = pytest.mark.gpu

NAMES = ["means", "scales", "quats", "densities", "sh"]


def run_case(scene, cam, opts, pix, sched_cap=64, params=None, label=None):
    r = gpu_render(scene, [cam], opts, sched_cap=sched_cap)
    assert r["status"] == 0
    ref = oracle.render(scene, cam, opts, pix=pix, sched_cap=sched_cap, params=params)
    agree = schedules_agree(r["sched"], r["sched_n"], ref["sched"], ref["sched_n"], pix)
    assert agree.mean() >= 0.99, f"only {agree.mean():.4f} of schedules agree"
    W = np.random.default_rng(11).normal(size=(len(pix), 4))
    W[~agree] = 0.0
    d_rgba = np.zeros((cam.n_rays, 4))
    d_rgba[pix] = W
    g = gpu_backward(r, d_rgba)
    assert g["status"] == 0, f"device status {g['status']}"
    gr = oracle.backward(scene, cam, opts, W, pix=pix, params=params)
    errs = {k: rel_l2(g[k], gr[k]) for k in NAMES}
    record_parity(f"{label or 'adjoint'} ({cam.width}x{cam.height}, {len(pix)} px)", "worst gradient rel L2",
                  max(errs.values()))
    for k in NAMES:
        assert np.linalg.norm(gr[k]) > 0, k
        assert errs[k] <= TOL_GRAD, f"{k}: rel L2 {errs[k]:.3g} ({errs})"
    return errs


def test_plain_2k_full_frame_gradients():
    w = synth.workload("plain_2k")
    cam = w.cameras[0]
    run_case(w.scene, cam, w.options, np.arange(cam.n_rays), label="plain_2k uniform")


def test_fast_options_small_gradients():
    w = synth.workload("plain_2k")
    cam = w.cameras[0]
    run_case(w.scene, cam, synth.fast_options(dt=0.01), np.arange(cam.n_rays), label="plain_2k fast options")


def test_torus_100k_bench_configuration_gradients():
    w = synth.workload("torus_100k")
    cam = w.cameras[0]
    pix = synth.pixel_subset(cam, 4096, seed=7)
    run_case(w.scene, cam, w.options, pix, params=oracle.Params(w.scene), label="torus_100k")


def test_outdoor_gradients_sampled():
    w = synth.workload("outdoor_3m", n=300_000)
    cam = w.cameras[0]
    pix = synth.pixel_subset(cam, 512, seed=9)
    run_case(w.scene, cam, w.options, pix, sched_cap=96, params=oracle.Params(w.scene))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_lower_sh_degrees_forward_and_gradients(deg):
    """sh_degree 0..2 (1, 4, 9 coefficients per channel): the CUDA path packs,
    colours and differentiates only the first (deg+1)^2 coefficients; image
    and gradients match the oracle of the same degree."""
    from helpers import TOL_RGBA, compare_rgba
    w = synth.workload("plain_2k", n=600)
    nk = (deg + 1) ** 2
    sc = synth.Scene(w.scene.means, w.scene.scales, w.scene.quats, w.scene.densities,
                     np.ascontiguousarray(w.scene.sh[:, :nk, :]), deg)
    cam = w.cameras[0]
    r = gpu_render(sc, [cam], w.options)
    assert r["status"] == 0
    err, ndiv = compare_rgba(r["rgba"], cam, sc, w.options)
    assert err <= TOL_RGBA and ndiv == 0
    errs = run_case(sc, cam, w.options, np.arange(cam.n_rays))
    assert all(e <= TOL_GRAD for e in errs.values())
