"""Tuning knobs, bounds and workspace limits of the C-ABI, on the GPU.

* hit_cap, the tile shape and N_S left at 0 select the defaults (512, 32x1,
  16) before the scene is autotuned and the autotuner's pick afterwards: the
  render is bit-identical to one with those values written out;
* with max_segments = 0 a ray's segment count is still bounded (2^20): a scene
  box vast next to the step stops every ray at the ceiling with
  RGX_ERR_ITER_LIMIT, in bounded time, instead of marching to the box's exit;
* the forward's tape of first chord lists may be capped or disabled
  (rgx_set_tape_limit): rays whose lists find no room are collected again by
  the adjoint, and the gradients do not change -- on a sparse view (first chord
  lists) and on a dense one (the sums records and the index tape with colours
  of chunked segments).
"""
import dataclasses
import time

import numpy as np
import pytest
import torch

from paper_2509_07782_b300 import rgx, synth
from helpers import gpu_backward, gpu_render

pytestmark = pytest.mark.gpu


def _render(sc, cams, o):
    rgba, _ = sc.forward(cams, o, want_state=False)
    assert sc.status() == 0
    return rgba


def test_zero_knobs_select_defaults_then_the_tuned_values():
    w = synth.workload("torus_100k", n=40_000, scale_res=0.2)
    sc = rgx.Scene()
    t = rgx.scene_tensors(w.scene)
    cams = rgx.Cameras(w.cameras)
    zero = rgx.make_opts(dataclasses.replace(w.options, hit_cap=0, tile_w=0, tile_h=0, n_s=0))
    sc.build(*t, zero)
    explicit = rgx.make_opts(dataclasses.replace(w.options, hit_cap=512, tile_w=32, tile_h=1, n_s=16))
    assert torch.equal(_render(sc, cams, zero), _render(sc, cams, explicit))
    best, _ = sc.autotune(cams, zero, tune_ns=True, with_backward=False)
    assert best.hit_cap in (32, 64, 96, 128, 192, 256, 384, 512, 640, 768) and best.n_s in (4, 8, 16, 32)
    tuned = rgx.make_opts(dataclasses.replace(w.options, hit_cap=best.hit_cap, tile_w=best.tile_w,
                                              tile_h=best.tile_h, n_s=best.n_s,
                                              lower_first=bool(best.flags & rgx.RGX_LOWER_FIRST)))
    assert torch.equal(_render(sc, cams, zero), _render(sc, cams, tuned))
    # forward and adjoint with zero knobs resolve alike: the replay reproduces T (no RGX_ERR_REPLAY)
    rgba, state = sc.forward(cams, zero)
    grads = [torch.zeros_like(x) for x in t]
    sc.backward(cams, zero, state, torch.randn_like(rgba), grads)
    assert sc.status() == 0
    # one of the two tile sides alone at 0 is an error
    bad = rgx.make_opts(dataclasses.replace(w.options, tile_w=0, tile_h=4))
    with pytest.raises(rgx.RgxError) as e:
        sc.forward(cams, bad)
    assert e.value.code == rgx.RGX_ERR_INVALID_ARG


def test_default_segment_ceiling_stops_rays_in_a_vast_box():
    # one faint Gaussian of enormous scale: its support (density just above sigma_eps) spans
    # ~1.2e6 units, so uniform segments of 16 x 0.05 would need ~1.5e6 segments per ray to
    # reach the box's exit; the default ceiling stops them at 2^20
    means = np.zeros((1, 3), np.float32)
    scales = np.full((1, 3), 1.0e6, np.float32)
    quats = np.array([[1.0, 0.0, 0.0, 0.0]], np.float32)
    dens = np.array([2.0e-6], np.float32)
    sh = np.zeros((1, 16, 3), np.float32)
    scene = synth.Scene(means, scales, quats, dens, sh, 3)
    cam = synth.look_at(np.array([0.0, 0.0, 3.0]), np.zeros(3), 50.0, 2, 2)
    o = synth.Options(dt=0.05, n_s=16, sigma_eps=1e-6, t_eps=1e-4)
    t0 = time.perf_counter()
    r = gpu_render(scene, [cam], o, sched_cap=1)
    dt = time.perf_counter() - t0
    assert r["status"] & rgx.RGX_ERR_ITER_LIMIT
    assert np.all(r["sched_n"] == 1 << 20)
    # the rays composited what they marched: T stayed high (a faint medium), RGB finite
    assert np.all(np.isfinite(r["rgba"])) and np.all(r["rgba"][:, 3] > 0.0)
    assert dt < 60.0
    # an explicit max_segments still wins
    r2 = gpu_render(scene, [cam], dataclasses.replace(o, max_segments=1000), sched_cap=1)
    assert r2["status"] & rgx.RGX_ERR_ITER_LIMIT and np.all(r2["sched_n"] == 1000)


@pytest.mark.parametrize("limit", [0, 3000])
def test_tape_limit_leaves_gradients_unchanged(limit):
    w = synth.workload("torus_100k", n=60_000, scale_res=0.3)
    d = np.random.default_rng(5).normal(size=(w.cameras[0].n_rays, 4))
    ref = gpu_backward(gpu_render(w.scene, w.cameras, w.options), d)
    assert ref["status"] == 0
    sc = rgx.Scene()
    sc.set_tape_limit(limit)
    r = gpu_render(w.scene, w.cameras, w.options, scene_obj=sc)
    g = gpu_backward(r, d)
    assert g["status"] == 0
    for k in ("means", "scales", "quats", "densities", "sh"):
        scale = np.abs(ref[k]).max() + 1e-30
        assert np.abs(g[k] - ref[k]).max() <= 1e-4 * scale, k
    cnt = sc.counters()
    # without room on the tape the adjoint collected the lists itself
    assert cnt["node_visits"] > 0


def test_dense_view_records_and_taped_colours_leave_gradients_unchanged():
    """A dense view (segments overflow a 32-entry list and are collected in chunks): the
    adjoint that reads the forward's sums records and its index tape -- each chunked chord's
    packed index with the colour the forward evaluated -- gives the gradients of the adjoint
    that collects, evaluates and colours every chunked segment itself (tape disabled), to
    rounding, with far fewer node visits; the forward image does not depend on the tape."""
    w = synth.workload("batch_1m", n=400_000)
    cam = synth.rescale_camera(w.cameras[3], 0.25)  # 256 x 192 of the 1024 x 768 view
    o = dataclasses.replace(w.options, hit_cap=32, n_s=32, tile_w=32, tile_h=1)
    d = np.random.default_rng(11).normal(size=(cam.n_rays, 4))
    ref = gpu_render(w.scene, [cam], o)
    assert ref["status"] == 0
    ref_fwd = ref["scene"].counters()
    g_ref = gpu_backward(ref, d)
    assert g_ref["status"] == 0
    taped = ref["scene"].counters()
    sc = rgx.Scene()
    sc.set_tape_limit(0)
    r = gpu_render(w.scene, [cam], o, scene_obj=sc)
    assert r["status"] == 0
    assert np.array_equal(r["rgba"], ref["rgba"])
    g = gpu_backward(r, d)
    assert g["status"] == 0
    untaped = sc.counters()
    # the view is dense: its segments average several lists of hits
    assert ref_fwd["hits"] > 4 * 32 * ref_fwd["segments"]
    for k in ("means", "scales", "quats", "densities", "sh"):
        scale = np.abs(g_ref[k]).max() + 1e-30
        assert np.abs(g[k] - g_ref[k]).max() <= 1e-4 * scale, k
    assert taped["node_visits"] < 0.5 * untaped["node_visits"]
