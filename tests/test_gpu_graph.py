"""CUDA-graph captured training step and the autotuner (batched multi-view
workload: several cameras of uneven resolution in one persistent launch).

* a captured build + forward + adjoint replays to the same RGBA (bit for bit)
  and the same gradients (up to float32 atomic order) as an eager step, also
  after the parameters are updated in place between replays;
* rgx_autotune returns one of its candidate configurations, and rendering with
  it matches the untuned render (it changes scheduling, not the method).
"""
import numpy as np
import pytest
import torch

from paper_2509_07782_b300 import graph, rgx, synth

pytestmark = pytest.mark.gpu


def eager_step(w, params, d_rgba, opts):
    sc = rgx.Scene()
    cams = rgx.Cameras(w.cameras)
    sc.build(*params, opts)
    rgba, state = sc.forward(cams, opts)
    grads = [torch.zeros_like(p) for p in params]
    sc.backward(cams, opts, state, d_rgba, grads)
    assert sc.status() == 0
    return rgba, grads


def test_captured_step_replays_like_eager():
    w = synth.workload("batch_1m", n=60_000, scale_res=0.15)
    opts = rgx.make_opts(w.options)
    params = list(rgx.scene_tensors(w.scene))
    cams = rgx.Cameras(w.cameras)
    d_rgba = torch.randn(cams.n_rays, 4, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    sc = rgx.Scene()
    step = graph.CapturedStep(sc, cams, opts, params, d_rgba)
    for it in range(2):
        if it == 1:
            with torch.no_grad():
                params[0].add_(0.002 * torch.randn_like(params[0]))   # in-place update between replays
                params[3].mul_(1.05)
        step.replay()
        torch.cuda.synchronize()
        assert sc.status() == 0
        rgba_e, grads_e = eager_step(w, params, d_rgba, opts)
        assert torch.equal(step.rgba, rgba_e)
        for g, ge in zip(step.grads, grads_e):
            scale = ge.abs().max().item() + 1e-30
            assert (g - ge).abs().max().item() <= 1e-4 * scale


def test_autotune_picks_a_candidate_that_renders_the_same():
    w = synth.workload("batch_1m", n=60_000, scale_res=0.1)
    base = rgx.make_opts(w.options)
    sc = rgx.Scene()
    t = rgx.scene_tensors(w.scene)
    sc.build(*t, base)
    cams = rgx.Cameras(w.cameras)
    best, ms = sc.autotune(cams, base, tune_ns=False, with_backward=True)
    assert ms > 0
    assert (best.tile_w, best.tile_h) in [(8, 4), (4, 8), (16, 2), (32, 1)]
    assert best.hit_cap in (32, 64, 96, 128, 192, 256, 384, 512, 640, 768) and best.n_s == base.n_s
    # the tuner may switch first-window lowering (scheduling only), nothing else of the flags
    assert (best.flags & ~rgx.RGX_LOWER_FIRST) == (base.flags & ~rgx.RGX_LOWER_FIRST) and best.dt_min == base.dt_min
    sc.build(*t, base)
    a, _ = sc.forward(cams, base)
    b, _ = sc.forward(cams, best)
    assert sc.status() == 0
    np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=0, atol=2e-6)
