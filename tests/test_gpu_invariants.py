"""GPU invariants that need no oracle value:

* determinism: two forward runs are bit-identical; the adjoint's replay
  reproduces every ray's T_final bit for bit (no RGX_ERR_REPLAY);
* Z-order storage (RGX_MORTON) changes memory order only: results are
  bit-identical with and without it;
* Z-order ray tiles (RGX_ZTILES) change which rays share a tile and so the
  tile's BVH cut, hence the traversal order and the order of the per-sample
  sums: results agree to float32 rounding;
* chord lists are windowed / chunked, never dropped: hit_cap 32 and 512 agree
  to float32 rounding;
* several cameras in one persistent launch equal one launch per camera;
* edge cases: empty scene -> background; a single Gaussian; ragged image
  sizes; host-side option checks; bad parameters and the segment limit
  are reported in the status word without a fault.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2509_07782_b300 import rgx, synth
from helpers import gpu_backward, gpu_render

pytestmark = pytest.mark.gpu


def opts_with(o, **kw):
    o = dataclasses.replace(o)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_forward_deterministic_and_replay_exact():
    w = synth.workload("torus_100k", n=30000, scale_res=0.25)
    r1 = gpu_render(w.scene, w.cameras, w.options)
    r2 = gpu_render(w.scene, w.cameras, w.options)
    np.testing.assert_array_equal(r1["rgba"], r2["rgba"])
    d = np.random.default_rng(0).normal(size=r1["rgba"].shape)
    g = gpu_backward(r1, d)
    assert g["status"] == 0  # no RGX_ERR_REPLAY: T_final reproduced bit for bit


def test_morton_storage_is_bit_identical():
    w = synth.workload("torus_100k", n=30000, scale_res=0.25)
    a = gpu_render(w.scene, w.cameras, opts_with(w.options, morton=True))
    b = gpu_render(w.scene, w.cameras, opts_with(w.options, morton=False))
    np.testing.assert_array_equal(a["rgba"], b["rgba"])


def test_ztiles_agree_to_rounding():
    w = synth.workload("torus_100k", n=30000, scale_res=0.25)
    a = gpu_render(w.scene, w.cameras, opts_with(w.options, ztiles=True))
    b = gpu_render(w.scene, w.cameras, opts_with(w.options, ztiles=False))
    assert a["status"] == 0 and b["status"] == 0
    np.testing.assert_allclose(a["rgba"], b["rgba"], rtol=0, atol=2e-6)
    d = np.random.default_rng(2).normal(size=a["rgba"].shape)
    ga, gb = gpu_backward(a, d), gpu_backward(b, d)
    assert ga["status"] == 0 and gb["status"] == 0
    for k in ("means", "scales", "quats", "densities", "sh"):
        np.testing.assert_allclose(ga[k], gb[k], rtol=1e-3, atol=1e-4 * np.abs(gb[k]).max())


def test_hit_cap_chunking_never_drops_hits():
    # hit_cap sets the chord-window capacity; 32 forces windows down to single
    # segments and chunked segments.  Summation order may change (float32
    # rounding) but no hit may be lost.
    w = synth.workload("torus_100k", n=60000, scale_res=0.2)
    a = gpu_render(w.scene, w.cameras, opts_with(w.options, hit_cap=32))
    b = gpu_render(w.scene, w.cameras, opts_with(w.options, hit_cap=512))
    assert a["status"] == 0 and b["status"] == 0
    np.testing.assert_allclose(a["rgba"], b["rgba"], rtol=0, atol=2e-6)
    d = np.random.default_rng(1).normal(size=a["rgba"].shape)
    ga, gb = gpu_backward(a, d), gpu_backward(b, d)
    for k in ("means", "scales", "quats", "densities", "sh"):
        np.testing.assert_allclose(ga[k], gb[k], rtol=1e-3, atol=1e-4 * np.abs(gb[k]).max())


def test_batch_launch_equals_single_launches():
    w = synth.workload("batch_1m", n=50000, scale_res=0.1)
    r = gpu_render(w.scene, w.cameras, w.options)
    off = 0
    for cam in w.cameras:
        s = gpu_render(w.scene, [cam], w.options)
        np.testing.assert_array_equal(r["rgba"][off:off + cam.n_rays], s["rgba"])
        off += cam.n_rays


def test_batched_adjoint_equals_the_sum_of_single_view_adjoints():
    # One persistent adjoint launch over several views of uneven size must add
    # up the per-view gradients (the loss is a sum over views); only the order
    # of the float atomics differs.
    w = synth.workload("batch_1m", n=50000, scale_res=0.1)
    r = gpu_render(w.scene, w.cameras, w.options)
    d = np.random.default_rng(3).normal(size=r["rgba"].shape)
    gb = gpu_backward(r, d)
    assert gb["status"] == 0
    total = {k: np.zeros_like(gb[k]) for k in ("means", "scales", "quats", "densities", "sh")}
    off = 0
    for cam in w.cameras:
        s = gpu_render(w.scene, [cam], w.options)
        gs = gpu_backward(s, d[off:off + cam.n_rays])
        assert gs["status"] == 0
        for k in total:
            total[k] += gs[k]
        off += cam.n_rays
    for k in total:
        assert np.abs(total[k]).max() > 0, k
        np.testing.assert_allclose(gb[k], total[k], rtol=1e-3, atol=1e-4 * np.abs(total[k]).max())


def test_empty_scene_and_single_gaussian():
    w = synth.workload("plain_2k")
    bg = (0.2, 0.3, 0.4)
    o = opts_with(w.options, bg=bg)
    empty = w.scene.subset(np.zeros(0, dtype=np.int64))
    r = gpu_render(empty, w.cameras, o)
    np.testing.assert_array_equal(r["rgba"], np.tile(np.array([*bg, 0.0], np.float32), (w.cameras[0].n_rays, 1)))
    one = w.scene.subset(np.array([5]))
    r1 = gpu_render(one, w.cameras, o)
    assert r1["status"] == 0
    assert np.all(r1["rgba"][:, 3] >= 0) and np.all(r1["rgba"][:, 3] <= 1)


def test_invalid_options_rejected_on_host():
    w = synth.workload("plain_2k", n=10)
    sc = rgx.Scene()
    t = rgx.scene_tensors(w.scene)
    sc.build(*t, rgx.make_opts(w.options))
    cb = rgx.Cameras(w.cameras)
    for bad in (dict(n_s=5), dict(dt=0.0), dict(hit_cap=16), dict(ztiles=True, tile_w=5, tile_h=5)):
        with pytest.raises(rgx.RgxError) as e:
            sc.forward(cb, rgx.make_opts(opts_with(w.options, **bad)))
        assert e.value.code == rgx.RGX_ERR_INVALID_ARG
    with pytest.raises(rgx.RgxError):
        sc.forward(rgx.Cameras([dataclasses.replace(w.cameras[0], width=0)]), rgx.make_opts(w.options))


def test_bad_parameters_and_segment_limit_reported():
    w = synth.workload("plain_2k", n=200)
    sc = w.scene
    means = sc.means.copy()
    means[3, 0] = np.nan
    bad = synth.Scene(means, sc.scales, sc.quats, sc.densities, sc.sh, 3)
    r = gpu_render(bad, w.cameras, w.options)
    assert r["status"] & rgx.RGX_ERR_BAD_PARAMS
    r2 = gpu_render(sc, w.cameras, opts_with(w.options, max_segments=2))
    assert r2["status"] & rgx.RGX_ERR_ITER_LIMIT
    torch.cuda.synchronize()


def test_adjoint_with_a_stale_state_collects_again_and_matches():
    # The scene's tape keeps the first chord lists of the LAST forward call only.
    # An adjoint given the state of an older call must notice (tag mismatch),
    # collect the lists again by traversal and replay the same march (no replay
    # error); gradients then agree up to the order of the float atomics.
    w = synth.workload("torus_100k", n=30000, scale_res=0.25)
    sc = rgx.Scene()
    t = rgx.scene_tensors(w.scene)
    o = rgx.make_opts(w.options)
    sc.build(*t, o)
    cb = rgx.Cameras(w.cameras)
    d = torch.as_tensor(np.random.default_rng(5).normal(size=(cb.n_rays, 4)), dtype=torch.float32, device="cuda")

    def adjoint(state):
        g = [torch.zeros_like(x) for x in t]
        sc.backward(cb, o, state, d, g)
        assert sc.status() == 0  # no RGX_ERR_REPLAY
        return [x.cpu().numpy() for x in g], sc.counters()["node_visits"]

    rgba1, st1 = sc.forward(cb, o)
    taped, visits_taped = adjoint(st1)
    other = rgx.Cameras([synth.rescale_camera(w.cameras[0], 0.5)])
    sc.forward(other, o)  # overwrites the tape
    again, visits_again = adjoint(st1)
    assert visits_again > 2 * visits_taped  # the lists were collected again
    for a, b in zip(taped, again):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(a).max())
