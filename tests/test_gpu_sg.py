"""The spherical-Gaussian appearance term on the GPU against the oracle (Eq. 1's
c_l "with SH/SG"; the supplementary's SH + SG model, Supp. Sec. 6.1: nine SH and
seven SG per primitive), through rgx_build_bvh_sg / rgx_render_backward_ex:

* forward max-abs 1e-4 per channel and opacity (full frame; sampled on the
  100k-Gaussian torus view with every speed option);
* gradients of all six tensors -- the five geometry / SH tensors and the lobes
  (raw axis, sharpness, amplitude) -- within relative L2 1e-3;
* a scene with zero lobe amplitudes renders exactly like the SH-only build,
  and rgx_render_backward_ex refuses a lobed scene without d_sg.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_07782_b300 import rgx, synth
from helpers import TOL_GRAD, TOL_RGBA, compare_rgba, gpu_backward, gpu_render, record_divergence, rel_l2, \
    schedules_agree

pytestmark = pytest.mark.gpu

NAMES = ["means", "scales", "quats", "densities", "sh", "sg"]


def _sg_scene(name, n=None, scale_res=None, seed=77):
    w = synth.workload(name, n=n, scale_res=scale_res)
    return w, synth.with_sg_appearance(w.scene, seed=seed)


@pytest.mark.parametrize("fast", [False, True])
def test_sg_forward_and_gradients_full_frame(fast):
    w, scene = _sg_scene("plain_2k")
    cam = w.cameras[0]
    o = synth.fast_options(dt=0.01) if fast else w.options
    r = gpu_render(scene, [cam], o, sched_cap=64)
    assert r["status"] == 0
    err, ndiv = compare_rgba(r["rgba"], cam, scene, o, gpu_sched=r["sched"], gpu_sched_n=r["sched_n"])
    record_divergence(f"plain_2k with 9 SH + 7 SG, {'fast' if fast else 'plain'}", ndiv, cam.n_rays)
    assert err <= TOL_RGBA
    pix = np.arange(cam.n_rays)
    ref = oracle.render(scene, cam, o, sched_cap=64)
    agree = schedules_agree(r["sched"], r["sched_n"], ref["sched"], ref["sched_n"], pix)
    assert agree.mean() >= 0.99
    W = np.random.default_rng(3).normal(size=(cam.n_rays, 4))
    W[~agree] = 0.0
    g = gpu_backward(r, W)
    assert g["status"] == 0
    gr = oracle.backward(scene, cam, o, W)
    errs = {k: rel_l2(g[k], gr[k]) for k in NAMES}
    for k in NAMES:
        assert np.linalg.norm(gr[k]) > 0, k
        assert errs[k] <= TOL_GRAD, f"{k}: rel L2 {errs[k]:.3g} ({errs})"


def test_sg_torus_sampled_forward_and_gradients():
    w, scene = _sg_scene("torus_100k", n=100_000, scale_res=0.5)
    cam = w.cameras[0]
    r = gpu_render(scene, [cam], w.options, sched_cap=64)
    assert r["status"] == 0
    params = oracle.Params(scene)
    pix = synth.pixel_subset(cam, 1024, seed=71)
    err, ndiv = compare_rgba(r["rgba"], cam, scene, w.options, pix=pix, gpu_sched=r["sched"],
                             gpu_sched_n=r["sched_n"], params=params)
    record_divergence("torus_100k (400x400) with 9 SH + 7 SG", ndiv, len(pix))
    assert err <= TOL_RGBA
    ref = oracle.render(scene, cam, w.options, pix=pix, sched_cap=64, params=params)
    agree = schedules_agree(r["sched"], r["sched_n"], ref["sched"], ref["sched_n"], pix)
    assert agree.mean() >= 0.99
    W = np.random.default_rng(72).normal(size=(len(pix), 4))
    W[~agree] = 0.0
    d = np.zeros((cam.n_rays, 4))
    d[pix] = W
    g = gpu_backward(r, d)
    assert g["status"] == 0
    gr = oracle.backward(scene, cam, w.options, W, pix=pix, params=params)
    for k in NAMES:
        e = rel_l2(g[k], gr[k])
        assert e <= TOL_GRAD, f"{k}: rel L2 {e:.3g}"


def test_zero_amplitude_lobes_render_like_sh_only():
    w, scene = _sg_scene("plain_2k", n=600)
    sg = np.array(scene.sg)
    sg[:, :, 4:] = 0.0
    lobed = synth.Scene(scene.means, scene.scales, scene.quats, scene.densities, scene.sh, scene.sh_degree, sg)
    plain = synth.Scene(scene.means, scene.scales, scene.quats, scene.densities, scene.sh, scene.sh_degree)
    a = gpu_render(lobed, w.cameras, w.options)
    b = gpu_render(plain, w.cameras, w.options)
    np.testing.assert_array_equal(a["rgba"], b["rgba"])
    d = torch.randn(w.cameras[0].n_rays, 4, device="cuda")
    grads = [torch.zeros_like(x) for x in a["tensors"]]
    with pytest.raises(rgx.RgxError) as e:
        rgx.rgx_render_backward_ex(a["scene"].h, a["cams"], a["opts"], a["state"], d, *grads,
                                   n=lobed.n, sh_degree=lobed.sh_degree, n_sg=7)
    assert e.value.code == rgx.RGX_ERR_INVALID_ARG
