"""The training step on the GPU against the oracle, through the C-ABI:

* image loss (1 - lambda) L1 + lambda DSSIM (Sec. 3.4) of three views of uneven
  size in one call: per-view loss (relative 1e-5) and dL/drgba (max-abs within
  1e-4 of the largest entry) against the oracle's FP64 loss and gradient;
* Adam, plain and log-parameterised: against the oracle's step (relative 1e-5);
* densification plan (bit-exact actions and offsets: decisions taken in float32
  on both sides) and apply (clones exact; split children to float32 rounding);
* a short training run on synthetic targets (views of a reference scene rendered
  by the library): the image loss falls, the statistic grows Gaussians at
  densification, and the device status stays clean.
"""
import numpy as np
import pytest
import torch

from oracle import losses
from oracle import train as otrain
from paper_2509_07782_b300 import rgx, synth
from paper_2509_07782_b300.train import Trainer

pytestmark = pytest.mark.gpu


def test_image_loss_matches_oracle_over_uneven_views():
    rng = np.random.default_rng(0)
    sizes = [(37, 23), (64, 48), (16, 90)]
    cams = rgx.Cameras([synth.Camera(np.eye(3, 4, dtype=np.float32), 50.0, 50.0, w / 2, h / 2, w, h)
                        for w, h in sizes])
    R = cams.n_rays
    pred = rng.uniform(0, 1, size=(R, 4)).astype(np.float32)
    # targets close to the prediction in places, far elsewhere (both L1 signs, varied SSIM)
    tgt = np.clip(pred[:, :3] + rng.normal(0, 0.2, size=(R, 3)), 0, 1).astype(np.float32)
    sc = rgx.Scene()
    loss = torch.zeros(3, device="cuda")
    d = torch.empty(R, 4, device="cuda")
    rgx.rgx_image_loss(sc.h, cams, torch.as_tensor(pred, device="cuda"), torch.as_tensor(tgt, device="cuda"), 0.2,
                       loss, d)
    torch.cuda.synchronize()
    d = d.cpu().numpy()
    off = 0
    for c, (w, h) in enumerate(sizes):
        sl = slice(off, off + w * h)
        L, g = losses.image_loss(pred[sl, :3].reshape(h, w, 3), tgt[sl].reshape(h, w, 3), lam=0.2)
        assert loss[c].item() == pytest.approx(L, rel=1e-5)
        gg = d[sl, :3].reshape(h, w, 3)
        assert np.abs(gg - g).max() <= 1e-4 * np.abs(g).max()
        assert np.all(d[sl, 3] == 0)
        off += w * h


@pytest.mark.parametrize("expo", [False, True])
def test_adam_matches_oracle(expo):
    rng = np.random.default_rng(1)
    n = 100_003
    p = rng.normal(-2 if expo else 0, 0.5, size=n).astype(np.float32)
    m = rng.normal(0, 0.01, size=n).astype(np.float32)
    v = rng.uniform(0, 1e-4, size=n).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    # the kernel receives its hyperparameters as float32: the oracle takes the same values
    f = lambda x: float(np.float32(x))  # noqa: E731
    ref = otrain.adam_step(p, g, m, v, lr=f(1e-2), step=7, b1=f(0.9), b2=f(0.999), eps=f(1e-15), exp_param=expo)
    tp, tm, tv, tg = (torch.as_tensor(x, device="cuda") for x in (p, m, v, g))
    act = torch.empty_like(tp)
    rgx.rgx_adam_step(tp, tg, tm, tv, 1e-2, 7, eps=1e-15, exp_param=expo, activated=act)
    torch.cuda.synchronize()
    # float32 against FP64: the moment updates cancel for entries near zero, so the absolute
    # tolerance scales with each tensor's magnitude
    for got, want in zip((tp, tm, tv, act), ref):
        want = np.asarray(want)
        np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-5, atol=1e-6 * np.abs(want).max())


def test_densify_plan_and_apply_match_oracle():
    rng = np.random.default_rng(2)
    w = synth.workload("torus_100k", n=50_000)
    sc_ = w.scene
    n = sc_.n
    stat = (rng.exponential(2e-4, size=n) * rng.integers(0, 4, size=n)).astype(np.float32)
    count = rng.integers(0, 4, size=n).astype(np.int32)
    stat[count == 0] = 0
    ref_a, ref_o, ref_n = otrain.densify_plan(stat, count, sc_.scales, 1.5e-4, 0.012)
    assert (ref_a == 1).sum() > 100 and (ref_a == 2).sum() > 100
    t = rgx.scene_tensors(sc_)
    scene = rgx.Scene()
    action = torch.empty(n, dtype=torch.int32, device="cuda")
    offset = torch.empty(n, dtype=torch.int32, device="cuda")
    n_out = rgx.rgx_densify_plan(scene.h, torch.as_tensor(stat, device="cuda"), torch.as_tensor(count, device="cuda"),
                                 t[1], 1.5e-4, 0.012, action, offset)
    assert n_out == ref_n
    np.testing.assert_array_equal(action.cpu().numpy(), ref_a)
    np.testing.assert_array_equal(offset.cpu().numpy(), ref_o)
    normals = rng.normal(size=(n, 2, 3)).astype(np.float32)
    outs = [torch.empty((n_out,) + tuple(x.shape[1:]), device="cuda") for x in t]
    src = torch.empty(n_out, dtype=torch.int32, device="cuda")
    rgx.rgx_densify_apply(action, offset, torch.as_tensor(normals, device="cuda"), t, outs, out_src=src)
    torch.cuda.synchronize()
    ref = otrain.densify_apply(ref_a, normals.astype(np.float64), sc_.means.astype(np.float64),
                               sc_.scales.astype(np.float64), sc_.quats.astype(np.float64),
                               sc_.densities.astype(np.float64), sc_.sh.astype(np.float64))
    np.testing.assert_array_equal(src.cpu().numpy(), ref["src"])
    for k, o in zip(["means", "scales", "quats", "densities", "sh"], outs):
        np.testing.assert_allclose(o.cpu().numpy(), ref[k], rtol=2e-6, atol=2e-6, err_msg=k)


def test_training_run_reduces_the_image_loss_and_densifies():
    truth = synth.workload("torus_100k", n=30_000, scale_res=0.15)
    views = [synth.orbit_camera(np.random.Generator(np.random.PCG64(900 + i)), 4.0, 120, 120) for i in range(4)]
    cams = rgx.Cameras(views)
    o = rgx.make_opts(truth.options)
    ref = rgx.Scene()
    ref.build(*rgx.scene_tensors(truth.scene), o)
    targets, _ = ref.forward(cams, o, want_state=False)
    targets = targets[:, :3].contiguous()
    # start: the same Gaussians with perturbed colours, densities and positions
    rng = np.random.default_rng(5)
    s0 = truth.scene
    start = synth.Scene(s0.means + rng.normal(0, 0.004, size=s0.means.shape).astype(np.float32), s0.scales,
                        s0.quats, (s0.densities * np.exp(rng.normal(0, 0.5, size=s0.n))).astype(np.float32),
                        (s0.sh + rng.normal(0, 0.15, size=s0.sh.shape)).astype(np.float32), 3)
    tr = Trainer(rgx.scene_tensors(start), cams, o, targets, size_threshold=0.02)
    first = None
    for it in range(60):
        loss, iso = tr.step()
        total = float(loss.sum())
        if first is None:
            first = total
    assert tr.scene.status() == 0
    assert total < 0.8 * first, (first, total)
    assert int(tr.count.max()) > 0
    n0 = tr.n
    tr.tau = float(np.quantile((tr.stat / tr.count.clamp(min=1)).cpu().numpy(), 0.95))  # densify the top 5 %
    n1 = tr.densify(torch.Generator(device="cuda").manual_seed(0))
    assert n1 > n0 and tr.n == n1
    loss, _ = tr.step()
    assert tr.scene.status() == 0 and np.isfinite(float(loss.sum()))
