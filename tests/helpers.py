"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
binding, run the FP64 oracle on the same seeded inputs, compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2509_07782_b300 import rgx, synth

TOL_RGBA = 1e-4      # max-abs per RGB channel and opacity, FP32 vs FP64
TOL_GRAD = 1e-3      # relative L2 per parameter tensor


def gpu_render(scene: synth.Scene, cams, opts, sched_cap: int = 0, scene_obj=None):
    sc = scene_obj or rgx.Scene()
    t = rgx.scene_tensors(scene)
    sg = rgx.sg_tensor(scene)
    o = rgx.make_opts(opts)
    sc.build(*t, o, sh_degree=scene.sh_degree, sg=sg)
    cb = rgx.Cameras(cams)
    out = sc.forward(cb, o, want_state=True, sched_cap=sched_cap)
    status = sc.status()
    res = dict(rgba=out[0].cpu().numpy().astype(np.float64), state=out[1], status=status, scene=sc,
               cams=cb, opts=o, tensors=t, sg=sg)
    if sched_cap:
        res["sched"] = out[2].cpu().numpy().astype(np.float64)
        res["sched_n"] = out[3].cpu().numpy().astype(np.int64)
    return res


def gpu_backward(res, d_rgba: np.ndarray):
    sc, cb, o, t = res["scene"], res["cams"], res["opts"], res["tensors"]
    grads = [torch.zeros_like(x) for x in t]
    up = torch.as_tensor(np.ascontiguousarray(d_rgba, dtype=np.float32), device=t[0].device)
    d_sg = None
    if res.get("sg") is not None:
        d_sg = torch.zeros_like(res["sg"])
        sc.backward_ex(cb, o, res["state"], up, grads, d_sg=d_sg)
    else:
        sc.backward(cb, o, res["state"], up, grads)
    status = sc.status()
    out = dict(means=grads[0].cpu().numpy(), scales=grads[1].cpu().numpy(), quats=grads[2].cpu().numpy(),
               densities=grads[3].cpu().numpy(), sh=grads[4].cpu().numpy(), status=status)
    if d_sg is not None:
        out["sg"] = d_sg.cpu().numpy()
    return out


# (test, divergent pixels, pixels compared) of every comparison in the session; printed in the
# terminal summary so that a drift in the number of rounding-divergent decisions shows
DIVERGENCE_LOG = []
# pixels allowed to exceed the tolerance through a rounding-divergent decision: at most one per
# comparison, or 0.1 % of the pixels compared when that is more
MAX_DIVERGENT_FRAC = 0.001


# (test, quantity, value) of the parity comparisons: max-abs RGBA error, worst relative L2 per gradient tensor
PARITY_LOG = []


def record_divergence(name: str, ndiv: int, n: int):
    DIVERGENCE_LOG.append((name, int(ndiv), int(n)))


def record_parity(name: str, quantity: str, value: float):
    PARITY_LOG.append((name, quantity, float(value)))


def compare_rgba(gpu_rgba: np.ndarray, cam, scene, opts, pix=None, gpu_sched=None, gpu_sched_n=None,
                 max_divergent_frac: float = MAX_DIVERGENT_FRAC, params=None):
    """Max-abs comparison with the oracle.  Pixels whose difference exceeds the
    tolerance are accepted only if (a) replaying the GPU's recorded schedule in
    the oracle reproduces the GPU value within tolerance -- i.e. the GPU took a
    discrete decision (skip / segment grid) that differs from the FP64 one only
    by rounding -- and (b) there are at most max(1, `max_divergent_frac` x the
    pixels compared) of them.  Returns (max_abs_err, n_divergent)."""
    ref = oracle.render(scene, cam, opts, pix=pix, params=params)
    g = gpu_rgba if pix is None else gpu_rgba[pix]
    err = np.abs(g - ref["rgba"]).max(axis=1)
    bad = np.nonzero(err > TOL_RGBA)[0]
    if len(bad) == 0:
        return float(err.max()) if err.size else 0.0, 0
    assert gpu_sched is not None, f"{len(bad)} pixels beyond {TOL_RGBA}: max {err.max():.3g}"
    assert len(bad) <= max(1.0, max_divergent_frac * len(err)) + 1e-9, \
        f"{len(bad)} of {len(err)} pixels beyond {TOL_RGBA} (max {err.max():.3g})"
    gp = np.arange(len(err)) if pix is None else np.asarray(pix)
    rows = gp[bad]
    cap = gpu_sched.shape[1]
    assert np.all(gpu_sched_n[rows] <= cap)
    rep = oracle.render(scene, cam, opts, pix=rows, sched=gpu_sched[rows], sched_n=gpu_sched_n[rows], params=params)
    err2 = np.abs(gpu_rgba[rows] - rep["rgba"]).max(axis=1)
    assert err2.max() <= TOL_RGBA, f"replayed GPU schedule still differs by {err2.max():.3g}"
    ok = err.copy()
    ok[bad] = 0
    return float(ok.max()), int(len(bad))


def schedules_agree(gpu_sched, gpu_n, ref_sched, ref_n, rows):
    """Per pixel: same number of evaluated segments and same (t_S, dt) within
    float32 rounding."""
    out = np.zeros(len(rows), dtype=bool)
    for i, r in enumerate(rows):
        if gpu_n[r] != ref_n[i]:
            continue
        m = int(min(gpu_n[r], gpu_sched.shape[1]))
        a, b = gpu_sched[r, :m], ref_sched[i, :m]
        out[i] = np.allclose(a, b, rtol=2e-5, atol=1e-6)
    return out


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
