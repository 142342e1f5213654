"""The Python binding checks what the C side cannot check on a plain pointer.

The C ABI takes raw device pointers, so a host array, a wrong element type or
a buffer shorter than the call writes would reach a kernel as a bad address.
The binding rejects such arguments with ValueError before anything is
enqueued.  The CPU tests here pass host tensors to every entry point; the GPU
test passes CUDA tensors of the wrong type, size or device and checks that no
call reaches the library.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2509_07782_b300 import rgx, synth


@pytest.fixture(scope="module")
def lib_built():
    from paper_2509_07782_b300 import build_lib
    build_lib.build()


def _setup(n=10):
    w = synth.workload("plain_2k", n=n)
    cams = rgx.Cameras(w.cameras)
    opts = rgx.make_opts(w.options)
    return w, cams, opts


def _host(shape, dtype=torch.float32):
    return torch.zeros(shape, dtype=dtype)


def test_every_entry_point_rejects_host_tensors(lib_built):
    w, cams, opts = _setup()
    n, R = w.scene.n, cams.n_rays
    params = [_host((n, 3)), _host((n, 3)), _host((n, 4)), _host(n), _host((n, 16, 3))]
    state = _host((R, rgx.rgx_fwd_state_bytes() // 4))
    calls = [
        lambda: rgx.rgx_build_bvh(None, *params, 3, opts),
        lambda: rgx.rgx_render_forward(None, cams, opts, _host((R, 4))),
        lambda: rgx.rgx_render_forward_sched(None, cams, opts, _host((R, 4)), state, _host((R, 8, 2)),
                                             _host(R, torch.int32)),
        lambda: rgx.rgx_render_backward(None, cams, opts, state, _host((R, 4)), *params, n=n),
        lambda: rgx.rgx_autotune(None, cams, opts, False, True, _host((R, 4)), state, _host((R, 4)), params),
        lambda: rgx.rgx_morton_sort_noalloc(params[0], False, _host(n, torch.int64), _host(n, torch.int32)),
        lambda: rgx.rgx_isotropic_loss(params[1], 10.0, 1.0, _host(1), _host((n, 3))),
        lambda: rgx.rgx_densify_accumulate(params[0], params[0], cams, _host(n), _host(n, torch.int32)),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()


def test_schedule_buffer_shape_is_checked(lib_built):
    _, cams, opts = _setup()
    R = cams.n_rays
    with pytest.raises(ValueError, match="sched"):
        rgx.rgx_render_forward_sched(None, cams, opts, _host((R, 4)), None, _host((R, 8)), _host(R, torch.int32))


def test_sh_degree_range_is_checked(lib_built):
    w, _, opts = _setup()
    n = w.scene.n
    params = [_host((n, 3)), _host((n, 3)), _host((n, 4)), _host(n), _host((n, 16, 3))]
    with pytest.raises(ValueError, match="sh_degree"):
        rgx.rgx_build_bvh(None, *params, 4, opts)


@pytest.mark.gpu
def test_wrong_dtype_size_or_device_never_reaches_the_library():
    w, cams, opts = _setup(n=50)
    n, R = w.scene.n, cams.n_rays
    sc = rgx.Scene()
    t = rgx.scene_tensors(w.scene)
    sc.build(*t, opts)
    rgba, state = sc.forward(cams, opts)
    torch.cuda.synchronize()
    good = [torch.zeros_like(x) for x in t]
    d = torch.zeros(R, 4, device="cuda")
    cases = [
        ("rgba", lambda: rgx.rgx_render_forward(sc.h, cams, opts, torch.empty(R, 4, dtype=torch.float64,
                                                                              device="cuda"))),
        ("rgba", lambda: rgx.rgx_render_forward(sc.h, cams, opts, torch.empty(R - 1, 4, device="cuda"))),
        ("fwd_state", lambda: rgx.rgx_render_forward(sc.h, cams, opts, rgba, state[: R // 2])),
        ("contiguous", lambda: rgx.rgx_render_forward(sc.h, cams, opts, torch.empty(4, R, device="cuda").t())),
        ("d_rgba", lambda: sc.backward(cams, opts, state, d[:-1], good)),
        ("d_sh", lambda: sc.backward(cams, opts, state, d, good[:4] + [torch.zeros(n, 9, 3, device="cuda")])),
        ("d_densities", lambda: sc.backward(cams, opts, state, d, good[:3] + [torch.zeros(n - 1, device="cuda"),
                                                                               good[4]])),
        ("different devices", lambda: sc.build(*[x.cpu() for x in t[:1]], *t[1:], opts)),
    ]
    for what, call in cases:
        with pytest.raises(ValueError, match=what):
            call()
    # the scene is untouched: a valid backward still runs and reports no device problem
    sc.backward(cams, opts, state, torch.randn(R, 4, device="cuda"), good)
    assert sc.status() == 0
    assert np.isfinite(good[0].cpu().numpy()).all()


def test_nvtx_ranges_are_opt_in_named_and_balanced(lib_built, monkeypatch):
    """With RGX_NVTX set, a call opens one NVTX range named after its entry
    point and closes it even when the call raises; without it, none."""
    _, cams, opts = _setup()
    pushed, popped = [], []
    monkeypatch.setattr(torch.cuda.nvtx, "range_push", lambda name: pushed.append(name))
    monkeypatch.setattr(torch.cuda.nvtx, "range_pop", lambda: popped.append(1))
    bad = _host((cams.n_rays, 4))
    with pytest.raises(ValueError):
        rgx.rgx_render_forward(None, cams, opts, bad)
    assert pushed == [] and popped == []
    monkeypatch.setattr(rgx, "NVTX", True)
    with pytest.raises(ValueError):
        rgx.rgx_render_forward(None, cams, opts, bad)
    with pytest.raises(ValueError):
        rgx.rgx_isotropic_loss(_host((4, 3)), 10.0, 1.0, _host(1), _host((4, 3)))
    assert pushed == ["rgx_render_forward", "rgx_isotropic_loss"] and len(popped) == 2
