"""Error behaviour of the C ABI that needs no GPU.

Every entry point checks its host-side arguments before any CUDA call and
returns an rgx_status (never crashes) with a description in rgx_last_error:
a null scene, null required pointers, out-of-range sizes and bad camera
intrinsics give RGX_ERR_INVALID_ARG, and empty work (n = 0) is RGX_OK
without a launch.  The calls go straight to the library through ctypes.
"""
import ctypes as C

import pytest

from paper_2509_07782_b300 import rgx


@pytest.fixture(scope="module")
def lib():
    from paper_2509_07782_b300 import build_lib
    build_lib.build()
    return rgx.lib()


def _msg(l, h=None):
    return l.rgx_last_error(h).decode()


def test_null_scene_is_rejected_by_every_scene_call(lib):
    o = rgx.RgxOpts()
    cam = (rgx.RgxCamera * 1)()
    best, ms = rgx.RgxOpts(), C.c_float()
    out8 = (C.c_uint64 * 8)()
    calls = {
        "rgx_build_bvh": lambda: lib.rgx_build_bvh(None, 0, 3, None, None, None, None, None, C.byref(o), None),
        "rgx_render_forward": lambda: lib.rgx_render_forward(None, cam, 1, C.byref(o), None, None, None),
        "rgx_render_forward_sched": lambda: lib.rgx_render_forward_sched(None, cam, 1, C.byref(o), None, None,
                                                                          None, 8, None, None),
        "rgx_render_backward": lambda: lib.rgx_render_backward(None, cam, 1, C.byref(o), None, None, None, None,
                                                               None, None, None, None),
        "rgx_sync_status": lambda: lib.rgx_sync_status(None, None),
        "rgx_get_bvh": lambda: lib.rgx_get_bvh(None, None, None, None, None, None),
        "rgx_get_counters": lambda: lib.rgx_get_counters(None, out8, None),
        "rgx_autotune": lambda: lib.rgx_autotune(None, cam, 1, C.byref(o), 0, 0, None, None, None, None, None,
                                                 None, None, None, C.byref(best), C.byref(ms), None),
    }
    for name, call in calls.items():
        assert call() == rgx.RGX_ERR_INVALID_ARG, name
        assert _msg(lib), name
    assert lib.rgx_scene_destroy(None) == rgx.RGX_OK


def test_scene_create_rejects_a_device_that_does_not_exist(lib):
    h = C.c_void_p()
    assert lib.rgx_scene_create(None, 0) == rgx.RGX_ERR_INVALID_ARG
    assert lib.rgx_scene_create(C.byref(h), -1) == rgx.RGX_ERR_INVALID_ARG
    assert h.value is None
    assert lib.rgx_scene_create(C.byref(h), 1 << 20) == rgx.RGX_ERR_INVALID_ARG
    assert "device" in _msg(lib)


def test_loss_and_statistic_argument_checks(lib):
    f = C.c_void_p(0x1000)  # never dereferenced: every call below returns before any launch
    assert lib.rgx_isotropic_loss(-1, None, 10.0, 1.0, None, None, None) == rgx.RGX_ERR_INVALID_ARG
    assert lib.rgx_isotropic_loss(5, None, 10.0, 1.0, f, f, None) == rgx.RGX_ERR_INVALID_ARG
    assert lib.rgx_isotropic_loss(0, None, 10.0, 1.0, None, None, None) == rgx.RGX_OK
    cam = rgx.RgxCamera()
    cam.fx = 0.0
    assert lib.rgx_densify_accumulate(0, None, None, None, None, None, None) == rgx.RGX_ERR_INVALID_ARG
    assert lib.rgx_densify_accumulate(0, None, None, C.byref(cam), None, None, None) == rgx.RGX_ERR_INVALID_ARG
    assert "fx" in _msg(lib)
    cam.fx = 500.0
    assert lib.rgx_densify_accumulate(0, None, None, C.byref(cam), None, None, None) == rgx.RGX_OK
    assert lib.rgx_densify_accumulate(3, f, None, C.byref(cam), f, f, None) == rgx.RGX_ERR_INVALID_ARG


def test_noalloc_sort_size_and_pointer_checks(lib):
    f = C.c_void_p(0x1000)
    assert lib.rgx_morton_sort_noalloc((1 << 18) + 1, f, 0, f, f, None) == rgx.RGX_ERR_INVALID_ARG
    assert "262144" in _msg(lib)
    assert lib.rgx_morton_sort_noalloc(-1, f, 0, f, f, None) == rgx.RGX_ERR_INVALID_ARG
    assert lib.rgx_morton_sort_noalloc(10, None, 0, f, f, None) == rgx.RGX_ERR_INVALID_ARG
    assert lib.rgx_morton_sort_noalloc(0, None, 0, None, None, None) == rgx.RGX_OK
