"""ctypes binding of librgx (see include/rgx.h).

Argument marshalling only: every step of the path runs in the CUDA library.
If ``librgx.so`` is missing or cannot be loaded, importing the functions
raises -- there is no CPU or PyTorch fallback.

Module-level functions carry the C names (``rgx_build_bvh``,
``rgx_render_forward``, ``rgx_render_backward`` ...) and take torch CUDA
tensors; ``Scene`` and ``Cameras`` are small owners of the opaque handle and
of the pinned camera array.  Before each call the binding checks what a plain
pointer cannot carry -- every tensor on the GPU, contiguous, of the element
type the header states and at least as long as the call reads or writes --
and raises ValueError instead of passing a bad address to a kernel.  A
``Cameras`` object must outlive the work enqueued with it: its pinned array is
read when the stream reaches the copy (``Scene`` keeps the last one alive).
"""
from __future__ import annotations

import ctypes as C
import functools
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librgx.so")

RGX_OK = 0
RGX_ERR_INVALID_ARG = 1
RGX_ERR_CUDA = 2
RGX_ERR_WORKSPACE = 3
RGX_ERR_STACK_OVERFLOW = 8
RGX_ERR_ITER_LIMIT = 16
RGX_ERR_BAD_PARAMS = 32
RGX_ERR_REPLAY = 64
RGX_ERR_NOT_BUILT = 128

RGX_SKIP, RGX_ADAPTIVE, RGX_MORTON, RGX_ZTILES, RGX_MORTON63, RGX_LOWER_FIRST = 1, 2, 4, 8, 16, 32
RGX_TUNE_NS, RGX_TUNE_EXHAUSTIVE = 1, 2

EXPORTS = ["rgx_scene_create", "rgx_scene_destroy", "rgx_build_bvh", "rgx_render_forward",
           "rgx_render_forward_sched", "rgx_render_backward", "rgx_sync_status", "rgx_fwd_state_bytes",
           "rgx_last_error", "rgx_get_bvh", "rgx_get_counters", "rgx_autotune",
           "rgx_morton_sort_noalloc", "rgx_isotropic_loss", "rgx_densify_accumulate", "rgx_set_tape_limit",
           "rgx_render_backward_ex", "rgx_build_bvh_sg", "rgx_image_loss", "rgx_adam_step", "rgx_densify_plan",
           "rgx_densify_apply"]


class RgxCamera(C.Structure):
    _fields_ = [("c2w", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("t_near", C.c_float), ("t_far", C.c_float)]


class RgxOpts(C.Structure):
    _fields_ = [("flags", C.c_int32), ("dt", C.c_float), ("dt_min", C.c_float), ("dt_max", C.c_float),
                ("beta", C.c_float), ("n_s", C.c_int32), ("t_eps", C.c_float), ("sigma_eps", C.c_float),
                ("bg", C.c_float * 3), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("hit_cap", C.c_int32), ("max_segments", C.c_int32)]


class RgxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rgx error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()

# RGX_NVTX=1: every call that enqueues work opens an NVTX range named after the
# entry point, so a profiler attributes the kernels it launches to that stage.
NVTX = os.environ.get("RGX_NVTX", "0") not in ("", "0")


def _traced(fn):
    name = fn.__name__

    @functools.wraps(fn)
    def call(*args, **kw):
        if not NVTX:
            return fn(*args, **kw)
        torch.cuda.nvtx.range_push(name)
        try:
            return fn(*args, **kw)
        finally:
            torch.cuda.nvtx.range_pop()
    return call


def lib() -> C.CDLL:
    """Load librgx.so (raises if it is missing: no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"librgx.so not built at {LIB_PATH}; run python -m paper_2509_07782_b300.build_lib")
            l = C.CDLL(LIB_PATH)
            vp, fp, i64 = C.c_void_p, C.c_void_p, C.c_int64
            l.rgx_scene_create.argtypes = [C.POINTER(vp), C.c_int32]
            l.rgx_scene_destroy.argtypes = [vp]
            l.rgx_build_bvh.argtypes = [vp, i64, C.c_int32, fp, fp, fp, fp, fp, C.POINTER(RgxOpts), vp]
            l.rgx_render_forward.argtypes = [vp, C.POINTER(RgxCamera), C.c_int32, C.POINTER(RgxOpts), fp, vp, vp]
            l.rgx_render_forward_sched.argtypes = [vp, C.POINTER(RgxCamera), C.c_int32, C.POINTER(RgxOpts), fp, vp,
                                                   fp, C.c_int32, vp, vp]
            l.rgx_render_backward.argtypes = [vp, C.POINTER(RgxCamera), C.c_int32, C.POINTER(RgxOpts), vp, fp,
                                              fp, fp, fp, fp, fp, vp]
            l.rgx_render_backward_ex.argtypes = [vp, C.POINTER(RgxCamera), C.c_int32, C.POINTER(RgxOpts), vp,
                                                 fp, fp, fp, fp, fp, fp, fp, fp, vp, vp]
            l.rgx_build_bvh_sg.argtypes = [vp, i64, C.c_int32, fp, fp, fp, fp, fp, C.c_int32, fp,
                                           C.POINTER(RgxOpts), vp]
            l.rgx_sync_status.argtypes = [vp, vp]
            l.rgx_fwd_state_bytes.restype = C.c_size_t
            l.rgx_fwd_state_bytes.argtypes = []
            l.rgx_last_error.restype = C.c_char_p
            l.rgx_last_error.argtypes = [vp]
            l.rgx_get_bvh.argtypes = [vp, vp, vp, vp, vp, vp]
            l.rgx_get_counters.argtypes = [vp, C.POINTER(C.c_uint64), vp]
            l.rgx_morton_sort_noalloc.argtypes = [i64, fp, C.c_int32, vp, vp, vp]
            l.rgx_isotropic_loss.argtypes = [i64, fp, C.c_float, C.c_float, fp, fp, vp]
            l.rgx_densify_accumulate.argtypes = [i64, fp, fp, C.POINTER(RgxCamera), fp, vp, vp]
            l.rgx_set_tape_limit.argtypes = [vp, i64]
            l.rgx_image_loss.argtypes = [vp, C.POINTER(RgxCamera), C.c_int32, fp, fp, C.c_float, fp, fp, vp]
            l.rgx_adam_step.argtypes = [i64, fp, fp, fp, fp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32,
                                        C.c_int32, fp, vp]
            l.rgx_densify_plan.argtypes = [vp, i64, fp, vp, fp, C.c_float, C.c_float, vp, vp,
                                           C.POINTER(C.c_int64), vp]
            l.rgx_densify_apply.argtypes = [i64, vp, vp, fp, fp, fp, fp, fp, fp, C.c_int32, fp, C.c_int32,
                                            fp, fp, fp, fp, fp, fp, vp, vp]
            l.rgx_autotune.argtypes = [vp, C.POINTER(RgxCamera), C.c_int32, C.POINTER(RgxOpts), C.c_int32,
                                       C.c_int32, fp, vp, fp, fp, fp, fp, fp, fp, C.POINTER(RgxOpts),
                                       C.POINTER(C.c_float), vp]
            for name in EXPORTS:
                f = getattr(l, name)
                if name not in ("rgx_fwd_state_bytes", "rgx_last_error"):
                    f.restype = C.c_int32
            _lib = l
    return _lib


def _check(code, handle=None):
    if code != RGX_OK:
        msg = lib().rgx_last_error(handle).decode(errors="replace")
        raise RgxError(code, msg)


def _ptr(t, name: str = "tensor", numel: int | None = None, dtype=torch.float32, nbytes: int | None = None,
         optional: bool = True):
    """Device pointer of a tensor after the checks the C side cannot make on a
    plain pointer: a contiguous CUDA tensor of the expected dtype holding at
    least `numel` elements (or `nbytes` bytes, for opaque buffers)."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    if nbytes is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{name} holds {t.numel() * t.element_size()} bytes, needs {nbytes}")
    return C.c_void_p(t.data_ptr())


def _same_device(*ts):
    devs = {t.device for t in ts if isinstance(t, torch.Tensor)}
    if len(devs) > 1:
        raise ValueError(f"tensors on different devices: {sorted(map(str, devs))}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ options
def make_opts(o) -> RgxOpts:
    """Convert a ``synth.Options``-like object into the C option struct."""
    x = RgxOpts()
    x.flags = ((RGX_SKIP if o.skip else 0) | (RGX_ADAPTIVE if o.adaptive else 0) |
               (RGX_MORTON if o.morton else 0) | (RGX_ZTILES if o.ztiles else 0) |
               (RGX_MORTON63 if o.morton63 else 0) | (RGX_LOWER_FIRST if getattr(o, "lower_first", False) else 0))
    x.dt, x.dt_min, x.dt_max, x.beta = o.dt, o.dt_min, o.dt_max, o.beta
    x.n_s, x.t_eps, x.sigma_eps = int(o.n_s), o.t_eps, o.sigma_eps
    for i in range(3):
        x.bg[i] = float(o.bg[i])
    x.tile_w, x.tile_h, x.hit_cap, x.max_segments = int(o.tile_w), int(o.tile_h), int(o.hit_cap), int(o.max_segments)
    return x


class Cameras:
    """Pinned host array of rgx_camera structs plus per-camera ray offsets."""

    def __init__(self, cams):
        self.cams = list(cams)
        n = len(self.cams)
        nbytes = C.sizeof(RgxCamera) * n
        self._buf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=torch.cuda.is_available())
        arr = (RgxCamera * n).from_address(self._buf.data_ptr())
        for i, c in enumerate(self.cams):
            m = np.asarray(c.c2w, dtype=np.float32).reshape(12)
            for k in range(12):
                arr[i].c2w[k] = float(m[k])
            arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = c.fx, c.fy, c.cx, c.cy
            arr[i].width, arr[i].height = int(c.width), int(c.height)
            arr[i].t_near, arr[i].t_far = c.t_near, c.t_far
        self.ptr = C.cast(C.c_void_p(self._buf.data_ptr()), C.POINTER(RgxCamera))
        self.count = n
        self.rays_per_cam = [c.width * c.height for c in self.cams]
        self.offsets = np.concatenate([[0], np.cumsum(self.rays_per_cam)]).astype(np.int64)
        self.n_rays = int(self.offsets[-1])


# ------------------------------------------------------------------ C names
def rgx_scene_create(device: int = 0):
    h = C.c_void_p()
    _check(lib().rgx_scene_create(C.byref(h), int(device)))
    return h


def rgx_scene_destroy(h):
    lib().rgx_scene_destroy(h)


def _param_ptrs(n, sh_degree, means, scales, quats, densities, sh, prefix=""):
    """Pointers of the five per-Gaussian arrays (parameters or their gradients)."""
    if not 0 <= int(sh_degree) <= 3:
        raise ValueError("sh_degree must be in 0..3")
    nk = (int(sh_degree) + 1) ** 2
    req = n > 0
    _same_device(means, scales, quats, densities, sh)
    return (_ptr(means, prefix + "means", 3 * n, optional=not req),
            _ptr(scales, prefix + "scales", 3 * n, optional=not req),
            _ptr(quats, prefix + "quats", 4 * n, optional=not req),
            _ptr(densities, prefix + "densities", n, optional=not req),
            _ptr(sh, prefix + "sh", nk * 3 * n, optional=not req))


@_traced
def rgx_build_bvh(h, means, scales, quats, densities, sh, sh_degree, opts, stream=None):
    n = int(means.shape[0])
    ptrs = _param_ptrs(n, sh_degree, means, scales, quats, densities, sh)
    _check(lib().rgx_build_bvh(h, n, int(sh_degree), *ptrs, C.byref(opts), _stream(stream)), h)


def _state_bytes(cams: Cameras) -> int:
    return cams.n_rays * rgx_fwd_state_bytes()


@_traced
def rgx_render_forward(h, cams: Cameras, opts, rgba, state=None, stream=None):
    R = cams.n_rays
    _same_device(rgba, state)
    p_rgba = _ptr(rgba, "rgba", 4 * R, optional=False)
    p_state = _ptr(state, "fwd_state", dtype=None, nbytes=_state_bytes(cams))
    _check(lib().rgx_render_forward(h, cams.ptr, cams.count, C.byref(opts), p_rgba, p_state, _stream(stream)), h)


@_traced
def rgx_render_forward_sched(h, cams: Cameras, opts, rgba, state, sched, sched_n, stream=None):
    R = cams.n_rays
    if sched is None or sched.dim() != 3 or sched.shape[2] != 2:
        raise ValueError("sched must be a [R, sched_cap, 2] tensor")
    cap = int(sched.shape[1])
    _same_device(rgba, state, sched, sched_n)
    p_rgba = _ptr(rgba, "rgba", 4 * R, optional=False)
    p_state = _ptr(state, "fwd_state", dtype=None, nbytes=_state_bytes(cams))
    p_sched = _ptr(sched, "sched", 2 * cap * R, optional=False)
    p_n = _ptr(sched_n, "sched_n", R, dtype=torch.int32, optional=False)
    _check(lib().rgx_render_forward_sched(h, cams.ptr, cams.count, C.byref(opts), p_rgba, p_state, p_sched, cap,
                                          p_n, _stream(stream)), h)


@_traced
def rgx_render_backward(h, cams: Cameras, opts, state, d_rgba, d_means, d_scales, d_quats, d_densities, d_sh,
                        stream=None, n=None, sh_degree: int = 3):
    """`n` (the scene's Gaussian count, when known) and `sh_degree` size-check the
    gradient arrays; without `n` only their dtype and placement are checked."""
    R = cams.n_rays
    _same_device(state, d_rgba, d_means, d_scales, d_quats, d_densities, d_sh)
    p_state = _ptr(state, "fwd_state", dtype=None, nbytes=_state_bytes(cams), optional=False)
    p_d = _ptr(d_rgba, "d_rgba", 4 * R, optional=False)
    g = _param_ptrs(int(n) if n is not None else 0, sh_degree, d_means, d_scales, d_quats, d_densities, d_sh,
                    prefix="d_")
    _check(lib().rgx_render_backward(h, cams.ptr, cams.count, C.byref(opts), p_state, p_d, *g, _stream(stream)), h)


@_traced
def rgx_render_backward_ex(h, cams: Cameras, opts, state, d_rgba, d_means, d_scales, d_quats, d_densities, d_sh,
                           d_sg=None, stat=None, count=None, stream=None, n=None, sh_degree: int = 3, n_sg: int = 0):
    """rgx_render_backward with the optional lobe gradients d_sg [n, n_sg, 7] and each
    camera's Eq. 11 statistic: stat [n] float32 and count [n] int32 (both or neither)."""
    R = cams.n_rays
    nn = int(n) if n is not None else 0
    _same_device(state, d_rgba, d_means, d_scales, d_quats, d_densities, d_sh, d_sg, stat, count)
    if (stat is None) != (count is None):
        raise ValueError("stat and count go together")
    p_state = _ptr(state, "fwd_state", dtype=None, nbytes=_state_bytes(cams), optional=False)
    p_d = _ptr(d_rgba, "d_rgba", 4 * R, optional=False)
    g = _param_ptrs(nn, sh_degree, d_means, d_scales, d_quats, d_densities, d_sh, prefix="d_")
    p_g = _ptr(d_sg, "d_sg", nn * int(n_sg) * 7)
    p_s = _ptr(stat, "stat", nn)
    p_c = _ptr(count, "count", nn, dtype=torch.int32)
    _check(lib().rgx_render_backward_ex(h, cams.ptr, cams.count, C.byref(opts), p_state, p_d, *g, p_g, p_s, p_c,
                                        _stream(stream)), h)


@_traced
def rgx_build_bvh_sg(h, means, scales, quats, densities, sh, sh_degree, sg, opts, stream=None):
    """rgx_build_bvh with spherical-Gaussian lobes sg [n, n_sg, 7] (float32)."""
    n = int(means.shape[0])
    ptrs = _param_ptrs(n, sh_degree, means, scales, quats, densities, sh)
    if sg.dim() != 3 or sg.shape[0] != n or sg.shape[2] != 7 or not 0 <= sg.shape[1] <= 7:
        raise ValueError("sg must be [n, n_sg <= 7, 7]")
    _same_device(means, sg)
    n_sg = int(sg.shape[1])
    p_sg = _ptr(sg, "sg", n * n_sg * 7, optional=n == 0)
    _check(lib().rgx_build_bvh_sg(h, n, int(sh_degree), *ptrs, n_sg, p_sg, C.byref(opts), _stream(stream)), h)


@_traced
def rgx_image_loss(h, cams: Cameras, rgba, target, lam, loss, d_rgba, stream=None):
    """loss [ncam] += (1 - lam) L1 + lam DSSIM per view; d_rgba [R,4] = dL/drgba (Sec. 3.4)."""
    R = cams.n_rays
    _same_device(rgba, target, loss, d_rgba)
    _check(lib().rgx_image_loss(h, cams.ptr, cams.count, _ptr(rgba, "rgba", 4 * R, optional=False),
                                _ptr(target, "target", 3 * R, optional=False), float(lam),
                                _ptr(loss, "loss", cams.count, optional=False),
                                _ptr(d_rgba, "d_rgba", 4 * R, optional=False), _stream(stream)), h)


@_traced
def rgx_adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15, exp_param=False, activated=None,
                  stream=None):
    """One Adam step in place on `param` (and its moments m, v); see include/rgx.h."""
    n = param.numel()
    _same_device(param, grad, m, v, activated)
    _check(lib().rgx_adam_step(n, _ptr(param, "param", n, optional=False), _ptr(grad, "grad", n, optional=False),
                               _ptr(m, "m", n, optional=False), _ptr(v, "v", n, optional=False), float(lr),
                               float(beta1), float(beta2), float(eps), int(step), int(bool(exp_param)),
                               _ptr(activated, "activated", n), _stream(stream)))


def rgx_densify_plan(h, stat, count, scales, tau, size_threshold, action, offset, stream=None) -> int:
    """Clone / split decision per Gaussian (Eq. 11 criterion); returns the new Gaussian count."""
    n = int(stat.numel())
    _same_device(stat, count, scales, action, offset)
    out = C.c_int64(0)
    _check(lib().rgx_densify_plan(h, n, _ptr(stat, "stat", n), _ptr(count, "count", n, dtype=torch.int32),
                                  _ptr(scales, "scales", 3 * n), float(tau), float(size_threshold),
                                  _ptr(action, "action", n, dtype=torch.int32),
                                  _ptr(offset, "offset", n, dtype=torch.int32), C.byref(out), _stream(stream)), h)
    return int(out.value)


@_traced
def rgx_densify_apply(action, offset, normals, params, outs, sg=None, out_sg=None, out_src=None, stream=None):
    """Write the kept, cloned and split Gaussians of a plan; params / outs are (means, scales,
    quats, densities, sh) tensors, normals [n, 2, 3]."""
    n = int(action.numel())
    means, scales, quats, dens, sh = params
    om, os_, oq, od, osh = outs
    _same_device(action, offset, normals, *params, *outs, sg, out_sg, out_src)
    shf = int(sh[0].numel()) if n > 0 else 0
    sgf = int(sg[0].numel()) if (sg is not None and n > 0) else 0
    _check(lib().rgx_densify_apply(n, _ptr(action, "action", n, dtype=torch.int32),
                                   _ptr(offset, "offset", n, dtype=torch.int32), _ptr(normals, "normals", 6 * n),
                                   _ptr(means, "means", 3 * n), _ptr(scales, "scales", 3 * n),
                                   _ptr(quats, "quats", 4 * n), _ptr(dens, "densities", n), _ptr(sh, "sh", shf * n),
                                   shf, _ptr(sg, "sg", sgf * n), sgf, _ptr(om, "out_means"), _ptr(os_, "out_scales"),
                                   _ptr(oq, "out_quats"), _ptr(od, "out_densities"), _ptr(osh, "out_sh"),
                                   _ptr(out_sg, "out_sg"), _ptr(out_src, "out_src", dtype=torch.int32),
                                   _stream(stream)))


def rgx_sync_status(h, stream=None) -> int:
    return int(lib().rgx_sync_status(h, _stream(stream)))


def rgx_fwd_state_bytes() -> int:
    return int(lib().rgx_fwd_state_bytes())


def new_state(n_rays: int, device) -> torch.Tensor:
    """An uninitialised forward-state buffer: n_rays x rgx_fwd_state_bytes(), as float32 words."""
    return torch.empty(n_rays, rgx_fwd_state_bytes() // 4, dtype=torch.float32, device=device)


def rgx_get_bvh(h, n, stream=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    codes = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    nodes = torch.empty(max(n - 1, 1), 16, dtype=torch.float32, device=dev)
    root = torch.empty(6, dtype=torch.float32, device=dev)
    _check(lib().rgx_get_bvh(h, _ptr(codes, dtype=torch.int64), _ptr(perm, dtype=torch.int32), _ptr(nodes),
                             _ptr(root), _stream(stream)), h)
    return codes[:n], perm[:n], nodes, root


def rgx_get_counters(h, stream=None):
    out = (C.c_uint64 * 8)()
    _check(lib().rgx_get_counters(h, out, _stream(stream)), h)
    keys = ["rays", "segments", "hits", "evals", "node_visits", "closest_hit", "skipped", "windows"]
    return dict(zip(keys, [int(v) for v in out]))


def rgx_set_tape_limit(h, max_entries: int):
    """Cap the forward's tape of first chord lists (0: no tape, < 0: default sizing)."""
    _check(lib().rgx_set_tape_limit(h, int(max_entries)), h)


@_traced
def rgx_autotune(h, cams: Cameras, base, mode, with_backward, rgba, state, d_rgba, grads, stream=None):
    """Returns (best RgxOpts, best time in ms).  `mode`: RGX_TUNE_NS | RGX_TUNE_EXHAUSTIVE
    (0 = tile shape and hit_cap, one knob at a time).  `grads` are scratch buffers."""
    best = RgxOpts()
    ms = C.c_float(0.0)
    R = cams.n_rays
    g = grads if grads is not None else [None] * 5
    _same_device(rgba, state, d_rgba, *g)
    p_rgba = _ptr(rgba, "rgba", 4 * R, optional=False)
    p_state = _ptr(state, "fwd_state", dtype=None, nbytes=_state_bytes(cams), optional=False)
    p_d = _ptr(d_rgba, "d_rgba", 4 * R, optional=not with_backward)
    p_g = [_ptr(x, "gradient scratch", optional=not with_backward) for x in g]
    _check(lib().rgx_autotune(h, cams.ptr, cams.count, C.byref(base), int(mode), int(with_backward),
                              p_rgba, p_state, p_d, *p_g, C.byref(best), C.byref(ms), _stream(stream)), h)
    return best, float(ms.value)


@_traced
def rgx_morton_sort_noalloc(means, wide, codes, perm, stream=None):
    """Sorted Morton codes / permutation of `means` with no device allocation
    (static scratch, n <= 262144).  codes: int64 [n] (uint64 bits), perm: int32 [n]."""
    n = int(means.shape[0])
    _same_device(means, codes, perm)
    p_m = _ptr(means, "means", 3 * n)
    p_c = _ptr(codes, "codes", n, dtype=torch.int64)
    p_p = _ptr(perm, "perm", n, dtype=torch.int32)
    _check(lib().rgx_morton_sort_noalloc(n, p_m, int(bool(wide)), p_c, p_p, _stream(stream)))


@_traced
def rgx_isotropic_loss(scales, r0, weight, loss, d_scales, stream=None):
    """loss (device float [1]) += weight * L_s; d_scales += weight * dL_s/ds (Eqs. 6-8)."""
    n = int(scales.shape[0])
    _same_device(scales, loss, d_scales)
    p_s = _ptr(scales, "scales", 3 * n)
    p_l = _ptr(loss, "loss", 1)
    p_g = _ptr(d_scales, "d_scales", 3 * n)
    _check(lib().rgx_isotropic_loss(n, p_s, float(r0), float(weight), p_l, p_g, _stream(stream)))


@_traced
def rgx_densify_accumulate(means, d_means, cams: Cameras, stat, count, stream=None):
    """Eq. 11 statistic of one view (cams holds exactly one camera)."""
    if cams.count != 1:
        raise ValueError("one camera per call")
    n = int(means.shape[0])
    _same_device(means, d_means, stat, count)
    p_m = _ptr(means, "means", 3 * n)
    p_d = _ptr(d_means, "d_means", 3 * n)
    p_s = _ptr(stat, "stat", n)
    p_c = _ptr(count, "count", n, dtype=torch.int32)
    _check(lib().rgx_densify_accumulate(n, p_m, p_d, cams.ptr, p_s, p_c, _stream(stream)))


# ------------------------------------------------------------------ convenience
class Scene:
    """Owner of one rgx_scene handle on the current CUDA device."""

    def __init__(self, device: int | None = None):
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.h = rgx_scene_create(self.device)
        self.n = 0
        self.sh_degree = 3
        self.n_sg = 0
        self._keep = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                rgx_scene_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def build(self, means, scales, quats, densities, sh, opts, sh_degree: int = 3, stream=None, sg=None):
        for t in (means, scales, quats, densities, sh, sg):
            if isinstance(t, torch.Tensor) and t.is_cuda and t.device.index != self.device:
                raise ValueError(f"parameters on {t.device}, scene on cuda:{self.device}")
        if sg is None:
            rgx_build_bvh(self.h, means, scales, quats, densities, sh, sh_degree, opts, stream)
            self.n_sg = 0
        else:
            rgx_build_bvh_sg(self.h, means, scales, quats, densities, sh, sh_degree, sg, opts, stream)
            self.n_sg = int(sg.shape[1])
        self.n = int(means.shape[0])
        self.sh_degree = int(sh_degree)

    def forward(self, cams: Cameras, opts, want_state: bool = True, stream=None, sched_cap: int = 0):
        dev = torch.device("cuda", self.device)
        rgba = torch.empty(cams.n_rays, 4, dtype=torch.float32, device=dev)
        state = new_state(cams.n_rays, dev) if want_state else None
        self._keep = cams
        if sched_cap > 0:
            sched = torch.zeros(cams.n_rays, sched_cap, 2, dtype=torch.float32, device=dev)
            sched_n = torch.zeros(cams.n_rays, dtype=torch.int32, device=dev)
            rgx_render_forward_sched(self.h, cams, opts, rgba, state, sched, sched_n, stream)
            return rgba, state, sched, sched_n
        rgx_render_forward(self.h, cams, opts, rgba, state, stream)
        return rgba, state

    def backward(self, cams: Cameras, opts, state, d_rgba, grads, stream=None):
        self._keep = cams
        rgx_render_backward(self.h, cams, opts, state, d_rgba, *grads, stream=stream, n=self.n,
                            sh_degree=self.sh_degree)

    def backward_ex(self, cams: Cameras, opts, state, d_rgba, grads, d_sg=None, stat=None, count=None, stream=None):
        """Adjoint with the lobe gradients (d_sg) and/or each camera's Eq. 11 statistic."""
        self._keep = cams
        rgx_render_backward_ex(self.h, cams, opts, state, d_rgba, *grads, d_sg=d_sg, stat=stat, count=count,
                               stream=stream, n=self.n, sh_degree=self.sh_degree, n_sg=self.n_sg)

    def status(self, stream=None) -> int:
        return rgx_sync_status(self.h, stream)

    def bvh(self, stream=None):
        return rgx_get_bvh(self.h, self.n, stream)

    def counters(self, stream=None):
        return rgx_get_counters(self.h, stream)

    def autotune(self, cams: Cameras, base, tune_ns: bool = False, with_backward: bool = True, stream=None,
                 exhaustive: bool = False):
        """Pick tile shape / hit_cap (/ N_S) by timing on this scene; returns (RgxOpts, ms).  The
        scene keeps the pick: later calls whose options leave those knobs at 0 use it."""
        dev = torch.device("cuda", self.device)
        rgba = torch.empty(cams.n_rays, 4, dtype=torch.float32, device=dev)
        state = new_state(cams.n_rays, dev)
        d_rgba, grads = None, None
        if with_backward:
            d_rgba = torch.randn(cams.n_rays, 4, dtype=torch.float32, device=dev)
            n = max(self.n, 1)
            grads = [torch.zeros(n, 3, device=dev), torch.zeros(n, 3, device=dev), torch.zeros(n, 4, device=dev),
                     torch.zeros(n, device=dev), torch.zeros(n, 16, 3, device=dev)]
        self._keep = cams
        mode = (RGX_TUNE_NS if tune_ns else 0) | (RGX_TUNE_EXHAUSTIVE if exhaustive else 0)
        return rgx_autotune(self.h, cams, base, mode, with_backward, rgba, state, d_rgba, grads, stream)

    def set_tape_limit(self, max_entries: int):
        rgx_set_tape_limit(self.h, max_entries)


def scene_tensors(scene, device="cuda"):
    """Upload a ``synth.Scene`` as contiguous float32 CUDA tensors."""
    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device).contiguous()
    nk = (scene.sh_degree + 1) ** 2
    return (t(scene.means).reshape(-1, 3), t(scene.scales).reshape(-1, 3), t(scene.quats).reshape(-1, 4),
            t(scene.densities).reshape(-1), t(scene.sh).reshape(-1, nk, 3))


def sg_tensor(scene, device="cuda"):
    """The scene's spherical-Gaussian lobes as a contiguous float32 CUDA tensor (or None)."""
    if getattr(scene, "sg", None) is None:
        return None
    return torch.as_tensor(np.ascontiguousarray(scene.sg, dtype=np.float32), device=device).contiguous()
