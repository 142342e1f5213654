"""FP64 CPU oracle for differentiable Gaussian volume ray marching.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The library's product path never
imports it, and it shares no code with the CUDA implementation.

The arithmetic lives in ``rgx_oracle.c`` (plain C, FP64, OpenMP over rays),
compiled on first use with gcc into ``oracle/_build/``.  This module only
marshals numpy arrays.  ``morton.py`` and ``lbvh.py`` hold the integer parts
(Z-order codes, Karras radix tree) in plain numpy / Python.

Every input array is promoted from the caller's float32 to float64 here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librgx_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=gnu11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class OxCamera(C.Structure):
    _fields_ = [("c2w", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32), ("t_near", C.c_double), ("t_far", C.c_double)]


class OxOpts(C.Structure):
    _fields_ = [("skip", C.c_int32), ("adaptive", C.c_int32), ("n_s", C.c_int32),
                ("max_segments", C.c_int32), ("dt", C.c_double), ("dt_min", C.c_double),
                ("dt_max", C.c_double), ("beta", C.c_double), ("t_eps", C.c_double),
                ("sigma_eps", C.c_double), ("bg", C.c_double * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int64)
            l.ox_render.restype = C.c_int64
            l.ox_render.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_int32, C.c_int32, dp,
                                    C.POINTER(OxCamera), C.POINTER(OxOpts), C.c_int64, ip,
                                    dp, dp, ip, ip, C.c_int64, dp, ip, C.c_int32, C.c_int32, C.c_int32]
            l.ox_backward.restype = C.c_int64
            l.ox_backward.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_int32, C.c_int32, dp,
                                      C.POINTER(OxCamera), C.POINTER(OxOpts), C.c_int64, ip, dp,
                                      dp, dp, dp, dp, dp, dp, C.c_int32]
            l.ox_sh_basis.restype = None
            l.ox_sh_basis.argtypes = [C.c_int, dp, dp]
            l.ox_quat_to_rot.restype = None
            l.ox_quat_to_rot.argtypes = [dp, dp]
            l.ox_prim_geometry.restype = None
            l.ox_prim_geometry.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_double, dp, dp, dp, dp]
            l.ox_ray.restype = None
            l.ox_ray.argtypes = [C.POINTER(OxCamera), C.c_int64, dp, dp]
            l.ox_chords.restype = None
            l.ox_chords.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_double, dp, dp, dp, dp]
            _lib = l
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(C.POINTER(C.c_double))
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def camera(cam) -> OxCamera:
    c = OxCamera()
    c2w = np.asarray(cam.c2w, dtype=np.float64).reshape(12)
    for i in range(12):
        c.c2w[i] = c2w[i]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.t_near, c.t_far = float(cam.t_near), float(cam.t_far)
    return c


def opts(o) -> OxOpts:
    x = OxOpts()
    x.skip, x.adaptive, x.n_s = int(bool(o.skip)), int(bool(o.adaptive)), int(o.n_s)
    x.max_segments = int(o.max_segments)
    x.dt, x.dt_min, x.dt_max, x.beta = float(o.dt), float(o.dt_min), float(o.dt_max), float(o.beta)
    x.t_eps, x.sigma_eps = float(o.t_eps), float(o.sigma_eps)
    for i in range(3):
        x.bg[i] = float(o.bg[i])
    return x


class Params:
    """FP64 copies of a scene's parameter arrays (the oracle's inputs)."""

    def __init__(self, scene):
        self.n = int(scene.means.shape[0])
        self.means = _d(scene.means).reshape(self.n, 3)
        self.scales = _d(scene.scales).reshape(self.n, 3)
        self.quats = _d(scene.quats).reshape(self.n, 4)
        self.dens = _d(scene.densities).reshape(self.n)
        self.sh_degree = int(scene.sh_degree)
        nk = (self.sh_degree + 1) ** 2
        self.sh = _d(scene.sh).reshape(self.n, nk, 3)
        sg = getattr(scene, "sg", None)
        # spherical-Gaussian lobes: (u_x, u_y, u_z, lambda, a_r, a_g, a_b) per lobe, or none
        self.sg = None if sg is None else _d(sg).reshape(self.n, -1, 7)
        self.n_sg = 0 if self.sg is None else int(self.sg.shape[1])

    def arrays(self):
        return [self.means, self.scales, self.quats, self.dens, self.sh]


def render(scene, cam, o, pix=None, sched_cap: int = 0, sched=None, sched_n=None,
           brute: bool = False, nthreads: int = 0, params: Params | None = None):
    """Forward render of one camera (all pixels, or the flat indices ``pix``).

    Returns dict(rgba[npix,4], state[npix,4]=(C,T), nseg[npix], active[npix,2],
    sched[npix,cap,2], sched_n[npix], n_iter_limit).  Passing ``sched`` and
    ``sched_n`` replays those evaluated segments instead of taking decisions.
    """
    P = params or Params(scene)
    pix_a = None if pix is None else np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    npix = cam.width * cam.height if pix_a is None else int(pix_a.shape[0])
    rgba = np.zeros((npix, 4))
    state = np.zeros((npix, 4))
    nseg = np.zeros(npix, dtype=np.int64)
    active = np.zeros((npix, 2), dtype=np.int64)
    replay = 0
    if sched is not None:
        sched = _d(sched)
        sched_n = np.ascontiguousarray(np.asarray(sched_n, dtype=np.int64))
        sched_cap = sched.shape[1]
        replay = 1
    elif sched_cap > 0:
        sched = np.zeros((npix, sched_cap, 2))
        sched_n = np.zeros(npix, dtype=np.int64)
    cm, op = camera(cam), opts(o)
    nerr = lib().ox_render(P.n, _ptr(P.means), _ptr(P.scales), _ptr(P.quats), _ptr(P.dens), _ptr(P.sh),
                           P.sh_degree, P.n_sg, _ptr(P.sg), C.byref(cm), C.byref(op), npix, _ptr(pix_a),
                           _ptr(rgba), _ptr(state), _ptr(nseg), _ptr(active),
                           int(sched_cap), _ptr(sched), _ptr(sched_n), replay, int(brute), int(nthreads))
    return dict(rgba=rgba, state=state, nseg=nseg, active=active, sched=sched, sched_n=sched_n,
                n_iter_limit=int(nerr))


def backward(scene, cam, o, d_rgba, pix=None, nthreads: int = 0, params: Params | None = None):
    """Analytic gradient of sum <d_rgba, rgba> w.r.t. the five parameter arrays."""
    P = params or Params(scene)
    pix_a = None if pix is None else np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    npix = cam.width * cam.height if pix_a is None else int(pix_a.shape[0])
    up = _d(d_rgba).reshape(npix, 4)
    g = [np.zeros_like(a) for a in P.arrays()]
    g_sg = np.zeros_like(P.sg) if P.sg is not None else None
    cm, op = camera(cam), opts(o)
    nerr = lib().ox_backward(P.n, _ptr(P.means), _ptr(P.scales), _ptr(P.quats), _ptr(P.dens), _ptr(P.sh),
                             P.sh_degree, P.n_sg, _ptr(P.sg), C.byref(cm), C.byref(op), npix, _ptr(pix_a), _ptr(up),
                             *[_ptr(x) for x in g], _ptr(g_sg), int(nthreads))
    out = dict(means=g[0], scales=g[1], quats=g[2], densities=g[3], sh=g[4], n_iter_limit=int(nerr))
    if g_sg is not None:
        out["sg"] = g_sg
    return out


def sh_basis(d, deg: int = 3) -> np.ndarray:
    d = _d(d).reshape(3)
    Y = np.zeros(16)
    lib().ox_sh_basis(int(deg), _ptr(d), _ptr(Y))
    return Y[: (deg + 1) ** 2]


def quat_to_rot(q) -> np.ndarray:
    q = _d(q).reshape(4)
    R = np.zeros(9)
    lib().ox_quat_to_rot(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def prim_geometry(scene, sigma_eps: float):
    """(R[N,3,3], M[N,3,3], Q_eps[N], AABB half-lengths[N,3]) in FP64."""
    P = Params(scene)
    R, M = np.zeros((P.n, 9)), np.zeros((P.n, 9))
    Qe, half = np.zeros(P.n), np.zeros((P.n, 3))
    lib().ox_prim_geometry(P.n, _ptr(P.means), _ptr(P.scales), _ptr(P.quats), _ptr(P.dens),
                           float(sigma_eps), _ptr(R), _ptr(M), _ptr(Qe), _ptr(half))
    return R.reshape(-1, 3, 3), M.reshape(-1, 3, 3), Qe, half


def ray(cam, pix: int):
    o, d = np.zeros(3), np.zeros(3)
    cm = camera(cam)
    lib().ox_ray(C.byref(cm), int(pix), _ptr(o), _ptr(d))
    return o, d


def chords(scene, sigma_eps: float, o, d):
    """(t_in[N], t_out[N]) of ray o + t d with every Gaussian; NaN when empty."""
    P = Params(scene)
    tin, tout = np.zeros(P.n), np.zeros(P.n)
    o, d = _d(o).reshape(3), _d(d).reshape(3)
    lib().ox_chords(P.n, _ptr(P.means), _ptr(P.scales), _ptr(P.quats), _ptr(P.dens), float(sigma_eps),
                    _ptr(o), _ptr(d), _ptr(tin), _ptr(tout))
    return tin, tout
