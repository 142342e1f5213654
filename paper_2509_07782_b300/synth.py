"""Seeded synthetic scenes and cameras for the Gaussian ray-marching path.

This module only *draws inputs*: Gaussian parameter arrays (means, linear
scales, (w,x,y,z) quaternions, densities, degree-3 SH coefficients) and pinhole
cameras.  It contains none of the rendering arithmetic, so both the FP64 oracle
and the CUDA library can consume its output without sharing method code.

The paper evaluates on NeRF-Synthetic, NSVF, Mip-NeRF360, Tanks&Temples and
Deep Blending captures, none of which are available here.  The five workloads
below stand in for them:

* ``plain_2k``    — 2,000 Gaussians in a cube, one 64x64 view, fixed step, no
                    skipping (the paper's uniform-sampling baseline).
* ``torus_100k``  — an object-centric scene (like the synthetic datasets, Sec. 4.3)
                    at 800x800, forward + adjoint with skipping + adaptive step.
* ``outdoor_3m``  — an unbounded scene (like Mip-NeRF360, Sec. 4.4) with a dense
                    central cluster and a background shell up to radius 100.
* ``batch_1m``    — 1M torus Gaussians, 8 views of uneven resolution in one launch.
* ``sweep_6m``    — 6M torus Gaussians, 64 views, forward only.

Distributions follow the workload recipes: log-normal scales/densities,
Shoemake-uniform rotations, SH coefficients ~ N(0, 0.2) (the +0.5 offset is
part of the colour activation, not of the coefficients).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

SH_COEFFS = 16  # degree 3


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV convention (+z forward, +y down, +x right).

    ``c2w`` is a row-major 3x4 camera-to-world matrix whose last column is the
    camera centre.  Pixel (u, v) looks through ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1).
    ``t_far <= 0`` means "exit of the scene bounding box".
    """
    c2w: np.ndarray  # (3, 4) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    t_near: float = 0.0
    t_far: float = 0.0

    @property
    def n_rays(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # (N, 3) float32
    scales: np.ndarray     # (N, 3) float32, linear, > 0
    quats: np.ndarray      # (N, 4) float32, (w, x, y, z), unnormalised allowed
    densities: np.ndarray  # (N,)   float32, > 0
    sh: np.ndarray         # (N, 16, 3) float32
    sh_degree: int = 3
    sg: np.ndarray | None = None  # (N, n_sg, 7) float32 spherical-Gaussian lobes: axis (raw), sharpness, RGB

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx], self.scales[idx], self.quats[idx],
                     self.densities[idx], self.sh[idx], self.sh_degree,
                     None if self.sg is None else self.sg[idx])

    def permuted(self, perm) -> "Scene":
        return self.subset(np.asarray(perm))


@dataclasses.dataclass
class Options:
    """Marching options (values of Alg. 1 / Eq. 5 inputs)."""
    skip: bool = False          # empty-space skipping (ClosestHit)
    adaptive: bool = False      # Eq. 5 segment size
    morton: bool = False        # store parameters in Z-order
    ztiles: bool = False        # Z-order 2D ray tiles
    morton63: bool = False      # 63-bit instead of 30-bit Morton codes
    lower_first: bool = False   # scheduling: lower an overflowing first window instead of giving up
    dt: float = 0.01
    dt_min: float = 0.005
    dt_max: float = 0.02
    beta: float = 1024.0
    n_s: int = 16
    t_eps: float = 1e-4
    sigma_eps: float = 1e-3
    bg: tuple = (0.0, 0.0, 0.0)
    tile_w: int = 8
    tile_h: int = 4
    hit_cap: int = 256
    max_segments: int = 0       # 0 = derived from the ray length


# ----------------------------------------------------------------------------
# primitive draws
# ----------------------------------------------------------------------------

def shoemake_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake 1992), as (w, x, y, z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1).astype(np.float32)


def _finish(rng, means, log_scale_mu, log_scale_sd, log_dens_mu, log_dens_sd) -> Scene:
    n = means.shape[0]
    log_s = rng.normal(0.0, 1.0, size=(n, 3)) * log_scale_sd + np.asarray(log_scale_mu).reshape(-1, 1)
    scales = np.exp(log_s).astype(np.float32)
    quats = shoemake_quats(rng, n)
    dens = np.exp(rng.normal(log_dens_mu, log_dens_sd, size=n)).astype(np.float32)
    sh = rng.normal(0.0, 0.2, size=(n, SH_COEFFS, 3)).astype(np.float32)
    return Scene(means.astype(np.float32), scales, quats, dens, sh, 3)


def with_sg_appearance(scene: Scene, seed: int, n_sg: int = 7, sh_degree: int = 2) -> Scene:
    """The scene with the appearance model of the SH/SG comparison (Supp. Sec. 6.1):
    SH up to ``sh_degree`` (9 coefficients per channel at degree 2) plus ``n_sg``
    spherical-Gaussian lobes per Gaussian.  Lobe draws: axis direction uniform on the
    sphere with a length in [0.5, 2] (the renderer normalises it), sharpness
    log-uniform in [0.5, 30], RGB amplitude ~ N(0, 0.15)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = scene.n
    nk = (sh_degree + 1) ** 2
    v = rng.normal(size=(n, n_sg, 3))
    v /= np.linalg.norm(v, axis=2, keepdims=True)
    v *= rng.uniform(0.5, 2.0, size=(n, n_sg, 1))
    lam = np.exp(rng.uniform(np.log(0.5), np.log(30.0), size=(n, n_sg, 1)))
    amp = rng.normal(0.0, 0.15, size=(n, n_sg, 3))
    sg = np.concatenate([v, lam, amp], axis=2).astype(np.float32)
    return Scene(scene.means, scene.scales, scene.quats, scene.densities,
                 np.ascontiguousarray(scene.sh[:, :nk, :]), sh_degree, sg)


def cube_scene(n: int, seed: int) -> Scene:
    """Means uniform in [-1,1]^3, log s ~ N(-3,0.5), log sigma ~ N(1,0.5)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    return _finish(rng, means, -3.0, 0.5, 1.0, 0.5)


def torus_scene(n: int, seed: int, major: float = 1.0, minor: float = 0.35) -> Scene:
    """Gaussians on a noise-perturbed torus surface around the z axis.

    The minor radius is perturbed by a sum of 8 periodic sinusoids in (u, v)
    of total amplitude 0.03; each point is pushed along the surface normal by
    N(0, 0.01).  log s ~ N(-4.5, 0.4), log sigma ~ N(2, 0.7).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ku = rng.integers(1, 7, size=8)
    kv = rng.integers(1, 7, size=8)
    ph = rng.uniform(0, 2 * np.pi, size=8)
    u = rng.uniform(0, 2 * np.pi, size=n)
    v = rng.uniform(0, 2 * np.pi, size=n)
    noise = np.zeros(n)
    for i in range(8):
        noise += np.sin(ku[i] * u + kv[i] * v + ph[i])
    r = minor + 0.03 * noise / 8.0
    r = r + rng.normal(0.0, 0.01, size=n)
    nx, ny, nz = np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)
    means = np.stack([major * np.cos(u) + r * nx, major * np.sin(u) + r * ny, r * nz], axis=1)
    return _finish(rng, means, -4.5, 0.4, 2.0, 0.7)


def outdoor_scene(n: int, seed: int) -> Scene:
    """Unbounded scene: 60% in 200 isotropic blobs inside the unit ball, 40% on a
    background shell with radius log-uniform in [1, 100].  log s grows with
    log-radius: N(-4.5 + ln max(r, 1), 0.4); log sigma ~ N(1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_fg = int(round(0.6 * n))
    n_bg = n - n_fg
    # blob centres uniform in the unit ball
    c = rng.normal(size=(200, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    c *= rng.random(200)[:, None] ** (1.0 / 3.0)
    sd = rng.uniform(0.03, 0.15, size=200)
    which = rng.integers(0, 200, size=n_fg)
    fg = c[which] + rng.normal(size=(n_fg, 3)) * sd[which, None]
    dirs = rng.normal(size=(n_bg, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = np.exp(rng.uniform(0.0, math.log(100.0), size=n_bg))
    bg = dirs * rad[:, None]
    means = np.concatenate([fg, bg], axis=0)
    rr = np.linalg.norm(means, axis=1)
    return _finish(rng, means, -4.5 + np.log(np.maximum(rr, 1.0)), 0.4, 1.0, 1.0)


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at(position, target, fov_deg: float, width: int, height: int) -> Camera:
    """Pinhole camera at ``position`` looking at ``target``; vertical fov."""
    p = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - p
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(f @ up) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    c2w = np.zeros((3, 4))
    c2w[:, 0], c2w[:, 1], c2w[:, 2], c2w[:, 3] = right, down, f, p
    focal = 0.5 * height / math.tan(math.radians(fov_deg) / 2.0)
    return Camera(c2w.astype(np.float32), float(focal), float(focal),
                  0.5 * width, 0.5 * height, int(width), int(height))


def orbit_camera(rng, radius: float, width: int, height: int, fov_deg: float = 50.0,
                 elev_deg=(-30.0, 60.0)) -> Camera:
    az = rng.uniform(0.0, 2 * np.pi)
    el = math.radians(rng.uniform(*elev_deg))
    pos = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return look_at(pos, np.zeros(3), fov_deg, width, height)


def sphere_camera(rng, radius: float, width: int, height: int, fov_deg: float = 50.0) -> Camera:
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return look_at(radius * d, np.zeros(3), fov_deg, width, height)


def inside_camera(rng, max_r: float, width: int, height: int, fov_deg: float = 50.0) -> Camera:
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    pos = d * max_r * rng.random() ** (1.0 / 3.0)
    look = rng.normal(size=3)
    look /= np.linalg.norm(look)
    return look_at(pos, pos + look, fov_deg, width, height)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

BATCH_RES = [(320, 240), (640, 480), (800, 800), (1024, 768), (1237, 822),
             (1600, 1200), (1920, 1080), (512, 512)]


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cameras: List[Camera]
    options: Options
    backward: bool

    @property
    def n_rays(self) -> int:
        return sum(c.n_rays for c in self.cameras)


def fast_options(**kw) -> Options:
    o = Options(skip=True, adaptive=True, morton=True, ztiles=True)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def workload(name: str, n: int | None = None, scale_res: float | None = None) -> Workload:
    """Build one of the five workloads.  ``n`` overrides the Gaussian count and
    ``scale_res`` scales every camera's resolution (both for quick tests)."""
    if name == "plain_2k":
        seed = 1001
        sc = cube_scene(n or 2000, seed)
        cams = [sphere_camera(np.random.Generator(np.random.PCG64(seed + 100)), 3.0, 64, 64)]
        opt = Options(skip=False, adaptive=False, dt=0.01, n_s=16)
        bw = False
    elif name == "torus_100k":
        seed = 1002
        sc = torus_scene(n or 100_000, seed)
        cams = [orbit_camera(np.random.Generator(np.random.PCG64(seed + 100)), 4.0, 800, 800)]
        opt = fast_options()
        bw = True
    elif name == "outdoor_3m":
        seed = 1003
        sc = outdoor_scene(n or 3_000_000, seed)
        cams = [inside_camera(np.random.Generator(np.random.PCG64(seed + 100)), 0.3, 1237, 822)]
        opt = fast_options(morton63=True)
        bw = True
    elif name == "batch_1m":
        seed = 1004
        sc = torus_scene(n or 1_000_000, seed)
        rng = np.random.Generator(np.random.PCG64(seed + 100))
        cams = [orbit_camera(rng, 4.0, w, h) for (w, h) in BATCH_RES]
        opt = fast_options()
        bw = True
    elif name == "sweep_6m":
        seed = 1005
        sc = torus_scene(n or 6_000_000, seed)
        rng = np.random.Generator(np.random.PCG64(seed + 100))
        cams = []
        for _ in range(64):
            w = int(rng.integers(256, 1921))
            h = int(rng.integers(256, 1081))
            cams.append(orbit_camera(rng, 4.0, w, h))
        opt = fast_options()
        bw = False
    else:
        raise KeyError(name)
    if scale_res is not None:
        cams = [rescale_camera(c, scale_res) for c in cams]
    return Workload(name, sc, cams, opt, bw)


def rescale_camera(cam: Camera, s: float) -> Camera:
    w = max(1, int(round(cam.width * s)))
    h = max(1, int(round(cam.height * s)))
    return Camera(cam.c2w.copy(), cam.fx * h / cam.height, cam.fy * h / cam.height,
                  0.5 * w, 0.5 * h, w, h, cam.t_near, cam.t_far)


def pixel_subset(cam: Camera, count: int, seed: int) -> np.ndarray:
    """Seeded subset of flat pixel indices (row-major) of one camera."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(count, cam.n_rays)
    return np.sort(rng.choice(cam.n_rays, size=count, replace=False)).astype(np.int64)
