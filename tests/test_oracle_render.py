"""Pins of the oracle's forward march (Eq. 1-5, Algorithm 1).

Independent references used here:
* the line integral of one truncated Gaussian has an erf closed form; the
  marched Eq. 3 must converge to the continuous Eq. 2 as the step shrinks
  (uniform and adaptive schedules, with and without skipping);
* two Gaussians that do not overlap along a ray composite in closed form;
* a scene whose Gaussians all share one colour c gives RGB = c (1 - T) + T bg;
* invariants: empty scene -> background; opacity in [0,1]; primitive order is
  irrelevant; skipping changes a uniform-step render by at most T_eps * max c;
  per-sample brute force over every Gaussian equals the chord pre-filter;
* Eq. 5 special cases (T = 1 gives max(t/beta, dt_min) clamped to dt_max);
* Algorithm 1's termination (stop once T <= T_eps at a segment start) and
  skipping (the first evaluated segment starts at the nearest chord entry).
Rays, rotations, chords and SH values are rebuilt here from their definitions
with scipy, not taken from the oracle.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import erf, sph_harm_y

import oracle
from paper_2509_07782_b300 import synth

SIG_EPS = 1e-3


# ---------------------------------------------------------------- helpers
def pinhole_ray(cam, pix):
    u, v = pix % cam.width, pix // cam.width
    dc = np.array([(u + 0.5 - cam.cx) / cam.fx, (v + 0.5 - cam.cy) / cam.fy, 1.0])
    c2w = np.asarray(cam.c2w, dtype=np.float64)
    d = c2w[:, :3] @ dc
    return c2w[:, 3].copy(), d / np.linalg.norm(d)


def real_sh(d):
    x, y, z = d
    th, ph = math.acos(max(-1, min(1, z))), math.atan2(y, x)
    out = []
    for l in range(4):
        for m in range(-l, l + 1):
            if m > 0:
                out.append(math.sqrt(2) * sph_harm_y(l, m, th, ph).real)
            elif m < 0:
                out.append(math.sqrt(2) * sph_harm_y(l, -m, th, ph).imag)
            else:
                out.append(sph_harm_y(l, 0, th, ph).real)
    return np.array(out)


def gauss_line_integral(mu, s, qwxyz, sig, o, d):
    """Optical depth of one Q_eps-truncated Gaussian along o + t d (Eq. 2):
    q(t) = a (t - t_c)^2 + q_min,  tau = sig e^{-q_min/2} sqrt(pi/(2a)) [erf(.)]_{t_in}^{t_out}."""
    R = Rotation.from_quat([qwxyz[1], qwxyz[2], qwxyz[3], qwxyz[0]]).as_matrix()
    Minv = np.diag(1.0 / np.asarray(s)) @ R.T
    y0, yd = Minv @ (o - mu), Minv @ d
    a = yd @ yd
    tc = -(y0 @ yd) / a
    qmin = (y0 + tc * yd) @ (y0 + tc * yd)
    Qe = 2 * math.log(sig / SIG_EPS)
    if qmin >= Qe:
        return 0.0, None
    h = math.sqrt((Qe - qmin) / a)
    k = math.sqrt(a / 2)
    tau = sig * math.exp(-qmin / 2) * math.sqrt(math.pi / (2 * a)) * (erf(k * h) - erf(-k * h))
    return tau, (tc - h, tc + h)


def one_gaussian_scene(seed=0, center=(0, 0, 0), sig=5.0, scale=0.08):
    rng = np.random.default_rng(seed)
    means = np.array([center], float)
    scales = scale * np.exp(rng.normal(0, 0.3, size=(1, 3)))
    quats = rng.normal(size=(1, 4))
    dens = np.array([sig])
    sh = rng.normal(0, 0.2, size=(1, 16, 3))
    return synth.Scene(means, scales, quats, dens, sh, 3)


def camera_at(pos, target=(0, 0, 0), w=12, h=12, fov=30.0):
    return synth.look_at(np.asarray(pos, float), np.asarray(target, float), fov, w, h)


def colour_of(scene, l, d):
    Y = real_sh(d)
    return np.maximum(0.0, 0.5 + Y @ scene.sh[l])


def opts(**kw):
    o = synth.Options(sigma_eps=SIG_EPS)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("mode", ["uniform", "uniform_skip", "adaptive_skip"])
def test_single_gaussian_erf_closed_form(mode):
    sc = one_gaussian_scene()
    cam = camera_at([0.3, -1.2, 1.5])
    if mode == "uniform":
        o_ = opts(dt=5e-5, n_s=16, t_eps=0.0)
    elif mode == "uniform_skip":
        o_ = opts(dt=5e-5, n_s=16, t_eps=0.0, skip=True)
    else:
        o_ = opts(adaptive=True, skip=True, dt_min=2e-5, dt_max=8e-5, beta=1e9, n_s=16, t_eps=0.0)
    r = oracle.render(sc, cam, o_)
    nhit = 0
    for p in range(cam.n_rays):
        o, d = pinhole_ray(cam, p)
        tau, ch = gauss_line_integral(sc.means[0], sc.scales[0], sc.quats[0], sc.densities[0], o, d)
        A = 1 - math.exp(-tau)
        c = colour_of(sc, 0, d)
        assert r["rgba"][p, 3] == pytest.approx(A, abs=2e-6)
        np.testing.assert_allclose(r["rgba"][p, :3], c * A, atol=2e-6)
        nhit += tau > 0
    assert nhit > cam.n_rays // 3


def test_explicit_bounds_integrate_only_between_them():
    """Algorithm 1 integrates over [t_n, t_f) only: with t_near and t_far cutting
    one Gaussian's chord at 10 % and 50 % of its length, the opacity is
    1 - exp(-tau) of the erf closed form taken between those two bounds, to
    within the one midpoint cell the far bound can split (density at t_f x dt/2)."""
    sc = one_gaussian_scene(seed=6)
    cam0 = camera_at([0.3, -1.2, 1.5], w=6, h=6)
    o_ = opts(dt=5e-5, n_s=16, t_eps=0.0)
    n = 0
    for p in range(cam0.n_rays):
        o, d = pinhole_ray(cam0, p)
        tau, ch = gauss_line_integral(sc.means[0], sc.scales[0], sc.quats[0], sc.densities[0], o, d)
        if ch is None or ch[1] - ch[0] < 0.02:
            continue
        t0 = ch[0] + 0.1 * (ch[1] - ch[0])
        t1 = ch[0] + 0.5 * (ch[1] - ch[0])
        cam = dataclasses.replace(cam0, t_near=float(t0), t_far=float(t1))
        tn, tf = float(np.float32(t0)), float(np.float32(t1))  # the camera stores float32 bounds
        r = oracle.render(sc, cam, o_, pix=np.array([p]))
        # partial integral: same q(t) = a (t - t_c)^2 + q_min as the whole-chord closed form
        R = Rotation.from_quat([sc.quats[0][1], sc.quats[0][2], sc.quats[0][3], sc.quats[0][0]]).as_matrix()
        Minv = np.diag(1.0 / np.asarray(sc.scales[0], np.float64)) @ R.T
        y0, yd = Minv @ (o - sc.means[0]), Minv @ d
        a = yd @ yd
        tc = -(y0 @ yd) / a
        qmin = (y0 + tc * yd) @ (y0 + tc * yd)
        k = math.sqrt(a / 2)
        part = sc.densities[0] * math.exp(-qmin / 2) * math.sqrt(math.pi / (2 * a)) * \
            (erf(k * (tf - tc)) - erf(k * (tn - tc)))
        assert 0.2 * tau < part < 0.55 * tau  # the bounds really cut the integral
        # midpoint cells start at t_n; the last counted one ends within dt/2 of t_f
        g_f = sc.densities[0] * math.exp(-(a * (tf - tc) ** 2 + qmin) / 2)
        assert r["rgba"][0, 3] == pytest.approx(1 - math.exp(-part), abs=g_f * o_.dt / 2 + 2e-6)
        n += 1
    assert n > 5


def test_erf_convergence_order():
    sc = one_gaussian_scene(seed=4)
    cam = camera_at([0.0, 0.9, 1.4], w=6, h=6)
    errs = []
    for dt in (4e-3, 1e-3, 2.5e-4):
        r = oracle.render(sc, cam, opts(dt=dt, n_s=8, t_eps=0.0))
        e = 0.0
        for p in range(cam.n_rays):
            o, d = pinhole_ray(cam, p)
            tau, _ = gauss_line_integral(sc.means[0], sc.scales[0], sc.quats[0], sc.densities[0], o, d)
            e = max(e, abs(r["rgba"][p, 3] - (1 - math.exp(-tau))))
        errs.append(e)
    # the truncation jump makes the error O(dt * sigma_eps); the smooth part is O(dt^2)
    assert errs[2] < errs[0] / 4
    assert errs[2] < 1e-5


def test_two_disjoint_gaussians_composite():
    sc1 = one_gaussian_scene(seed=1, center=(0, 0, 0.4), sig=3.0)
    sc2 = one_gaussian_scene(seed=2, center=(0, 0, -0.4), sig=8.0)
    sc = synth.Scene(*(np.concatenate([a, b]) for a, b in
                       zip([sc1.means, sc1.scales, sc1.quats, sc1.densities, sc1.sh],
                           [sc2.means, sc2.scales, sc2.quats, sc2.densities, sc2.sh])), 3)
    cam = camera_at([0.0, 0.05, 2.5], w=10, h=10, fov=8.0)
    bg = (0.2, 0.4, 0.9)
    r = oracle.render(sc, cam, opts(dt=5e-5, n_s=16, t_eps=0.0, bg=bg))
    both = 0
    for p in range(cam.n_rays):
        o, d = pinhole_ray(cam, p)
        t1, ch1 = gauss_line_integral(sc.means[0], sc.scales[0], sc.quats[0], sc.densities[0], o, d)
        t2, ch2 = gauss_line_integral(sc.means[1], sc.scales[1], sc.quats[1], sc.densities[1], o, d)
        if ch1 and ch2:
            assert ch1[1] < ch2[0]  # disjoint, Gaussian 0 first
            both += 1
        c1, c2 = colour_of(sc, 0, d), colour_of(sc, 1, d)
        T = math.exp(-t1 - t2)
        C = c1 * (1 - math.exp(-t1)) + math.exp(-t1) * c2 * (1 - math.exp(-t2))
        np.testing.assert_allclose(r["rgba"][p, :3], C + T * np.array(bg), atol=3e-6)
        assert r["rgba"][p, 3] == pytest.approx(1 - T, abs=3e-6)
    assert both > 10


def test_equal_colour_scene_identity():
    w = synth.workload("plain_2k", n=400)
    sc = w.scene
    col = np.array([0.3, 0.7, 0.55])
    sh = np.zeros_like(sc.sh, dtype=np.float64)
    sh[:, 0, :] = (col - 0.5) / (0.5 / math.sqrt(math.pi))  # Y_0 = 1 / (2 sqrt(pi))
    sc = synth.Scene(sc.means, sc.scales, sc.quats, sc.densities, sh, 3)
    bg = (0.1, 0.2, 0.3)
    r = oracle.render(sc, w.cameras[0], opts(dt=0.01, n_s=16, bg=bg))
    T = 1 - r["rgba"][:, 3]
    np.testing.assert_allclose(r["rgba"][:, :3], col[None] * (1 - T[:, None]) + T[:, None] * np.array(bg),
                               atol=1e-12)
    assert (r["rgba"][:, 3] > 0.5).mean() > 0.3


# ---------------------------------------------------------------- invariants
def test_empty_scene_returns_background():
    bg = (0.25, 0.5, 0.75)
    cam = camera_at([0, 0, 3])
    empty = synth.Scene(np.zeros((0, 3)), np.ones((0, 3)), np.ones((0, 4)), np.ones(0),
                        np.zeros((0, 16, 3)), 3)
    for sk in (False, True):
        r = oracle.render(empty, cam, opts(skip=sk, bg=bg))
        np.testing.assert_array_equal(r["rgba"], np.tile([*bg, 0.0], (cam.n_rays, 1)))
    # Gaussians whose peak density is below sigma_eps have empty support
    sc = one_gaussian_scene(sig=SIG_EPS * 0.5)
    r = oracle.render(sc, cam, opts(bg=bg))
    np.testing.assert_array_equal(r["rgba"], np.tile([*bg, 0.0], (cam.n_rays, 1)))


def test_rays_missing_everything_and_opacity_range():
    w = synth.workload("plain_2k", n=300)
    r = oracle.render(w.scene, w.cameras[0], w.options)
    A = r["rgba"][:, 3]
    assert np.all(A >= 0) and np.all(A <= 1)
    assert np.all(r["rgba"][:, :3] >= 0)
    miss = r["active"][:, 0] == 0
    assert miss.any()
    np.testing.assert_array_equal(r["rgba"][miss], 0.0)


def test_permutation_invariance():
    w = synth.workload("plain_2k", n=500)
    perm = np.random.default_rng(0).permutation(w.scene.n)
    r0 = oracle.render(w.scene, w.cameras[0], w.options)
    r1 = oracle.render(w.scene.permuted(perm), w.cameras[0], w.options)
    np.testing.assert_allclose(r0["rgba"], r1["rgba"], atol=1e-12)


def test_skipping_changes_uniform_render_at_most_teps():
    w = synth.workload("plain_2k")
    cam = w.cameras[0]
    o0 = w.options
    o1 = opts(dt=o0.dt, n_s=o0.n_s, skip=True)
    r0 = oracle.render(w.scene, cam, o0)
    r1 = oracle.render(w.scene, cam, o1)
    cmax = 0.5 + np.abs(w.scene.sh).sum(axis=1).max() * 0.5  # |Y_k| <= 0.5 generously bounds c
    diff = np.abs(r0["rgba"] - r1["rgba"])
    assert diff[:, 3].max() <= o0.t_eps + 1e-12
    assert diff[:, :3].max() <= o0.t_eps * cmax + 1e-12


def test_brute_force_samples_equal_chord_prefilter():
    w = synth.workload("plain_2k", n=30)
    cam = synth.rescale_camera(w.cameras[0], 8 / 64)
    for o_ in (w.options, synth.fast_options(dt_min=0.005, sigma_eps=SIG_EPS)):
        r0 = oracle.render(w.scene, cam, o_)
        r1 = oracle.render(w.scene, cam, o_, brute=True)
        np.testing.assert_allclose(r0["rgba"], r1["rgba"], atol=1e-13)


# ---------------------------------------------------------------- Alg. 1 / Eq. 5
def test_adaptive_step_special_cases():
    sc = one_gaussian_scene(sig=0.5)  # tau small, T stays near 1 for one segment
    cam = camera_at([0, 0, 30.0], w=4, h=4, fov=0.5)
    beta = 1024.0
    # far camera: t/beta = ~0.029 > dt_max -> clamped to dt_max
    r = oracle.render(sc, cam, opts(adaptive=True, skip=True, beta=beta, dt_min=0.005, dt_max=0.02),
                      sched_cap=64)
    seen = False
    for p in range(cam.n_rays):
        if r["sched_n"][p] > 0:
            assert r["sched"][p, 0, 1] == 0.02
            seen = True
    assert seen
    # t/beta in (dt_min, dt_max): first segment has T = 1 exactly -> dt = t_S / beta
    r = oracle.render(sc, cam, opts(adaptive=True, skip=True, beta=beta, dt_min=0.005, dt_max=0.2),
                      sched_cap=64)
    for p in range(cam.n_rays):
        if r["sched_n"][p] > 0:
            tS, dtk = r["sched"][p, 0]
            assert dtk == pytest.approx(tS / beta, rel=1e-15)
            # later segments: dt grows like T^{-1/3} (T < 1) but never below t/beta
            for s in range(1, r["sched_n"][p]):
                assert r["sched"][p, s, 1] >= r["sched"][p, s, 0] / beta * (1 - 1e-15)


def test_adaptive_step_follows_transmittance():
    """Eq. 5 away from T = 1: for every evaluated segment i the step is
    min(max(t_S,i / beta, dt_min) * T_i^(-1/3), dt_max), with T_i the
    transmittance at the segment's start, read by replaying the ray's first i
    segments.  The scene is dense enough that T falls well below 1 and dt_max
    is wide enough that the T factor is not clamped away."""
    w = synth.workload("plain_2k", n=400)
    sc = synth.Scene(w.scene.means, w.scene.scales, w.scene.quats, w.scene.densities * 4.0, w.scene.sh, 3)
    cam = synth.rescale_camera(w.cameras[0], 16 / 64)
    o_ = opts(adaptive=True, skip=True, dt_min=0.004, dt_max=0.5, beta=200.0, t_eps=1e-4)
    r = oracle.render(sc, cam, o_, sched_cap=256)
    n = r["sched_n"]
    checked, low_T = 0, 0
    for i in range(1, 12):
        idx = np.nonzero(n > i)[0]
        if idx.size == 0:
            continue
        rr = oracle.render(sc, cam, o_, pix=idx, sched=r["sched"][idx], sched_n=np.full(idx.size, i))
        T = rr["state"][:, 3]
        tS, dtk = r["sched"][idx, i, 0], r["sched"][idx, i, 1]
        want = np.minimum(np.maximum(tS / o_.beta, o_.dt_min) * T ** (-1.0 / 3.0), o_.dt_max)
        np.testing.assert_allclose(dtk, want, rtol=1e-12)
        checked += idx.size
        low_T += int((T < 0.7).sum())
    assert checked > 200 and low_T > 50


def test_skipping_jumps_the_gap_between_two_gaussians():
    """After the last segment touching one Gaussian, an empty segment sends the
    march to ClosestHit of its end: with adaptive steps the next evaluated
    segment starts exactly at the second Gaussian's chord entry, and with the
    uniform lattice one step of guard below it.  Chord ends come from the erf
    helper's closed-form quadratic, not from the oracle."""
    s1, s2 = one_gaussian_scene(seed=1, center=(0, 0, 0.6)), one_gaussian_scene(seed=2, center=(0, 0, -0.6))
    sc = synth.Scene(np.concatenate([s1.means, s2.means]), np.concatenate([s1.scales, s2.scales]),
                     np.concatenate([s1.quats, s2.quats]), np.concatenate([s1.densities, s2.densities]) * 0.2,
                     np.concatenate([s1.sh, s2.sh]), 3)
    cam = camera_at([0.01, 0.02, 3.0], w=6, h=6, fov=2.0)
    oa = opts(adaptive=True, skip=True, dt_min=0.005, dt_max=0.02, t_eps=0.0)
    ou = opts(dt=0.01, skip=True, t_eps=0.0)
    ra, ru = oracle.render(sc, cam, oa, sched_cap=256), oracle.render(sc, cam, ou, sched_cap=256)
    n = 0
    for p in range(cam.n_rays):
        o, d = pinhole_ray(cam, p)
        c = [gauss_line_integral(sc.means[l], sc.scales[l], sc.quats[l], sc.densities[l], o, d)[1] for l in (0, 1)]
        if c[0] is None or c[1] is None:
            continue
        (a0, a1), (b0, b1) = sorted(c)
        assert b0 - a1 > 0.2
        n += 1
        starts = ra["sched"][p, :ra["sched_n"][p], 0]
        after = starts[starts > a1]
        assert after.size and after[0] == pytest.approx(b0, abs=1e-9)
        su = ru["sched"][p, :ru["sched_n"][p], 0]
        after_u = su[su > a1]
        assert after_u.size and b0 - 2 * ou.dt - 1e-9 <= after_u[0] <= b0 - ou.dt + 1e-9
    assert n > 10


def test_skipping_from_inside_a_gaussian():
    """A camera inside a Gaussian's support: ClosestHit(t_n) is t_n itself (the
    enclosing chord already contains it), so the first segment starts at t_n,
    and the skipping render equals the plain one within T_eps * max c."""
    sc = one_gaussian_scene(sig=3.0, scale=0.5)
    cam = camera_at([0.05, 0.02, 0.1], target=(1, 0.3, 0.2), w=8, h=8, fov=40.0)
    o_ = opts(adaptive=True, skip=True, dt_min=0.005, dt_max=0.02)
    r = oracle.render(sc, cam, o_, sched_cap=64)
    assert np.all(r["sched_n"] > 0)
    np.testing.assert_array_equal(r["sched"][:, 0, 0], cam.t_near)
    ou, ou_skip = opts(dt=0.01), opts(dt=0.01, skip=True)
    r0, r1 = oracle.render(sc, cam, ou), oracle.render(sc, cam, ou_skip)
    assert r0["rgba"][:, 3].min() > 0.05
    cmax = 0.5 + np.abs(sc.sh).sum(axis=1).max()
    assert np.abs(r0["rgba"] - r1["rgba"]).max() <= ou.t_eps * cmax + 1e-12


def test_closest_hit_starts_at_first_chord_entry():
    sc = one_gaussian_scene()
    cam = camera_at([0.3, -1.2, 1.5])
    o_ = opts(adaptive=True, skip=True, dt_min=0.005, dt_max=0.02)
    r = oracle.render(sc, cam, o_, sched_cap=16)
    ou = opts(dt=0.01, skip=True)
    ru = oracle.render(sc, cam, ou, sched_cap=16)
    n = 0
    for p in range(cam.n_rays):
        o, d = pinhole_ray(cam, p)
        tau, ch = gauss_line_integral(sc.means[0], sc.scales[0], sc.quats[0], sc.densities[0], o, d)
        if ch is None:
            assert r["sched_n"][p] == 0 and ru["sched_n"][p] == 0
            continue
        n += 1
        assert r["sched"][p, 0, 0] == pytest.approx(ch[0], abs=1e-9)
        # uniform: snapped to the lattice, one step of guard below the entry
        t0 = ru["sched"][p, 0, 0]
        assert ch[0] - 2 * ou.dt - 1e-9 <= t0 <= ch[0] - ou.dt + 1e-9
        assert abs(t0 / ou.dt - round(t0 / ou.dt)) < 1e-6
    assert n > 10


def test_termination_at_segment_granularity():
    w = synth.workload("plain_2k")
    cam = w.cameras[0]
    sc = w.scene
    w.scene = synth.Scene(sc.means, sc.scales, sc.quats, sc.densities * 30.0, sc.sh, 3)  # opaque
    r = oracle.render(w.scene, cam, w.options, sched_cap=256)
    T = r["state"][:, 3]
    stopped = T <= w.options.t_eps
    assert stopped.sum() > 100
    # replaying all but the last evaluated segment leaves T above T_eps
    idx = np.nonzero(stopped)[0][:60]
    sched = r["sched"][idx]
    n_short = r["sched_n"][idx] - 1
    rr = oracle.render(w.scene, cam, w.options, pix=idx, sched=sched, sched_n=n_short)
    assert np.all(rr["state"][:, 3] > w.options.t_eps)
    # and replaying the full schedule reproduces the render exactly
    rf = oracle.render(w.scene, cam, w.options, pix=idx, sched=sched, sched_n=r["sched_n"][idx])
    np.testing.assert_allclose(rf["rgba"], r["rgba"][idx], atol=1e-14)


def test_segment_limit_is_reported():
    w = synth.workload("plain_2k", n=300)
    o_ = opts(dt=0.01, max_segments=3)
    r = oracle.render(w.scene, w.cameras[0], o_)
    assert r["n_iter_limit"] > 0


# ---------------------------------------------------------------- rays and bounds
def test_rays_pass_through_the_pixel_they_project_to():
    """Ray generation pinned by its inverse: projecting any point of pixel (u, v)'s
    ray back through the camera (world to camera by the inverse of the c2w
    rotation, perspective division, intrinsics) lands on that pixel's centre
    (u + 1/2, v + 1/2) in front of the camera; the ray starts at the camera
    centre and has unit length.  Random rotations, off-centre principal points
    and unequal focal lengths, so a swapped axis or intrinsic fails."""
    rng = np.random.default_rng(21)
    for _ in range(5):
        rot = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        centre = rng.normal(size=3) * 2
        c2w = np.concatenate([rot, centre[:, None]], 1).astype(np.float32)
        W, H = int(rng.integers(5, 40)), int(rng.integers(5, 40))
        cam = synth.Camera(c2w, float(rng.uniform(20, 80)), float(rng.uniform(20, 80)),
                           float(rng.uniform(0, W)), float(rng.uniform(0, H)), W, H)
        R64, C64 = c2w[:, :3].astype(np.float64), c2w[:, 3].astype(np.float64)
        for pix in rng.integers(0, W * H, size=20):
            o, d = oracle.ray(cam, int(pix))
            np.testing.assert_allclose(o, C64, atol=1e-12)
            assert abs(np.linalg.norm(d) - 1.0) < 1e-12
            for t in (0.5, 3.0, 40.0):
                pc = np.linalg.solve(R64, o + t * d - C64)
                assert pc[2] > 0
                u = cam.fx * pc[0] / pc[2] + cam.cx
                v = cam.fy * pc[1] / pc[2] + cam.cy
                assert abs(u - (pix % W + 0.5)) < 1e-9 and abs(v - (pix // W + 0.5)) < 1e-9


@pytest.mark.parametrize("mode", ["uniform", "adaptive_skip"])
def test_far_bound_at_the_scene_box_exit_changes_nothing(mode):
    """t_far <= 0 stands for the exit of the scene box (the union of the
    ellipsoid boxes).  Density is zero outside that box, so an explicit far
    bound beyond it must give the same render, for a camera outside the box
    (rays cross the whole sparse scene, so an exit computed too early would cut
    density off), a camera inside it, and rays that miss it."""
    w = synth.workload("plain_2k", n=200)
    o_ = w.options if mode == "uniform" else synth.fast_options(dt_min=0.005, sigma_eps=w.options.sigma_eps)
    inside = synth.look_at(np.zeros(3), np.array([1.0, 0.3, 0.2]), 60.0, 10, 10)
    away = synth.look_at(np.array([0.0, 0.0, 3.0]), np.array([0.0, 0.0, 6.0]), 30.0, 6, 6)
    for cam in (synth.rescale_camera(w.cameras[0], 12 / 64), inside, away):
        r_far = oracle.render(w.scene, dataclasses.replace(cam, t_far=20.0), o_)
        r_auto = oracle.render(w.scene, dataclasses.replace(cam, t_far=0.0), o_)
        np.testing.assert_allclose(r_auto["rgba"], r_far["rgba"], atol=1e-14)
        if cam is not away:
            assert (r_auto["rgba"][:, 3] > 1e-3).sum() > cam.n_rays // 4
    np.testing.assert_array_equal(r_auto["rgba"], np.tile([*o_.bg, 0.0], (away.n_rays, 1)))
