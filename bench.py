#!/usr/bin/env python3
"""Benchmark of the differentiable Gaussian ray-marching step on B300.

One step = the whole hot path on one batch: rgx_build_bvh (bounds, Morton
codes, radix sort, radix tree, refit, packing) + rgx_render_forward (skip +
adaptive step + Z-order storage + Z-order ray tiles) + rgx_render_backward
(replayed adjoint + per-Gaussian finalisation), on the torus workload:
100,000 seeded Gaussians, one 800x800 view on a radius-4 orbit.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  ``value`` is whole-job Mrays/s of the step
with inputs resident in HBM, timed with CUDA events per step on the launching
stream, L2 flushed (256 MiB write) between steps outside the events.
``e2e`` repeats the step through the same C-ABI with host (pinned) buffers:
every step uploads its parameters and upstream gradient and downloads its
gradients and image inside the timed region, the copies on a second stream
overlapping the neighbouring steps' kernels.  ``roofline`` relates the dominant
kernel's counted FP32/SFU work to the derived ALU peak, ``hbm_roofline`` its
algorithmic bytes (and the profiled DRAM bytes) to the measured copy bandwidth,
and ``cpu_baseline`` times the FP64 oracle on all host cores and on one.
``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
pixel sample instead.
Multi-GPU (torchrun): each rank renders its own seeded camera of the same
scene (weak scaling); ranks share nothing on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "torus_100k"
# one-view forward + adjoint workloads (run_rgx) and their descriptions
STEP_WORKLOADS = {
    "torus_100k": "100,000 Gaussians on a noise-perturbed torus, one 800x800 view on a radius-4 orbit, BVH rebuild + "
                  "forward + adjoint (skip + adaptive Eq.5 + Z-order + Z-tiles, N_S=16)",
    "plain_2k": "2,000 Gaussians uniform in [-1,1]^3, one 64x64 view at radius 3, BVH rebuild + forward + adjoint "
                "(uniform dt=0.01, no skipping, N_S=16)",
    "outdoor_3m": "3,000,000 Gaussians (200-blob cluster + log-radius shell to r=100), one 1237x822 view from inside "
                  "the cluster, BVH rebuild (63-bit codes) + forward + adjoint (skip + adaptive Eq.5 + Z-order + "
                  "Z-tiles, N_S=16)",
}
METRIC = "Mrays/s render & fwd+bwd ms/iter vs plain marcher at ≤1e-4 err; % HBM peak"


def workload_label(name: str, fallback: str = "") -> str:
    """The config's workload string; both arms (the CUDA path and the oracle)
    print the same one for the same workload."""
    return f"{name}: " + STEP_WORKLOADS.get(name, fallback)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="rgx", choices=["rgx", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-tune", action="store_true",
                   help="skip rgx_autotune (tile shape and hit_cap; N_S fixed) before the timed steps")
    p.add_argument("--tile", default=None, help="fixed ray-tile shape WxH (skips rgx_autotune)")
    p.add_argument("--hit-cap", type=int, default=None, help="fixed hit-list capacity (skips rgx_autotune)")
    p.add_argument("--workload", default=WORKLOAD, choices=list(STEP_WORKLOADS) + ["batch_1m", "sweep_6m"],
                   help="torus_100k (default), plain_2k, outdoor_3m: one view, build + forward + adjoint; "
                        "batch_1m = 8 uneven views, autotuned, CUDA-graph captured fwd+bwd; sweep_6m = 64 views "
                        "forward, one persistent launch vs one launch per view")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    for path in (os.path.join(ROOT, "MEASURED_PEAKS.json"),):
        try:
            with open(path) as f:
                d = json.load(f)
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------------------------
def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summaries, or None when there is none for that pair or the kernel source
    changed since the counters were taken."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_2509_07782_b300", "csrc", "march.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.split()
            if len(parts) == 6 and parts[0] == "traffic_bytes_per_launch" and parts[1] == workload \
                    and parts[2] == kernel and parts[4] == "src_sha256" and parts[5] == sha:
                return int(parts[3])
    return None


def launches_per_step(opts) -> int:
    passes = 8 if opts.morton63 else 4
    build = 2 + 3 * passes + 1 + 3       # bounds, morton, sort passes, pack, karras + refit + widen
    return build + 1 + 2                  # forward march; backward march + finalize


def touched_gaussians(grads) -> int:
    """Gaussians with a non-zero entry in any of the five gradient tensors of a
    dense random upstream gradient: the Gaussians the march had to read (a lower
    bound, since a Gaussian whose every sample falls outside its truncation
    contributes nothing)."""
    import torch
    n = grads[0].shape[0]
    return int(torch.cat([g.reshape(n, -1) for g in grads], 1).ne(0).any(1).sum())


def hbm_roofline(n_touched: int, rays: int, seconds: float, backward: bool, peak_gbs: float, traffic=None,
                 ray_bytes: int = 32):
    """Algorithmic HBM bytes of one march launch and the bandwidth they imply.

    Forward: each touched Gaussian's 236-byte parameter record and one 32-byte
    BVH node per touched Gaussian read once, 16 B RGBA + 16 B state per ray
    written (`ray_bytes` = 16 for a forward that keeps no state).  Adjoint: the
    same reads, 16 B dL/dRGBA + 16 B state per ray, and each touched Gaussian's
    236 bytes of gradient read and written once.  Beside them the measured DRAM
    bytes of the same kernel (ncu), when known.
    """
    per_g = 236 + 32 + (2 * 236 if backward else 0)
    alg = n_touched * per_g + rays * ray_bytes
    out = {"algorithmic_bytes": alg, "achieved": alg / seconds / 1e9, "peak": peak_gbs, "unit": "GB/s",
           "frac": alg / seconds / 1e9 / peak_gbs, "touched_gaussians": n_touched}
    if traffic is not None:
        out["dram_bytes"] = traffic
        out["dram_gbs"] = traffic / seconds / 1e9
        out["dram_frac"] = traffic / seconds / 1e9 / peak_gbs
    return out


def alu_model(evals, hits, segs, rays, ns, backward: bool):
    """FP32 FLOP-equivalents of the algorithmic work of one march launch.

    Per (sample, Gaussian) evaluation: sample offset (FMA), quadratic form
    (MUL + FMA), exponent (FMA), 1 ex2 on the SFU, density add, 3 colour FMA
    -> 14 FP32 FLOPs + 1 ex2; the adjoint evaluates twice (the replayed sums,
    then its own sample loop) and adds the dL/dg product (3 FMA + mul), 3
    moment FMA (+2 mul) and 3 colour-gradient FMA -> 2 x 30 + 22.  Per (ray,
    segment, Gaussian) hit: chord solve (~60 FLOPs) and SH colour (48 FMA = 96
    FLOPs) in the forward; in the adjoint, whose lists come from the forward's
    tape, the local frame and moment expansion (~60) and the SH gradient
    (48 MUL x 2 = 96), added with 15 float4 atomics.  One ex2 is counted as
    16 FLOP-equivalents (128 FP32 lanes x 2 vs 16 SFU results per SM per
    clock), so the FP32 pipe peak is the single denominator.
    """
    per_eval = 14 + 16
    per_hit = 60 + 96
    if backward:
        per_eval = 2 * per_eval + 22
        per_hit = 60 + 96
    return evals * per_eval + hits * per_hit


def rank_workload(name: str, rank: int):
    """The workload as rank `rank` renders it: rank 0 the named view, every other
    rank its own seeded view of the same scene (weak scaling, nothing shared on
    the data path)."""
    from paper_2509_07782_b300 import synth
    w = synth.workload(name)
    if rank > 0:
        cam0 = w.cameras[0]
        rng = np.random.Generator(np.random.PCG64(5000 + rank))
        if name == "outdoor_3m":
            w.cameras = [synth.inside_camera(rng, 0.3, cam0.width, cam0.height)]
        elif name == "plain_2k":
            w.cameras = [synth.sphere_camera(rng, 3.0, cam0.width, cam0.height)]
        else:
            w.cameras = [synth.orbit_camera(rng, 4.0, cam0.width, cam0.height)]
    return w


def max_over_ranks(values, world: int, device=None):
    """Element-wise maximum of per-rank timings (ms) over all ranks."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def whole_job_mrays(world: int, rays_per_rank: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: rays of all ranks over the slowest rank's time."""
    return world * rays_per_rank * steps / (total_ms / 1e3) / 1e6


def run_rgx(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_2509_07782_b300 import rgx, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = rank_workload(args.workload, rank)
    opts = rgx.make_opts(w.options)
    cams = rgx.Cameras(w.cameras)
    R = cams.n_rays
    t = rgx.scene_tensors(w.scene, device=dev)
    sc = rgx.Scene(local)
    stream = torch.cuda.current_stream()
    upstream = torch.randn(R, 4, device=dev, generator=torch.Generator(device=dev).manual_seed(1 + rank))
    grads = [torch.zeros_like(x) for x in t]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tuned = None
    if args.tile or args.hit_cap:
        if args.tile:
            opts.tile_w, opts.tile_h = (int(x) for x in args.tile.lower().split("x"))
        if args.hit_cap:
            opts.hit_cap = args.hit_cap
        tuned = {"tile": [opts.tile_w, opts.tile_h], "hit_cap": opts.hit_cap, "fixed": True}
    elif not args.no_tune:
        # implementation knobs only (tile shape, hit-list capacity); N_S stays the workload's
        sc.build(*t, opts)
        best, tune_ms = sc.autotune(cams, opts, tune_ns=False, with_backward=True)
        opts = best
        tuned = {"tile": [best.tile_w, best.tile_h], "hit_cap": best.hit_cap, "tuning_ms": tune_ms}

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        sc.build(*t, opts)
        if ev is not None:
            ev[1].record(stream)
        rgba, state = sc.forward(cams, opts)
        if ev is not None:
            ev[2].record(stream)
        for g in grads:
            g.zero_()
        sc.backward(cams, opts, state, upstream, grads)
        if ev is not None:
            ev[3].record(stream)
        return rgba

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st = sc.status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        step(evs[i])
        flush.fill_(float(i))  # L2 flush between steps, outside the events
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    fwd_ms = [e[1].elapsed_time(e[2]) for e in evs]
    bwd_ms = [e[2].elapsed_time(e[3]) for e in evs]
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    total_ms = float(sum(step_ms))
    st = sc.status()

    # work counters of one forward and one backward (separate, untimed calls)
    rgba, state = sc.forward(cams, opts)
    cf = sc.counters()
    for g in grads:
        g.zero_()
    sc.backward(cams, opts, state, upstream, grads)
    cb = sc.counters()
    torch.cuda.synchronize()
    n_touched = touched_gaussians(grads)

    # e2e through the C-ABI with host buffers: every step uploads its parameters and upstream
    # gradient from pinned host memory and downloads its gradients and image.  The copies run
    # on a copy stream with two buffer slots, so step i+1's upload and step i's download overlap
    # the kernels of the neighbouring steps; the timed region runs from before the first upload
    # to after the last download.
    host_in = [x.cpu().pin_memory() for x in t] + [upstream.cpu().pin_memory()]
    cs = torch.cuda.Stream(device=dev)
    slots = [dict(dev_in=[torch.empty_like(x) for x in t] + [torch.empty_like(upstream)],
                  grads=[torch.empty_like(x) for x in t],
                  rgba=torch.empty(R, 4, dtype=torch.float32, device=dev), state=rgx.new_state(R, dev),
                  host_out=[torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in t] +
                           [torch.empty(R, 4, dtype=torch.float32, pin_memory=True)],
                  loaded=torch.cuda.Event(), computed=torch.cuda.Event(), unloaded=torch.cuda.Event(),
                  used=False) for _ in range(2)]
    h2d = sum(x.numel() * x.element_size() for x in host_in)
    d2h = sum(x.numel() * x.element_size() for x in slots[0]["host_out"])
    n_g = int(t[0].shape[0])

    def upload(sl):
        with torch.cuda.stream(cs):
            if sl["used"]:
                cs.wait_event(sl["computed"])  # the slot's previous step has consumed its inputs
            for d, h in zip(sl["dev_in"], host_in):
                d.copy_(h, non_blocking=True)
            sl["loaded"].record(cs)

    def compute(sl):
        stream.wait_event(sl["loaded"])
        if sl["used"]:
            stream.wait_event(sl["unloaded"])  # the slot's previous results have left the device
        d = sl["dev_in"]
        rgx.rgx_build_bvh(sc.h, *d[:5], 3, opts, stream=stream)
        rgx.rgx_render_forward(sc.h, cams, opts, sl["rgba"], sl["state"], stream=stream)
        for g in sl["grads"]:
            g.zero_()
        rgx.rgx_render_backward(sc.h, cams, opts, sl["state"], d[5], *sl["grads"], stream=stream, n=n_g)
        sl["computed"].record(stream)
        sl["used"] = True

    def download(sl):
        with torch.cuda.stream(cs):
            cs.wait_event(sl["computed"])
            for h, d in zip(sl["host_out"], sl["grads"] + [sl["rgba"]]):
                h.copy_(d, non_blocking=True)
            sl["unloaded"].record(cs)

    def e2e_run(nsteps, e0=None, e1=None):
        if e0 is not None:
            e0.record(stream)
        cs.wait_stream(stream)
        upload(slots[0])
        for i in range(nsteps):
            if i + 1 < nsteps:
                upload(slots[(i + 1) % 2])
            compute(slots[i % 2])
            download(slots[i % 2])
        stream.wait_event(slots[(nsteps - 1) % 2]["unloaded"])
        if e1 is not None:
            e1.record(stream)
        return slots[(nsteps - 1) % 2]["host_out"]

    e2e_run(2)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    last = e2e_run(args.steps, e0, e1)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    # the downloaded results must be the step's: the image bit for bit, the gradients (float
    # atomics, summation order free) to rounding; reported on the line, and on stderr if not
    e2e_ok = bool(torch.equal(last[5], rgba.cpu()))
    for h, g in zip(last[:5], grads):
        ref = g.cpu()
        e2e_ok &= float((h - ref).norm()) <= 1e-4 * max(float(ref.norm()), 1e-30)
    if not e2e_ok:
        print("warning: end-to-end results differ from the device-resident step's", file=sys.stderr)

    # the plain single-view marcher on the same GPU (uniform step = dt_min, no skip,
    # caller-order storage, scanline rays): forward and forward+adjoint
    plain = None
    if not args.no_plain:
        po = synth.Options(dt=w.options.dt_min if w.options.adaptive else w.options.dt, n_s=w.options.n_s,
                           sigma_eps=w.options.sigma_eps, hit_cap=w.options.hit_cap, morton63=w.options.morton63)
        popts = rgx.make_opts(po)
        sp = rgx.Scene(local)
        for _ in range(2):
            sp.build(*t, popts)
            _, pst = sp.forward(cams, popts)
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        fm, fb = [], []
        for i in range(3):
            sp.build(*t, popts)
            a.record(stream)
            _, pst = sp.forward(cams, popts)
            b.record(stream)
            gl = [torch.zeros_like(x) for x in t]
            sp.backward(cams, popts, pst, upstream, gl)
            c.record(stream)
            torch.cuda.synchronize()
            fm.append(a.elapsed_time(b))
            fb.append(b.elapsed_time(c))
            flush.fill_(0.0)
        plain = {"fwd_ms": statistics.median(fm), "bwd_ms": statistics.median(fb),
                 "render_mrays_s": R / statistics.median(fm) / 1e3,
                 "options": f"uniform dt={po.dt}, N_S={po.n_s}, no skip, caller order, scanline rays"}
        if sp.status() != 0:
            plain["status"] = "device status nonzero"

    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_mrays(world, R, args.steps, total_ms)
    return dict(R=R, ms_per_step=ms_per_step, value=value, build_ms=statistics.median(build_ms),
                fwd_ms=statistics.median(fwd_ms), bwd_ms=statistics.median(bwd_ms), wall_s=wall,
                e2e=dict(value=whole_job_mrays(world, R, 1, e2e_ms), unit="Mrays/s", h2d_bytes_per_step=h2d,
                         d2h_bytes_per_step=d2h, ms_per_step=e2e_ms, matches_device_step=e2e_ok,
                         copies="pinned host buffers; uploads and downloads on a copy stream, two buffer "
                                "slots, overlapping the neighbouring steps' kernels"),
                counters_fwd=cf, counters_bwd=cb, clocks=clocks, status=st, plain=plain, opts=w.options, tuned=tuned,
                n=w.scene.n, n_touched=n_touched, steps_launches=launches_per_step(w.options) * args.steps)


def _oracle_rate(w, cam, P, threads: int, max_seconds: float, npix_start: int):
    """Oracle forward + adjoint on a seeded pixel sample of ``cam`` with
    ``threads`` OpenMP threads, the sample grown 4x until a pass takes about a
    quarter of ``max_seconds``.  Returns (rays/s, pixels, seconds)."""
    import oracle
    from paper_2509_07782_b300 import synth
    npix = npix_start
    while True:
        pix = synth.pixel_subset(cam, npix, seed=3)
        W = np.random.default_rng(4).normal(size=(len(pix), 4))
        t0 = time.perf_counter()
        oracle.render(w.scene, cam, w.options, pix=pix, params=P, nthreads=threads)
        oracle.backward(w.scene, cam, w.options, W, pix=pix, params=P, nthreads=threads)
        dt = time.perf_counter() - t0
        if dt > max_seconds / 4 or npix >= cam.n_rays:
            return len(pix) / dt, len(pix), dt
        npix = min(cam.n_rays, npix * 4)


def cpu_baseline(workload=WORKLOAD, max_seconds=12.0, npix_start=256):
    """FP64 oracle (as it stands) on the host cores: forward + adjoint on a
    seeded pixel sample of the same view, grown until ~max_seconds; then once
    more on one core (a smaller sample, ~max_seconds / 2)."""
    import oracle
    from paper_2509_07782_b300 import synth
    w = synth.workload(workload)
    cam = w.cameras[0]
    P = oracle.Params(w.scene)
    cores = os.cpu_count() or 1
    rate, n, dt = _oracle_rate(w, cam, P, cores, max_seconds, npix_start)
    out = {"value": rate / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
           "sample": f"{n} seeded pixels of the {cam.width}x{cam.height} view, forward + adjoint, {dt:.2f} s"}
    rate1, n1, dt1 = _oracle_rate(w, cam, P, 1, max_seconds / 2, max(16, npix_start // 16))
    out["single_core"] = {"value": rate1 / 1e6, "unit": "Mrays/s", "cores": 1,
                          "sample": f"{n1} seeded pixels, forward + adjoint, {dt1:.2f} s"}
    return out


def run_batch(args):
    """batch_1m: 1M Gaussians, 8 views of uneven resolution, one persistent
    forward + adjoint launch each, tuned by rgx_autotune, captured in a CUDA graph."""
    import torch

    from paper_2509_07782_b300 import graph, rgx, synth
    dev = torch.device("cuda", 0)
    w = synth.workload("batch_1m")
    base = rgx.make_opts(w.options)
    cams = rgx.Cameras(w.cameras)
    params = list(rgx.scene_tensors(w.scene, device=dev))
    sc = rgx.Scene(0)
    sc.build(*params, base)
    best, tune_ms = sc.autotune(cams, base, tune_ns=False, with_backward=True)
    d_rgba = torch.randn(cams.n_rays, 4, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    for name, opts in (("autotuned", best), ("default", base)):
        step = graph.CapturedStep(sc, cams, opts, params, d_rgba)
        for _ in range(max(args.warmup, 3)):
            step.replay()
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(step.stream)
            step.replay()
            e1.record(step.stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            flush.fill_(0.0)
        out[name] = statistics.median(times)
        if sc.status(step.stream) != 0:
            out[name + "_status"] = "device status nonzero"
    ms = out["autotuned"]
    return {"metric": METRIC, "value": cams.n_rays / ms / 1e3, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_1m: 1M torus Gaussians, 8 views {320x240 ... 1920x1080}, "
                                   "BVH rebuild + persistent forward + adjoint, CUDA-graph captured",
                       "rays_per_step": cams.n_rays, "l2": "flushed between steps"},
            "autotuned": {"tile": [best.tile_w, best.tile_h], "hit_cap": best.hit_cap, "n_s": best.n_s,
                          "tuning_ms": tune_ms},
            "graph_ms_autotuned": out["autotuned"], "graph_ms_default": out["default"]}


def run_sweep(args):
    """sweep_6m: 6M Gaussians, 64 views, forward only: one persistent launch
    for all views vs one launch per view; FPS per view size."""
    import torch

    from paper_2509_07782_b300 import rgx, synth
    dev = torch.device("cuda", 0)
    w = synth.workload("sweep_6m")
    opts = rgx.make_opts(w.options)
    t = rgx.scene_tensors(w.scene, device=dev)
    sc = rgx.Scene(0)
    sc.build(*t, opts)
    cams_all = rgx.Cameras(w.cameras)
    singles = [rgx.Cameras([c]) for c in w.cameras]
    rgba = torch.empty(cams_all.n_rays, 4, device=dev)
    st = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):
        rgx.rgx_render_forward(sc.h, cams_all, opts, rgba)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        rgx.rgx_render_forward(sc.h, cams_all, opts, rgba)
    e1.record(st)
    torch.cuda.synchronize()
    ms_persistent = e0.elapsed_time(e1) / args.steps
    per_view = []
    outs = [torch.empty(c.n_rays, 4, device=dev) for c in singles]
    for c, o in zip(singles, outs):
        rgx.rgx_render_forward(sc.h, c, opts, o)
    torch.cuda.synchronize()
    for c, o in zip(singles, outs):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        rgx.rgx_render_forward(sc.h, c, opts, o)
        b.record(st)
        torch.cuda.synchronize()
        per_view.append((c.cams[0].width, c.cams[0].height, a.elapsed_time(b)))
    ms_per_view_total = sum(x[2] for x in per_view)
    fps = sorted(((wd * ht, 1e3 / ms) for wd, ht, ms in per_view))
    q = [fps[0], fps[len(fps) // 2], fps[-1]]
    # forward only: no gradient tells which Gaussians were read, so all of them count (an upper bound)
    peaks, src = load_peaks()
    hbm = hbm_roofline(w.scene.n, cams_all.n_rays, ms_persistent / 1e3, False, float(peaks.get("hbm_gbs", 6400.0)),
                       ray_bytes=16)
    hbm.update(kernel="k_march<16,0>", peak_source=f"{src} copy bandwidth",
               touched_note="every Gaussian counted as read (upper bound; forward only)")
    return {"metric": METRIC, "value": cams_all.n_rays / ms_persistent / 1e3, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_persistent, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep_6m: 6M torus Gaussians, 64 seeded views 256..1920 x 256..1080, forward "
                                   "only", "rays_per_step": cams_all.n_rays},
            "one_launch_per_view": {"ms_total": ms_per_view_total,
                                    "mrays_s": cams_all.n_rays / ms_per_view_total / 1e3},
            "fps_per_view": {"smallest": {"pixels": q[0][0], "fps": q[0][1]},
                             "median": {"pixels": q[1][0], "fps": q[1][1]},
                             "largest": {"pixels": q[2][0], "fps": q[2][1]}},
            "hbm_roofline": hbm,
            "device_status": sc.status()}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload not in STEP_WORKLOADS and args.impl != "reference":
        if rank == 0:
            print(json.dumps(run_batch(args) if args.workload == "batch_1m" else run_sweep(args)))
        return
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        from paper_2509_07782_b300 import synth
        w = synth.workload(args.workload)
        cam = w.cameras[0]
        P = oracle.Params(w.scene)
        cores = os.cpu_count() or 1
        # the oracle brute-forces every Gaussian per ray: the sample shrinks with N
        npix = int(min(2048, max(64, 2048 * 100_000 // max(w.scene.n, 1))))
        pix = synth.pixel_subset(cam, min(npix, cam.n_rays), seed=3)
        with_bwd = args.workload != "sweep_6m"
        W = np.random.default_rng(4).normal(size=(len(pix), 4))
        for _ in range(max(args.warmup, 0)):
            oracle.render(w.scene, cam, w.options, pix=pix[:16], params=P, nthreads=cores)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            oracle.render(w.scene, cam, w.options, pix=pix, params=P, nthreads=cores)
            if with_bwd:
                oracle.backward(w.scene, cam, w.options, W, pix=pix, params=P, nthreads=cores)
            times.append(time.perf_counter() - t0)
        tot = sum(times)
        v = len(pix) * args.steps / tot / 1e6
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mrays/s", "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": workload_label(args.workload,
                                                     f"{w.scene.n} Gaussians, first of {len(w.cameras)} views"),
                          "sample": f"{len(pix)} seeded pixels of the {cam.width}x{cam.height} view per step"},
               "cpu_baseline": {"value": v, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                                "sample": f"{len(pix)} seeded pixels per step, forward"
                                          + (" + adjoint" if with_bwd else "")},
               "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    r = run_rgx(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    peaks, src = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    fp32_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2
    cb, cf = r["counters_bwd"], r["counters_fwd"]
    ns = r["opts"].n_s
    flops_b = alu_model(cb["evals"], cb["hits"], cb["segments"], cb["rays"], ns, True)
    flops_f = alu_model(cf["evals"], cf["hits"], cf["segments"], cf["rays"], ns, False)
    # dominant kernel: the backward march (its call also zeroes the accumulators and finalises)
    bwd_s = r["bwd_ms"] / 1e3
    fwd_s = r["fwd_ms"] / 1e3
    dominant_is_bwd = r["bwd_ms"] >= r["fwd_ms"]
    achieved = (flops_b / bwd_s if dominant_is_bwd else flops_f / fwd_s) / 1e12
    kname = "k_march<16,1>" if dominant_is_bwd else "k_march<16,0>"
    roofline = {"bound": "alu", "kernel": kname,
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": profiled_traffic(kname, args.workload),
                "peak_source": f"148 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (derived), HBM {src} "
                               f"{peaks.get('hbm_gbs')} GB/s"}
    hbm = hbm_roofline(r["n_touched"], r["R"], bwd_s if dominant_is_bwd else fwd_s, dominant_is_bwd,
                       float(peaks.get("hbm_gbs", 6400.0)), roofline["traffic"])
    hbm["kernel"] = kname
    hbm["peak_source"] = f"{src} copy bandwidth"
    out = {
        "metric": METRIC, "value": r["value"], "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(args.workload),
                   "knobs": "tile shape and hit_cap from rgx_autotune unless fixed",
                   "rays_per_step_per_gpu": r["R"], "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"{world} independent views, no data-path collective",
                   "autotuned": r["tuned"]},
        "fwd_bwd_ms": r["fwd_ms"] + r["bwd_ms"], "build_ms": r["build_ms"], "fwd_ms": r["fwd_ms"],
        "bwd_ms": r["bwd_ms"], "render_mrays_s": r["R"] / r["fwd_ms"] / 1e3,
        "plain_marcher": r["plain"],
        "speedup_vs_plain": {"render": (r["plain"]["fwd_ms"] / r["fwd_ms"]) if r["plain"] else None,
                             "fwd_bwd": ((r["plain"]["fwd_ms"] + r["plain"]["bwd_ms"]) / (r["fwd_ms"] + r["bwd_ms"]))
                             if r["plain"] else None},
        "roofline": roofline,
        "hbm_roofline": hbm,
        "work": {"fwd": cf, "bwd": cb},
        "e2e": r["e2e"], "gpu_launches": r["steps_launches"], "clocks": r["clocks"],
        "device_status": r["status"],
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
