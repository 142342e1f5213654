#!/usr/bin/env python3
"""Benchmark of the differentiable Gaussian ray-marching step on B300.

One step = the whole hot path on one batch: rgx_build_bvh (bounds, Morton
codes, radix sort, radix tree, refit, packing) + rgx_render_forward (skip +
adaptive Eq. 5 step + Z-order storage + Z-order ray tiles, every camera in one
persistent launch) + rgx_render_backward (replayed adjoint + per-Gaussian
finalisation).  Default workload ``batch_1m``: 1,000,000 seeded torus
Gaussians, 8 views of uneven resolution {320x240 ... 1920x1080} (7,082,990
rays), tile shape, hit-list capacity and N_S picked by rgx_autotune, the step
captured in CUDA graphs (build, forward, adjoint).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

Prints one JSON line (rank 0).  ``value`` is whole-job Mrays/s of the step
with inputs resident in HBM, timed with CUDA events per replay on the graph's
stream, L2 flushed (256 MiB write) between steps outside the events.  Events
between the build, forward and adjoint graphs split each step into stages.
The single-view ``torus_100k`` and ``outdoor_3m`` steps and the forward-only
``sweep_6m`` ride along as sub-objects, each beside its plain marcher.
``e2e`` repeats the step through the C-ABI with host (pinned) buffers: every
step uploads its parameters and upstream gradient and downloads its gradients
and image inside the timed region.  ``plain_marcher`` times the plain
single-view marcher (uniform step = dt_min, no skipping, caller order,
scanline rays, one launch per view) on the same views.  ``roofline`` relates
the dominant march kernel's counted FP32 work to the FP32 peak derived from the
SM count and clock, ``hbm_roofline`` its algorithmic bytes to the measured
copy bandwidth, ``cpu_baseline`` times the FP64 oracle on the host cores.
``--impl reference`` times the FP64 CPU oracle on a bounded pixel sample of the
same workload instead.  Multi-GPU (torchrun): each rank renders its own seeded
views of the same scene and the ranks sum their gradients with one all-reduce
inside the timed step (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batch_1m"
# forward + adjoint step workloads and their descriptions
STEP_WORKLOADS = {
    "batch_1m": "1,000,000 Gaussians on a noise-perturbed torus, 8 views of uneven resolution {320x240, 640x480, "
                "800x800, 1024x768, 1237x822, 1600x1200, 1920x1080, 512x512} on radius-4 orbits (7,082,990 rays), "
                "BVH rebuild + one persistent forward + one persistent adjoint launch captured in CUDA graphs "
                "(skip + adaptive Eq.5 + Z-order + Z-tiles; tile shape, hit_cap and N_S autotuned)",
    "torus_100k": "100,000 Gaussians on a noise-perturbed torus, one 800x800 view on a radius-4 orbit, BVH rebuild + "
                  "forward + adjoint (skip + adaptive Eq.5 + Z-order + Z-tiles, N_S=16)",
    "plain_2k": "2,000 Gaussians uniform in [-1,1]^3, one 64x64 view at radius 3, BVH rebuild + forward + adjoint "
                "(uniform dt=0.01, no skipping, N_S=16)",
    "outdoor_3m": "3,000,000 Gaussians (200-blob cluster + log-radius shell to r=100), one 1237x822 view from inside "
                  "the cluster, BVH rebuild (63-bit codes) + forward + adjoint (skip + adaptive Eq.5 + Z-order + "
                  "Z-tiles, N_S=16)",
}
SWEEP = ("sweep_6m: 6,000,000 torus Gaussians, 64 seeded views 256..1920 x 256..1080, forward only, one "
         "persistent launch (and one launch per view beside it)")
METRIC = "Mrays/s render & fwd+bwd ms/iter vs plain marcher at ≤1e-4 err; % HBM peak"
# workloads whose autotuning includes N_S (the batched training step names all three knobs)
TUNE_NS = {"batch_1m"}
# seconds of oracle work the reference arm's timed steps take in all (its sample is sized to it)
REF_BUDGET_S = 90.0


def workload_label(name: str, fallback: str = "") -> str:
    """The config's workload string; both arms (the CUDA path and the oracle)
    print the same one for the same workload."""
    if name == "sweep_6m":
        return SWEEP
    return f"{name}: " + STEP_WORKLOADS.get(name, fallback)


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="rgx", choices=["rgx", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=list(STEP_WORKLOADS) + ["sweep_6m"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="leave out the torus_100k, outdoor_3m and sweep_6m sub-objects of the default line")
    p.add_argument("--no-tune", action="store_true", help="skip rgx_autotune (the workload's own knobs)")
    p.add_argument("--tune-exhaustive", action="store_true", help="rgx_autotune over the full candidate grid")
    p.add_argument("--tile", default=None, help="fixed ray-tile shape WxH (skips rgx_autotune)")
    p.add_argument("--hit-cap", type=int, default=None, help="fixed hit-list capacity (skips rgx_autotune)")
    p.add_argument("--n-s", type=int, default=None, help="fixed samples per segment (skips rgx_autotune)")
    p.add_argument("--scale-res", type=float, default=None,
                   help="scale every view's resolution (a smaller case of the same scene, e.g. for a profiler "
                        "capture; the line's config records it)")
    return p.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
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
def kernel_version() -> str:
    """Version tag of the march kernels (RGX_MARCH_VERSION in march.cu): ncu counters
    taken on another version no longer describe the kernel."""
    src = open(os.path.join(ROOT, "paper_2509_07782_b300", "csrc", "march.cu")).read()
    m = re.search(r'#define\s+RGX_MARCH_VERSION\s+"([^"]+)"', src)
    return m.group(1) if m else "unversioned"


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summaries (lines ``traffic_bytes_per_launch <workload> <kernel> <bytes>
    kernel_version <v>``), or None when there is none for that pair or the
    kernel version changed since the counters were taken."""
    import glob
    ver = kernel_version()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.split()
            if len(parts) == 6 and parts[0] == "traffic_bytes_per_launch" and parts[1] == workload \
                    and parts[2] == kernel and parts[4] == "kernel_version" and parts[5] == ver:
                return int(parts[3])
    return None


def launches_per_step(opts, ncam_launches: int = 1) -> int:
    """Kernels of this library one step launches: the build (bounds, Morton codes, 3 per
    radix pass, pack, radix tree, refit, 4-wide records) and per march launch one kernel,
    plus the adjoint's finalisation."""
    passes = 8 if opts.flags & 16 else 4
    build = 2 + 3 * passes + 1 + 3
    return build + ncam_launches + ncam_launches + 1


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


def alu_model(evals, hits, backward: bool):
    """FP32 FLOPs of the arithmetic one march launch performs (no SFU weighting).

    Per (sample, listed Gaussian) pair: sample offset (FMA), quadratic form
    (MUL + FMA), truncation compare, exponent argument (FMA) and, where the
    sample lies inside the truncation, density add and 3 colour FMA: counted as
    14 FLOPs for every listed pair (an upper bound on the in-support pairs) plus
    one ex2 on the SFU, which is not counted here.  The adjoint evaluates each
    pair twice (the replayed sums, then its own loop) and adds the dL/dg
    product, 3 moment terms and 3 colour-gradient FMA: 2 x 14 + 22.  Per (ray,
    segment, Gaussian) hit: chord solve (~60) and SH colour (48 FMA = 96) in
    the forward; local frame and moment expansion (~60) and SH gradient (96)
    in the adjoint.
    """
    per_eval = 2 * 14 + 22 if backward else 14
    per_hit = 60 + 96
    return evals * per_eval + hits * per_hit


def fp32_peak_tflops(sm_mhz: float, sms: int = 148) -> float:
    """FP32 peak derived from the unit counts: SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def batch_cameras(rank: int):
    """Rank r > 0's own 8 views: the batch's resolutions on seeded radius-4 orbits."""
    from paper_2509_07782_b300 import synth
    rng = np.random.Generator(np.random.PCG64(5000 + rank))
    return [synth.orbit_camera(rng, 4.0, w, h) for (w, h) in synth.BATCH_RES]


def rank_workload(name: str, rank: int, scale_res=None):
    """The workload as rank `rank` renders it: rank 0 the named views, every other
    rank its own seeded views of the same scene (weak scaling)."""
    from paper_2509_07782_b300 import synth
    w = synth.workload(name)
    if rank > 0:
        cam0 = w.cameras[0]
        rng = np.random.Generator(np.random.PCG64(5000 + rank))
        if name == "outdoor_3m":
            w.cameras = [synth.inside_camera(rng, 0.3, cam0.width, cam0.height)]
        elif name == "plain_2k":
            w.cameras = [synth.sphere_camera(rng, 3.0, cam0.width, cam0.height)]
        elif name == "batch_1m":
            w.cameras = batch_cameras(rank)
        else:
            w.cameras = [synth.orbit_camera(rng, 4.0, cam0.width, cam0.height)]
    if scale_res is not None:
        w.cameras = [synth.rescale_camera(c, scale_res) for c in w.cameras]
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


def plain_options(w):
    """The plain single-view marcher's options: uniform step = the workload's dt_min (its
    dt in uniform mode), no skipping, caller-order storage, scanline rays."""
    from paper_2509_07782_b300 import synth
    return synth.Options(dt=w.options.dt_min if w.options.adaptive else w.options.dt, n_s=w.options.n_s,
                         sigma_eps=w.options.sigma_eps, hit_cap=w.options.hit_cap, morton63=w.options.morton63)


# ---------------------------------------------------------------------------------------------
def _tune(args, name, sc, cams, t, opts):
    """Tuning knobs of the step: fixed from the command line, rgx_autotune, or the
    workload's own.  Returns (opts, description)."""
    import torch
    if args.tile or args.hit_cap or args.n_s:
        if args.tile:
            opts.tile_w, opts.tile_h = (int(x) for x in args.tile.lower().split("x"))
        if args.hit_cap:
            opts.hit_cap = args.hit_cap
        if args.n_s:
            opts.n_s = args.n_s
        return opts, {"tile": [opts.tile_w, opts.tile_h], "hit_cap": opts.hit_cap, "n_s": opts.n_s, "fixed": True}
    if args.no_tune:
        return opts, {"tile": [opts.tile_w, opts.tile_h], "hit_cap": opts.hit_cap, "n_s": opts.n_s,
                      "tuned": False}
    sc.build(*t, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, best_ms = sc.autotune(cams, opts, tune_ns=name in TUNE_NS, with_backward=True,
                                exhaustive=args.tune_exhaustive)
    wall = (time.perf_counter() - t0) * 1e3
    return best, {"tile": [best.tile_w, best.tile_h], "hit_cap": best.hit_cap, "n_s": best.n_s,
                  "lower_first": bool(best.flags & 32),
                  "tuned_knobs": "tile shape, hit_cap" + (", N_S" if name in TUNE_NS else "") +
                                 ", first-window lowering",
                  "search": "exhaustive grid" if args.tune_exhaustive else "one knob at a time",
                  "best_candidate_ms": best_ms, "tuning_wall_ms": wall}


def run_plain(sc_factory, w, t, up, opts_tuned, stream, reps=3):
    """The plain single-view marcher: one launch per view, forward and forward + adjoint."""
    import torch
    from paper_2509_07782_b300 import rgx
    po = plain_options(w)
    popts = rgx.make_opts(po)
    popts.hit_cap = opts_tuned.hit_cap
    sp = sc_factory()
    singles = [rgx.Cameras([c]) for c in w.cameras]
    offs = np.concatenate([[0], np.cumsum([c.n_rays for c in w.cameras])]).astype(np.int64)
    ups = [up[int(offs[i]):int(offs[i + 1])] for i in range(len(singles))]
    grads = [torch.zeros_like(x) for x in t]

    def once(timed):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        sp.build(*t, popts)
        fm = bm = 0.0
        for cb, u in zip(singles, ups):
            ev[0].record(stream)
            _, pst = sp.forward(cb, popts)
            ev[1].record(stream)
            sp.backward(cb, popts, pst, u, grads)
            ev[2].record(stream)
            torch.cuda.synchronize()
            fm += ev[0].elapsed_time(ev[1])
            bm += ev[1].elapsed_time(ev[2])
        return fm, bm

    once(False)
    res = [once(True) for _ in range(reps)]
    fm = statistics.median(r[0] for r in res)
    bm = statistics.median(r[1] for r in res)
    # work counters of one untimed forward per view, summed over the views
    work = {}
    for cb in singles:
        sp.forward(cb, popts)
        for k, v in sp.counters(stream).items():
            work[k] = work.get(k, 0) + v
    R = sum(c.n_rays for c in w.cameras)
    out = {"fwd_ms": fm, "bwd_ms": bm, "fwd_bwd_ms": fm + bm, "render_mrays_s": R / fm / 1e3,
           "fwd_bwd_mrays_s": R / (fm + bm) / 1e3,
           "options": f"uniform dt={po.dt}, N_S={po.n_s}, hit_cap={popts.hit_cap}, no skip, caller order, "
                      f"scanline rays, one launch per view ({len(singles)} views)",
           "work_fwd": work}
    if sp.status() != 0:
        out["status"] = "device status nonzero"
    return out


def run_e2e(sc, cams, opts, t, upstream, steps, stream, ref_rgba, ref_grads):
    """The step through the C-ABI with host buffers: every step uploads its parameters and
    upstream gradient from pinned host memory and downloads its gradients and image.  The
    copies run on a copy stream with two buffer slots, so step i+1's upload and step i's
    download overlap the kernels of the neighbouring steps; the timed region runs from
    before the first upload to after the last download."""
    import torch
    from paper_2509_07782_b300 import rgx
    dev = t[0].device
    R = cams.n_rays
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

    with torch.cuda.stream(stream):
        e2e_run(2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        last = e2e_run(steps, e0, e1)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the downloaded results must be the step's: the image bit for bit, the gradients (float
    # atomics, summation order free) to rounding
    ok = bool(torch.equal(last[5], ref_rgba.cpu()))
    for h, g in zip(last[:5], ref_grads):
        ref = g.cpu()
        ok &= float((h - ref).norm()) <= 1e-4 * max(float(ref.norm()), 1e-30)
    if not ok:
        print("warning: end-to-end results differ from the device-resident step's", file=sys.stderr)
    return dict(ms_per_step=ms, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, matches_device_step=ok,
                copies="pinned host buffers; uploads and downloads on a copy stream, two buffer slots, "
                       "overlapping the neighbouring steps' kernels")


def run_step(args, name, rank, world, local, plain=True, e2e=True):
    """Forward + adjoint step of one workload (one or several views), captured in a CUDA graph."""
    import torch
    import torch.distributed as dist

    from paper_2509_07782_b300 import dist as rdist
    from paper_2509_07782_b300 import graph, rgx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = rank_workload(name, rank, getattr(args, "scale_res", None))
    opts = rgx.make_opts(w.options)
    cams = rgx.Cameras(w.cameras)
    R = cams.n_rays
    t = list(rgx.scene_tensors(w.scene, device=dev))
    sc = rgx.Scene(local)
    upstream = torch.randn(R, 4, device=dev, generator=torch.Generator(device=dev).manual_seed(1 + rank))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts, tuned = _tune(args, name, sc, cams, t, opts)
    step = graph.CapturedStep(sc, cams, opts, t, upstream)
    stream = step.stream

    def one(events=None):
        step.replay(events)
        if world > 1:
            with torch.cuda.stream(stream):
                rdist.allreduce_gradients(step.grad_flat, world)

    for _ in range(max(args.warmup, 3)):
        one()
    torch.cuda.synchronize()
    st = sc.status(stream)
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    # per step: events before the build, the forward and the adjoint graphs, after the adjoint,
    # and after the gradient all-reduce (multi-GPU)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        one(evs[i][:4])
        evs[i][4].record(stream)
        with torch.cuda.stream(stream):
            flush.fill_(float(i))  # L2 flush between steps, outside the events
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [e[0].elapsed_time(e[4]) for e in evs]
    total_ms = float(sum(step_ms))
    st = sc.status(stream)
    build_ms = statistics.median(e[0].elapsed_time(e[1]) for e in evs)
    fwd_ms = statistics.median(e[1].elapsed_time(e[2]) for e in evs)
    bwd_ms = statistics.median(e[2].elapsed_time(e[3]) for e in evs)
    grads = [g.clone() for g in step.grads]
    rgba = step.rgba.clone()

    # work counters of one forward and one backward (separate, untimed eager calls)
    with torch.cuda.stream(stream):
        r2, state = sc.forward(cams, opts, stream=stream)
        cf = sc.counters(stream)
        g2 = [torch.zeros_like(x) for x in t]
        sc.backward(cams, opts, state, upstream, g2, stream=stream)
        cb = sc.counters(stream)
    torch.cuda.synchronize()
    n_touched = touched_gaussians(g2)

    e2e_out = None
    if e2e:
        # single-rank step (no all-reduce), compared with that rank's own gradients
        e2e_out = run_e2e(sc, cams, opts, t, upstream, args.steps, torch.cuda.current_stream(dev), r2, g2)
    plain_out = run_plain(lambda: rgx.Scene(local), w, t, upstream, opts, torch.cuda.current_stream(dev)) \
        if plain else None

    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_out["ms_per_step"] if e2e_out else 0.0], world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_mrays(world, R, args.steps, total_ms)
    if e2e_out:
        e2e_out = dict(value=whole_job_mrays(world, R, 1, e2e_ms), unit="Mrays/s", **e2e_out)
        e2e_out["ms_per_step"] = e2e_ms
    return dict(R=R, ncam=len(w.cameras), ms_per_step=ms_per_step, value=value, build_ms=build_ms,
                fwd_ms=fwd_ms, bwd_ms=bwd_ms, wall_s=wall, e2e=e2e_out, counters_fwd=cf, counters_bwd=cb,
                clocks=clocks, status=st, plain=plain_out, opts=opts, tuned=tuned, n=w.scene.n,
                n_touched=n_touched, steps_launches=launches_per_step(opts) * args.steps,
                rgba_mean=float(rgba[:, 3].mean()), grad_norm=float(sum(float(g.norm()) for g in grads)))


def _oracle_rate(w, cams_pix, P, threads: int, max_seconds: float, per_cam_start: int):
    """Oracle forward + adjoint on seeded pixel samples of each view with ``threads``
    OpenMP threads, the samples grown 4x until a pass takes about a quarter of
    ``max_seconds``.  Returns (rays/s, pixels, seconds)."""
    import oracle
    from paper_2509_07782_b300 import synth
    k = per_cam_start
    while True:
        tot, t0 = 0, time.perf_counter()
        for ci, cam in enumerate(cams_pix):
            pix = synth.pixel_subset(cam, k, seed=3 + ci)
            W = np.random.default_rng(4 + ci).normal(size=(len(pix), 4))
            oracle.render(w.scene, cam, w.options, pix=pix, params=P, nthreads=threads)
            oracle.backward(w.scene, cam, w.options, W, pix=pix, params=P, nthreads=threads)
            tot += len(pix)
        dt = time.perf_counter() - t0
        if dt > max_seconds / 4 or all(k >= c.n_rays for c in cams_pix):
            return tot / dt, tot, dt
        k *= 4


def cpu_baseline(workload=WORKLOAD, max_seconds=12.0):
    """FP64 oracle (as it stands) on the host cores: forward + adjoint on seeded pixel
    samples of the workload's views, grown until ~max_seconds / 4 per pass; then once
    more on one core (a smaller sample)."""
    import oracle
    from paper_2509_07782_b300 import synth
    w = synth.workload(workload)
    P = oracle.Params(w.scene)
    cores = os.cpu_count() or 1
    start = max(4, int(256 * 100_000 / max(w.scene.n, 1)) // len(w.cameras))
    rate, n, dt = _oracle_rate(w, w.cameras, P, cores, max_seconds, start)
    out = {"value": rate / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
           "sample": f"{n} seeded pixels over the {len(w.cameras)} view(s), forward + adjoint, {dt:.2f} s"}
    rate1, n1, dt1 = _oracle_rate(w, w.cameras, P, 1, max_seconds / 2, max(1, start // 16))
    out["single_core"] = {"value": rate1 / 1e6, "unit": "Mrays/s", "cores": 1,
                          "sample": f"{n1} seeded pixels, forward + adjoint, {dt1:.2f} s"}
    return out


def run_sweep(args, steps=None):
    """sweep_6m: 6M Gaussians, 64 views, forward only: one persistent launch for all views
    vs one launch per view; FPS per view size."""
    import torch

    from paper_2509_07782_b300 import rgx, synth
    dev = torch.device("cuda", 0)
    steps = steps or args.steps
    w = synth.workload("sweep_6m")
    wo = w.options
    t = rgx.scene_tensors(w.scene, device=dev)
    sc = rgx.Scene(0)
    if args.tile or args.hit_cap or args.n_s:
        if args.tile:
            wo.tile_w, wo.tile_h = (int(x) for x in args.tile.lower().split("x"))
        if args.hit_cap:
            wo.hit_cap = args.hit_cap
        if args.n_s:
            wo.n_s = args.n_s
        opts = rgx.make_opts(wo)
        knobs = {"tile": [wo.tile_w, wo.tile_h], "hit_cap": wo.hit_cap, "n_s": wo.n_s, "fixed": True}
    elif args.no_tune:
        opts = rgx.make_opts(wo)
        knobs = {"tile": [wo.tile_w, wo.tile_h], "hit_cap": wo.hit_cap, "n_s": wo.n_s, "tuned": False}
    else:
        # rgx_autotune (forward only) on every 8th view: a sample of the sizes in one launch
        sc.build(*t, rgx.make_opts(wo))
        sub = rgx.Cameras(w.cameras[::8])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opts, best_ms = sc.autotune(sub, rgx.make_opts(wo), tune_ns=True, with_backward=False)
        knobs = {"tile": [opts.tile_w, opts.tile_h], "hit_cap": opts.hit_cap, "n_s": opts.n_s,
                 "lower_first": bool(opts.flags & 32), "tuned_knobs": "tile shape, hit_cap, N_S, first-window lowering",
                 "tuned_on": f"every 8th view ({len(w.cameras[::8])} of {len(w.cameras)}), forward only",
                 "best_candidate_ms": best_ms, "tuning_wall_ms": (time.perf_counter() - t0) * 1e3}
    sc.build(*t, opts)
    cams_all = rgx.Cameras(w.cameras)
    singles = [rgx.Cameras([c]) for c in w.cameras]
    rgba = torch.empty(cams_all.n_rays, 4, device=dev)
    st = torch.cuda.current_stream()
    rgx.rgx_render_forward(sc.h, cams_all, opts, rgba)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        rgx.rgx_render_forward(sc.h, cams_all, opts, rgba)
    e1.record(st)
    torch.cuda.synchronize()
    ms_persistent = e0.elapsed_time(e1) / steps
    per_view = []
    outs = [torch.empty(c.n_rays, 4, device=dev) for c in singles]
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
    peaks, src = load_peaks()
    # forward only: no gradient tells which Gaussians were read, so all of them count (an upper bound)
    kname = f"k_march<{int(opts.n_s)},0>"
    hbm = hbm_roofline(w.scene.n, cams_all.n_rays, ms_persistent / 1e3, False, float(peaks.get("hbm_gbs", 6400.0)),
                       traffic=profiled_traffic(kname, "sweep_6m"), ray_bytes=16)
    hbm.update(kernel=kname, peak_source=f"{src} copy bandwidth",
               touched_note="every Gaussian counted as read (upper bound; forward only)")
    return {"workload": SWEEP, "rays_per_step": cams_all.n_rays, "render_mrays_s": cams_all.n_rays / ms_persistent / 1e3,
            "ms_per_render": ms_persistent, "steps": steps,
            "knobs": knobs,
            "one_launch_per_view": {"ms_total": ms_per_view_total,
                                    "mrays_s": cams_all.n_rays / ms_per_view_total / 1e3},
            "fps_per_view": {"smallest": {"pixels": q[0][0], "fps": q[0][1]},
                             "median": {"pixels": q[1][0], "fps": q[1][1]},
                             "largest": {"pixels": q[2][0], "fps": q[2][1]}},
            "hbm_roofline": hbm, "device_status": sc.status()}


def reference_line(args):
    """The FP64 oracle on the host cores (as it stands), on a bounded pixel sample of
    every view of the workload, forward + adjoint (forward only for the sweep)."""
    import oracle
    from paper_2509_07782_b300 import synth
    w = synth.workload(args.workload)
    P = oracle.Params(w.scene)
    cores = os.cpu_count() or 1
    cams = w.cameras if args.workload != "sweep_6m" else w.cameras[:8]
    with_bwd = args.workload != "sweep_6m"
    # the oracle brute-forces every Gaussian per ray: the per-step sample is sized from its measured
    # rate so that the timed steps take about REF_BUDGET_S seconds in all (at least one pixel per view)
    # (one call with a pixel per core, so that every OpenMP thread works as in the timed steps)
    # (a pixel per core of every view, one call per view: every OpenMP thread busy, as in the timed
    # steps, whose per-view sample is a multiple of the core count where the budget allows)
    probe = [(cam, synth.pixel_subset(cam, cores, seed=900 + i)) for i, cam in enumerate(cams)]
    t0 = time.perf_counter()
    for cam, pix in probe:
        oracle.render(w.scene, cam, w.options, pix=pix, params=P, nthreads=cores)
        if with_bwd:
            oracle.backward(w.scene, cam, w.options, np.ones((len(pix), 4)), pix=pix, params=P, nthreads=cores)
    dt_probe = max(time.perf_counter() - t0, 1e-6)  # seconds for `cores` pixels of every view
    budget = REF_BUDGET_S / max(args.steps, 1)
    per = cores * int(budget // dt_probe) if budget >= dt_probe else int(cores * budget / dt_probe)
    per = int(min(max(per, 1), max(1, 2048 // len(cams))))
    samples = [(cam, synth.pixel_subset(cam, min(per, cam.n_rays), seed=3 + i)) for i, cam in enumerate(cams)]
    Ws = [np.random.default_rng(4 + i).normal(size=(len(p), 4)) for i, (_, p) in enumerate(samples)]
    for _ in range(max(args.warmup, 0)):
        cam, pix = samples[0]
        oracle.render(w.scene, cam, w.options, pix=pix[:4], params=P, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for (cam, pix), W in zip(samples, Ws):
            oracle.render(w.scene, cam, w.options, pix=pix, params=P, nthreads=cores)
            if with_bwd:
                oracle.backward(w.scene, cam, w.options, W, pix=pix, params=P, nthreads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    rays = sum(len(p) for _, p in samples)
    v = rays * args.steps / tot / 1e6
    desc = f"{rays} seeded pixels over {len(samples)} view(s) per step, forward" + (" + adjoint" if with_bwd else "")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(args.workload, f"{w.scene.n} Gaussians"), "sample": desc},
            "cpu_baseline": {"value": v, "unit": "Mrays/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def step_line(args, r, world):
    """The JSON line of a forward + adjoint step workload."""
    peaks, src = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    fp32_peak = fp32_peak_tflops(sm_mhz)
    cb, cf = r["counters_bwd"], r["counters_fwd"]
    flops_b = alu_model(cb["evals"], cb["hits"], True)
    flops_f = alu_model(cf["evals"], cf["hits"], False)
    ns = int(r["opts"].n_s)
    dominant_is_bwd = r["bwd_ms"] >= r["fwd_ms"]
    kname = f"k_march<{ns},{1 if dominant_is_bwd else 0}>"
    k_s = (r["bwd_ms"] if dominant_is_bwd else r["fwd_ms"]) / 1e3
    flops = flops_b if dominant_is_bwd else flops_f
    achieved = flops / k_s / 1e12
    # ncu's DRAM bytes describe the full-size workload: none for a scaled-down view
    traffic = profiled_traffic(kname, args.workload) if not args.scale_res else None
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic,
                "peak_source": f"derived (not measured): 148 SMs x 128 FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz; "
                               "FP32 FLOPs only, ex2 (SFU) not counted",
                "duration": "median over the timed steps of its graph's replay (CUDA events on the launching stream)",
                "work": "per (sample, listed Gaussian) pair 14 FLOPs (2x14+22 in the adjoint), per (ray, "
                        "segment, Gaussian) hit 156, from device counters"}
    hbm = hbm_roofline(r["n_touched"], r["R"], k_s, dominant_is_bwd, float(peaks.get("hbm_gbs", 6400.0)), traffic)
    hbm["kernel"] = kname
    hbm["peak_source"] = f"{src} copy bandwidth"
    out = {
        "metric": METRIC, "value": r["value"], "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(args.workload) +
                   (f" (views scaled by {args.scale_res})" if args.scale_res else ""),
                   "rays_per_step_per_gpu": r["R"], "views": r["ncam"], "gaussians": r["n"],
                   "l2": "flushed (256 MiB write) between steps",
                   "parallelism": (f"{world} ranks, each its own seeded views of one scene; one all-reduce "
                                   "(sum) of the gradients per step") if world > 1 else "1 GPU",
                   "knobs": r["tuned"]},
        "fwd_bwd_ms": r["fwd_ms"] + r["bwd_ms"], "build_ms": r["build_ms"], "fwd_ms": r["fwd_ms"],
        "bwd_ms": r["bwd_ms"], "render_mrays_s": r["R"] / r["fwd_ms"] / 1e3,
        "stage_timing": "CUDA events between the build, forward and adjoint graphs of each timed step, median",
        "plain_marcher": r["plain"],
        "speedup_vs_plain": {"render": (r["plain"]["fwd_ms"] / r["fwd_ms"]) if r["plain"] else None,
                             "fwd_bwd": (r["plain"]["fwd_bwd_ms"] / (r["fwd_ms"] + r["bwd_ms"]))
                             if r["plain"] else None},
        "roofline": roofline,
        "hbm_roofline": hbm,
        "work": {"fwd": cf, "bwd": cb},
        "e2e": r["e2e"], "gpu_launches": r["steps_launches"], "clocks": r["clocks"],
        "device_status": r["status"],
    }
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_line(args)))
        return
    import torch
    if args.workload == "sweep_6m":
        if rank == 0:
            s = run_sweep(args)
            print(json.dumps({"metric": METRIC, "value": s["render_mrays_s"], "unit": "Mrays/s", "n_gpus": 1,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": s["ms_per_render"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic", "config": {"workload": SWEEP}, "sweep": s}))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    r = run_step(args, args.workload, rank, world, local, plain=not args.no_plain, e2e=not args.no_e2e)
    extras = {}
    if rank == 0 and args.workload == WORKLOAD and not args.no_extras:
        # the single-view workloads beside the batch: the sparse object view and the dense
        # outdoor view, each with the plain marcher on the same view
        for name, steps in (("torus_100k", "10"), ("outdoor_3m", "5")):
            sub = parse(["--steps", steps, "--warmup", "3"])
            c = run_step(sub, name, 0, 1, local, plain=True, e2e=False)
            extras[name] = {"workload": workload_label(name), "value": c["value"], "unit": "Mrays/s",
                            "steps": int(steps), "ms_per_step": c["ms_per_step"], "build_ms": c["build_ms"],
                            "fwd_ms": c["fwd_ms"], "bwd_ms": c["bwd_ms"], "render_mrays_s": c["R"] / c["fwd_ms"] / 1e3,
                            "knobs": c["tuned"], "plain_marcher": c["plain"],
                            "speedup_vs_plain": {"render": c["plain"]["fwd_ms"] / c["fwd_ms"],
                                                 "fwd_bwd": c["plain"]["fwd_bwd_ms"] / (c["fwd_ms"] + c["bwd_ms"])},
                            "device_status": c["status"]}
        extras["sweep_6m"] = run_sweep(args, steps=2)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    out = step_line(args, r, world)
    out.update(extras)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
