"""Host-side arithmetic of bench.py that needs no GPU: the count of Gaussians a
march touched (from its gradients) and the algorithmic-HBM roofline built on it."""
from __future__ import annotations

import numpy as np
import torch

import bench


def _grads(n, nk=16):
    return [torch.zeros(n, 3), torch.zeros(n, 3), torch.zeros(n, 4), torch.zeros(n), torch.zeros(n, nk, 3)]


def test_touched_counts_gaussians_with_any_nonzero_gradient_entry():
    g = _grads(7)
    assert bench.touched_gaussians(g) == 0
    g[3][2] = 1.0          # density only
    g[4][5, 15, 2] = -3.0  # last SH coefficient of the last channel only
    g[0][5, 0] = 2.0       # same Gaussian again: counted once
    g[2][6, 3] = 1e-30     # tiny but non-zero
    assert bench.touched_gaussians(g) == 3


def test_touched_count_does_not_broadcast_between_tensor_shapes():
    # a (N,) tensor beside (N,3) ones must not form an N x N mask
    n = 1000
    g = _grads(n)
    g[3][:] = 1.0
    assert bench.touched_gaussians(g) == n


def test_hbm_roofline_counts_the_method_bytes():
    f = bench.hbm_roofline(1000, 64, 1e-3, False, 6505.6)
    assert f["algorithmic_bytes"] == 1000 * (236 + 32) + 64 * 32
    b = bench.hbm_roofline(1000, 64, 1e-3, True, 6505.6, traffic=10_000_000)
    assert b["algorithmic_bytes"] == 1000 * (236 + 32 + 2 * 236) + 64 * 32
    assert np.isclose(b["achieved"], b["algorithmic_bytes"] / 1e-3 / 1e9)
    assert np.isclose(b["frac"], b["achieved"] / 6505.6)
    assert np.isclose(b["dram_gbs"], 10.0) and np.isclose(b["dram_frac"], 10.0 / 6505.6)
    assert "dram_bytes" not in f
    # a forward that keeps no per-ray state writes only RGBA
    g = bench.hbm_roofline(1000, 64, 1e-3, False, 6505.6, ray_bytes=16)
    assert g["algorithmic_bytes"] == 1000 * (236 + 32) + 64 * 16


def test_profiled_traffic_is_keyed_on_workload_kernel_and_kernel_version(monkeypatch, tmp_path):
    src = tmp_path / "paper_2509_07782_b300" / "csrc"
    src.mkdir(parents=True)
    (src / "march.cu").write_text('// kernels\n#define RGX_MARCH_VERSION "v7"\n')
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "a.md").write_text(
        "traffic_bytes_per_launch torus_100k k_march<16,1> 123 kernel_version v7\n"
        "traffic_bytes_per_launch outdoor_3m k_march<16,1> 456 kernel_version v7\n"
        "traffic_bytes_per_launch outdoor_3m k_march<16,0> 789 kernel_version v6\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_version() == "v7"
    assert bench.profiled_traffic("k_march<16,1>", "torus_100k") == 123
    assert bench.profiled_traffic("k_march<16,1>", "outdoor_3m") == 456
    assert bench.profiled_traffic("k_march<16,1>", "plain_2k") is None
    # counters taken on another kernel version do not count
    assert bench.profiled_traffic("k_march<16,0>", "outdoor_3m") is None


def test_the_repository_kernel_version_is_declared():
    assert bench.kernel_version() not in ("", "unversioned")


def test_alu_model_and_fp32_peak():
    assert bench.alu_model(10, 2, False) == 10 * 14 + 2 * 156
    assert bench.alu_model(10, 2, True) == 10 * 50 + 2 * 156
    assert np.isclose(bench.fp32_peak_tflops(2032.0), 148 * 128 * 2 * 2.032e9 / 1e12)


def test_launch_count_per_step():
    from paper_2509_07782_b300 import rgx, synth
    o30 = rgx.make_opts(synth.fast_options())
    o63 = rgx.make_opts(synth.fast_options(morton63=True))
    # build: bounds, morton, 3 per radix pass, pack, karras, refit, widen; forward march; adjoint march + finalise
    assert bench.launches_per_step(o30) == 2 + 12 + 1 + 3 + 1 + 2
    assert bench.launches_per_step(o63) == 2 + 24 + 1 + 3 + 1 + 2


def test_reference_arm_prints_the_contract_line_on_the_host():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and
    prints one JSON line with the same metric, unit and workload as the CUDA
    arm, its own cpu_baseline and an e2e object with no device copies."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "plain_2k",
                          "--steps", "1", "--warmup", "1"], cwd=root, capture_output=True, text=True,
                         timeout=600, check=True).stdout.strip().splitlines()
    d = json.loads(out[-1])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "Mrays/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.workload_label("plain_2k")
    assert d["steps"] == 1 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["dtype"] == "f64" and d["data"] == "synthetic"


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """Launched the way multi-GPU runs are (torchrun, two ranks, 127.0.0.1),
    the reference arm runs on rank 0 only: exactly one JSON line comes out and
    both ranks exit 0."""
    import json
    import os
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                          "--workload", "plain_2k", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                         cwd=root, capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_clock_sampler_summarises_rows_and_reasons():
    """The clocks object of the JSON line: median SM clock under load, the
    maximum clock, and every throttle reason seen active in any sample."""
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["unsampled"]
    row = "0, {sm}, 2032, 900.5, 0x0, {hw}, Not Active, Not Active, {cap}"
    s.rows = [[x.strip() for x in row.format(sm=sm, hw=hw, cap=cap).split(",")]
              for sm, hw, cap in ((2032, "Not Active", "Not Active"), (1980, "Not Active", "Active"),
                                  (2032, "Not Active", "Not Active"), ("[N/A]", "Active", "Not Active"))]
    c = s.stop()
    assert c["sm_mhz"] == 2032.0 and c["sm_max_mhz"] == 2032.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert c["samples"] == 4


def test_step_line_attaches_profiled_traffic_only_at_full_size(monkeypatch, tmp_path):
    """The DRAM bytes ncu counted describe the full-size workload: a line built on
    views scaled down for a profiler's small case carries none."""
    import types
    src = tmp_path / "paper_2509_07782_b300" / "csrc"
    src.mkdir(parents=True)
    (src / "march.cu").write_text('#define RGX_MARCH_VERSION "v9"\n')
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "b.md").write_text(
        "traffic_bytes_per_launch batch_1m k_march<32,0> 1000000 kernel_version v9\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    cnt = {"evals": 10_000, "hits": 100, "segments": 10, "rays": 50}
    r = dict(R=50, ncam=1, ms_per_step=3.0, value=1.0, build_ms=0.1, fwd_ms=2.0, bwd_ms=1.0, e2e=None,
             counters_fwd=cnt, counters_bwd=cnt, clocks={}, status=0, plain=None, opts=types.SimpleNamespace(n_s=32),
             tuned={}, n=10, n_touched=10, steps_launches=21)
    full = bench.step_line(bench.parse(["--workload", "batch_1m"]), r, 1)
    assert full["roofline"]["kernel"] == "k_march<32,0>"
    assert full["roofline"]["traffic"] == 1_000_000
    assert full["hbm_roofline"]["dram_bytes"] == 1_000_000
    small = bench.step_line(bench.parse(["--workload", "batch_1m", "--scale-res", "0.12"]), r, 1)
    assert small["roofline"]["traffic"] is None and "dram_bytes" not in small["hbm_roofline"]
    assert "scaled by 0.12" in small["config"]["workload"]
