"""Multi-GPU host logic of bench.py, run as two gloo ranks on the CPU.

The path shards by view: every rank renders its own seeded camera of the same
scene, so the data path has no collective.  What the ranks share is the timing
protocol: the step time is the maximum over ranks and the whole-job value
counts the rays of every rank over that time.  These tests run that logic in
two processes (world size 2, gloo, 127.0.0.1) without any GPU.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w = bench.rank_workload("plain_2k", rank)
        cam = w.cameras[0]
        # rank-dependent local timings (ms): step total and end-to-end
        local = [10.0 + 5.0 * rank, 30.0 - 7.0 * rank]
        mx = bench.max_over_ranks(local, world)
        q.put((rank, np.asarray(cam.c2w, np.float64).tolist(), cam.width, cam.height, int(w.scene.n), mx))
    finally:
        dist.destroy_process_group()


def _run(world: int):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return {o[0]: o for o in out}


def test_two_ranks_render_distinct_views_of_one_scene_and_agree_on_the_max_time():
    res = _run(2)
    r0, r1 = res[0], res[1]
    # one scene, two different seeded views of the same size
    assert r0[4] == r1[4] == 2000
    assert (r0[2], r0[3]) == (r1[2], r1[3]) == (64, 64)
    assert not np.allclose(r0[1], r1[1])
    # rank 0 renders the workload's own view
    import bench
    from paper_2509_07782_b300 import synth
    assert np.allclose(r0[1], synth.workload("plain_2k").cameras[0].c2w)
    # deterministic per rank
    assert np.allclose(r1[1], bench.rank_workload("plain_2k", 1).cameras[0].c2w)
    # every rank sees the maximum over ranks of each timing
    assert r0[5] == r1[5] == [15.0, 30.0]


def test_whole_job_value_counts_every_rank_over_the_slowest_time():
    import bench
    one = bench.whole_job_mrays(1, 640_000, 10, 250.0)
    assert np.isclose(one, 640_000 * 10 / 0.25 / 1e6)
    # two ranks, same per-rank work, slowest rank took longer: value uses that time
    two = bench.whole_job_mrays(2, 640_000, 10, 300.0)
    assert np.isclose(two, 2 * 640_000 * 10 / 0.3 / 1e6)
    assert two < 2 * one


def _allreduce_main(rank: int, world: int, port: int, q) -> None:
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2509_07782_b300 import dist as rdist
    from paper_2509_07782_b300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.workload("plain_2k", n=300)
        cam = synth.rescale_camera(_rank_camera(rank), 0.25)  # 16x16
        W = np.random.default_rng(10 + rank).normal(size=(cam.n_rays, 4))
        g = oracle.backward(w.scene, cam, w.options, W)
        parts = [torch.as_tensor(g[k], dtype=torch.float64) for k in ("means", "scales", "quats", "densities", "sh")]
        flat, views = rdist.flat_views(parts, "cpu", dtype=torch.float64)
        for v, p in zip(views, parts):
            v.copy_(p)
        rdist.allreduce_gradients(flat, world)
        q.put((rank, flat.numpy().copy()))
    finally:
        dist.destroy_process_group()


def _rank_camera(rank: int):
    import bench
    return bench.rank_workload("plain_2k", rank).cameras[0]


def test_view_sharded_gradients_sum_over_ranks_with_one_allreduce():
    """Each rank differentiates its own view (the oracle, on the host) and the
    five gradient tensors, views of one flat buffer, are summed over the ranks
    with one all-reduce: every rank ends with the gradient of both views."""
    import oracle
    from paper_2509_07782_b300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_allreduce_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.workload("plain_2k", n=300)
    total = []
    for rank in range(2):
        cam = synth.rescale_camera(_rank_camera(rank), 0.25)
        W = np.random.default_rng(10 + rank).normal(size=(cam.n_rays, 4))
        g = oracle.backward(w.scene, cam, w.options, W)
        total.append(np.concatenate([g[k].ravel() for k in ("means", "scales", "quats", "densities", "sh")]))
    ref = total[0] + total[1]
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(out[0], ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out[1], ref, rtol=1e-12, atol=1e-12)
