"""The view-sharded multi-GPU step, emulated as two processes on one GPU.

Each rank builds its own BVH from the same parameters, renders and
differentiates its own views with the CUDA library, and the ranks sum their
gradients with one all-reduce (gloo, over host copies: there is one GPU).  The
result must equal the single-process adjoint of all the views in one batched
launch, within the gradient tolerance (relative L2 1e-3 per tensor).  The two
processes' kernels never wait on each other; only the host all-reduce joins them.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

NAMES = ["means", "scales", "quats", "densities", "sh"]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _views():
    from paper_2509_07782_b300 import synth
    w = synth.workload("batch_1m", n=80_000, scale_res=0.2)
    return w, w.cameras[:4]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    try:
        import torch.distributed as dist

        from paper_2509_07782_b300 import dist as rdist
        from paper_2509_07782_b300 import rgx

        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        try:
            torch.cuda.set_device(0)
            w, cams = _views()
            idx = list(range(rank, len(cams), world))
            mine = [cams[i] for i in idx]
            t = rgx.scene_tensors(w.scene)
            o = rgx.make_opts(w.options)
            sc = rgx.Scene(0)
            sc.build(*t, o)
            cb = rgx.Cameras(mine)
            rgba, state = sc.forward(cb, o)
            d = torch.cat([_upstream(i, cams[i].n_rays) for i in idx])
            flat, grads = rdist.flat_views(t, "cuda")
            sc.backward(cb, o, state, d, grads)
            assert sc.status() == 0
            host = flat.cpu()
            rdist.allreduce_gradients(host, world)
            q.put((rank, host.numpy().copy()))
        finally:
            dist.destroy_process_group()
    except BaseException as e:  # report instead of leaving the parent waiting
        q.put((rank, repr(e)))
        raise


def _upstream(i: int, n: int) -> torch.Tensor:
    g = torch.Generator().manual_seed(100 + i)
    return torch.randn(n, 4, generator=g).cuda()


def test_two_ranks_allreduced_gradients_equal_the_batched_adjoint():
    from paper_2509_07782_b300 import rgx
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
    for r in range(2):
        assert not isinstance(out[r], str), f"rank {r}: {out[r]}"
    for p in procs:
        assert p.exitcode == 0
    # single process: all four views in one persistent launch, in the ranks' order of views
    w, cams = _views()
    order = list(range(0, len(cams), 2)) + list(range(1, len(cams), 2))
    t = rgx.scene_tensors(w.scene)
    o = rgx.make_opts(w.options)
    sc = rgx.Scene()
    sc.build(*t, o)
    cb = rgx.Cameras([cams[i] for i in order])
    rgba, state = sc.forward(cb, o)
    d = torch.cat([_upstream(i, cams[i].n_rays) for i in order])
    grads = [torch.zeros_like(x) for x in t]
    sc.backward(cb, o, state, d, grads)
    assert sc.status() == 0
    ref = np.concatenate([g.cpu().numpy().ravel() for g in grads])
    np.testing.assert_array_equal(out[0], out[1])
    off = 0
    for name, g in zip(NAMES, grads):
        n = g.numel()
        a, b = out[0][off:off + n].astype(np.float64), ref[off:off + n].astype(np.float64)
        assert np.linalg.norm(b) > 0, name
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-3, name
        off += n
