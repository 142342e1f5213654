"""One training step -- BVH rebuild, forward march, adjoint -- captured in a CUDA graph.

The step works on persistent tensors: the caller updates the five parameter
tensors (and, if it wants, the upstream gradient) in place between replays and
reads ``rgba`` / ``grads`` after each replay.  Capture happens after one eager
warm-up step, which grows the scene's workspace and caches every launch
configuration, so the captured calls allocate nothing and make no attribute
queries.  Cameras are copied from their pinned host buffer at every replay, so
their contents (not their number or sizes) may change between replays.

With ``stage_events=True`` four CUDA events are recorded inside the graph
(external event-record nodes) around the build, the forward and the adjoint,
so every replay also yields the time of each stage (``stage_ms()``).
"""
from __future__ import annotations

import torch

from . import dist, rgx


class _StageEvents:
    """Four timing events recorded by graph nodes (cudaEventRecordExternal)."""

    def __init__(self):
        from cuda.bindings import runtime as rt
        self.rt = rt
        self.ev = []
        for _ in range(4):
            err, e = rt.cudaEventCreate()
            if err != rt.cudaError_t.cudaSuccess:
                raise RuntimeError(f"cudaEventCreate: {err}")
            self.ev.append(e)

    def record(self, i: int, stream: torch.cuda.Stream):
        rt = self.rt
        (err,) = rt.cudaEventRecordWithFlags(self.ev[i], stream.cuda_stream, rt.cudaEventRecordExternal)
        if err != rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaEventRecordWithFlags: {err}")

    def elapsed(self, i: int, j: int) -> float:
        err, ms = self.rt.cudaEventElapsedTime(self.ev[i], self.ev[j])
        if err != self.rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaEventElapsedTime: {err}")
        return float(ms)

    def __del__(self):
        try:
            for e in self.ev:
                self.rt.cudaEventDestroy(e)
        except Exception:
            pass


class CapturedStep:
    def __init__(self, scene: rgx.Scene, cams: rgx.Cameras, opts: rgx.RgxOpts, params, d_rgba: torch.Tensor,
                 sh_degree: int = 3, backward: bool = True, stage_events: bool = False):
        self.scene, self.cams, self.opts = scene, cams, opts
        self.params = list(params)
        self.sh_degree = sh_degree
        self.backward = backward
        dev = self.params[0].device
        self.rgba = torch.empty(cams.n_rays, 4, dtype=torch.float32, device=dev)
        self.state = rgx.new_state(cams.n_rays, dev)
        self.d_rgba = d_rgba
        # the five gradient tensors are views of one flat buffer, so that a multi-GPU step
        # sums them over ranks with a single all-reduce
        self.grad_flat, self.grads = dist.flat_views(self.params, dev)
        self.stream = torch.cuda.Stream(device=dev)
        self.events = _StageEvents() if stage_events else None
        # eager warm-up on the capture stream (workspace growth, launch-config cache)
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(self.stream):
            self._body()
        self.stream.synchronize()
        st = scene.status(self.stream)
        if st != 0:
            raise rgx.RgxError(st, "device status after warm-up")
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._body()

    def _mark(self, i: int):
        if self.events is not None:
            self.events.record(i, self.stream)

    def _body(self):
        s = self.stream
        h = self.scene.h
        self._mark(0)
        rgx.rgx_build_bvh(h, *self.params, self.sh_degree, self.opts, stream=s)
        self._mark(1)
        rgx.rgx_render_forward(h, self.cams, self.opts, self.rgba, self.state, stream=s)
        self._mark(2)
        if self.backward:
            self.grad_flat.zero_()
            rgx.rgx_render_backward(h, self.cams, self.opts, self.state, self.d_rgba, *self.grads, stream=s)
        self._mark(3)

    def replay(self):
        """Replay on the step's own stream (the stream the graph was captured on)."""
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def stage_ms(self):
        """(build, forward, adjoint) milliseconds of the last replay (after it has finished)."""
        e = self.events
        return e.elapsed(0, 1), e.elapsed(1, 2), e.elapsed(2, 3)
