"""One training step -- BVH rebuild, forward march, adjoint -- captured in CUDA graphs.

The step works on persistent tensors: the caller updates the five parameter
tensors (and, if it wants, the upstream gradient) in place between replays and
reads ``rgba`` / ``grads`` after each replay.  Capture happens after one eager
warm-up step, which grows the scene's workspace and caches every launch
configuration, so the captured calls allocate nothing and make no attribute
queries.  Cameras are copied from their pinned host buffer at every replay, so
their contents (not their number or sizes) may change between replays.

The three stages are captured as three graphs replayed back to back on the
step's stream, so that CUDA events recorded between them (``replay(events)``)
time each stage of every replay.
"""
from __future__ import annotations

import torch

from . import dist, rgx


class CapturedStep:
    def __init__(self, scene: rgx.Scene, cams: rgx.Cameras, opts: rgx.RgxOpts, params, d_rgba: torch.Tensor,
                 sh_degree: int = 3, backward: bool = True):
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
        stages = [self._build, self._forward] + ([self._adjoint] if backward else [])
        # eager warm-up on the capture stream (workspace growth, launch-config cache)
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(self.stream):
            for f in stages:
                f()
        self.stream.synchronize()
        st = scene.status(self.stream)
        if st != 0:
            raise rgx.RgxError(st, "device status after warm-up")
        self.graphs = []
        for f in stages:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                f()
            self.graphs.append(g)

    def _build(self):
        rgx.rgx_build_bvh(self.scene.h, *self.params, self.sh_degree, self.opts, stream=self.stream)

    def _forward(self):
        rgx.rgx_render_forward(self.scene.h, self.cams, self.opts, self.rgba, self.state, stream=self.stream)

    def _adjoint(self):
        self.grad_flat.zero_()
        rgx.rgx_render_backward(self.scene.h, self.cams, self.opts, self.state, self.d_rgba, *self.grads,
                                stream=self.stream)

    def replay(self, events=None):
        """Replay the step on its own stream (the stream the graphs were captured on).
        ``events``: len(stages) + 1 CUDA events, recorded before each stage and after
        the last (elapsed times between neighbours: build, forward, adjoint)."""
        with torch.cuda.stream(self.stream):
            for i, g in enumerate(self.graphs):
                if events is not None:
                    events[i].record(self.stream)
                g.replay()
            if events is not None:
                events[len(self.graphs)].record(self.stream)
