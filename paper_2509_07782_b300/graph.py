"""One training step -- BVH rebuild, forward march, adjoint -- captured in a CUDA graph.

The step works on persistent tensors: the caller updates the five parameter
tensors (and, if it wants, the upstream gradient) in place between replays and
reads ``rgba`` / ``grads`` after each replay.  Capture happens after one eager
warm-up step, which grows the scene's workspace and caches every launch
configuration, so the captured calls allocate nothing and make no attribute
queries.  Cameras are copied from their pinned host buffer at every replay, so
their contents (not their number or sizes) may change between replays.
"""
from __future__ import annotations

import torch

from . import rgx


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
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.stream = torch.cuda.Stream(device=dev)
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

    def _body(self):
        s = self.stream
        h = self.scene.h
        rgx.rgx_build_bvh(h, *self.params, self.sh_degree, self.opts, stream=s)
        rgx.rgx_render_forward(h, self.cams, self.opts, self.rgba, self.state, stream=s)
        if self.backward:
            for g in self.grads:
                g.zero_()
            rgx.rgx_render_backward(h, self.cams, self.opts, self.state, self.d_rgba, *self.grads, stream=s)

    def replay(self):
        """Replay on the step's own stream (the stream the graph was captured on)."""
        with torch.cuda.stream(self.stream):
            self.graph.replay()
