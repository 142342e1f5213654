"""torch.autograd.Function around the CUDA forward march and its adjoint.

``render(scene, cams, opts, means, scales, quats, densities, sh)`` rebuilds the
BVH (the paper rebuilds it at every optimisation step, Sec. 3.2), renders every
camera in one persistent launch and returns RGBA [R, 4].  Its backward calls
``rgx_render_backward`` and returns gradients for the five parameter tensors.
"""
from __future__ import annotations

import torch

from . import rgx


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, densities, sh, scene: rgx.Scene, cams: rgx.Cameras, opts):
        tensors = [x.detach().contiguous().float() for x in (means, scales, quats, densities, sh)]
        sh_degree = int(round(tensors[4].shape[1] ** 0.5)) - 1
        scene.build(*tensors, opts, sh_degree=sh_degree)
        rgba, state = scene.forward(cams, opts, want_state=True)
        ctx.scene, ctx.cams, ctx.opts = scene, cams, opts
        ctx.shapes = [t.shape for t in tensors]
        ctx.save_for_backward(state)
        return rgba

    @staticmethod
    def backward(ctx, d_rgba):
        (state,) = ctx.saved_tensors
        dev = state.device
        grads = [torch.zeros(s, dtype=torch.float32, device=dev) for s in ctx.shapes]
        ctx.scene.backward(ctx.cams, ctx.opts, state, d_rgba.contiguous().float(), grads)
        return (*grads, None, None, None)


def render(scene: rgx.Scene, cams: rgx.Cameras, opts, means, scales, quats, densities, sh):
    return RenderFunction.apply(means, scales, quats, densities, sh, scene, cams, opts)
