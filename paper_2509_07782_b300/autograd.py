"""torch.autograd.Function around the CUDA forward march and its adjoint.

``render(scene, cams, opts, means, scales, quats, densities, sh, sg=None)``
rebuilds the BVH (the paper rebuilds it at every optimisation step, Sec. 3.2),
renders every camera in one persistent launch and returns RGBA [R, 4].  Its
backward calls ``rgx_render_backward`` (``rgx_render_backward_ex`` when the
Gaussians carry spherical-Gaussian lobes ``sg`` [n, n_sg, 7]) and returns the
gradients of the parameter tensors.
"""
from __future__ import annotations

import torch

from . import rgx


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, densities, sh, sg, scene: rgx.Scene, cams: rgx.Cameras, opts):
        tensors = [x.detach().contiguous().float() for x in (means, scales, quats, densities, sh)]
        sg_t = sg.detach().contiguous().float() if sg is not None else None
        sh_degree = int(round(tensors[4].shape[1] ** 0.5)) - 1
        scene.build(*tensors, opts, sh_degree=sh_degree, sg=sg_t)
        rgba, state = scene.forward(cams, opts, want_state=True)
        ctx.scene, ctx.cams, ctx.opts = scene, cams, opts
        ctx.shapes = [t.shape for t in tensors]
        ctx.sg_shape = sg_t.shape if sg_t is not None else None
        ctx.save_for_backward(state)
        return rgba

    @staticmethod
    def backward(ctx, d_rgba):
        (state,) = ctx.saved_tensors
        dev = state.device
        grads = [torch.zeros(s, dtype=torch.float32, device=dev) for s in ctx.shapes]
        d_sg = None
        if ctx.sg_shape is not None:
            d_sg = torch.zeros(ctx.sg_shape, dtype=torch.float32, device=dev)
            ctx.scene.backward_ex(ctx.cams, ctx.opts, state, d_rgba.contiguous().float(), grads, d_sg=d_sg)
        else:
            ctx.scene.backward(ctx.cams, ctx.opts, state, d_rgba.contiguous().float(), grads)
        return (*grads, d_sg, None, None, None)


def render(scene: rgx.Scene, cams: rgx.Cameras, opts, means, scales, quats, densities, sh, sg=None):
    return RenderFunction.apply(means, scales, quats, densities, sh, sg, scene, cams, opts)
