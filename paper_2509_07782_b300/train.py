"""One training iteration of the method through the C-ABI (Sec. 3.4, 3.5, 4.2).

``Trainer.step()``: rebuild the BVH from the current parameters, render every view
of the batch in one persistent launch, the image loss (1 - lambda) L1 + lambda DSSIM
against the targets and its gradient, the adjoint (which also accumulates each
camera's densification statistic, Eq. 11), the isotropic loss on the scales
(Eqs. 6-8, lambda_s = 2.5e-4, r0 = 10), and one Adam step per parameter tensor --
scales and densities optimised as logarithms.  ``Trainer.densify()`` applies the
clone / split rule to Gaussians over the threshold tau (1.5e-4, Sec. 4.2) and
resets the statistic.  Every step runs in the library's kernels; this class only
owns the tensors.
"""
from __future__ import annotations

import torch

from . import rgx


class Trainer:
    def __init__(self, params, cams: rgx.Cameras, opts, targets: torch.Tensor, sg=None, lr=None, lam: float = 0.2,
                 lambda_s: float = 2.5e-4, r0: float = 10.0, tau: float = 1.5e-4, size_threshold: float = 0.01,
                 sh_degree: int = 3, device=None):
        means, scales, quats, dens, sh = [p.detach().contiguous().float().clone() for p in params]
        self.dev = means.device if device is None else torch.device(device)
        # the optimiser's variables; scales and densities as logarithms
        self.raw = {"means": means, "log_scales": scales.log(), "quats": quats, "log_dens": dens.log(), "sh": sh}
        if sg is not None:
            self.raw["sg"] = sg.detach().contiguous().float().clone()
        self.act = {"log_scales": scales.clone(), "log_dens": dens.clone()}
        self.lr = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "log_dens": 5e-2, "sh": 2.5e-3, "sg": 2.5e-3}
        if lr:
            self.lr.update(lr)
        self.cams, self.opts, self.targets = cams, opts, targets
        self.lam, self.lambda_s, self.r0, self.tau, self.size_threshold = lam, lambda_s, r0, tau, size_threshold
        self.sh_degree = sh_degree
        self.scene = rgx.Scene(self.dev.index if self.dev.index is not None else torch.cuda.current_device())
        self.t = 0
        self._alloc()

    # ---------------------------------------------------------------------------------
    def _alloc(self):
        n = self.n
        self.m = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.grads = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.stat = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.count = torch.zeros(n, dtype=torch.int32, device=self.dev)
        R = self.cams.n_rays
        self.rgba = torch.empty(R, 4, dtype=torch.float32, device=self.dev)
        self.state = rgx.new_state(R, self.dev)
        self.d_rgba = torch.empty(R, 4, dtype=torch.float32, device=self.dev)
        self.loss = torch.zeros(self.cams.count, dtype=torch.float32, device=self.dev)
        self.iso = torch.zeros(1, dtype=torch.float32, device=self.dev)

    @property
    def n(self) -> int:
        return int(self.raw["means"].shape[0])

    def params(self):
        """The values the renderer takes: (means, scales, quats, densities, sh)."""
        return (self.raw["means"], self.act["log_scales"], self.raw["quats"], self.act["log_dens"], self.raw["sh"])

    # ---------------------------------------------------------------------------------
    def step(self, stream=None):
        """One iteration; returns the device loss tensor [ncam] (image loss per view) and the
        isotropic loss [1] of this step."""
        h, s = self.scene.h, stream
        sg = self.raw.get("sg")
        self.scene.build(*self.params(), self.opts, sh_degree=self.sh_degree, sg=sg, stream=s)
        rgx.rgx_render_forward(h, self.cams, self.opts, self.rgba, self.state, stream=s)
        self.loss.zero_()
        self.iso.zero_()
        rgx.rgx_image_loss(h, self.cams, self.rgba, self.targets, self.lam, self.loss, self.d_rgba, stream=s)
        for g in self.grads.values():
            g.zero_()
        g = self.grads
        rgx.rgx_render_backward_ex(h, self.cams, self.opts, self.state, self.d_rgba, g["means"], g["log_scales"],
                                   g["quats"], g["log_dens"], g["sh"], d_sg=g.get("sg"), stat=self.stat,
                                   count=self.count, stream=s, n=self.n, sh_degree=self.sh_degree,
                                   n_sg=int(sg.shape[1]) if sg is not None else 0)
        rgx.rgx_isotropic_loss(self.act["log_scales"], self.r0, self.lambda_s, self.iso, g["log_scales"], stream=s)
        self.t += 1
        for k in self.raw:
            expo = k in ("log_scales", "log_dens")
            rgx.rgx_adam_step(self.raw[k], g[k], self.m[k], self.v[k], self.lr[k], self.t, exp_param=expo,
                              activated=self.act[k] if expo else None, stream=s)
        return self.loss, self.iso

    def densify(self, generator: torch.Generator | None = None, stream=None) -> int:
        """Clone / split the Gaussians over the threshold; returns the new count.  Split
        children draw their offsets from `generator` (standard normals)."""
        n = self.n
        action = torch.empty(n, dtype=torch.int32, device=self.dev)
        offset = torch.empty(n, dtype=torch.int32, device=self.dev)
        n_out = rgx.rgx_densify_plan(self.scene.h, self.stat, self.count, self.act["log_scales"], self.tau,
                                     self.size_threshold, action, offset, stream=stream)
        normals = torch.randn(n, 2, 3, device=self.dev, generator=generator)
        outs = [torch.empty((n_out,) + tuple(t.shape[1:]), dtype=torch.float32, device=self.dev)
                for t in self.params()]
        sg = self.raw.get("sg")
        out_sg = torch.empty((n_out,) + tuple(sg.shape[1:]), device=self.dev) if sg is not None else None
        src = torch.empty(n_out, dtype=torch.int32, device=self.dev)
        rgx.rgx_densify_apply(action, offset, normals, self.params(), outs, sg=sg, out_sg=out_sg, out_src=src,
                              stream=stream)
        means, scales, quats, dens, sh = outs
        self.raw = {"means": means, "log_scales": scales.log(), "quats": quats, "log_dens": dens.log(), "sh": sh}
        if sg is not None:
            self.raw["sg"] = out_sg
        self.act = {"log_scales": scales, "log_dens": dens}
        self._alloc()
        return n_out
