"""The one exchange of a view-sharded multi-GPU step: a sum of the gradients.

Rays and cameras are independent given the scene, so each rank renders and
differentiates its own views against a replica of the parameters (each rank
rebuilds its own BVH).  What ranks must share is the gradient of the loss over
all views: the five gradient tensors (236 B per Gaussian) summed over ranks.
``CapturedStep`` keeps them as views of one flat buffer, so the exchange is a
single all-reduce (NCCL on GPUs, gloo on the host).
"""
from __future__ import annotations

import torch


def allreduce_gradients(flat: torch.Tensor, world: int, group=None) -> torch.Tensor:
    """Sum `flat` (all five gradient tensors, contiguous) over the ranks in place."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return flat


def flat_views(tensors, device, dtype=torch.float32):
    """One zeroed flat buffer and views of it shaped like `tensors`."""
    flat = torch.zeros(sum(t.numel() for t in tensors), dtype=dtype, device=device)
    views, off = [], 0
    for t in tensors:
        views.append(flat[off:off + t.numel()].view(t.shape))
        off += t.numel()
    return flat, views
