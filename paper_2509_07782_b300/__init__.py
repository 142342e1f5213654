"""B300-native differentiable volume ray marching through elliptical Gaussians.

The compute path is the C-ABI library ``librgx.so`` (hand-written sm_103a CUDA,
``csrc/``); ``rgx`` is its thin ctypes binding and ``autograd`` wraps it in a
``torch.autograd.Function``.  ``synth`` draws seeded synthetic scenes.
"""
__all__ = ["rgx", "autograd", "synth"]
