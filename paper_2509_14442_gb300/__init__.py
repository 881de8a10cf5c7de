"""GB300 (sm_103a) implementation of the differentiable BOS forward model of
single-view physics-informed BOS tomography (arxiv 2509.14442).

- ``bos``: ctypes binding of the C ABI (include/bos.h) of the CUDA library.
- ``torch_ops``: ``torch.autograd.Function`` over render / backward.
- ``scenes``: seeded synthetic scenes (inputs only).
"""
__all__ = ["bos", "scenes"]
