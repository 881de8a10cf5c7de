"""torch.autograd.Function over the BOS render and its hand-written adjoint.

    ctx = bos.Context(0); ctx.set_geometry(...)
    I = render(T, ctx, grid)          # forward: bos_set_grid + bos_render(save_for_backward=1)
    loss = ((target - I) ** 2).sum()
    loss.backward()                   # backward: bos_backward -> T.grad

Both directions run in the CUDA library; PyTorch only owns the tensors and the stream.
"""
from __future__ import annotations

import torch

from . import bos


class BOSRender(torch.autograd.Function):
    @staticmethod
    def forward(fctx, T, ctx: "bos.Context", grid, prec: int):
        T = T.detach().contiguous()
        ctx.set_grid(grid, T, prec)
        I, _, _ = ctx.render(disp=False, save_for_backward=True)
        fctx.bos = ctx
        fctx.T = T                      # the adjoint's chain rule reads T
        return I

    @staticmethod
    def backward(fctx, gI):
        dT = fctx.bos.backward(gI.contiguous().to(torch.float32))
        return dT, None, None, None


def render(T, ctx: "bos.Context", grid, prec: int = bos.BOS_PREC_FP32_COMP):
    """Differentiable I_flow(T) for the geometry already set on `ctx`."""
    return BOSRender.apply(T, ctx, grid, prec)
