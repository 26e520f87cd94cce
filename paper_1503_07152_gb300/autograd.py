"""torch.autograd.Function over the factored HODLR apply and its hand-written
adjoint (both CUDA kernels of libhm.so)."""
from __future__ import annotations

import torch

from . import _lib


class HodlrApply(torch.autograd.Function):
    """y = H x for H given by factors U, V (L x N x k, level-major, column-major
    per level), D (leaves x nmax x nmax, column-major per leaf) on ``tree``.
    Gradients flow to x, U, V and D through hm_hodlr_factored_adjoint."""

    @staticmethod
    def forward(ctx, x, U, V, D, tree, k):
        for t in (x, U, V, D):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("x, U, V, D must be contiguous float32 CUDA tensors")
        y = torch.empty_like(x)
        _lib.hm_hodlr_factored_apply(tree, k, U, V, D, x, y)
        ctx.save_for_backward(x, U, V, D)
        ctx.tree, ctx.k = tree, k
        return y

    @staticmethod
    def backward(ctx, g):
        x, U, V, D = ctx.saved_tensors
        g = g.contiguous()
        need = ctx.needs_input_grad
        gx = torch.empty_like(x) if need[0] else None
        gU = torch.empty_like(U) if need[1] else None
        gV = torch.empty_like(V) if need[2] else None
        gD = torch.empty_like(D) if need[3] else None
        _lib.hm_hodlr_factored_adjoint(ctx.tree, ctx.k, U, V, D, x, g, 1.0, gx, gU, gV, gD)
        return gx, gU, gV, gD, None, None
