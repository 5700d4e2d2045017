"""The H^2 product as a differentiable torch operation in x.

For P = Q with a symmetric kernel the represented matrix is symmetric (the
symmetric shortcut V_B = U_B of Sec. 5 makes the H^2 matrix itself symmetric),
so dL/dx = A^T dL/dy = A dL/dy is one more product with the same handle.
Derivatives in the points or the kernel parameters are not provided.
"""
from __future__ import annotations

from . import nnca


def _function():
    import torch

    class H2Product(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, h, precision):
            ctx.h = h
            ctx.precision = precision
            return h.matvec(x.detach(), precision)

        @staticmethod
        def backward(ctx, g):
            return ctx.h.matvec(g.contiguous(), ctx.precision), None, None

    return H2Product


_FN = None


def h2_matvec(h: "nnca.H2", x, precision: int = nnca.PREC_FP64):
    """y = A x with autograd support in x (x: CUDA tensor (n,) or (nrhs, n))."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(x, h, precision)
