"""The H^2 product as a differentiable torch operation.

For P = Q with a symmetric kernel the represented matrix is symmetric (the
symmetric shortcut V_B = U_B of Sec. 5 makes the H^2 matrix itself symmetric),
so dL/dx = A^T dL/dy = A dL/dy is one more product with the same handle.

The derivatives in the points and in the kernel parameter h (kparam[1], the
Gaussian's bandwidth) are taken with the pivots held fixed: every index set of
the build (tree, lists, pivots) stays, and A~ moves through its kernel entries
and its bases (Sec. 2.3.1, Eqs. 11 and 14). They come from the library's adjoint
kernels (nnca_gradient), in FP64.
"""
from __future__ import annotations

from . import nnca


def _function():
    import torch

    class H2Product(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, points, bandwidth, h, precision):
            ctx.h = h
            ctx.precision = precision
            ctx.save_for_backward(x)
            ctx.want = (points is not None and points.requires_grad,
                        bandwidth is not None and bandwidth.requires_grad)
            ctx.pshape = None if points is None else points.shape
            return h.matvec(x.detach(), precision)

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            g = g.contiguous()
            dx = ctx.h.matvec(g, ctx.precision)
            dp = dh = None
            if any(ctx.want):
                n = ctx.h.n
                xd = x.detach().to(torch.float64).contiguous()
                gd = g.to(torch.float64).contiguous()
                nrhs = 1 if xd.dim() == 1 else xd.shape[0]
                gp = torch.empty(ctx.pshape, dtype=torch.float64, device=x.device)
                gh = torch.zeros(1, dtype=torch.float64, device=x.device)
                nnca.nnca_gradient(ctx.h.handle, xd, gd, nrhs, n, gp, gh)
                dp = gp if ctx.want[0] else None
                dh = gh.reshape(()) if ctx.want[1] else None
            return dx, dp, dh, None, None

    return H2Product


_FN = None


def h2_matvec(h: "nnca.H2", x, precision: int = nnca.PREC_FP64, points=None, bandwidth=None):
    """y = A~ x with autograd support in x (x: CUDA tensor (n,) or (nrhs, n)), and,
    with the pivots held fixed, in `points` (the (n, d) FP64 CUDA tensor the handle
    was built from) and `bandwidth` (a 0-d FP64 tensor equal to kparam[1]) when
    they are given with requires_grad."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(x, points, bandwidth, h, precision)
