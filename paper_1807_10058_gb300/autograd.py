"""torch.autograd wrapper of the forward transform.

y = DCT_n x is linear, so its vector-Jacobian product is the adjoint: for a
real loss L and PyTorch's complex-gradient convention g = dL/dRe(y) +
i dL/dIm(y), the gradient is D^H g for complex x and Re(D^H g) for real x --
exactly what fcc_dct_adjoint returns for the plan's dtype.  Both directions
run in the library's CUDA kernels.
"""
import torch

from . import binding


class FccDct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint(g.contiguous()), None


def fcc_dct(x, plan):
    """Differentiable y = DCT_n x for a flat tensor x of plan.points values."""
    return FccDct.apply(x, plan)


__all__ = ["FccDct", "fcc_dct", "binding"]
