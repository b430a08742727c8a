"""torch.autograd wrappers of the forward transform and its adjoint.

y = DCT_n x is linear, so its vector-Jacobian product is the adjoint: for a
real loss L and PyTorch's complex-gradient convention g = dL/dRe(y) +
i dL/dIm(y), the gradient is D^H g for complex x and Re(D^H g) for real x --
exactly what fcc_dct_adjoint returns for the plan's dtype.  The adjoint is
linear too, and its vector-Jacobian product is the forward: for
r = Re(D^H g) (real plans) and an upstream real gradient h, dL/dRe(g) +
i dL/dIm(g) = D h; for complex plans (D^H)^H = D.  Each backward calls the
other Function, so derivatives of any order (Hessian-vector products of a
reconstruction loss, gradgradcheck) stay in the library's CUDA kernels.
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
        return FccDctAdjoint.apply(g.contiguous(), ctx.plan), None


class FccDctAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, plan):
        ctx.plan = plan
        return plan.adjoint(g.contiguous())

    @staticmethod
    def backward(ctx, h):
        return FccDct.apply(h.contiguous(), ctx.plan), None


def fcc_dct(x, plan):
    """Differentiable y = DCT_n x for a flat tensor x of plan.points values."""
    return FccDct.apply(x, plan)


def fcc_dct_adjoint(g, plan):
    """Differentiable D^H g (real plans: Re D^H g) for a flat complex tensor g."""
    return FccDctAdjoint.apply(g, plan)


__all__ = ["FccDct", "FccDctAdjoint", "fcc_dct", "fcc_dct_adjoint", "binding"]
