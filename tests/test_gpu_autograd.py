"""Differentiation through the C ABI: the backward pass is the adjoint."""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_10058_gb300 import binding, inputs
from paper_1807_10058_gb300.autograd import fcc_dct, fcc_dct_adjoint

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("dtype,n", [("r64", 4), ("c64", 3), ("r64", 8)])
def test_gradcheck_fp64(dtype, n):
    real = dtype == "r64"
    with binding.Plan(n, 2, dtype) as p:
        t = torch.float64 if real else torch.complex128
        x = torch.randn(2 * n ** 3, dtype=t, device=DEV, requires_grad=True)
        assert torch.autograd.gradcheck(lambda v: fcc_dct(v, p), (x,), eps=1e-6, atol=1e-7, rtol=1e-7)


@pytest.mark.parametrize("dtype,n", [("r64", 4), ("c64", 3)])
def test_adjoint_gradcheck_and_second_order(dtype, n):
    """The adjoint as a differentiable function (its backward is the forward),
    and second derivatives through both: gradgradcheck runs the backward of
    each backward in the library's kernels."""
    real = dtype == "r64"
    with binding.Plan(n, 2, dtype) as p:
        t = torch.float64 if real else torch.complex128
        g = torch.randn(2 * n ** 3, dtype=torch.complex128, device=DEV, requires_grad=True)
        assert torch.autograd.gradcheck(lambda v: fcc_dct_adjoint(v, p), (g,), eps=1e-6, atol=1e-7, rtol=1e-7)
        x = torch.randn(2 * n ** 3, dtype=t, device=DEV, requires_grad=True)
        assert torch.autograd.gradgradcheck(lambda v: fcc_dct(v, p), (x,), eps=1e-6, atol=1e-7, rtol=1e-7)
        assert torch.autograd.gradgradcheck(lambda v: fcc_dct_adjoint(v, p), (g,), eps=1e-6, atol=1e-7, rtol=1e-7)


def test_hessian_vector_product_of_a_reconstruction_loss():
    """L = ||D x - b||^2 has Hessian 2 Re(D^H D) (real x): the double-backward
    product H v equals 2 Re(D^H (D v)) from the oracle's dense matrix."""
    n, batch = 6, 2
    rng = np.random.default_rng(11)
    x0 = rng.standard_normal(batch * n ** 3)
    v = rng.standard_normal(batch * n ** 3)
    b = oracle.forward_dense(rng.standard_normal((batch, n, n, n)), n).reshape(-1)
    with binding.Plan(n, batch, "r64") as p:
        x = torch.from_numpy(x0).to(DEV).requires_grad_(True)
        bt = torch.from_numpy(b).to(DEV)
        L = torch.sum(torch.abs(fcc_dct(x, p) - bt) ** 2)
        (gx,) = torch.autograd.grad(L, x, create_graph=True)
        (hv,) = torch.autograd.grad(gx, x, grad_outputs=torch.from_numpy(v).to(DEV))
    Dv = oracle.forward_dense(v.reshape(batch, n, n, n), n)
    ref = 2 * oracle.adjoint_dense(Dv, n).real.reshape(-1)
    got = hv.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_masked_reconstruction_gradient_matches_oracle():
    """L = ||M . (D x) - b||^2, grad = 2 Re D^H (M . (M . D x - b))."""
    n, batch = 8, 2
    x0 = inputs.phantom(n, batch, seed=3)
    xt = inputs.phantom(n, batch, seed=9)
    M = inputs.bernoulli_mask(n, batch, seed=4, p=0.1).astype(np.float64)
    b = M * oracle.forward_dense(xt, n)
    with binding.Plan(n, batch, "r64") as p:
        x = torch.from_numpy(x0.reshape(-1)).to(DEV).requires_grad_(True)
        Mt = torch.from_numpy(M.reshape(-1)).to(DEV)
        bt = torch.from_numpy(b.reshape(-1)).to(DEV)
        L = torch.sum(torch.abs(Mt * fcc_dct(x, p) - bt) ** 2)
        L.backward()
        g = x.grad.cpu().numpy().reshape(x0.shape)
    r = M * (M * oracle.forward_dense(x0, n) - b)
    ref = 2 * oracle.adjoint_dense(r, n).real
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("dtype", ["r32", "r32_bf16x3", "r32_tf32x3"])
def test_adjoint_dot_product_fp32_large(dtype):
    """<D x, g> = <x, Re D^H g>, the difference measured against the
    Cauchy-Schwarz scale ||g|| ||D x|| (the inner product itself may cancel);
    the tensor-core forms run both the forward and the adjoint on tcgen05."""
    n, batch = 64, 2
    gen = torch.Generator(device=DEV)
    gen.manual_seed(12)
    with binding.Plan(n, batch, dtype) as p:
        x = torch.randn(batch * n ** 3, device=DEV, generator=gen)
        g = torch.randn(batch * n ** 3, device=DEV, dtype=torch.complex64, generator=gen)
        y = p.forward(x)
        lhs = torch.sum((torch.conj(g).to(torch.complex128) * y.to(torch.complex128)).real)
        rhs = torch.sum(x.double() * p.adjoint(g).double())
        scale = torch.linalg.vector_norm(g.to(torch.complex128)) * torch.linalg.vector_norm(y.to(torch.complex128))
        assert abs(lhs - rhs) / scale < 1e-6
