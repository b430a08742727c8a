"""The paper's radix-2x2x2 recursion (Sec. 4.B, eq. FastAlgorithm) on the GPU
(fcc_dct_plan_radix2): FP64 evaluation against the dense matrix of Def. 2 and
against the oracle's own FP64 recursion; the FP32 form's error grows with the
order (the instability that keeps the recursion off the fast path); the
non-zeros of the derived basis change B_n agree with the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from oracle import radix2 as oracle_radix2
from paper_1807_10058_gb300 import binding

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SKEWS = [((1, 0, 3), 8), ((1, 0, 11), 16)]


def _run(n, batch, dtype, skew, x):
    with binding.Plan(n, batch, dtype, skew=skew, radix2=True) as p:
        xd = torch.from_numpy(x.reshape(-1).astype(np.complex128 if dtype == "c64" else np.complex64)).to(DEV)
        y = p.forward(xd)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.complex128).reshape(x.shape), p


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("skew", SKEWS)
@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_radix2_fp64_matches_dense_definition(n, skew):
    rng = np.random.default_rng(n)
    batch = 3
    x = rng.standard_normal((batch, n ** 3)) + 1j * rng.standard_normal((batch, n ** 3))
    y, _ = _run(n, batch, "c64", skew, x)
    ref = x @ oracle.dct_matrix(n, skew).T
    assert _rel(y, ref) < 1e-11, _rel(y, ref)


def test_radix2_fp64_matches_the_oracles_recursion():
    n, skew = 8, SKEWS[0]
    x = np.random.default_rng(3).standard_normal((2, n ** 3)) + 0j
    y, _ = _run(n, 2, "c64", skew, x)
    assert _rel(y, oracle_radix2.forward_radix2(x, n, skew)) < 1e-12


def test_radix2_fp32_error_grows_with_the_order():
    """The recursion rounded in FP32 (B_n, DCT_2 and every product in FP32):
    the error against the FP64 dense matrix grows from level to level,
    unlike the F S form (~1e-7 at every order)."""
    err = {}
    for n in (4, 8, 16):
        x = np.random.default_rng(10 + n).standard_normal((2, n ** 3)) + 0j
        y, _ = _run(n, 2, "c32", SKEWS[0], x)
        err[n] = _rel(y, x @ oracle.dct_matrix(n).T)
    assert err[4] < 1e-5 and err[16] < 1e-2, err
    assert err[16] > 3 * err[4], err


def test_radix2_basis_change_statistics_match_the_oracle():
    for n in (4, 8):
        with binding.Plan(n, 1, "c64", radix2=True) as p:
            nz, mx, shifts = p.radix2_stats(n)
            assert shifts == 1
            B = oracle_radix2.basis_change(n)
            assert abs(nz - oracle_radix2.nonzeros_per_row(B)) < 1e-9, (n, nz)
            assert abs(mx - np.abs(B).max()) < 1e-9 * mx
            assert abs(p.radix2_stats(0) * n ** 3 - oracle_radix2.recursion_macs(n)) < 1e-6
    with binding.Plan(16, 1, "c64", radix2=True) as p:
        nz16, _, _ = p.radix2_stats(16)
        assert nz16 > 6   # not O(1): the rows of B_n fill up with the order
        assert p.radix2_stats(8)[2] == 8 and p.radix2_stats(4)[2] == 64


def test_radix2_plan_serves_the_forward_only():
    n = 4
    L = binding.lib()
    with binding.Plan(n, 2, "c64", radix2=True) as p:
        y = torch.zeros(2 * n ** 3, dtype=torch.complex128, device=DEV)
        with pytest.raises(binding.FccError) as e:
            p.inverse(y)
        assert e.value.status == binding.FCC_ERR_UNSUPPORTED
        with pytest.raises(binding.FccError) as e:
            p.adjoint(y)
        assert e.value.status == binding.FCC_ERR_UNSUPPORTED
        assert p.launches(0) == 3 + 8 and p.launches(1) == 0
