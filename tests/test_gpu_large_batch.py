"""Batches past the 65,535-block limit of a launch's grid.y.

Every pass launches one grid row per volume (or per pair of real volumes),
so a chunk of more than 65,535 of them is split into several launches.  At
orders 2 and 4 a chunk holds hundreds of thousands of volumes: order 2 with
140,001 volumes is one chunk of 70,000 pairs plus the odd volume left over;
order 4 with 131,075 volumes and 64 MB chunks is a chunk of 65,536 pairs (one
more than a launch takes) and a chunk of one pair and one single volume.
Checked against the oracle's dense matrix (Def. 2, Sec. 4.A) on every volume.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = {"r64": 1e-12, "c64": 1e-12, "r32": 1e-5, "c32": 1e-5, "r32_bf16x3": 1e-6}
INV_TOL = {"r64": 4e-12, "c64": 4e-12, "r32": 4e-5, "c32": 4e-5, "r32_bf16x3": 4e-5}   # the inverse's bars elsewhere
CASES = [(2, 140001, 0), (4, 131075, 64)]


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def worst_volume(a, b, n):
    """Largest per-volume relative error (a split launch that skipped or
    repeated volumes shows up here even when the batch-wide norm hides it)."""
    a = np.asarray(a).reshape(-1, n ** 3)
    b = np.asarray(b).reshape(-1, n ** 3)
    num = np.linalg.norm(a - b, axis=1)
    den = np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    return float((num / den).max())


def recorded_launches(p, call):
    """Kernel launches of one call as the plan's per-launch timer records them."""
    p.profile(True)
    call()
    torch.cuda.synchronize()
    rec = p.profile_read()
    p.profile(False)
    return sum(c for _, c in rec.values())


@pytest.mark.parametrize("dtype", ["r32", "c32", "r64", "c64", "r32_bf16x3"])
@pytest.mark.parametrize("n,batch,chunk_mb", CASES)
def test_batch_beyond_grid_limit(dtype, n, batch, chunk_mb):
    complex_in = dtype.startswith("c")
    fp64 = dtype in ("r64", "c64")
    rt, ct = (np.float64, np.complex128) if fp64 else (np.float32, np.complex64)
    x = inputs.uniform(n, batch, seed=n, complex_=complex_in).astype(ct if complex_in else rt)
    y_ref = oracle.forward_dense(x.astype(np.complex128), n)
    g = inputs.uniform(n, batch, seed=50 + n, complex_=True).astype(ct)
    a_ref = oracle.adjoint_dense(g.astype(np.complex128), n)
    if not complex_in:
        a_ref = a_ref.real
    with binding.Plan(n, batch, dtype) as p:
        if chunk_mb:
            p.set_schedule(chunk_mb=chunk_mb)
        xd = torch.from_numpy(x.reshape(-1)).to(DEV)
        yd = torch.from_numpy(y_ref.astype(ct).reshape(-1)).to(DEV)
        gd = torch.from_numpy(g.reshape(-1)).to(DEV)
        y = p.forward(xd).cpu().numpy()
        xi = p.inverse(yd).cpu().numpy()
        a = p.adjoint(gd).cpu().numpy()
        p.check()
        # the launch counts the library reports include the split launches
        for which, call in ((0, lambda: p.forward(xd)), (1, lambda: p.inverse(yd)), (2, lambda: p.adjoint(gd))):
            assert recorded_launches(p, call) == p.launches(which), (which, p.launches(which))
    tol = TOL[dtype]
    assert worst_volume(y, y_ref, n) < 10 * tol and rel(y, y_ref) < tol, (worst_volume(y, y_ref, n), rel(y, y_ref))
    itol = INV_TOL[dtype]
    assert worst_volume(xi, x, n) < 10 * itol and rel(xi, x) < itol, (worst_volume(xi, x, n), rel(xi, x))
    assert worst_volume(a, a_ref, n) < 10 * tol and rel(a, a_ref) < tol, (worst_volume(a, a_ref, n), rel(a, a_ref))


@pytest.mark.parametrize("n,batch,chunk_mb", CASES)
def test_packed_batch_beyond_grid_limit(n, batch, chunk_mb):
    """The Hermitian-packed forward and inverse of the same batches (pairs of
    real volumes; the odd volume goes through the single-volume branch)."""
    x = inputs.uniform(n, batch, seed=7 + n).astype(np.float32)
    y_ref = oracle.forward_dense(x.astype(np.complex128), n)
    pk_ref = oracle.pack_hermitian(y_ref, n)
    with binding.Plan(n, batch, "r32") as p:
        if chunk_mb:
            p.set_schedule(chunk_mb=chunk_mb)
        xd = torch.from_numpy(x.reshape(-1)).to(DEV)
        pd = torch.from_numpy(pk_ref.astype(np.float32).reshape(-1)).to(DEV)
        pk = p.forward_packed(xd).cpu().numpy()
        xi = p.inverse_packed(pd).cpu().numpy()
        p.check()
        for which, call in ((3, lambda: p.forward_packed(xd)), (4, lambda: p.inverse_packed(pd))):
            assert recorded_launches(p, call) == p.launches(which), (which, p.launches(which))
    assert worst_volume(pk, pk_ref, n) < 1e-4 and rel(pk, pk_ref) < 1e-5, (worst_volume(pk, pk_ref, n), rel(pk, pk_ref))
    assert worst_volume(xi, x, n) < 4e-4 and rel(xi, x) < 4e-5, (worst_volume(xi, x, n), rel(xi, x))
