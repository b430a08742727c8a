"""Whole-volume parity at the headline configuration: order 128, batch 64,
CT-like phantoms, FP32 storage, each dtype with the schedule the library's
autotuner picks (as bench.py times it).

Two whole volumes of the batch (2,097,152 points each) are compared element
by element with the oracle's FP64 exchanged-sum form of Def. 2 (itself
pinned against the row-by-row definition at this order in
tests/test_oracle_pins.py).  Bars: relative L2 over the volume 1e-6 for the
tensor-core dtypes and 1e-5 for the plain FP32 form; per element the error
is bounded by a fraction of the RMS of the volume plus the RMS of the
output's own pencil along the slow axis (the last DFT pass sums that
pencil, so its FP32 rounding is absolute at the pencil's scale: CT-like
phantoms put a large share of the energy into the pencils through the
low frequencies), plus 1e-6 of the entry itself.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N, BATCH = 128, 64
CHECKED = (0, 37)
REL = {"r32_bf16x3": 1e-6, "r32_tf32x3": 1e-6, "r32": 1e-5}
ELEM = {"r32_bf16x3": 5e-6, "r32_tf32x3": 5e-6, "r32": 1e-5}


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def headline():
    """The batch on the device (checked volumes from the seeded host
    generator, the rest device noise of the same scale) and the oracle's
    values of the checked volumes."""
    gen = torch.Generator(device=DEV)
    gen.manual_seed(2024)
    x = torch.rand(BATCH * N ** 3, generator=gen, device=DEV, dtype=torch.float32)
    host = {}
    for v in CHECKED:
        vol = inputs.phantom(N, 1, seed=500 + v)[0].astype(np.float32)
        host[v] = vol
        x[v * N ** 3:(v + 1) * N ** 3] = torch.from_numpy(vol.reshape(-1)).to(DEV)
    ref = {v: oracle.forward_sum_fft(host[v].astype(np.float64), N) for v in CHECKED}
    return x, host, ref


def _check_volume(got, ref, rel_bar, elem_bar, what):
    got = got.reshape(N, N, N)
    ref = ref.reshape(N, N, N)
    err = np.abs(got - ref)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    pencil = np.sqrt(np.mean(np.abs(ref) ** 2, axis=0, keepdims=True))   # slow-axis pencils
    r = _rel(got, ref)
    assert r < rel_bar, (what, "rel L2", r)
    ratio = err / (elem_bar * (rms + pencil) + 1e-6 * np.abs(ref))
    at = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    worst = float(ratio[at])
    assert worst <= 1.0, (what, "per element", worst, "rel L2", r, "max err / rms", float(err.max() / rms),
                          "at", tuple(int(v) for v in at), "|ref| / rms", float(np.abs(ref[at]) / rms),
                          "pencil rms / rms", float(pencil[(0,) + at[1:]] / rms))
    return r


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3", "r32"])
def test_headline_forward_whole_volumes(headline, dtype):
    x, host, ref = headline
    with binding.Plan(N, BATCH, dtype) as p:
        y = torch.empty(BATCH * N ** 3, dtype=torch.complex64, device=DEV)
        p.autotune(x, y)
        y = p.forward(x, out=y)
        p.check()
        for v in CHECKED:
            got = y[v * N ** 3:(v + 1) * N ** 3].cpu().numpy().reshape(N, N, N)
            _check_volume(got.astype(np.complex128), ref[v], REL[dtype], ELEM[dtype], (dtype, v))


def test_headline_packed_forward_whole_volumes(headline):
    """The Hermitian-packed output of the headline form: n^3 reals per volume,
    against the oracle's packing of its own values."""
    x, host, ref = headline
    with binding.Plan(N, BATCH, "r32_bf16x3") as p:
        pk = p.forward_packed(x)
        p.check()
        for v in CHECKED:
            got = pk[v * N ** 3:(v + 1) * N ** 3].cpu().numpy().astype(np.float64)
            want = oracle.pack_hermitian(ref[v].reshape(-1), N)[0]
            _check_volume(got, want, 1e-6, 5e-6, ("packed", v))


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3"])
def test_headline_inverse_and_adjoint_whole_volumes(headline, dtype):
    """Inverse: the residual ||D x^ - y|| / ||y|| of the returned volumes,
    with D x^ from the oracle in FP64 (the exact inverse has residual 0), and
    the distance to the original phantom.  Adjoint: Re(D^H g) against the
    oracle for a seeded complex g."""
    x, host, ref = headline
    y = torch.empty(BATCH * N ** 3, dtype=torch.complex64, device=DEV)
    gen = torch.Generator(device=DEV)
    gen.manual_seed(77)
    y.real.copy_(torch.randn(BATCH * N ** 3, generator=gen, device=DEV))
    y.imag.copy_(torch.randn(BATCH * N ** 3, generator=gen, device=DEV))
    g = y.clone()
    gh = {}
    for i, v in enumerate(CHECKED):
        y[v * N ** 3:(v + 1) * N ** 3] = torch.from_numpy(ref[v].reshape(-1).astype(np.complex64)).to(DEV)
        rng = np.random.default_rng(900 + i)
        gv = (rng.standard_normal(N ** 3) + 1j * rng.standard_normal(N ** 3)).astype(np.complex64)
        gh[v] = gv
        g[v * N ** 3:(v + 1) * N ** 3] = torch.from_numpy(gv).to(DEV)
    with binding.Plan(N, BATCH, dtype) as p:
        xi = p.inverse(y)
        ad = p.adjoint(g)
        p.check()
        for v in CHECKED:
            xv = xi[v * N ** 3:(v + 1) * N ** 3].cpu().numpy().astype(np.float64).reshape(N, N, N)
            y32 = ref[v].astype(np.complex64).astype(np.complex128)
            res = _rel(oracle.forward_sum_fft(xv, N), y32)
            assert res < REL[dtype], (dtype, v, "inverse residual", res)
            assert _rel(xv, host[v].astype(np.float64)) < 4e-6, (dtype, v)
            av = ad[v * N ** 3:(v + 1) * N ** 3].cpu().numpy().astype(np.float64)
            aref = oracle.adjoint_sum_fft(gh[v].astype(np.complex128).reshape(N, N, N), N).real.reshape(-1)
            _check_volume(av, aref, REL[dtype], ELEM[dtype], (dtype, v, "adjoint"))


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32"])
def test_order_96_whole_volumes(dtype):
    """Order 96 (the gradient-descent configuration's order and the top of the
    ragged range; register-radix shape 24 x 4): two whole volumes of a batch
    of 8 phantoms against the oracle, forward, and the inverse residual."""
    n, batch = 96, 8
    vols = {v: inputs.phantom(n, 1, seed=700 + v)[0].astype(np.float32) for v in (0, 5)}
    gen = torch.Generator(device=DEV)
    gen.manual_seed(96)
    x = torch.rand(batch * n ** 3, generator=gen, device=DEV, dtype=torch.float32)
    for v, vol in vols.items():
        x[v * n ** 3:(v + 1) * n ** 3] = torch.from_numpy(vol.reshape(-1)).to(DEV)
    with binding.Plan(n, batch, dtype) as p:
        y = p.forward(x)
        xi = p.inverse(y)
        p.check()
        for v, vol in vols.items():
            ref = oracle.forward_sum_fft(vol.astype(np.float64), n)
            got = y[v * n ** 3:(v + 1) * n ** 3].cpu().numpy().astype(np.complex128)
            assert _rel(got, ref.reshape(-1)) < REL[dtype], (dtype, v)
            back = xi[v * n ** 3:(v + 1) * n ** 3].cpu().numpy().astype(np.float64)
            assert _rel(back, vol.reshape(-1).astype(np.float64)) < 4 * REL["r32"], (dtype, v)
