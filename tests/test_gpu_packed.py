"""Hermitian-packed forward / inverse of real plans through the C ABI.

For a real volume the n^3 complex values y = D x come in conjugate pairs
y[pi(a)] = conj(y[a]); the packed layout keeps n^3 reals (oracle.pack_hermitian
states it, pinned on the CPU in test_oracle_pins).  Expected values are the
oracle's y packed by the oracle; tolerances as for the complex outputs:
FP64 1e-12, FP32 1e-5, tensor-core forms 1e-6 relative L2.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {"r64": 1e-12, "r32": 1e-5, "r32_bf16x3": 1e-6, "r32_tf32x3": 1e-6, "r32_bf16x6": 1e-6}
RT = {"r64": np.float64}


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype).reshape(-1)).to(DEV)


def _oracle_forward(x, n):
    return oracle.forward_dense(x, n) if n <= 8 else oracle.forward_sum_fft(x, n)


@pytest.mark.parametrize("dtype", ["r64", "r32", "r32_bf16x3", "r32_tf32x3"])
@pytest.mark.parametrize("n,batch", [(1, 3), (2, 2), (3, 3), (5, 1), (7, 2), (8, 2), (8, 3), (12, 2), (16, 4),
                                     (24, 3)])
def test_packed_forward_and_inverse_against_oracle(dtype, n, batch):
    if n == 1 and dtype.startswith("r32_"):
        pytest.skip("tensor-core plans start at n = 2")
    rt = RT.get(dtype, np.float32)
    x = inputs.smoothed_noise(n, batch, seed=n) if n > 2 else inputs.uniform(n, batch, seed=n)
    x = x.astype(rt).astype(np.float64)
    y_ref = _oracle_forward(x, n)
    pk_ref = oracle.pack_hermitian(y_ref, n)
    with binding.Plan(n, batch, dtype) as p:
        pk = p.forward_packed(dev(x, rt))
        xi = p.inverse_packed(dev(pk_ref, rt)).cpu().numpy()
        rt_back = p.inverse_packed(pk).cpu().numpy()
        y_c = p.forward(dev(x, rt)).cpu().numpy()
        p.check()
    pk = pk.cpu().numpy()
    assert rel(pk, pk_ref) < TOL[dtype], rel(pk, pk_ref)
    # the packed values are the complex form's values, re-laid out
    assert rel(pk, oracle.pack_hermitian(y_c, n)) < TOL[dtype], rel(pk, oracle.pack_hermitian(y_c, n))
    assert rel(xi, x) < 4 * max(TOL[dtype], 1e-5 if rt == np.float32 else 0), rel(xi, x)
    assert rel(rt_back, x) < 4 * max(TOL[dtype], 1e-5 if rt == np.float32 else 0), rel(rt_back, x)


@pytest.mark.parametrize("dtype", ["r32", "r32_bf16x3"])
@pytest.mark.parametrize("n,batch", [(64, 3), (96, 2), (128, 2)])
def test_packed_full_volumes_and_sampled_rows(dtype, n, batch):
    """Fast paired path (and, at odd batch, the unpaired last volume):
    packed output equals the packed complex output of the same plan, sampled
    rows match the oracle, the packed round trip returns the input."""
    gen = torch.Generator(device=DEV)
    gen.manual_seed(n)
    x = torch.rand(batch * n ** 3, generator=gen, device=DEV, dtype=torch.float32) * 2 - 1
    vol0 = inputs.phantom(n, 1, seed=3)[0].astype(np.float32)
    x[:n ** 3] = torch.from_numpy(vol0.reshape(-1)).to(DEV)
    rng = np.random.default_rng(n)
    with binding.Plan(n, batch, dtype) as p:
        pk = p.forward_packed(x)
        y = p.forward(x)
        back = p.inverse_packed(pk)
        p.check()
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        want = oracle.pack_hermitian(yh, n).reshape(-1)
        got = pk.cpu().numpy()
        # the same FP32 arithmetic up to the order of the split's additions
        assert rel(got, want) < 1e-6, rel(got, want)
        err_rt = (torch.linalg.vector_norm(back - x) / torch.linalg.vector_norm(x)).item()
        assert err_rt < 1e-5, err_rt
    # sampled points of volume 0 against the oracle's rows (real part at
    # primary points, -imaginary part elsewhere)
    rows = rng.integers(0, n ** 3, size=24)
    ref = oracle.forward_rows(vol0.astype(np.float64), n, rows)
    prim = oracle.packed_primary(n)[rows]
    ref_pk = np.where(prim, ref.real, -ref.imag)
    rms = np.sqrt(np.mean(np.abs(yh[:n ** 3]) ** 2))
    est = np.sqrt(np.mean((got[rows] - ref_pk) ** 2)) / rms
    assert est < TOL[dtype] * 2, est


def test_packed_ragged_plan():
    orders = [8, 8, 5, 16, 16, 16, 1, 24]
    vols = [inputs.smoothed_noise(n, 1, seed=i)[0] if n > 2 else inputs.uniform(n, 1, seed=i)[0]
            for i, n in enumerate(orders)]
    flat = np.concatenate([v.reshape(-1) for v in vols]).astype(np.float32)
    with binding.Plan(orders=orders, dtype="r32") as p:
        pk = p.forward_packed(dev(flat, np.float32))
        back = p.inverse_packed(pk).cpu().numpy()
        pk = pk.cpu().numpy()
    off = 0
    for v, n in zip(vols, orders):
        ref = oracle.pack_hermitian(_oracle_forward(v.astype(np.float32).astype(np.float64), n), n).reshape(-1)
        assert rel(pk[off:off + n ** 3], ref) < 1e-5, n
        assert rel(back[off:off + n ** 3], v) < 4e-5, n
        off += n ** 3


def test_packed_host_forms_match_device_forms():
    n, batch = 32, 6
    x = inputs.smoothed_noise(n, batch, seed=4).astype(np.float32).reshape(-1)
    with binding.Plan(n, batch, "r32_bf16x3") as p:
        pk_dev = p.forward_packed(dev(x, np.float32)).cpu()
        xh = torch.from_numpy(x).pin_memory()
        pkh = torch.empty(x.size, dtype=torch.float32).pin_memory()
        p.forward_packed_host(xh, pkh)
        backh = torch.empty(x.size, dtype=torch.float32).pin_memory()
        p.inverse_packed_host(pkh, backh)
        torch.cuda.synchronize()
    assert torch.equal(pkh, pk_dev)
    assert rel(backh.numpy(), x) < 4e-5


def test_packed_launch_counts_match_recorded_launches():
    for n, batch, dtype in [(64, 5, "r32"), (16, 2, "r32_bf16x3"), (12, 3, "r32"), (8, 1, "r64")]:
        rt = np.float64 if dtype == "r64" else np.float32
        x = dev(inputs.uniform(n, batch, seed=1), rt)
        with binding.Plan(n, batch, dtype) as p:
            p.forward_packed(x)   # first call allocates the workspace
            for which, call in ((3, p.forward_packed), (4, p.inverse_packed)):
                p.profile(True)
                call(x)
                torch.cuda.synchronize()
                rec = p.profile_read()
                p.profile(False)
                assert sum(c for _, c in rec.values()) == p.launches(which), (n, batch, dtype, which, rec)


def test_packed_calls_refuse_what_they_do_not_serve():
    L = binding.lib()
    with binding.Plan(8, 2, "c32") as p:
        a = torch.zeros(2 * 8 ** 3, dtype=torch.float32, device=DEV)
        b = torch.zeros(2 * 8 ** 3, dtype=torch.float32, device=DEV)
        for f in (L.fcc_dct_forward_packed, L.fcc_dct_inverse_packed):
            assert f(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), None) \
                == binding.FCC_ERR_UNSUPPORTED
    with binding.Plan(8, 2, "r32", skew=((1, 0, 11), 16)) as p:
        for f in (L.fcc_dct_forward_packed, L.fcc_dct_inverse_packed):
            assert f(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), None) \
                == binding.FCC_ERR_UNSUPPORTED
    with binding.Plan(8, 2, "r32") as p:
        # overlapping and misaligned buffers
        assert L.fcc_dct_forward_packed(p.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr() + 16),
                                        None) == binding.FCC_ERR_INVALID_ARG
        assert L.fcc_dct_forward_packed(p.handle, ctypes.c_void_p(a.data_ptr() + 4), ctypes.c_void_p(b.data_ptr()),
                                        None) == binding.FCC_ERR_INVALID_ARG
