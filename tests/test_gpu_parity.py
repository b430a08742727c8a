"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over the whole output): FP64 dtypes 1e-12, FP32
dtypes 1e-5 (the bar the FP32 transform must meet).  Element-wise maxima are
reported in the assertion messages.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL = {"r64": 1e-12, "c64": 1e-12, "r32": 1e-5, "c32": 1e-5}
RT = {"r64": np.float64, "c64": np.float64, "r32": np.float32, "c32": np.float32}
CT = {"r64": np.complex128, "c64": np.complex128, "r32": np.complex64, "c32": np.complex64}
DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype).reshape(-1)).to(DEV)


def host(t, shape):
    return t.cpu().numpy().reshape(shape)


def _input(dtype, n, batch, seed):
    return inputs.uniform(n, batch, seed=seed, complex_=dtype.startswith("c"))


@pytest.mark.parametrize("dtype", ["r64", "c64", "r32", "c32"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 10, 12])
def test_small_orders_against_dense_definition(dtype, n):
    batch = 3
    x = _input(dtype, n, batch, seed=n)
    y_ref = oracle.forward_dense(x, n)
    g = inputs.uniform(n, batch, seed=100 + n, complex_=True)
    a_ref = oracle.adjoint_dense(g, n)
    real = dtype.startswith("r")
    with binding.Plan(n, batch, dtype) as p:
        xd = dev(x, RT[dtype] if real else CT[dtype])
        y = host(p.forward(xd), x.shape)
        xi = host(p.inverse(dev(y_ref, CT[dtype])), x.shape)
        a = host(p.adjoint(dev(g, CT[dtype])), x.shape)
    assert rel(y, y_ref) < TOL[dtype], (rel(y, y_ref), np.abs(y - y_ref).max())
    assert rel(xi, x) < TOL[dtype] * 4, rel(xi, x)
    a_want = a_ref.real if real else a_ref
    assert rel(a, a_want) < TOL[dtype], rel(a, a_want)


@pytest.mark.parametrize("dtype", ["r64", "r32", "c32"])
@pytest.mark.parametrize("n", [16, 24, 40, 64])
def test_medium_orders_full_volumes(dtype, n):
    batch = 2
    x = inputs.smoothed_noise(n, batch, seed=7) if dtype.startswith("r") else _input(dtype, n, batch, 3)
    y_ref = oracle.forward_sum_fft(x, n)
    real = dtype.startswith("r")
    with binding.Plan(n, batch, dtype) as p:
        y = host(p.forward(dev(x, RT[dtype] if real else CT[dtype])), x.shape)
        xi = host(p.inverse(dev(y_ref, CT[dtype])), x.shape)
        g = y_ref / np.linalg.norm(y_ref)
        a = host(p.adjoint(dev(g, CT[dtype])), x.shape)
    assert rel(y, y_ref) < TOL[dtype], rel(y, y_ref)
    assert rel(xi, x) < TOL[dtype] * 4, rel(xi, x)
    a_ref = oracle.adjoint_sum_fft(g, n)
    assert rel(a, a_ref.real if real else a_ref) < TOL[dtype]


def _full_size(n, batch, checked, seed, maker):
    """Batch of `batch` volumes of order n on the device; the volumes listed
    in `checked` come from the seeded host generator, the rest are device
    noise of the same scale.  Returns (device tensor, {v: host volume})."""
    gen = torch.Generator(device=DEV)
    gen.manual_seed(seed)
    x = torch.rand(batch * n ** 3, generator=gen, device=DEV, dtype=torch.float32) * 2 - 1
    hv = {}
    for v in checked:
        vol = maker(n, 1, seed=seed + v)[0]
        hv[v] = vol
        x[v * n ** 3:(v + 1) * n ** 3] = torch.from_numpy(vol.astype(np.float32).reshape(-1)).to(DEV)
    return x, hv


@pytest.mark.parametrize("n,batch,maker", [(128, 64, inputs.phantom), (64, 256, inputs.smoothed_noise),
                                           (96, 32, inputs.phantom)])
def test_full_size_sampled_rows_and_round_trip(n, batch, maker):
    checked = [0, batch // 2, batch - 1]
    x, hv = _full_size(n, batch, checked, seed=11, maker=maker)
    rng = np.random.default_rng(n)
    with binding.Plan(n, batch, "r32") as p:
        y = p.forward(x)
        xr = p.inverse(y)
        torch.cuda.synchronize()
        # round trip on every volume (property at any size)
        err_rt = (torch.linalg.vector_norm(xr - x) / torch.linalg.vector_norm(x)).item()
        assert err_rt < 1e-5, err_rt
        for v in checked:
            # uniform rows estimate the whole-output relative L2 without bias;
            # the first and last point are checked element-wise as well
            rows = rng.integers(0, n ** 3, size=24)
            edge = np.array([0, n ** 3 - 1])
            allrows = np.concatenate([rows, edge])
            ref = oracle.forward_rows(hv[v].astype(np.float32).astype(np.float64), n, allrows)
            got = y[v * n ** 3 + torch.from_numpy(allrows).to(DEV)].cpu().numpy()
            rms = torch.sqrt(torch.mean(torch.abs(y[v * n ** 3:(v + 1) * n ** 3]) ** 2)).item()
            err = np.abs(got - ref)
            est = np.sqrt(np.mean(err[:24] ** 2)) / rms
            assert est < 1e-5, (v, est)
            # per element: FFT rounding is absolute (scale of the whole output)
            # plus a relative part for the few very large (DC-like) entries
            assert (err <= 1e-5 * rms + 1e-6 * np.abs(ref)).all(), (v, err / (rms + np.abs(ref)))


@pytest.mark.parametrize("dtype", ["r64", "r32"])
def test_ragged_plan_matches_per_volume_oracle(dtype):
    orders = [8, 5, 12, 8, 1, 16, 3]
    vols = [inputs.uniform(n, 1, seed=i)[0] for i, n in enumerate(orders)]
    flat = np.concatenate([v.reshape(-1) for v in vols])
    with binding.Plan(orders=orders, dtype=dtype) as p:
        y = p.forward(dev(flat, RT[dtype])).cpu().numpy()
        back = p.inverse(p.forward(dev(flat, RT[dtype]))).cpu().numpy()
    off = 0
    for v, n in zip(vols, orders):
        ref = oracle.forward_dense(v, n).reshape(-1) if n <= 12 else oracle.forward_sum_fft(v, n).reshape(-1)
        assert rel(y[off:off + n ** 3], ref) < TOL[dtype]
        assert rel(back[off:off + n ** 3], v) < TOL[dtype] * 4
        off += n ** 3


def test_host_buffer_entry_point_matches_device_call():
    n, batch = 16, 4
    x = inputs.smoothed_noise(n, batch, seed=2).astype(np.float32)
    with binding.Plan(n, batch, "r32") as p:
        yd = p.forward(dev(x, np.float32)).cpu()
        xh = torch.from_numpy(x.reshape(-1)).pin_memory()
        yh = torch.empty(batch * n ** 3, dtype=torch.complex64).pin_memory()
        p.forward_host(xh, yh)
        torch.cuda.synchronize()
    assert torch.equal(yd, yh)


def test_bad_device_arguments_are_rejected():
    n = 8
    L = binding.lib()
    with binding.Plan(n, 2, "r32") as p:
        x = torch.zeros(2 * n ** 3 + 8, device=DEV)
        y = torch.zeros(2 * n ** 3, device=DEV, dtype=torch.complex64)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        mis = ctypes.c_void_p(x.data_ptr() + 4)
        assert L.fcc_dct_forward(p.handle, mis, ctypes.c_void_p(y.data_ptr()), st) == binding.FCC_ERR_INVALID_ARG
        # overlapping input and output
        yy = torch.zeros(4 * n ** 3, device=DEV, dtype=torch.complex64)
        assert L.fcc_dct_forward(p.handle, ctypes.c_void_p(yy.data_ptr()), ctypes.c_void_p(yy.data_ptr() + 16),
                                 st) == binding.FCC_ERR_INVALID_ARG
        assert L.fcc_dct_forward(p.handle, None, ctypes.c_void_p(y.data_ptr()), st) == binding.FCC_ERR_INVALID_ARG


def test_unsupported_order_reports_status():
    with pytest.raises(binding.FccError) as e:
        binding.Plan(37, 1, "r32")
    assert e.value.status == binding.FCC_ERR_UNSUPPORTED


# --- tensor-core form: the forward orbit cores on tcgen05 ----------------------

TC_TOL = 1e-6   # relative L2 against the FP64 oracle


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3"])
@pytest.mark.parametrize("n,batch", [(2, 2), (5, 3), (8, 2), (16, 4), (24, 2), (64, 2)])
def test_tensor_core_forward_full_volumes(dtype, n, batch):
    x = inputs.smoothed_noise(n, batch, seed=5).astype(np.float32)
    ref = oracle.forward_sum_fft(x.astype(np.float64), n)
    with binding.Plan(n, batch, dtype) as p:
        y = host(p.forward(dev(x, np.float32)), x.shape)
        xi = host(p.inverse(dev(ref, np.complex64)), x.shape)
        p.check()
    assert rel(y, ref) < TC_TOL, rel(y, ref)
    assert rel(xi, x) < 4e-5


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3"])
def test_tensor_core_forward_order_128_sampled(dtype):
    n, batch = 128, 4
    checked = [0, 3]
    x, hv = _full_size(n, batch, checked, seed=21, maker=inputs.phantom)
    rng = np.random.default_rng(3)
    with binding.Plan(n, batch, dtype) as p, binding.Plan(n, batch, "r32") as q:
        y = p.forward(x)
        y32 = q.forward(x)
        p.check()
        for v in checked:
            rows = rng.integers(0, n ** 3, size=24)
            ref = oracle.forward_rows(hv[v].astype(np.float32).astype(np.float64), n, rows)
            got = y[v * n ** 3 + torch.from_numpy(rows).to(DEV)].cpu().numpy()
            rms = torch.sqrt(torch.mean(torch.abs(y[v * n ** 3:(v + 1) * n ** 3]) ** 2)).item()
            est = np.sqrt(np.mean(np.abs(got - ref) ** 2)) / rms
            assert est < TC_TOL, (v, est)
        # the tensor-core and SIMT forms agree to FP32 rounding everywhere
        d = (torch.linalg.vector_norm(y - y32) / torch.linalg.vector_norm(y32)).item()
        assert d < TC_TOL, d


def test_tensor_core_form_in_a_fresh_process():
    """The tensor-core plan is usable as the first thing a process does (no
    state left behind by other paths)."""
    import subprocess
    import sys
    code = ("import torch, sys; sys.path.insert(0, '.');"
            "from paper_1807_10058_gb300 import binding;"
            "p = binding.Plan(64, 4, 'r32_bf16x3'); q = binding.Plan(64, 4, 'r32');"
            "x = torch.rand(4 * 64 ** 3, device='cuda');"
            "a = p.forward(x); b = q.forward(x); p.check();"
            "print((torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item())")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert float(out.stdout.strip().splitlines()[-1]) < 1e-6


# --- ragged batches and CUDA-graph capture -------------------------------------

def _ragged_volumes(orders, seed):
    vols = [inputs.smoothed_noise(n, 1, seed=seed + i)[0] for i, n in enumerate(orders)]
    return vols, np.concatenate([v.reshape(-1) for v in vols])


@pytest.mark.parametrize("dtype", ["r32", "c32"])
def test_ragged_orders_8_to_96_grouped_by_order(dtype):
    orders = inputs.ragged_orders(30, seed=4)
    vols, flat = _ragged_volumes(orders, seed=100)
    if dtype == "c32":
        flat = flat + 1j * np.roll(flat, 7)
    with binding.Plan(orders=orders, dtype=dtype) as p:
        y = p.forward(dev(flat, np.float32 if dtype == "r32" else np.complex64)).cpu().numpy()
        assert p.launches(0) < 5 * len(set(orders))   # per-order launches, not per volume
    off = 0
    for i, n in enumerate(orders):
        v = flat[off:off + n ** 3].reshape(n, n, n).astype(np.complex64 if dtype == "c32" else np.float32)
        ref = oracle.forward_sum_fft(v.astype(np.complex128 if dtype == "c32" else np.float64), n).reshape(-1)
        assert rel(y[off:off + n ** 3], ref) < TOL[dtype], (i, n)
        off += n ** 3


def test_ragged_odd_offsets_fall_back_correctly():
    orders = [5, 8, 24, 3, 16]   # the even orders start at odd point offsets
    vols, flat = _ragged_volumes(orders, seed=7)
    with binding.Plan(orders=orders, dtype="r32") as p:
        y = p.forward(dev(flat, np.float32)).cpu().numpy()
    off = 0
    for v, n in zip(vols, orders):
        ref = oracle.forward_sum_fft(v.astype(np.float32).astype(np.float64), n).reshape(-1)
        assert rel(y[off:off + n ** 3], ref) < TOL["r32"]
        off += n ** 3


@pytest.mark.parametrize("orders", [[64] * 4, [8, 16, 24, 32, 40, 48, 56, 64, 72, 80, 88, 96]])
def test_forward_captured_in_cuda_graph(orders):
    vols, flat = _ragged_volumes(orders, seed=3)
    with binding.Plan(orders=orders, dtype="r32") as p:
        x = dev(flat, np.float32)
        y = torch.empty(p.points, dtype=torch.complex64, device=DEV)
        p.forward(x, out=y)            # warm-up outside the capture (sets kernel attributes)
        ref = y.clone()
        y.zero_()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.forward(x, out=y)
        torch.cuda.current_stream().wait_stream(s)
        y.zero_()
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, ref)


@pytest.mark.parametrize("batch", [18, 7])
def test_host_entry_points_in_several_chunks(batch):
    """Host-buffer calls pipeline chunks of volumes through copy-in, transform
    and copy-out streams; results equal the device calls bit for bit."""
    n = 128
    x = inputs.phantom(n, batch, seed=12).astype(np.float32)
    with binding.Plan(n, batch, "r32") as p:
        xd = dev(x, np.float32)
        yd = p.forward(xd)
        back = p.inverse(yd).cpu()
        yd = yd.cpu()
        xh = torch.from_numpy(x.reshape(-1)).pin_memory()
        yh = torch.empty(batch * n ** 3, dtype=torch.complex64).pin_memory()
        p.forward_host(xh, yh)
        xb = torch.empty(batch * n ** 3, dtype=torch.float32).pin_memory()
        p.inverse_host(yh, xb)
        torch.cuda.synchronize()
    assert torch.equal(yd, yh)
    assert torch.equal(back, xb)


def test_bf16x6_equals_bf16x3():
    """A 3-way split of the exact core has zero low parts: the 6-product form
    is the 3-product form, bit for bit."""
    n, batch = 48, 6
    x = dev(inputs.phantom(n, batch, seed=31).astype(np.float32), np.float32)
    with binding.Plan(n, batch, "r32_bf16x3") as a, binding.Plan(n, batch, "r32_bf16x6") as b:
        assert torch.equal(a.forward(x), b.forward(x))


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3", "r32_bf16x6"])
@pytest.mark.parametrize("n,batch", [(8, 4), (16, 3), (24, 2), (48, 4), (64, 2)])
def test_tensor_core_inverse_and_adjoint(dtype, n, batch):
    """Inverse and adjoint of the tensor-core dtypes: the class blocks on
    tcgen05 in the six-product BF16 form (FP32-level accuracy).  The adjoint
    against the oracle's D^H; the inverse against the exact inverse of the
    same complex64 input (dense oracle at n <= 16) or, beyond, against the
    plain FP32 inverse and the original volume."""
    x = inputs.smoothed_noise(n, batch, seed=17).astype(np.float32)
    ref = oracle.forward_sum_fft(x.astype(np.float64), n)
    y32 = ref.astype(np.complex64)
    g = (inputs.uniform(n, batch, seed=18) + 1j * inputs.uniform(n, batch, seed=19)).astype(np.complex64)
    with binding.Plan(n, batch, dtype) as p:
        xi = host(p.inverse(dev(y32, np.complex64)), x.shape)
        ad = host(p.adjoint(dev(g, np.complex64)), x.shape)
        p.check()
    with binding.Plan(n, batch, "r32") as q:
        xi32 = host(q.inverse(dev(y32, np.complex64)), x.shape)
    aref = oracle.adjoint_sum_fft(g.astype(np.complex128), n).real
    assert rel(ad, aref) < TC_TOL, rel(ad, aref)
    if n <= 16:
        xref = np.stack([oracle.inverse_dense(y32[b].astype(np.complex128), n).real for b in range(batch)])
        assert rel(xi, xref) < TC_TOL, rel(xi, xref)
    assert rel(xi, xi32) < 2e-6, rel(xi, xi32)
    assert rel(xi, x) < 4e-5


def test_tensor_core_forward_bench_configuration():
    """The headline configuration as bench.py times it: order 128, batch 64,
    BF16 terms, 8 MB chunks over 3 internal streams (the autotuner's pick on
    GB300), row phase in the DFT passes; sampled rows of three volumes
    against the oracle, and agreement with the plain FP32 form everywhere."""
    n, batch = 128, 64
    checked = [0, 31, 63]
    x, hv = _full_size(n, batch, checked, seed=41, maker=inputs.phantom)
    rng = np.random.default_rng(41)
    with binding.Plan(n, batch, "r32_bf16x3") as p, binding.Plan(n, batch, "r32") as q:
        p.set_schedule(chunk_mb=8, streams=3)
        assert p.schedule()["tc_fold"] == 1
        y = p.forward(x)
        y32 = q.forward(x)
        p.check()
        for v in checked:
            rows = rng.integers(0, n ** 3, size=24)
            ref = oracle.forward_rows(hv[v].astype(np.float32).astype(np.float64), n, rows)
            got = y[v * n ** 3 + torch.from_numpy(rows).to(DEV)].cpu().numpy()
            rms = torch.sqrt(torch.mean(torch.abs(y[v * n ** 3:(v + 1) * n ** 3]) ** 2)).item()
            est = np.sqrt(np.mean(np.abs(got - ref) ** 2)) / rms
            assert est < TC_TOL, (v, est)
        d = (torch.linalg.vector_norm(y - y32) / torch.linalg.vector_norm(y32)).item()
        assert d < TC_TOL, d


def test_maximum_order_sampled_rows_and_round_trip():
    """The largest order a plan accepts (512: generic mixed-radix passes, 5.7 M
    orbits), a pair of real volumes: sampled rows of the first against the
    oracle and the round trip of both."""
    n, batch = 512, 2
    x, hv = _full_size(n, batch, [0], seed=5, maker=inputs.uniform)
    rng = np.random.default_rng(512)
    with binding.Plan(n, batch, "r32") as p:
        y = p.forward(x)
        back = p.inverse(y)
        torch.cuda.synchronize()
        err_rt = (torch.linalg.vector_norm(back - x) / torch.linalg.vector_norm(x)).item()
        rows = rng.integers(0, n ** 3, size=8)
        ref = oracle.forward_rows(hv[0].astype(np.float32).astype(np.float64), n, rows)
        got = y[torch.from_numpy(rows).to(DEV)].cpu().numpy()
        rms = torch.sqrt(torch.mean(torch.abs(y[:n ** 3]) ** 2)).item()
    assert err_rt < 1e-5, err_rt
    est = np.sqrt(np.mean(np.abs(got - ref) ** 2)) / rms
    assert est < 1e-5, est
