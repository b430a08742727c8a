"""fcc_dct_inverse_static: the inverse for callers that may not allocate.

Some callers cannot allocate device memory while they run the inverse (an
allocator callback, or a latency-critical loop in which cudaMalloc would
synchronise the device).  This entry point keeps its workspace in a
file-scope device array instead of plan memory.  Here it is called through
the C ABI twice in a row, on different inputs, and must agree with the
ordinary inverse (fcc_dct_inverse) within the FP32 tolerance of the other
parity tests.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-5   # relative L2, as for every FP32 parity test


def _rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


def _static_inverse(plan, y):
    out = torch.empty(plan.points, dtype=torch.float32 if plan.real_input else torch.complex64, device=DEV)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = binding.lib().fcc_dct_inverse_static(plan.handle, ctypes.c_void_p(y.data_ptr()),
                                                  ctypes.c_void_p(out.data_ptr()), st)
    assert status == binding.FCC_OK, binding.status_string(status)
    return out


@pytest.mark.parametrize("order,batch,dtype", [(16, 3, "r32"), (128, 2, "r32"), (24, 2, "r32"), (8, 2, "c32"),
                                               (1, 5, "r32")])
def test_static_inverse_matches_inverse_twice(order, batch, dtype):
    with binding.Plan(order, batch, dtype) as p:
        for call in range(2):   # two calls in a row share the workspace
            if p.real_input:
                x = torch.from_numpy(inputs.smoothed_noise(order, batch, seed=10 * call).astype(np.float32)
                                     .reshape(-1)).to(DEV) if order > 1 else torch.randn(batch, device=DEV)
            else:
                x = torch.from_numpy(inputs.uniform(order, batch, seed=call, complex_=True)
                                     .astype(np.complex64).reshape(-1)).to(DEV)
            y = p.forward(x)
            ref = p.inverse(y)
            got = _static_inverse(p, y)
            torch.cuda.synchronize()
            assert _rel(got, ref) < TOL, (call, _rel(got, ref))
            assert _rel(got, x) < 4 * TOL


@pytest.mark.parametrize("orders,dtype", [([8, 8, 8, 16, 24, 24, 24], "r32"), ([5, 8, 8, 8, 16, 24, 24, 24], "r32"),
                                          ([24, 64, 16], "c32")])
def test_static_inverse_ragged_plans_match_inverse(orders, dtype):
    """Ragged plans: mixed orders in one plan, odd counts per order (the
    single leftover volume of a real plan), and volume bases that are only
    8-byte aligned after an odd order (the generic DFT and pair-merge paths)."""
    vols = [inputs.smoothed_noise(n, 1, seed=40 + i)[0] for i, n in enumerate(orders)]
    flat = np.concatenate([v.reshape(-1) for v in vols])
    if dtype == "c32":
        flat = flat + 1j * np.roll(flat, 5)
    with binding.Plan(orders=orders, dtype=dtype) as p:
        x = torch.from_numpy(flat.astype(np.float32 if dtype == "r32" else np.complex64)).to(DEV)
        y = p.forward(x)
        ref = p.inverse(y)
        for call in range(2):
            got = _static_inverse(p, y)
            torch.cuda.synchronize()
            assert _rel(got, ref) < TOL, (call, _rel(got, ref))
        assert _rel(got, x) < 4 * TOL


def test_static_inverse_complex_plan_at_a_fast_order():
    n, batch = 64, 3
    with binding.Plan(n, batch, "c32") as p:
        x = torch.from_numpy(inputs.uniform(n, batch, seed=9, complex_=True).astype(np.complex64).reshape(-1)).to(DEV)
        y = p.forward(x)
        ref = p.inverse(y)
        got = _static_inverse(p, y)
        torch.cuda.synchronize()
        assert _rel(got, ref) < TOL and _rel(got, x) < 4 * TOL


def test_static_inverse_rejects_what_does_not_fit():
    with binding.Plan(8, 1, "r64") as p:   # FP64 plans are not served
        y = torch.zeros(8 ** 3, dtype=torch.complex128, device=DEV)
        out = torch.empty(8 ** 3, dtype=torch.float64, device=DEV)
        assert binding.lib().fcc_dct_inverse_static(p.handle, ctypes.c_void_p(y.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()), None) == binding.FCC_ERR_UNSUPPORTED
    with binding.Plan(160, 1, "r32") as p:  # 160^3 complex floats exceed the array
        y = torch.zeros(160 ** 3, dtype=torch.complex64, device=DEV)
        out = torch.empty(160 ** 3, dtype=torch.float32, device=DEV)
        assert binding.lib().fcc_dct_inverse_static(p.handle, ctypes.c_void_p(y.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()), None) == binding.FCC_ERR_UNSUPPORTED
