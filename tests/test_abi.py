"""The C ABI library loads, exports what include/fcc_dct.h declares, and
rejects bad arguments before touching the GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1807_10058_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fcc_dct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcc_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = binding.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    assert set(binding.EXPORTS) == set(names)


def test_status_strings():
    for s in range(6):
        assert binding.status_string(s)


@pytest.mark.parametrize("order,batch,dtype", [(0, 1, 2), (-3, 1, 2), (513, 1, 2), (8, 0, 2), (8, 1, 99), (8, 1, -1)])
def test_invalid_plan_arguments(order, batch, dtype):
    L = binding.lib()
    assert not L.fcc_dct_plan(order, batch, dtype)
    assert L.fcc_dct_last_error() == binding.FCC_ERR_INVALID_ARG


def test_invalid_ragged_arguments():
    L = binding.lib()
    assert not L.fcc_dct_plan_ragged(None, 3, 2)
    assert L.fcc_dct_last_error() == binding.FCC_ERR_INVALID_ARG
    arr = (ctypes.c_int * 2)(8, 0)
    assert not L.fcc_dct_plan_ragged(arr, 2, 2)
    assert L.fcc_dct_last_error() == binding.FCC_ERR_INVALID_ARG


@pytest.mark.parametrize("v,d,dtype,status", [
    ((1, 0, 3), 0, 2, binding.FCC_ERR_INVALID_ARG),          # d < 1
    ((1, 0, 3), 1025, 2, binding.FCC_ERR_INVALID_ARG),       # d > FCC_MAX_SHIFT_DEN
    ((1, 70000, 3), 8, 2, binding.FCC_ERR_INVALID_ARG),      # |v| > FCC_MAX_SHIFT_NUM
    ((1, 0, 11), 16, 9, binding.FCC_ERR_INVALID_ARG),        # dtype
    ((1, 0, 11), 16, 5, binding.FCC_ERR_UNSUPPORTED),        # tensor-core dtype, other shift
    ((9, 0, 3), 8, 4, binding.FCC_ERR_UNSUPPORTED),
])
def test_invalid_skew_plan_arguments(v, d, dtype, status):
    L = binding.lib()
    arr = (ctypes.c_int * 3)(*v)
    assert not L.fcc_dct_plan_skew(8, 2, dtype, arr, d)
    assert L.fcc_dct_last_error() == status
    assert not L.fcc_dct_plan_skew(8, 2, 2, None, 8)
    assert L.fcc_dct_last_error() == binding.FCC_ERR_INVALID_ARG


def test_null_plan_calls():
    L = binding.lib()
    for f in (L.fcc_dct_forward, L.fcc_dct_inverse, L.fcc_dct_adjoint, L.fcc_dct_forward_host,
              L.fcc_dct_inverse_host, L.fcc_dct_forward_packed, L.fcc_dct_inverse_packed,
              L.fcc_dct_forward_packed_host, L.fcc_dct_inverse_packed_host):
        assert f(None, None, None, None) == binding.FCC_ERR_INVALID_ARG
    assert L.fcc_dct_batch(None) == 0 and L.fcc_dct_points(None) == 0
    L.fcc_dct_destroy(None)


def test_describe_rejects_bad_order():
    L = binding.lib()
    n = ctypes.c_int64()
    assert L.fcc_dct_describe(0, ctypes.byref(n), None, None, None, None, None, None, None, None, None) \
        == binding.FCC_ERR_INVALID_ARG


def test_schedule_calls_reject_null_plan():
    L = binding.lib()
    assert L.fcc_dct_set_schedule(None, 0, 32) == binding.FCC_ERR_INVALID_ARG
    assert L.fcc_dct_get_schedule(None, 0) == -1
    assert L.fcc_dct_autotune(None, None, None, None, 3, None) == binding.FCC_ERR_INVALID_ARG


def test_wait_timeout_hook_rejects_null_plan():
    assert binding.lib().fcc_dct_test_wait_timeout(None, 1) == binding.FCC_ERR_INVALID_ARG


def test_injected_allocation_failure_of_the_plan_object():
    """The first allocation of plan creation (the host plan object) fails on
    request: NULL, FCC_ERR_ALLOC, no plan left alive, the hook disarmed.
    Runs without a GPU: nothing before that allocation touches the device."""
    L = binding.lib()
    assert L.fcc_dct_test_fail_alloc(-1) == binding.FCC_ERR_INVALID_ARG
    seq0, plans0, dev0 = binding.allocations()
    assert L.fcc_dct_test_fail_alloc(1) == binding.FCC_OK
    assert not L.fcc_dct_plan(8, 2, 2)
    assert L.fcc_dct_last_error() == binding.FCC_ERR_ALLOC
    seq1, plans1, dev1 = binding.allocations()
    assert seq1 == seq0 + 1 and plans1 == plans0 and dev1 == dev0
    # disarmed: the next failure (if any) is not an allocation failure
    assert L.fcc_dct_test_fail_alloc(0) == binding.FCC_OK
    h = L.fcc_dct_plan(8, 2, 2)
    if h:
        L.fcc_dct_destroy(h)
    else:
        assert L.fcc_dct_last_error() != binding.FCC_ERR_ALLOC
    assert binding.allocations()[1] == plans0


@pytest.mark.parametrize("order,dtype", [(32, 1), (6, 1), (0, 1), (8, 2), (8, 5)])
def test_radix2_plan_arguments(order, dtype):
    """The radix-2 recursion takes orders 2, 4, 8, 16 and complex dtypes only
    (checked before touching the GPU)."""
    L = binding.lib()
    assert not L.fcc_dct_plan_radix2(order, 1, dtype, None, 8)
    assert L.fcc_dct_last_error() == binding.FCC_ERR_INVALID_ARG
    assert L.fcc_dct_radix2_stats(None, 0, None, None, None) == -1
