"""Host-side allocation failure (injected through fcc_dct_test_fail_alloc,
no GPU fault): every allocation of plan creation, of the first packed call
and of the first host-buffer call can fail; the call reports FCC_ERR_ALLOC,
releases what it had allocated (no plan alive, no device bytes held, the
device's free memory back where it was) and the library works afterwards."""
import numpy as np
import pytest
import torch

from paper_1807_10058_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("order,batch,dtype", [(64, 4, "r32_bf16x3"), (24, 3, "r32"), (8, 2, "c64")])
def test_every_allocation_of_plan_creation_can_fail(order, batch, dtype):
    L = binding.lib()
    # warm-up: the first use of the library loads its kernels (and the
    # module's static device array) once per process; that is not a leak
    with binding.Plan(order, batch, dtype) as w:
        w.forward(torch.zeros(w.points, dtype=torch.float32 if w.real_input else
                              (torch.complex128 if dtype == "c64" else torch.complex64), device=DEV))
    seq0, plans0, dev0 = binding.allocations()
    free0 = _free_bytes()
    failures = 0
    for nth in range(1, 400):
        assert L.fcc_dct_test_fail_alloc(nth) == binding.FCC_OK
        h = L.fcc_dct_plan(order, batch, binding.DTYPES[dtype])
        if h:   # nth is beyond the plan's allocations: it succeeded
            L.fcc_dct_test_fail_alloc(0)
            L.fcc_dct_destroy(h)
            break
        failures += 1
        assert L.fcc_dct_last_error() == binding.FCC_ERR_ALLOC, nth
        _, plans, dev = binding.allocations()
        assert plans == plans0 and dev == dev0, (nth, plans, dev)
        assert abs(_free_bytes() - free0) < 8 << 20, nth
    assert failures >= 3   # the plan object, the status word, device tables
    assert binding.allocations()[1:] == (plans0, dev0)
    assert abs(_free_bytes() - free0) < 8 << 20


def test_first_packed_and_host_buffer_calls_report_allocation_failure():
    n, batch = 32, 4
    L = binding.lib()
    x = torch.from_numpy(inputs.phantom(n, batch, seed=4).astype(np.float32)).to(DEV).reshape(-1)
    with binding.Plan(n, batch, "r32") as p:
        _, plans0, dev0 = binding.allocations()
        # the packed workspace is allocated by the first packed call
        assert L.fcc_dct_test_fail_alloc(1) == binding.FCC_OK
        with pytest.raises(binding.FccError) as e:
            p.forward_packed(x)
        assert e.value.status == binding.FCC_ERR_ALLOC
        assert binding.allocations()[1:] == (plans0, dev0)
        pk = p.forward_packed(x)            # allocates now and runs
        y = p.forward(x)
        idx = torch.arange(n ** 3, device=DEV)
        l, q = (idx // n) % n, idx % n
        prim = ((2 * l < n) | ((2 * l == n) & (2 * q < n))).repeat(batch)
        assert torch.equal(pk, torch.where(prim, y.real, -y.imag))
        # the staging buffers of the host-buffer calls
        xh = x.cpu().pin_memory()
        yh = torch.empty(batch * n ** 3, dtype=torch.complex64).pin_memory()
        _, _, dev1 = binding.allocations()
        assert L.fcc_dct_test_fail_alloc(1) == binding.FCC_OK
        with pytest.raises(binding.FccError) as e:
            p.forward_host(xh, yh)
        assert e.value.status == binding.FCC_ERR_ALLOC
        assert binding.allocations()[2] == dev1
        p.forward_host(xh, yh)
        torch.cuda.synchronize()
        assert torch.equal(yh, y.cpu())
