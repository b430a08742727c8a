"""The skew transform DCT_n(r,s,t) of Def. 2 on the GPU, through the C ABI,
against the oracle evaluated at the same shift (r, s, t) = v / d.

Tolerances as for the canonical transform: relative L2 1e-12 (FP64 dtypes),
1e-5 (FP32 dtypes); the inverse of an ill-conditioned shift is allowed its
condition number on top.
"""
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
C0 = ((1, 0, 3), 8)
# the halved shifts (c0 + a)/2 of the radix-2 step of Sec. 4.B: invertible
HALVED = [((1, 0, 11), 16), ((9, 8, 11), 16), ((1, 0, 3), 16)]
SINGULAR = [((0, 0, 0), 1), ((1, 1, 1), 4)]
# cond(D) = the largest condition number of a class block (F / n^1.5 is
# unitary), the same at every order >= 8 (host plan tables)
COND = {HALVED[0]: 12.9, HALVED[1]: 12.9, HALVED[2]: 135.0, ((1, 0, 3), 32): 1.27e4}


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


@pytest.mark.parametrize("skew", HALVED[:2])
@pytest.mark.parametrize("dtype", ["r64", "c64", "r32", "c32"])
@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_skew_small_orders_against_dense_definition(n, dtype, skew):
    batch = 3
    x = _input(dtype, n, batch, seed=n)
    D = oracle.dct_matrix(n, skew)
    cond = np.linalg.cond(D)
    y_ref = oracle.forward_dense(x, n, skew)
    g = inputs.uniform(n, batch, seed=200 + n, complex_=True)
    a_ref = oracle.adjoint_dense(g, n, skew)
    real = dtype.startswith("r")
    with binding.Plan(n, batch, dtype, skew=skew) as p:
        y = host(p.forward(dev(x, RT[dtype] if real else CT[dtype])), x.shape)
        xi = host(p.inverse(dev(y_ref, CT[dtype])), x.shape)
        a = host(p.adjoint(dev(g, CT[dtype])), x.shape)
    assert rel(y, y_ref) < TOL[dtype], rel(y, y_ref)
    assert rel(xi, x) < TOL[dtype] * cond, (rel(xi, x), cond)
    assert rel(a, a_ref.real if real else a_ref) < TOL[dtype]


@pytest.mark.parametrize("skew", [HALVED[0], HALVED[2], ((1, 0, 3), 32)])
@pytest.mark.parametrize("dtype", ["r64", "r32", "c32"])
@pytest.mark.parametrize("n", [16, 27, 40, 64])
def test_skew_medium_orders_full_volumes(n, dtype, skew):
    """n = 27 runs the generic DFT passes, the others the register-radix ones."""
    batch = 3
    x = inputs.smoothed_noise(n, batch, seed=11) if dtype.startswith("r") else _input(dtype, n, batch, 4)
    y_ref = oracle.forward_sum_fft(x, n, skew)
    real = dtype.startswith("r")
    with binding.Plan(n, batch, dtype, skew=skew) as p:
        y = host(p.forward(dev(x, RT[dtype] if real else CT[dtype])), x.shape)
        back = host(p.inverse(dev(y, CT[dtype])), x.shape)
        g = y_ref / np.linalg.norm(y_ref)
        a = host(p.adjoint(dev(g, CT[dtype])), x.shape)
    assert rel(y, y_ref) < TOL[dtype], rel(y, y_ref)
    # the round trip is allowed a fraction of cond(D) on top of the forward's bar
    rt_tol = TOL[dtype] * max(4.0, COND[skew] / 4)
    assert rel(back, x) < rt_tol, rel(back, x)
    a_ref = oracle.adjoint_sum_fft(g, n, skew)
    assert rel(a, a_ref.real if real else a_ref) < TOL[dtype]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("dtype", ["r32", "c32", "r64"])
def test_shift_by_one_grid_step_rolls_the_canonical_transform(axis, dtype):
    """theta moves by one grid step along `axis` when c0 -> c0 + e_axis, so
    D(c0 + e) = P D(c0) with P the cyclic roll of the point index: the skew
    path (generic mixing) against the canonical fast path."""
    n, batch = 32, 4
    v = [1, 0, 3]
    v[axis] += 8
    x = inputs.smoothed_noise(n, batch, seed=3) if dtype.startswith("r") else _input(dtype, n, batch, 5)
    real = dtype.startswith("r")
    xd = dev(x, RT[dtype] if real else CT[dtype])
    g = inputs.uniform(n, batch, seed=77, complex_=True)
    ax = axis + 1
    with binding.Plan(n, batch, dtype) as p0, binding.Plan(n, batch, dtype, skew=(tuple(v), 8)) as p1:
        y0 = host(p0.forward(xd), x.shape)
        y1 = host(p1.forward(xd), x.shape)
        assert rel(y1, np.roll(y0, -1, axis=ax)) < TOL[dtype]
        # D(c0 + e)^{-1} y = D(c0)^{-1} P^T y and D(c0 + e)^H g = D(c0)^H P^T g
        yd = dev(y1, CT[dtype])
        xi1 = host(p1.inverse(yd), x.shape)
        assert rel(xi1, x) < 4 * TOL[dtype]
        a1 = host(p1.adjoint(dev(g, CT[dtype])), x.shape)
        a0 = host(p0.adjoint(dev(np.roll(g, 1, axis=ax), CT[dtype])), x.shape)
        assert rel(a1, a0) < TOL[dtype]


@pytest.mark.parametrize("skew", SINGULAR)
def test_singular_shift_forward_and_adjoint_work_inverse_is_refused(skew):
    n, batch = 12, 2
    x = inputs.smoothed_noise(n, batch, seed=21)
    g = inputs.uniform(n, batch, seed=22, complex_=True)
    with binding.Plan(n, batch, "r32", skew=skew) as p:
        y = host(p.forward(dev(x, np.float32)), x.shape)
        a = host(p.adjoint(dev(g, np.complex64)), x.shape)
        yd = dev(y, np.complex64)
        with pytest.raises(binding.FccError) as e:
            p.inverse(yd)
        assert e.value.status == binding.FCC_ERR_UNSUPPORTED
        xh = torch.empty(p.points, dtype=torch.float32).pin_memory()
        with pytest.raises(binding.FccError) as e:
            p.inverse_host(yd.cpu().pin_memory(), xh)
        assert e.value.status == binding.FCC_ERR_UNSUPPORTED
        xo = torch.empty(p.points, dtype=torch.float32, device=DEV)
        assert binding.lib().fcc_dct_inverse_static(p.handle, yd.data_ptr(), xo.data_ptr(), None) \
            == binding.FCC_ERR_UNSUPPORTED
    assert rel(y, oracle.forward_sum_fft(x, n, skew)) < 1e-5
    assert rel(a, oracle.adjoint_sum_fft(g, n, skew).real) < 1e-5


@pytest.mark.parametrize("dtype", ["r32", "r32_bf16x3"])
def test_canonical_shift_in_other_terms_is_the_canonical_plan(dtype):
    n, batch = 24, 4
    x = dev(inputs.smoothed_noise(n, batch, seed=8), np.float32)
    with binding.Plan(n, batch, dtype) as p0, binding.Plan(n, batch, dtype, skew=((2, 0, 6), 16)) as p1:
        assert p1.launches(0) == p0.launches(0)
        assert torch.equal(p0.forward(x), p1.forward(x))


def test_skew_host_entry_points():
    n, batch, skew = 32, 6, HALVED[1]
    x = inputs.smoothed_noise(n, batch, seed=30).astype(np.float32)
    with binding.Plan(n, batch, "r32", skew=skew) as p:
        yd = p.forward(dev(x, np.float32))
        yh = torch.empty(p.points, dtype=torch.complex64).pin_memory()
        p.forward_host(torch.from_numpy(x.reshape(-1)).pin_memory(), yh)
        torch.cuda.synchronize()
        xh = torch.empty(p.points, dtype=torch.float32).pin_memory()
        p.inverse_host(yh.clone().pin_memory(), xh)
        torch.cuda.synchronize()
        assert torch.equal(yh, yd.cpu())
        assert rel(xh.numpy(), x) < 4e-5


@pytest.mark.parametrize("case", ["fast_fwd", "fast_inv", "generic_fwd", "generic_adj"])
def test_skew_launch_count_matches_recorded_launches(case):
    n = 64 if case.startswith("fast") else 27
    which = {"fwd": 0, "inv": 1, "adj": 2}[case.split("_")[1]]
    with binding.Plan(n, 5, "r32", skew=HALVED[0]) as p:
        x = torch.zeros(p.points, dtype=torch.float32 if which == 0 else torch.complex64, device=DEV)
        p.profile(True)
        (p.forward, p.inverse, p.adjoint)[which](x)
        torch.cuda.synchronize()
        rec = p.profile_read()
        p.profile(False)
        assert sum(c for _, c in rec.values()) == p.launches(which), rec
        assert "mix_skew_" + ("fwd", "inv", "adj")[which] in rec


def test_skew_full_size_sampled_rows():
    """Order 128, batch 8 (the bench's launch shape for the skew line), rows of
    D(c) x sampled uniformly and computed one by one by the oracle."""
    n, batch, skew = 128, 8, HALVED[0]
    rng = np.random.default_rng(4)
    checked = [0, 5]
    gen = torch.Generator(device=DEV)
    gen.manual_seed(12)
    xd = torch.rand(batch * n ** 3, generator=gen, device=DEV, dtype=torch.float32)
    vols = {}
    for v in checked:
        vols[v] = inputs.phantom(n, 1, seed=40 + v)[0].astype(np.float32)
        xd[v * n ** 3:(v + 1) * n ** 3] = torch.from_numpy(vols[v].reshape(-1)).to(DEV)
    with binding.Plan(n, batch, "r32", skew=skew) as p:
        y = p.forward(xd)
        ys = {v: y[v * n ** 3:(v + 1) * n ** 3].cpu().numpy() for v in checked}
    for v in checked:
        rows = rng.integers(0, n ** 3, size=16)
        ref = oracle.forward_rows(vols[v].astype(np.float64), n, rows, skew)
        got = ys[v][rows]
        scale = np.sqrt(np.mean(np.abs(ys[v]) ** 2))
        assert rel(got, ref) < 1e-5, rel(got, ref)
        assert np.abs(got - ref).max() < 1e-5 * scale + 1e-6 * np.abs(ref).max()
