"""Execution schedules on the GPU: the persistent ragged launch, the schedule
knobs and the autotuner change how the work runs, never what it computes.
Results are compared with the oracle (or, across schedules, with each other
to FP32 rounding), through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1807_10058_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _ragged(orders, seed, complex_in=False):
    vols = [inputs.smoothed_noise(n, 1, seed=seed + i)[0] for i, n in enumerate(orders)]
    flat = np.concatenate([v.reshape(-1) for v in vols])
    if complex_in:
        flat = flat + 1j * np.roll(flat, 11)
    return flat


def _check_against_oracle(y, flat, orders, tol):
    off = 0
    for i, n in enumerate(orders):
        v = flat[off:off + n ** 3].reshape(n, n, n)
        ref = oracle.forward_sum_fft(v.astype(np.complex128 if np.iscomplexobj(v) else np.float64), n).reshape(-1)
        assert rel(y[off:off + n ** 3], ref) < tol, (i, n)
        off += n ** 3


@pytest.mark.parametrize("dtype", ["r32", "c32"])
def test_persistent_ragged_launch_matches_oracle(dtype):
    orders = inputs.ragged_orders(24, seed=9)
    flat = _ragged(orders, seed=300, complex_in=dtype == "c32")
    x = torch.from_numpy(flat.astype(np.float32 if dtype == "r32" else np.complex64)).to(DEV)
    with binding.Plan(orders=orders, dtype=dtype) as p:
        p.set_schedule(ragged=1)
        assert p.schedule()["ragged"] == 1
        assert p.launches(0) == 1
        p.profile(True)
        y = p.forward(x)
        torch.cuda.synchronize()
        rec = p.profile_read()
        p.profile(False)
        assert set(rec) == {"ragged_persistent"} and rec["ragged_persistent"][1] == 1
        y = y.cpu().numpy()
        p.set_schedule(ragged=0)
        y0 = p.forward(x).cpu().numpy()
    _check_against_oracle(y, flat, orders, 1e-5)
    assert rel(y, y0) < 1e-6


@pytest.mark.parametrize("dtype", ["r32", "r32_bf16x3"])
def test_ragged_pairs_of_scattered_volumes(dtype):
    """Per-order launches pair the real volumes of each order in their order of
    appearance (the two volumes of a pair sit anywhere in the batch), and an
    odd count leaves one volume single: checked against the oracle volume by
    volume, against the per-run schedule and the persistent launch (neither
    pairs across the batch), and the launch count the plan reports."""
    orders = [16, 8, 16, 24, 8, 16, 32, 24, 16, 8, 40]
    flat = _ragged(orders, seed=77)
    x = torch.from_numpy(flat.astype(np.float32)).to(DEV)
    with binding.Plan(orders=orders, dtype=dtype) as p:
        p.set_schedule(ragged=0)
        p.profile(True)
        y = p.forward(x)
        torch.cuda.synchronize()
        rec = p.profile_read()
        p.profile(False)
        assert sum(c for _, c in rec.values()) == p.launches(0), (rec, p.launches(0))
        assert "fft_pencil_pair" in rec, rec
        # the same launches captured in a CUDA graph and replayed
        yg = torch.empty_like(y)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.forward(x, out=yg)
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(yg, y)
        y = y.cpu().numpy()
        p.set_schedule(ragged=2)
        y_run = p.forward(x).cpu().numpy()
        p.set_schedule(ragged=1)
        y_pers = p.forward(x).cpu().numpy()
    _check_against_oracle(y, flat, orders, 1e-5)
    assert rel(y, y_run) < 1e-6 and rel(y, y_pers) < 1e-6, (rel(y, y_run), rel(y, y_pers))


@pytest.mark.parametrize("dtype", ["r32", "r32_bf16x3"])
def test_ragged_inverse_and_adjoint_pair_scattered_volumes(dtype):
    """Inverse and adjoint of a ragged batch of real volumes run per order over
    the pairs of its volumes (read and written at their own offsets), with an
    odd leftover alone: the inverse returns the coefficients, the adjoint
    matches the oracle volume by volume, both match the per-run schedule, and
    the launch counts are the reported ones."""
    orders = [16, 8, 16, 24, 8, 16, 32, 24, 16, 8, 40]
    flat = _ragged(orders, seed=91)
    rng = np.random.default_rng(5)
    g = (rng.standard_normal(flat.size) + 1j * rng.standard_normal(flat.size)).astype(np.complex64)
    x = torch.from_numpy(flat.astype(np.float32)).to(DEV)
    gd = torch.from_numpy(g).to(DEV)
    with binding.Plan(orders=orders, dtype=dtype) as p:
        y = p.forward(x)
        for which, call in ((1, lambda: p.inverse(y)), (2, lambda: p.adjoint(gd))):
            p.profile(True)
            call()
            torch.cuda.synchronize()
            rec = p.profile_read()
            p.profile(False)
            assert sum(c for _, c in rec.values()) == p.launches(which), (which, rec, p.launches(which))
            assert "fft_pencil_merge" in rec, rec
        xi = p.inverse(y).cpu().numpy()
        a = p.adjoint(gd).cpu().numpy()
        p.set_schedule(ragged=2)
        xi_run = p.inverse(y).cpu().numpy()
        a_run = p.adjoint(gd).cpu().numpy()
    assert rel(xi, flat) < 4e-5, rel(xi, flat)
    assert rel(xi, xi_run) < 1e-5 and rel(a, a_run) < 1e-5, (rel(xi, xi_run), rel(a, a_run))
    off = 0
    for i, n in enumerate(orders):
        gv = g[off:off + n ** 3].reshape(n, n, n).astype(np.complex128)
        ref = oracle.adjoint_sum_fft(gv, n).real.reshape(-1)
        assert rel(a[off:off + n ** 3], ref) < 1e-5, (i, n)
        off += n ** 3


def test_persistent_ragged_launch_in_cuda_graph():
    orders = [96, 8, 40, 64, 16, 88, 24]
    flat = _ragged(orders, seed=17)
    with binding.Plan(orders=orders, dtype="r32") as p:
        p.set_schedule(ragged=1)
        x = torch.from_numpy(flat.astype(np.float32)).to(DEV)
        y = torch.empty(p.points, dtype=torch.complex64, device=DEV)
        p.forward(x, out=y)            # outside the capture: kernel attributes
        ref = y.clone()
        y.zero_()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.forward(x, out=y)
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, ref)


def test_schedule_arguments_are_checked():
    with binding.Plan(32, 2, "r32") as p:
        L = binding.lib()
        for key, bad in ((0, 0), (0, 2000), (1, 0), (1, 5), (2, 3), (3, 5), (4, 2), (4, -1), (9, 1)):
            assert L.fcc_dct_set_schedule(p.handle, key, bad) == binding.FCC_ERR_INVALID_ARG
        # one persistent launch is for ragged plans only
        assert L.fcc_dct_set_schedule(p.handle, 2, 1) == binding.FCC_ERR_UNSUPPORTED
        assert L.fcc_dct_get_schedule(p.handle, 9) == -1
        assert p.schedule() == {"chunk_mb": 32, "streams": 2, "ragged": 0, "tc_blocks": 0, "tc_fold": 1}


@pytest.mark.parametrize("dtype", ["r32", "r32_bf16x3"])
def test_schedules_agree_on_uniform_batches(dtype):
    n, batch = 64, 10
    x = torch.from_numpy(inputs.phantom(n, batch, seed=5).astype(np.float32)).to(DEV)
    with binding.Plan(n, batch, dtype) as p:
        y0 = p.forward(x).cpu().numpy()
        for sched in ({"chunk_mb": 4, "streams": 1}, {"chunk_mb": 64, "streams": 3}, {"streams": 4, "tc_blocks": 1}):
            p.set_schedule(**sched)
            y = p.forward(x).cpu().numpy()
            assert rel(y, y0) < 1e-6, sched
        # inverse and adjoint keep within the workspace sized at plan creation
        back = p.inverse(p.forward(x)).cpu().numpy()
        assert rel(back, x.cpu().numpy().reshape(-1)) < 1e-5


@pytest.mark.parametrize("ragged", [False, True])
def test_autotune_keeps_a_valid_schedule(ragged):
    if ragged:
        orders = inputs.ragged_orders(16, seed=21)
        p = binding.Plan(orders=orders, dtype="r32")
        flat = _ragged(orders, seed=50)
    else:
        p = binding.Plan(48, 8, "r32_bf16x3")
        flat = inputs.phantom(48, 8, seed=6).reshape(-1)
    with p:
        x = torch.from_numpy(flat.astype(np.float32)).to(DEV)
        y0 = p.forward(x).cpu().numpy()
        out = torch.empty(p.points, dtype=torch.complex64, device=DEV)
        ms, sched = p.autotune(x, out, reps=2)
        assert ms > 0
        assert 1 <= sched["streams"] <= 4 and sched["chunk_mb"] >= 1 and sched["ragged"] in (0, 1, 2)
        y = p.forward(x).cpu().numpy()
        assert rel(y, y0) < 1e-6


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3"])
def test_mixing_replay_runs_in_the_forward_geometry(dtype):
    """The measurement aid replays the forward mixing's launches (same count,
    same chunks) on one stream and refuses what it does not serve."""
    n, batch = 64, 6
    x = torch.from_numpy(inputs.phantom(n, batch, seed=4).reshape(-1).astype(np.float32)).to(DEV)
    out = torch.empty(n ** 3 * batch, dtype=torch.complex64, device=DEV)
    with binding.Plan(n, batch, dtype) as p:
        p.set_schedule(streams=1, chunk_mb=2)   # one pair per chunk: three mixing launches
        y0 = p.forward(x).cpu().numpy()
        p.profile(True)
        p.forward(x, out=out)
        torch.cuda.synchronize()
        fwd = p.profile_read()
        p.mixing_replay(x, out)
        torch.cuda.synchronize()
        rep = p.profile_read()
        p.profile(False)
        p.check()
        assert set(rep) == {"mix_replay"}, rep
        assert rep["mix_replay"][1] == fwd["mix_tc_fwd"][1] == 3, (rep, fwd)
        # the plan is untouched: the forward still gives the same values
        assert rel(p.forward(x).cpu().numpy(), y0) == 0.0
    with binding.Plan(n, batch, "r32") as q, pytest.raises(binding.FccError):
        q.mixing_replay(x, out)


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    """FCC_AUTOTUNE_CACHE: the first search appends its result as a JSON line;
    a plan of the same key takes the cached schedule without a search (no new
    line); another key searches and appends; malformed lines are skipped."""
    import json
    cache = tmp_path / "autotune.jsonl"
    monkeypatch.setenv("FCC_AUTOTUNE_CACHE", str(cache))
    n, batch = 24, 6
    flat = inputs.smoothed_noise(n, batch, seed=8).reshape(-1).astype(np.float32)
    x = torch.from_numpy(flat).to(DEV)
    out = torch.empty(n ** 3 * batch, dtype=torch.complex64, device=DEV)
    with binding.Plan(n, batch, "r32") as p:
        y0 = p.forward(x).cpu().numpy()
        ms, sched = p.autotune(x, out, reps=2)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1, lines
    rec = json.loads(lines[0])
    assert "order=24 batch=6 dtype=" in rec["key"] and "gpu=" in rec["key"], rec
    assert (rec["chunk_mb"], rec["streams"], rec["ragged"]) == (sched["chunk_mb"], sched["streams"], sched["ragged"])
    with binding.Plan(n, batch, "r32") as q:
        # a different schedule first: the cached one must replace it
        q.set_schedule(chunk_mb=sched["chunk_mb"] + 7, streams=1 if sched["streams"] != 1 else 2)
        ms2, sched2 = q.autotune(x, out, reps=2)
        assert ms2 > 0 and sched2 == sched, (sched2, sched)
        assert rel(q.forward(x).cpu().numpy(), y0) < 1e-6
    assert len(cache.read_text().splitlines()) == 1
    # malformed lines, then a new key (another batch): searched and appended
    with open(cache, "a") as f:
        f.write("not json at all\n{\"key\": \"order=24 batch=4\n")
    with binding.Plan(n, 4, "r32") as r:
        r.autotune(x[: 4 * n ** 3], out[: 4 * n ** 3], reps=2)
    lines = cache.read_text().splitlines()
    assert len(lines) == 4 and "order=24 batch=4 dtype=" in json.loads(lines[-1])["key"], lines


@pytest.mark.parametrize("case", ["r32_n128", "bf16_n64", "ragged", "ragged_persistent", "inverse", "odd_n", "odd_n_inverse",
                                  "bf16_inverse"])
def test_launch_count_matches_recorded_launches(case):
    if case.startswith("ragged"):
        orders = inputs.ragged_orders(12, seed=2)
        p = binding.Plan(orders=orders, dtype="r32")
        if case == "ragged_persistent":
            p.set_schedule(ragged=1)
    else:
        n, batch, dtype = {"r32_n128": (128, 5, "r32"), "bf16_n64": (64, 9, "r32_bf16x3"), "inverse": (64, 6, "r32"),
                           "odd_n": (27, 5, "r32"), "odd_n_inverse": (27, 5, "r32"), "bf16_inverse": (64, 7, "r32_bf16x3")}[case]
        p = binding.Plan(n, batch, dtype)
    with p:
        which = 1 if case.endswith("inverse") else 0
        x = torch.zeros(p.points, dtype=torch.float32 if which == 0 else torch.complex64, device=DEV)
        p.profile(True)
        (p.forward if which == 0 else p.inverse)(x)
        torch.cuda.synchronize()
        rec = p.profile_read()
        p.profile(False)
        assert sum(c for _, c in rec.values()) == p.launches(which), rec


def test_tensor_core_wait_timeout_is_reported_and_the_context_survives():
    """The bounded MMA-completion wait runs out (test hook: no MMA, no signal):
    the host reads FCC_ERR_TIMEOUT, and the next call is correct."""
    n, batch = 32, 4
    L = binding.lib()
    x = torch.from_numpy(inputs.phantom(n, batch, seed=8).astype(np.float32)).to(DEV)
    with binding.Plan(n, batch, "r32_bf16x3") as p:
        ref = p.forward(x).clone()
        assert L.fcc_dct_check(p.handle) == binding.FCC_OK
        assert L.fcc_dct_test_wait_timeout(p.handle, 1) == binding.FCC_OK
        p.forward(x)
        assert L.fcc_dct_check(p.handle) == binding.FCC_ERR_TIMEOUT
        assert L.fcc_dct_check(p.handle) == binding.FCC_OK   # the status word was cleared
        # the plan's next call reports a timeout recorded by an earlier one
        p.forward(x)
        torch.cuda.synchronize()
        with pytest.raises(binding.FccError) as e:
            p.forward(x)
        assert e.value.status == binding.FCC_ERR_TIMEOUT
        assert L.fcc_dct_check(p.handle) == binding.FCC_OK
        assert L.fcc_dct_test_wait_timeout(p.handle, 0) == binding.FCC_OK
        y = p.forward(x)
        assert L.fcc_dct_check(p.handle) == binding.FCC_OK
        assert torch.equal(y, ref)
    with binding.Plan(n, batch, "r32") as q:
        assert L.fcc_dct_test_wait_timeout(q.handle, 1) == binding.FCC_ERR_UNSUPPORTED


@pytest.mark.parametrize("dtype", ["r32_bf16x3", "r32_tf32x3"])
@pytest.mark.parametrize("n,batch", [(128, 4), (64, 5), (24, 3), (8, 2)])
def test_row_phase_in_dft_passes_matches_mixing_epilogue(dtype, n, batch):
    """FCC_SCHED_TC_FOLD: the row phase applied by the slab / pencil passes
    (default) or in the mixing epilogue gives the same transform to FP32
    rounding, complex and packed, with the same launch count."""
    gen = torch.Generator(device=DEV)
    gen.manual_seed(n)
    x = torch.rand(batch * n ** 3, generator=gen, device=DEV, dtype=torch.float32) * 2 - 1
    with binding.Plan(n, batch, dtype) as p:
        assert p.schedule()["tc_fold"] == 1
        y1 = p.forward(x)
        k1 = p.forward_packed(x)
        l1 = (p.launches(0), p.launches(3))
        p.set_schedule(tc_fold=0)
        y0 = p.forward(x)
        k0 = p.forward_packed(x)
        assert (p.launches(0), p.launches(3)) == l1
        p.check()
    d = (torch.linalg.vector_norm(y1 - y0) / torch.linalg.vector_norm(y0)).item()
    dk = (torch.linalg.vector_norm(k1 - k0) / torch.linalg.vector_norm(k0)).item()
    assert d < 5e-7 and dk < 5e-7, (d, dk)
