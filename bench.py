#!/usr/bin/env python
"""Throughput of the FCC cosine transform on one GB300 (or N replicas).

One step = the forward transform y = DCT_n x of a batch of synthetic
volumes (order n = 128, batch 64 by default: CT-like phantoms, FP32 real
coefficients -> complex64 point values).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fcc|reference]

N > 1 runs under torchrun: every rank transforms its own batch (replicas,
no collective), the timed region is bracketed by barriers and the slowest
rank's time is used.  --impl reference times the FP64 oracle on the host
cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FCC-DCT Gpoints/s + %roofline (n=128, batch 64), TC form vs FP32 at 1e-6 err"
UNIT = "Gpoints/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def l2_copy_peak(device):
    """Copy rate of an L2-resident buffer (read + write bytes per second, GB/s):
    torch's copy kernel over two buffers of 16-32 MB each (together below the
    126 MB L2), timed with CUDA events after a warm-up; the best size."""
    import torch
    best = 0.0
    for mb in (16, 24, 32):
        n = mb * 2 ** 20 // 4
        a = torch.rand(n, device=device)
        b = torch.empty_like(a)
        for _ in range(20):
            b.copy_(a)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * n * 4 * 200 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        del a, b
    return best


def slowest_rank_ms(ms, dist, device):
    """Replicas: every rank times its own batch; the job's time is the slowest
    rank's (no data-path collective, only this reduction)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def rank_seed(rank):
    """Seed of a rank's synthetic batch (ranks transform different volumes)."""
    return 1000 * int(rank)


# the sources of the kernels whose DRAM traffic profiles/kernel_traffic.json
# records (the mixing, slab and pencil passes, what they include, and the plan
# builder that lays out the tiles the mixing walks)
TRAFFIC_KERNEL_SOURCES = ("mix_tc.cuh", "mix_tiled.cuh", "kernels.cuh", "plan.h", "plan.cpp", "weyl_const.h",
                          "fft_fast.cuh", "fft_slab128.cuh", "dft_reg.cuh")


def kernel_sources_digest():
    """sha256 over the code of the files that define the kernels of the
    traffic table (TRAFFIC_KERNEL_SOURCES) with comments and whitespace
    removed; the host orchestration (*.cu, *.cpp) and the comments do not
    change what a kernel does."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1807_10058_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(TRAFFIC_KERNEL_SOURCES):
        with open(os.path.join(csrc, name)) as f:
            code = f.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(name.encode())
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()


def _traffic(kernel, points_per_launch):
    """DRAM bytes per launch of `kernel` from the committed ncu capture
    (profiles/kernel_traffic.json), scaled to the launch size; None when the
    kernel sources changed since the capture or the kernel was not captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "kernel_traffic.json")) as f:
            d = json.load(f)
        if kernel_sources_digest() != d["kernel_sources_sha256"] or kernel not in d["kernels"]:
            return None
        k = d["kernels"][kernel]
        return (k["dram_read"] + k["dram_write"]) * points_per_launch / d["points_per_launch"]
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler for the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n, seconds=12.0):
    """The FP64 oracle (direct definition, exact phases) timed on the host
    cores on a bounded sample: whole output rows of one phantom volume."""
    import numpy as np
    import oracle
    from paper_1807_10058_gb300 import inputs
    cores = len(os.sched_getaffinity(0))
    x = inputs.phantom(n, 1, seed=0)[0]
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    oracle.forward_rows(x, n, rng.integers(0, n ** 3, size=cores), nthreads=cores)
    t1 = time.perf_counter() - t0
    reps = max(1, int(seconds / max(t1, 1e-3)))
    rows = rng.integers(0, n ** 3, size=cores * reps)
    t0 = time.perf_counter()
    oracle.forward_rows(x, n, rows, nthreads=cores)
    dt = time.perf_counter() - t0
    # the oracle's exchanged-sum form (orbit sums, then numpy's FFT) on one
    # whole volume: the CPU counterpart of the F S factorisation, FP64
    t0 = time.perf_counter()
    oracle.forward_sum_fft(x, n)
    dtf = time.perf_counter() - t0
    return {"value": len(rows) / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d output points (whole rows of D, 24 n^3 terms each) of one n=%d phantom volume, "
                      "FP64 direct definition in C/OpenMP, %.1f s" % (len(rows), n, dt),
            "fft_form": {"value": n ** 3 / dtf / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one whole n=%d phantom volume, FP64 orbit sums + numpy FFT (one thread), "
                                   "%.1f s" % (n, dtf)}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1807_10058_gb300 import inputs
    n = args.order
    cores = len(os.sched_getaffinity(0))
    x = inputs.phantom(n, 1, seed=0)[0]
    rng = np.random.default_rng(1)
    # size one step so that the whole run stays within a few minutes
    t0 = time.perf_counter()
    oracle.forward_rows(x, n, rng.integers(0, n ** 3, size=cores), nthreads=cores)
    per = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)
    rows_per_step = cores * max(1, int(budget / max(per, 1e-3)))
    for _ in range(args.warmup):
        oracle.forward_rows(x, n, rng.integers(0, n ** 3, size=cores), nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forward_rows(x, n, rng.integers(0, n ** 3, size=rows_per_step), nthreads=cores)
    dt = time.perf_counter() - t0
    value = rows_per_step * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic CT-like phantom (seeded)",
            "config": {"workload": "FCC-DCT forward, order n=%d, batch %d (bounded sample: %d output points "
                                   "per step)" % (n, args.batch, rows_per_step), "order": n, "batch": args.batch},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d output rows per step, FP64 direct definition" % rows_per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


FORM_NAMES = {"r32": "plain FP32 (SIMT orbit cores)",
              "r32_bf16x3": "tensor-core (tcgen05 BF16, 3-term split inputs) orbit-core",
              "r32_tf32x3": "tensor-core (tcgen05 TF32, 2-term split inputs, exact core) orbit-core",
              "r32_bf16x6": "tensor-core (tcgen05 BF16, 6-product form = 3 products, exact core) orbit-core"}


def sampled_accuracy(x, y, n, dev, rows=24, skew=None):
    """An accuracy probe of a GPU result: the first input volume, uniformly
    sampled output rows and the GPU's values there, and the RMS of the first
    output volume.  The oracle evaluates probes in the CPU leg
    (evaluate_probes); uniform rows give an unbiased estimate of the
    whole-output relative L2."""
    import numpy as np
    import torch
    r = np.random.default_rng(3).integers(0, n ** 3, size=rows)
    return {"vol": x[:n ** 3].double().cpu().numpy(), "rows": r, "n": n, "skew": skew,
            "got": y[torch.from_numpy(r).to(dev)].cpu().numpy(),
            "rms": torch.sqrt(torch.mean(torch.abs(y[:n ** 3].to(torch.complex128)) ** 2)).item()}


def evaluate_probes(probes):
    """CPU leg: the FP64 oracle's rows for each accuracy probe; relative L2
    estimate and the largest sampled error (over the output RMS)."""
    import numpy as np
    import oracle
    out = {}
    for name, pr in probes.items():
        try:
            ref = oracle.forward_rows(pr["vol"], pr["n"], pr["rows"], skew=pr["skew"] or oracle.CANONICAL_SKEW,
                                      nthreads=len(os.sched_getaffinity(0)))
            err = np.abs(pr["got"] - ref)
            out[name] = {"rel_l2_est": float(np.sqrt(np.mean(err ** 2)) / pr["rms"]),
                         "max_err_over_rms": float(err.max() / pr["rms"]), "rows": len(pr["rows"]),
                         "oracle": "FP64 direct definition"}
        except Exception as exc:  # accuracy is reported, never required
            out[name] = {"error": str(exc)}
    return out


WHOLE_FORMS = ("r32", "r32_bf16x3", "r32_tf32x3", "r32_bf16x6")


def whole_volume_outputs(x, n, dev):
    """Volume 0 of the bench input through every form (a plan over the first
    pair of volumes), for the whole-volume comparison of the CPU leg."""
    from paper_1807_10058_gb300 import binding
    n3 = n ** 3
    outs = {}
    for form in WHOLE_FORMS:
        with binding.Plan(n, 2, form) as q:
            outs[form] = q.forward(x[:2 * n3])[:n3].cpu().numpy()
    return {"vol": x[:n3].double().cpu().numpy(), "n": n, "outs": outs}


def evaluate_whole_volume(w):
    """CPU leg: every output of volume 0 against the oracle's FP64 exchanged-sum
    form (orbit sums, then numpy's FFT): relative L2 and largest error over the
    output RMS, element by element over the whole volume."""
    import numpy as np
    import oracle
    try:
        t0 = time.perf_counter()
        ref = oracle.forward_sum_fft(w["vol"], w["n"]).ravel()
        dt = time.perf_counter() - t0
        rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
        forms = {}
        for form, got in w["outs"].items():
            err = np.abs(got.astype(np.complex128) - ref)
            forms[form] = {"rel_l2": float(np.linalg.norm(err) / np.linalg.norm(ref)),
                           "max_err_over_rms": float(err.max() / rms)}
        return {"oracle": "FP64 exchanged-sum form (orbit sums + FFT), whole volume 0 (%d points, %.1f s)"
                          % (ref.size, dt), "forms": forms}
    except Exception as exc:  # accuracy is reported, never required
        return {"error": str(exc)}


def _time(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def secondary_configs(dev):
    """The other workloads, each short: order 64 x 256 round trip; a ragged
    batch of 1000 volumes (orders 8..96) under each ragged schedule; order
    96 x 32 masked-reconstruction gradient descent through the autograd
    wrapper; the skew transform at order 128 x 64."""
    import numpy as np
    import torch
    from paper_1807_10058_gb300 import binding, inputs
    from paper_1807_10058_gb300.autograd import fcc_dct
    out = {}
    # round trip, n = 64, batch 256 (smoothed noise)
    n, b = 64, 256
    x = torch.randn(b * n ** 3, device=dev)
    with binding.Plan(n, b, "r32") as p:
        y = torch.empty(b * n ** 3, dtype=torch.complex64, device=dev)
        xr = torch.empty_like(x)
        ms = _time(lambda: (p.forward(x, out=y), p.inverse(y, out=xr)), 5, 3)
        rt = (torch.linalg.vector_norm(xr - x) / torch.linalg.vector_norm(x)).item()
    out["roundtrip_n64_b256"] = {"value": b * n ** 3 / (ms * 1e-3) / 1e9, "unit": "Gpoints/s (forward + inverse)",
                                 "ms_per_step": ms, "roundtrip_rel_l2": rt, "data": "i.i.d. N(0,1) coefficients"}
    # the same round trip in the tensor-core form (context: its inverse runs the
    # six-product BF16 blocks)
    with binding.Plan(n, b, "r32_bf16x3") as p:
        ms = _time(lambda: (p.forward(x, out=y), p.inverse(y, out=xr)), 5, 3)
        rt = (torch.linalg.vector_norm(xr - x) / torch.linalg.vector_norm(x)).item()
    out["roundtrip_n64_b256_tensor_core"] = {"value": b * n ** 3 / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                                             "roundtrip_rel_l2": rt, "form": "r32_bf16x3"}
    # ragged, 1000 volumes: per-order launches and the single persistent
    # launch, each captured in a CUDA graph; one launch set per run of equal
    # orders (no graph); then the autotuner's pick
    orders = inputs.ragged_orders(1000, seed=0)
    tot = sum(o ** 3 for o in orders)
    x = torch.randn(tot, device=dev)
    y = torch.empty(tot, dtype=torch.complex64, device=dev)

    def graph_ms(p):
        p.forward(x, out=y)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.forward(x, out=y)
        torch.cuda.current_stream().wait_stream(s)
        return _time(g.replay, 5, 2)

    rag = {"points": tot, "unit": "Gpoints/s", "data": "i.i.d. N(0,1) coefficients, orders U{8..96}"}
    with binding.Plan(orders=orders, dtype="r32") as p:
        ms = graph_ms(p)
        ref = y.clone()
        rag["grouped_graph"] = {"value": tot / (ms * 1e-3) / 1e9, "ms": ms, "launches": p.launches(0)}
        p.set_schedule(ragged=1)
        ms = graph_ms(p)
        diff = (torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item()
        rag["persistent_graph"] = {"value": tot / (ms * 1e-3) / 1e9, "ms": ms, "launches": p.launches(0),
                                   "rel_diff": diff}
        p.set_schedule(ragged=2)
        ms = _time(lambda: p.forward(x, out=y), 3, 1)
        diff = (torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item()
        rag["per_volume"] = {"value": tot / (ms * 1e-3) / 1e9, "ms": ms, "launches": p.launches(0), "rel_diff": diff}
        ms, sched = p.autotune(x, y, reps=2)
        rag["autotuned"] = {"value": tot / (ms * 1e-3) / 1e9, "ms": ms, "schedule": sched, "launches": p.launches(0)}
        # the inverse of the same batch: per-order launches over the pairs of
        # each order's volumes, and one launch set per run (no graph)
        xr = torch.empty_like(x)
        p.set_schedule(ragged=0)
        p.forward(x, out=y)
        ms = _time(lambda: p.inverse(y, out=xr), 5, 2)
        rt = (torch.linalg.vector_norm(xr - x) / torch.linalg.vector_norm(x)).item()
        rag["inverse_grouped"] = {"value": tot / (ms * 1e-3) / 1e9, "ms": ms, "launches": p.launches(1),
                                  "roundtrip_rel_l2": rt}
        p.set_schedule(ragged=2)
        ms = _time(lambda: p.inverse(y, out=xr), 3, 1)
        rag["inverse_per_volume"] = {"value": tot / (ms * 1e-3) / 1e9, "ms": ms, "launches": p.launches(1)}
        p.set_schedule(**{k: v for k, v in sched.items() if k in ("chunk_mb", "streams", "ragged")})
    out["ragged_1000"] = rag
    # autograd: 50 gradient-descent steps of ||M . (D x) - b||^2, n = 96, batch 32
    n, b = 96, 32
    xt = inputs.phantom_device(n, b, seed=9, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    M = (torch.rand(b * n ** 3, generator=gen, device=dev) < 0.1).float()
    with binding.Plan(n, b, "r32") as p:
        bt = M * p.forward(xt)
        x = torch.zeros(b * n ** 3, device=dev, requires_grad=True)

        def step():
            loss = torch.sum(torch.abs(M * fcc_dct(x, p) - bt) ** 2)
            loss.backward()
            with torch.no_grad():
                x.sub_(1e-6 * x.grad)
            x.grad = None
            return loss
        ms_gd = _time(step, 50, 3)
        with torch.no_grad():
            l0 = torch.sum(torch.abs(bt) ** 2).item()
        final = step().item()
    out["autograd_gd_n96_b32"] = {"ms_per_gd_step": ms_gd, "steps_timed": 50, "loss_ratio_after": final / l0,
                                  "note": "forward + adjoint backward per step, step size 1e-6"}
    # the skew transform DCT_n(1/16, 0, 11/16) of Def. 2 (a halved shift of the
    # radix-2 step), order 128 x 64, FP32: tiled orbit mixing on the staged
    # class cores with the plan's row phases + the register-radix DFT passes,
    # no pairing
    n, b, skew = 128, 64, ((1, 0, 11), 16)
    x = inputs.phantom_device(n, b, seed=5, device=dev)
    y = torch.empty(b * n ** 3, dtype=torch.complex64, device=dev)
    with binding.Plan(n, b, "r32", skew=skew) as p:
        ms = _time(lambda: p.forward(x, out=y), 10, 3)
        launches = p.launches(0)
        p.profile(True)
        p.forward(x, out=y)
        torch.cuda.synchronize()
        kern = {k: round(v[0], 4) for k, v in p.profile_read().items()}
        p.profile(False)
    pts = b * n ** 3
    peak, kind = _peaks()
    out["skew_n128_b64"] = {"value": pts / (ms * 1e-3) / 1e9, "unit": "Gpoints/s", "ms_per_step": ms,
                            "shift": "(1, 0, 11) / 16", "launches": launches,
                            "step_roofline_frac": pts * 12 / (ms * 1e-3) / (peak * 1e9), "peak_kind": kind,
                            "kernels_ms": kern, "accuracy_probe": sampled_accuracy(x, y, n, dev, skew=skew),
                            "form": "r32: tiled orbit mixing on staged class cores + register-radix DFT passes"}
    del x, y
    # the paper's radix-2x2x2 recursion (Sec. 4.B) at order 16: the GPU
    # evaluation in FP64 and FP32 beside the F S form on the same complex
    # inputs, its operation counts and how its FP32 form rounds
    n, b = 16, 64
    gen = torch.Generator(device=dev)
    gen.manual_seed(16)
    xc = torch.randn(b * n ** 3, dtype=torch.complex128, device=dev, generator=gen)
    r2 = {"order": n, "batch": b}
    with binding.Plan(n, b, "c64") as q:
        yf = q.forward(xc)
        r2["fs_c64_ms"] = _time(lambda: q.forward(xc, out=yf), 10, 3)
    with binding.Plan(n, b, "c64", radix2=True) as q:
        y64 = q.forward(xc)
        r2["radix2_c64_ms"] = _time(lambda: q.forward(xc, out=y64), 10, 3)
        r2["launches"] = q.launches(0)
        r2["macs_per_point"] = q.radix2_stats(0)
        r2["nnz_per_row_B"] = {k: q.radix2_stats(k)[0] for k in (4, 8, 16)}
        r2["max_abs_B"] = {k: q.radix2_stats(k)[1] for k in (4, 8, 16)}
    with binding.Plan(n, b, "c32", radix2=True) as q:
        x32 = xc.to(torch.complex64)
        y32 = q.forward(x32)
        r2["radix2_c32_ms"] = _time(lambda: q.forward(x32, out=y32), 10, 3)
    r2["rel_diff_radix2_c64_vs_fs_c64"] = (torch.linalg.vector_norm(y64 - yf) / torch.linalg.vector_norm(yf)).item()
    r2["rel_diff_radix2_c32_vs_radix2_c64"] = (torch.linalg.vector_norm(y32.to(torch.complex128) - y64)
                                               / torch.linalg.vector_norm(y64)).item()
    out["radix2_n16_b64"] = r2
    # the voxel rendering of Sec. 5 (Fig. 4): one n = 128 phantom volume drawn as
    # cubes and as the FCC lattice's rhombic dodecahedra, 1024 x 1024 pixels
    n = 128
    vol = inputs.phantom_device(n, 1, seed=7, device=dev)
    vol = (vol / vol.max()).clamp(0, 1)
    img = torch.empty(1024 * 1024, device=dev)
    ren = {"order": n, "pixels": 1024 * 1024, "step": 0.25, "kappa": 0.5}
    for cells in ("cube", "rhombic_dodecahedron"):
        fn = lambda: binding.render_cells(vol, n, cells, azimuth=0.6, elevation=0.4, kappa=0.5, step=0.25,
                                          width=1024, height=1024, image=img)
        ren[cells + "_ms"] = _time(fn, 5, 2)
        ren[cells + "_mean_grey"] = img.mean().item()
    out["render_n128_1024px"] = ren
    return out


def host_link_rates(dev, nbytes):
    """Pinned host <-> device copy rates (GB/s) for a buffer of nbytes, CUDA
    events around 3 copies each way after one warm-up copy: the link that
    bounds the end-to-end numbers."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name, fn in (("h2d_gbs", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_gbs", lambda: h.copy_(d, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = 3 * nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del h, d
    return out


def packed_vs_complex(pk, y, n, batch, dev):
    """Relative L2 between the packed output and the complex output of the
    same plan re-laid out (primary points keep Re y, the others -Im y)."""
    import torch
    idx = torch.arange(n ** 3, device=dev)
    l, q = (idx // n) % n, idx % n
    prim = ((2 * l < n) | ((2 * l == n) & (2 * q < n))).repeat(batch)
    want = torch.where(prim, y.real, -y.imag)
    return (torch.linalg.vector_norm(pk - want) / torch.linalg.vector_norm(want)).item()


def packed_config(plan, x, y, n, batch, args, dev, st):
    """The headline form with the Hermitian-packed output (n^3 reals per
    volume, fcc_dct_forward_packed) on the same inputs: device-timed, its
    kernels, the packed round trip, agreement with the complex output
    re-laid out, and end to end with host buffers (half the D2H bytes)."""
    import torch
    pts = batch * n ** 3
    pk = torch.empty(pts, dtype=torch.float32, device=dev)
    plan.forward_packed(x, out=pk)   # first call allocates the packed workspace
    ms = _time(lambda: plan.forward_packed(x, out=pk), args.steps, args.warmup)
    kept = plan.schedule()
    plan.set_schedule(streams=1)
    plan.profile(True)
    plan.forward_packed(x, out=pk)
    torch.cuda.synchronize()
    kern = {k: round(v[0], 4) for k, v in plan.profile_read().items()}
    plan.profile(False)
    plan.set_schedule(streams=kept["streams"])
    # the layout (primary points keep Re y, the others -Im y) applied to the
    # complex output of the same plan
    plan.forward(x, out=y)
    diff = packed_vs_complex(pk, y, n, batch, dev)
    back = torch.empty_like(x)
    plan.inverse_packed(pk, out=back)
    rt = (torch.linalg.vector_norm(back - x) / torch.linalg.vector_norm(x)).item()
    del back
    xh = x.cpu().pin_memory()
    pkh = torch.empty(pts, dtype=torch.float32).pin_memory()
    plan.forward_packed_host(xh, pkh)
    torch.cuda.synchronize()
    ke = max(3, args.steps // 4)
    runs = []
    for _ in range(3):   # three timings in the same run: the spread shows how steady the link is
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(ke):
            plan.forward_packed_host(xh, pkh)
        e1.record(st)
        torch.cuda.synchronize()
        runs.append(e0.elapsed_time(e1) / ke)
    ms_e2e = statistics.median(runs)
    link = host_link_rates(dev, pts * 4)
    peak, kind = _peaks()
    return {"value": pts / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "form": args.dtype,
            "output": "Hermitian-packed reals (n^3 per volume)", "bytes_per_point": 8,
            "step_roofline_frac": pts * 8 / (ms * 1e-3) / (peak * 1e9), "peak_kind": kind,
            "launches": plan.launches(3), "kernels_ms": kern, "rel_diff_vs_complex_output": diff,
            "roundtrip_rel_l2": rt,
            "e2e": {"value": pts / (ms_e2e * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": pts * 4,
                    "d2h_bytes_per_step": pts * 4, "ms_per_step_runs": runs,
                    "pinned_copy_gbs": link,
                    "link_bound_ms": pts * 4 / (min(link["h2d_gbs"], link["d2h_gbs"]) * 1e9) * 1e3}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fcc", choices=["fcc", "reference"])
    ap.add_argument("--order", type=int, default=128)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--dtype", default="r32_bf16x3",
                    help="form timed for the headline value (r32_bf16x3 = tensor-core form)")
    ap.add_argument("--compare", default="r32", help="second form timed beside it ('' to skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary configurations")
    ap.add_argument("--autotune", type=int, default=1, help="run fcc_dct_autotune before timing (1) or not (0)")
    ap.add_argument("--sched", default="",
                    help="schedule keys applied after the autotuner, e.g. 'streams=1,chunk_mb=32'")
    ap.add_argument("--output", default="complex", choices=["complex", "packed"],
                    help="forward output: complex64 point values, or the Hermitian-packed reals of real plans")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_1807_10058_gb300 import binding, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n, batch = args.order, args.batch
    pts = batch * n ** 3
    dev = torch.device("cuda", local)

    x = inputs.phantom_device(n, batch, seed=rank_seed(rank), device=dev)
    plan = binding.Plan(n, batch, args.dtype)
    y = torch.empty(pts, dtype=torch.complex64, device=dev)
    st = torch.cuda.current_stream(dev)
    packed = args.output == "packed"
    pk = torch.empty(pts, dtype=torch.float32, device=dev) if packed else None
    step_bytes = 8 if packed else 12   # algorithmic bytes per point of a whole forward step

    def fwd(p=plan):
        return p.forward_packed(x, out=pk) if packed else p.forward(x, out=y)

    def barrier():
        if dist is not None:
            dist.barrier()

    # the library's autotuner picks the execution schedule once (untimed)
    sched = plan.autotune(x, y, reps=3)[1] if args.autotune else plan.schedule()
    if args.sched:
        plan.set_schedule(**{k: int(v) for k, v in (kv.split("=") for kv in args.sched.split(","))})
        sched = plan.schedule()
    for _ in range(args.warmup):
        fwd()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        fwd()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ck = clocks.stop()
    ms = slowest_rank_ms(ms, dist, dev)

    # per-kernel durations: the same K steps again with per-launch events on
    # one internal stream, so that each kernel is timed alone
    kept = plan.schedule()
    plan.set_schedule(streams=1)
    plan.profile(True)
    for _ in range(args.steps):
        fwd()
    torch.cuda.synchronize()
    kern = plan.profile_read()
    # the mixing's access-pattern ceiling: its launches replayed with no
    # arithmetic, same chunks, geometry and stream (tensor-core forms)
    replay_ms = None
    if args.dtype.startswith("r32_") and batch >= 2:
        for _ in range(args.steps):
            plan.mixing_replay(x, y)
        torch.cuda.synchronize()
        rec = plan.profile_read()
        if "mix_replay" in rec:
            replay_ms = rec["mix_replay"][0] / args.steps
    plan.profile(False)
    plan.set_schedule(streams=kept["streams"])
    # algorithmic bytes per real point of each kernel.  Real plans pair two
    # volumes per complex transform: the mixing reads x (4 B) and writes half a
    # complex value (4 B); each DFT pass reads and writes half a complex value;
    # the split (alone, or fused into the last DFT pass) reads half a complex
    # value and writes one complex output (8 B).
    paired = args.dtype.startswith("r") and batch >= 2
    if paired:
        algo_bytes = {"mix_tiled_fwd": 8, "mix_tc_fwd": 8, "fft_slab": 8, "fft_pencil": 8, "pair_split": 12,
                      "fft_pencil_pair": 12, "fft_pencil_pair_packed": 8}
    else:
        algo_bytes = {"mix_tiled_fwd": 12, "fft_slab": 16, "fft_pencil": 16, "orbit_mix_fwd": 12,
                      "fft_axis0": 16, "fft_axis1": 16, "fft_axis2": 16}
    top = max(kern.items(), key=lambda kv: kv[1][0])
    top_name, (top_ms, top_cnt) = top
    per_launch_ms = top_ms / top_cnt
    per_launch_pts = pts * args.steps / top_cnt
    peak, peak_kind = _peaks()
    l2_peak = l2_copy_peak(dev)
    # the roofline unit is the whole forward's algorithmic bytes per point
    # (12: FP32 in, complex64 out; 8 with the packed output), charged to the
    # dominant kernel per point it processes; the kernel's own paired bytes
    # (what it reads and writes itself) are reported beside it
    achieved = step_bytes * per_launch_pts / (per_launch_ms * 1e-3) / 1e9
    own_gbs = algo_bytes.get(top_name, 12) * per_launch_pts / (per_launch_ms * 1e-3) / 1e9
    traffic = _traffic(top_name, per_launch_pts) if n == 128 else None
    step_gbs = step_bytes * pts / (ms * 1e-3) / 1e9

    # accuracy on sampled rows of one volume (outside the timed region)
    probes = {}
    relayout = None
    if packed:   # the packed values are the complex output re-laid out
        plan.forward(x, out=y)
        relayout = packed_vs_complex(pk, y, n, batch, dev)
    whole = None
    if rank == 0:
        probes["headline"] = sampled_accuracy(x, y, n, dev)
        if world == 1 and not args.no_cpu_baseline and batch >= 2:
            whole = whole_volume_outputs(x, n, dev)

    # end to end through the C ABI with host buffers
    xh = x.cpu().pin_memory()
    yh = torch.empty(pts, dtype=torch.float32 if packed else torch.complex64).pin_memory()
    fwd_host = plan.forward_packed_host if packed else plan.forward_host
    fwd_host(xh, yh)
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    ke = max(3, args.steps // 4)
    barrier()
    e2.record(st)
    for _ in range(ke):
        fwd_host(xh, yh)
    e3.record(st)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3) / ke
    link = host_link_rates(dev, pts * 4)

    # the comparison form on the same inputs (same timing rules)
    compare = None
    if args.compare and args.compare != args.dtype:
        with binding.Plan(n, batch, args.compare) as q:
            q_sched = q.autotune(x, y, reps=3)[1] if args.autotune else q.schedule()
            for _ in range(args.warmup):
                fwd(q)
            torch.cuda.synchronize()
            barrier()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(st)
            for _ in range(args.steps):
                fwd(q)
            c1.record(st)
            torch.cuda.synchronize()
            ms_c = c0.elapsed_time(c1) / args.steps
            if packed:
                q.forward(x, out=y)
            if rank == 0:
                probes["compare"] = sampled_accuracy(x, y, n, dev)
            compare = {"form": args.compare, "value": world * pts / (ms_c * 1e-3) / 1e9, "unit": UNIT,
                       "ms_per_step": ms_c, "schedule": q_sched}

    extra = None
    if rank == 0 and not args.no_extra and n == 128 and batch == 64:
        extra = secondary_configs(dev)
        if not packed:
            extra["packed_n%d_b%d" % (n, batch)] = packed_config(plan, x, y, n, batch, args, dev, st)

    # the CPU leg (rank 0, one GPU): the oracle timed on the host cores, and the
    # oracle's rows for the accuracy probes taken above
    cpu = None
    if extra and "skew_n128_b64" in extra:
        probes["skew"] = extra["skew_n128_b64"].pop("accuracy_probe")
    acc = {k: {"skipped": "oracle leg not run (--no-cpu-baseline or N > 1)"} for k in probes}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)
        acc = evaluate_probes(probes)
        if whole is not None:
            whole = evaluate_whole_volume(whole)
    if compare is not None and "compare" in acc:
        compare["accuracy"] = acc["compare"]
    if extra and "skew" in acc:
        extra["skew_n128_b64"]["accuracy"] = acc["skew"]
    accuracy = acc.get("headline")

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * pts / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"r32": "f32", "r32_bf16x3": "bf16x3/f32", "r32_tf32x3": "tf32x3/f32",
                      "r32_bf16x6": "bf16x6/f32"}.get(args.dtype, args.dtype),
            "data": "synthetic CT-like phantoms (10-30 random ellipsoids, densities U[0,1], +N(0,1e-3^2)), seeded",
            "config": {"workload": "FCC-DCT forward y = DCT_n x, order n=%d, batch %d, FP32 real -> %s, "
                                   "%s form" % (n, batch, "Hermitian-packed FP32 reals" if packed else "complex64",
                                                FORM_NAMES.get(args.dtype, args.dtype)),
                       "output": args.output, "packed_equals_complex_relaid": relayout,
                       "order": n, "batch": batch, "points_per_step": pts, "form": args.dtype,
                       "schedule": sched, "autotuned": bool(args.autotune),
                       "l2": "inputs %.0f MB + outputs %.0f MB per step exceed the 126 MB L2"
                             % (pts * 4 / 1e6, pts * (step_bytes - 4) / 1e6)},
            "roofline": {"bound": "hbm", "kernel": top_name, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "algorithmic_bytes_per_point": step_bytes,
                         "kernel_own_bytes_per_point": algo_bytes.get(top_name, 12),
                         "kernel_own_achieved": own_gbs, "kernel_own_frac": own_gbs / peak,
                         "l2": {"peak": l2_peak, "unit": "GB/s", "frac": own_gbs / l2_peak,
                                "kind": "measured copy of an L2-resident buffer (read + write)"},
                         "access_pattern": None if replay_ms is None or top_name not in ("mix_tc_fwd",) else {
                             "replay_ms_per_step": replay_ms, "kernel_ms_per_step": top_ms / args.steps,
                             "frac": replay_ms / (top_ms / args.steps),
                             "kind": "the kernel's own gathers and stores replayed with no arithmetic "
                                     "(fcc_dct_diag_mixing_replay; same chunks, grid and stream)"}},
            "step_roofline": {"achieved": step_gbs, "frac": step_gbs / peak, "bytes_per_point": step_bytes},
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kern.items()},
            "kernels": {k: {"launches_per_step": v[1] / args.steps, "ms_per_launch": v[0] / v[1],
                            "achieved_gbs": algo_bytes.get(k, 12) * pts / (v[0] / args.steps * 1e-3) / 1e9,
                            "frac": algo_bytes.get(k, 12) * pts / (v[0] / args.steps * 1e-3) / 1e9 / peak,
                            "frac_l2": algo_bytes.get(k, 12) * pts / (v[0] / args.steps * 1e-3) / 1e9 / l2_peak}
                        for k, v in kern.items()},
            "kernel_timing": "CUDA events around each launch, one internal stream (each kernel alone)",
            "e2e": {"value": world * pts / (ms_e2e * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(xh.numel() * 4), "d2h_bytes_per_step": int(yh.numel() * yh.element_size()),
                    "pinned_copy_gbs": link,
                    # the slower direction alone, at its measured one-way rate
                    "link_bound_ms": max(xh.numel() * 4 / (link["h2d_gbs"] * 1e9),
                                         yh.numel() * yh.element_size() / (link["d2h_gbs"] * 1e9)) * 1e3},
            "gpu_launches": plan.launches(3 if packed else 0) * args.steps,
            "clocks": ck,
            "accuracy": accuracy,
            "accuracy_whole_volume": whole if whole is None or "outs" not in whole else None,
            "compare": compare,
            "secondary": extra,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
