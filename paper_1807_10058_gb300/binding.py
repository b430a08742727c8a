"""Thin ctypes binding of libfccdct (include/fcc_dct.h).

Argument marshalling only: tensors are passed as device pointers together
with torch's current CUDA stream; every step of the transform runs in the
library's CUDA kernels.  If the library is missing this module raises --
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfccdct.so")

FCC_OK, FCC_ERR_INVALID_ARG, FCC_ERR_UNSUPPORTED, FCC_ERR_ALLOC, FCC_ERR_CUDA, FCC_ERR_TIMEOUT = range(6)
DTYPES = {"r64": 0, "c64": 1, "r32": 2, "c32": 3, "r32_tf32x3": 4, "r32_bf16x3": 5, "r32_bf16x6": 6}
EXPORTS = [
    "fcc_dct_plan", "fcc_dct_plan_ragged", "fcc_dct_forward", "fcc_dct_inverse", "fcc_dct_adjoint",
    "fcc_dct_forward_host", "fcc_dct_inverse_host", "fcc_dct_batch", "fcc_dct_points",
    "fcc_dct_in_bytes", "fcc_dct_out_bytes", "fcc_dct_launches", "fcc_dct_last_error",
    "fcc_status_string", "fcc_dct_destroy", "fcc_dct_describe", "fcc_dct_weyl_group",
    "fcc_dct_profile_enable", "fcc_dct_profile_read", "fcc_dct_inverse_static", "fcc_dct_check",
    "fcc_dct_set_schedule", "fcc_dct_get_schedule", "fcc_dct_autotune", "fcc_dct_test_wait_timeout",
    "fcc_dct_plan_skew", "fcc_dct_describe_skew", "fcc_dct_forward_packed", "fcc_dct_inverse_packed",
    "fcc_dct_forward_packed_host", "fcc_dct_inverse_packed_host", "fcc_dct_test_fail_alloc",
    "fcc_dct_test_allocations", "fcc_dct_plan_radix2", "fcc_dct_radix2_stats",
    "fcc_render_cells", "fcc_dct_diag_mixing_replay", "fcc_dct_describe_tiles",
]

# execution-schedule keys (fcc_sched_key)
SCHED = {"chunk_mb": 0, "streams": 1, "ragged": 2, "tc_blocks": 3, "tc_fold": 4}

_LIB = None


class FccError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_string(status), status))


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfccdct.so is not built (run __graft_entry__.build()); "
                               "there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.fcc_dct_plan.argtypes = [i32, i32, i32]
        L.fcc_dct_plan.restype = vp
        L.fcc_dct_plan_ragged.argtypes = [ctypes.POINTER(i32), i32, i32]
        L.fcc_dct_plan_ragged.restype = vp
        L.fcc_dct_plan_skew.argtypes = [i32, i32, i32, ctypes.POINTER(i32), i32]
        L.fcc_dct_plan_skew.restype = vp
        L.fcc_dct_plan_radix2.argtypes = [i32, i32, i32, ctypes.POINTER(i32), i32]
        L.fcc_dct_plan_radix2.restype = vp
        L.fcc_dct_radix2_stats.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]
        L.fcc_dct_radix2_stats.restype = i32
        f32 = ctypes.c_float
        L.fcc_render_cells.argtypes = [vp, i32, i32, f32, f32, f32, f32, i32, i32, vp, vp]
        L.fcc_render_cells.restype = i32
        L.fcc_dct_describe_skew.argtypes = [i32, ctypes.POINTER(i32), i32, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                            ctypes.POINTER(i32), ctypes.POINTER(i32)] + [vp] * 7
        L.fcc_dct_describe_skew.restype = i32
        for f in ("fcc_dct_forward", "fcc_dct_inverse", "fcc_dct_adjoint", "fcc_dct_forward_host",
                  "fcc_dct_inverse_host", "fcc_dct_inverse_static", "fcc_dct_forward_packed",
                  "fcc_dct_inverse_packed", "fcc_dct_forward_packed_host", "fcc_dct_inverse_packed_host",
                  "fcc_dct_diag_mixing_replay"):
            getattr(L, f).argtypes = [vp, vp, vp, vp]
            getattr(L, f).restype = i32
        L.fcc_dct_batch.argtypes = [vp]
        L.fcc_dct_batch.restype = i32
        for f in ("fcc_dct_points", "fcc_dct_in_bytes", "fcc_dct_out_bytes"):
            getattr(L, f).argtypes = [vp]
            getattr(L, f).restype = i64
        L.fcc_dct_launches.argtypes = [vp, i32]
        L.fcc_dct_launches.restype = i32
        L.fcc_dct_check.argtypes = [vp]
        L.fcc_dct_check.restype = i32
        L.fcc_dct_last_error.argtypes = []
        L.fcc_dct_last_error.restype = i32
        L.fcc_status_string.argtypes = [i32]
        L.fcc_status_string.restype = ctypes.c_char_p
        L.fcc_dct_destroy.argtypes = [vp]
        L.fcc_dct_destroy.restype = None
        L.fcc_dct_describe.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                       vp, vp, vp, vp, vp, vp, vp]
        L.fcc_dct_describe.restype = i32
        L.fcc_dct_describe_tiles.argtypes = [i32, vp, vp, vp, vp]
        L.fcc_dct_describe_tiles.restype = i32
        L.fcc_dct_weyl_group.argtypes = [vp]
        L.fcc_dct_weyl_group.restype = i32
        L.fcc_dct_profile_enable.argtypes = [vp, i32]
        L.fcc_dct_profile_enable.restype = i32
        L.fcc_dct_profile_read.argtypes = [vp, vp, vp, vp, i32]
        L.fcc_dct_profile_read.restype = i32
        L.fcc_dct_set_schedule.argtypes = [vp, i32, i32]
        L.fcc_dct_set_schedule.restype = i32
        L.fcc_dct_get_schedule.argtypes = [vp, i32]
        L.fcc_dct_get_schedule.restype = i32
        L.fcc_dct_autotune.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(ctypes.c_float)]
        L.fcc_dct_autotune.restype = i32
        L.fcc_dct_test_wait_timeout.argtypes = [vp, i32]
        L.fcc_dct_test_wait_timeout.restype = i32
        L.fcc_dct_test_fail_alloc.argtypes = [i32]
        L.fcc_dct_test_fail_alloc.restype = i32
        L.fcc_dct_test_allocations.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.fcc_dct_test_allocations.restype = i64
        _LIB = L
    return _LIB


def status_string(s):
    return lib().fcc_status_string(int(s)).decode()


def last_error():
    return lib().fcc_dct_last_error()


def _check(status, what):
    if status != FCC_OK:
        raise FccError(status, what)


def describe(order, skew=None):
    """Host-side orbit tables of the plan builder (no GPU needed).  skew:
    ((v0, v1, v2), d) for the shift v / d of DCT_n(r,s,t), None for (1/8, 0, 3/8)."""
    L = lib()
    v, d = skew if skew is not None else ((1, 0, 3), 8)
    varr = (ctypes.c_int * 3)(*[int(a) for a in v])
    inv_ok = ctypes.c_int()
    no, nc, fc = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    _check(L.fcc_dct_describe_skew(order, varr, int(d), ctypes.byref(inv_ok), ctypes.byref(no), ctypes.byref(nc),
                                   ctypes.byref(fc), None, None, None, None, None, None, None), "describe")
    reps = np.zeros(no.value, dtype=np.uint32)
    cls = np.zeros(no.value, dtype=np.int32)
    wrap = np.zeros(nc.value * 72, dtype=np.int32)
    canon = np.zeros(nc.value * 24, dtype=np.int32)
    mats = [np.zeros(nc.value * 576 * 2) for _ in range(3)]
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(L.fcc_dct_describe_skew(order, varr, int(d), ctypes.byref(inv_ok), ctypes.byref(no), ctypes.byref(nc),
                                   ctypes.byref(fc), ptr(reps), ptr(cls), ptr(wrap), ptr(canon), ptr(mats[0]),
                                   ptr(mats[1]), ptr(mats[2])), "describe")
    cx = [(m[0::2] + 1j * m[1::2]).reshape(nc.value, 24, 24) for m in mats]
    k = np.stack([reps & 1023, (reps >> 10) & 1023, (reps >> 20) & 1023], 1).astype(np.int64)
    return {"reps": k, "cls": cls, "free_class": fc.value, "wrap": wrap.reshape(-1, 24, 3),
            "canon": canon.reshape(-1, 24), "fwd": cx[0], "inv": cx[1], "adj": cx[2],
            "invertible": bool(inv_ok.value)}


def describe_tiles(order):
    """Host-side tile layout of the mixing kernels at the canonical shift (no
    GPU needed): (tile offsets, free-class tile count, representatives (k1, k2,
    k3) in tile order)."""
    L = lib()
    nt, nf = ctypes.c_int32(), ctypes.c_int32()
    _check(L.fcc_dct_describe_tiles(order, ctypes.byref(nt), ctypes.byref(nf), None, None), "describe_tiles")
    off = np.zeros(nt.value + 1, dtype=np.int32)
    _check(L.fcc_dct_describe_tiles(order, None, None, off.ctypes.data_as(ctypes.c_void_p), None), "describe_tiles")
    reps = np.zeros(int(off[-1]), dtype=np.uint32)
    _check(L.fcc_dct_describe_tiles(order, None, None, None, reps.ctypes.data_as(ctypes.c_void_p)), "describe_tiles")
    k = np.stack([reps & 1023, (reps >> 10) & 1023, (reps >> 20) & 1023], 1).astype(np.int64)
    return off, nf.value, k


def allocations():
    """(allocations made so far, live plans, device bytes the live plans own)."""
    plans, dev = ctypes.c_int64(), ctypes.c_int64()
    seq = lib().fcc_dct_test_allocations(ctypes.byref(plans), ctypes.byref(dev))
    return seq, plans.value, dev.value


CELLS = {"cube": 0, "rhombic_dodecahedron": 1}


def render_cells(volume, n, cells="rhombic_dodecahedron", azimuth=0.6, elevation=0.4, kappa=4.0, step=0.05,
                 width=256, height=256, image=None):
    """Grey-level image of an n^3 FP32 device volume drawn as lattice cells
    (fcc_render_cells): cubes or the rhombic dodecahedra of the FCC lattice."""
    import torch
    if image is None:
        image = torch.empty(height * width, dtype=torch.float32, device=volume.device)
    st = torch.cuda.current_stream(volume.device).cuda_stream
    _check(lib().fcc_render_cells(ctypes.c_void_p(volume.data_ptr()), int(n), CELLS[cells], float(azimuth),
                                  float(elevation), float(kappa), float(step), int(width), int(height),
                                  ctypes.c_void_p(image.data_ptr()), ctypes.c_void_p(st)), "fcc_render_cells")
    return image


def weyl_group():
    out = np.zeros(216, dtype=np.int32)
    _check(lib().fcc_dct_weyl_group(out.ctypes.data_as(ctypes.c_void_p)), "weyl_group")
    return out.reshape(24, 3, 3).astype(np.int64)


_REAL_T = {0: "float64", 1: "float64", 2: "float32", 3: "float32", 4: "float32", 5: "float32", 6: "float32"}


class Plan:
    """A device plan for `batch` volumes of order `order` (or a ragged list of
    orders).  skew = ((v0, v1, v2), d): the skew transform DCT_n(r,s,t) with
    (r, s, t) = v / d (uniform batches).  Owns the library handle; release
    with close() or `with`."""

    def __init__(self, order=None, batch=1, dtype="r32", orders=None, skew=None, radix2=False):
        import torch  # noqa: F401  (initialises the CUDA context torch uses)
        L = lib()
        self.dtype_code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        if radix2:
            v, d = skew if skew is not None else ((1, 0, 3), 8)
            varr = (ctypes.c_int * 3)(*[int(a) for a in v])
            h = L.fcc_dct_plan_radix2(int(order), int(batch), self.dtype_code, varr, int(d))
            self.orders = [int(order)] * int(batch)
        elif orders is not None:
            arr = (ctypes.c_int * len(orders))(*[int(o) for o in orders])
            h = L.fcc_dct_plan_ragged(arr, len(orders), self.dtype_code)
            self.orders = [int(o) for o in orders]
        elif skew is not None:
            v, d = skew
            varr = (ctypes.c_int * 3)(*[int(a) for a in v])
            h = L.fcc_dct_plan_skew(int(order), int(batch), self.dtype_code, varr, int(d))
            self.orders = [int(order)] * int(batch)
        else:
            h = L.fcc_dct_plan(int(order), int(batch), self.dtype_code)
            self.orders = [int(order)] * int(batch)
        if not h:
            raise FccError(L.fcc_dct_last_error(), "fcc_dct_plan")
        self.handle = ctypes.c_void_p(h)
        self.batch = L.fcc_dct_batch(self.handle)
        self.points = L.fcc_dct_points(self.handle)
        self.real_input = self.dtype_code not in (1, 3)
        self.real_type = _REAL_T[self.dtype_code]

    def close(self):
        if getattr(self, "handle", None):
            lib().fcc_dct_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def radix2_stats(self, level):
        """Radix-2 plans: (non-zeros per row of B_level, its largest |entry|,
        shifts at that level), or the complex multiply-adds per point of one
        transform for level 0."""
        nz, mx, macs = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        r = lib().fcc_dct_radix2_stats(self.handle, int(level), ctypes.byref(nz), ctypes.byref(mx), ctypes.byref(macs))
        if r < 0:
            raise FccError(last_error(), "fcc_dct_radix2_stats")
        return macs.value if level == 0 else (nz.value, mx.value, r)

    def check(self):
        """Synchronise and raise if a device-side wait of an earlier call timed out."""
        _check(lib().fcc_dct_check(self.handle), "fcc_dct_check")

    def launches(self, which=0):
        return lib().fcc_dct_launches(self.handle, which)

    def set_schedule(self, **kw):
        """Execution schedule knobs: chunk_mb, streams, ragged (0 per-order
        launches, 1 one persistent launch, 2 per run of equal orders), tc_blocks."""
        for k, v in kw.items():
            _check(lib().fcc_dct_set_schedule(self.handle, SCHED[k], int(v)), "set_schedule(%s)" % k)

    def schedule(self):
        return {k: lib().fcc_dct_get_schedule(self.handle, v) for k, v in SCHED.items()}

    def autotune(self, x, out, reps=3):
        """Time the forward transform under the candidate schedules, keep the
        fastest; returns (ms per call, schedule).  Synchronises the stream."""
        import torch
        best = ctypes.c_float(0.0)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().fcc_dct_autotune(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(st), int(reps), ctypes.byref(best)), "autotune")
        return best.value, self.schedule()

    def profile(self, enable=True):
        _check(lib().fcc_dct_profile_enable(self.handle, 1 if enable else 0), "profile_enable")

    def profile_read(self, cap=32):
        """{kernel name: (total ms, launches)} recorded since the last read."""
        names = ctypes.create_string_buffer(48 * cap)
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_int * cap)()
        k = lib().fcc_dct_profile_read(self.handle, names, ms, cnt, cap)
        if k < 0:
            raise FccError(last_error(), "profile_read")
        raw = names.raw
        return {raw[48 * i:48 * i + 48].split(b"\0")[0].decode(): (ms[i], cnt[i]) for i in range(min(k, cap))}

    # -- tensor helpers -------------------------------------------------------
    def _torch_types(self):
        import torch
        rt = torch.float64 if self.real_type == "float64" else torch.float32
        ct = torch.complex128 if rt == torch.float64 else torch.complex64
        return rt, ct

    def _shape_out(self, t, complex_):
        import torch
        rt, ct = self._torch_types()
        return torch.empty(self.points, dtype=ct if complex_ else rt, device=t.device)

    def _call(self, fn, what, x, out, out_complex):
        import torch
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("input must be a contiguous CUDA tensor")
        if out is None:
            out = self._shape_out(x, out_complex)
        else:   # the C ABI takes plain pointers: the sizes are checked here
            rt, ct = self._torch_types()
            want = ct if out_complex else rt
            if not out.is_cuda or not out.is_contiguous() or out.dtype != want or out.numel() != self.points:
                raise ValueError("%s: out must be a contiguous CUDA %s tensor with %d elements"
                                 % (what, want, self.points))
        st = torch.cuda.current_stream(x.device).cuda_stream
        _check(fn(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                  ctypes.c_void_p(st)), what)
        return out

    def forward(self, x, out=None):
        rt, ct = self._torch_types()
        want = rt if self.real_input else ct
        if x.dtype != want or x.numel() != self.points:
            raise ValueError("forward input must be %s with %d elements" % (want, self.points))
        return self._call(lib().fcc_dct_forward, "fcc_dct_forward", x, out, True)

    def inverse(self, y, out=None):
        rt, ct = self._torch_types()
        if y.dtype != ct or y.numel() != self.points:
            raise ValueError("inverse input must be %s with %d elements" % (ct, self.points))
        return self._call(lib().fcc_dct_inverse, "fcc_dct_inverse", y, out, not self.real_input)

    def adjoint(self, g, out=None):
        rt, ct = self._torch_types()
        if g.dtype != ct or g.numel() != self.points:
            raise ValueError("adjoint input must be %s with %d elements" % (ct, self.points))
        return self._call(lib().fcc_dct_adjoint, "fcc_dct_adjoint", g, out, not self.real_input)

    def mixing_replay(self, x, out):
        """Measurement aid: the forward tensor-core mixing's memory accesses with
        no arithmetic (fcc_dct_diag_mixing_replay); `out` (the forward's output
        size) receives meaningless values."""
        rt, _ = self._torch_types()
        if not self.real_input or x.dtype != rt or x.numel() != self.points:
            raise ValueError("replay input must be %s with %d elements (real plans)" % (rt, self.points))
        return self._call(lib().fcc_dct_diag_mixing_replay, "fcc_dct_diag_mixing_replay", x, out, True)

    def forward_packed(self, x, out=None):
        """Hermitian-packed forward of a real plan: n^3 reals per volume
        (fcc_dct_forward_packed; layout in include/fcc_dct.h)."""
        rt, _ = self._torch_types()
        if not self.real_input or x.dtype != rt or x.numel() != self.points:
            raise ValueError("packed forward input must be %s with %d elements (real plans)" % (rt, self.points))
        return self._call(lib().fcc_dct_forward_packed, "fcc_dct_forward_packed", x, out, False)

    def inverse_packed(self, pk, out=None):
        """Inverse of forward_packed (fcc_dct_inverse_packed)."""
        rt, _ = self._torch_types()
        if not self.real_input or pk.dtype != rt or pk.numel() != self.points:
            raise ValueError("packed inverse input must be %s with %d elements (real plans)" % (rt, self.points))
        return self._call(lib().fcc_dct_inverse_packed, "fcc_dct_inverse_packed", pk, out, False)

    def _need_host(self, t, what, complex_):
        """A host buffer of the plan's size (the C ABI cannot check it)."""
        rt, ct = self._torch_types()
        want = ct if complex_ else rt
        if t.is_cuda or not t.is_contiguous() or t.dtype != want or t.numel() != self.points:
            raise ValueError("%s: host buffers must be contiguous CPU %s tensors with %d elements"
                             % (what, want, self.points))

    def forward_packed_host(self, x_host, pk_host):
        """forward_packed with host tensors (as forward_host)."""
        import torch
        self._need_host(x_host, "fcc_dct_forward_packed_host", False)
        self._need_host(pk_host, "fcc_dct_forward_packed_host", False)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().fcc_dct_forward_packed_host(self.handle, ctypes.c_void_p(x_host.data_ptr()),
                                                 ctypes.c_void_p(pk_host.data_ptr()), ctypes.c_void_p(st)),
               "fcc_dct_forward_packed_host")
        return pk_host

    def inverse_packed_host(self, pk_host, x_host):
        """inverse_packed with host tensors (as forward_host)."""
        import torch
        self._need_host(pk_host, "fcc_dct_inverse_packed_host", False)
        self._need_host(x_host, "fcc_dct_inverse_packed_host", False)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().fcc_dct_inverse_packed_host(self.handle, ctypes.c_void_p(pk_host.data_ptr()),
                                                 ctypes.c_void_p(x_host.data_ptr()), ctypes.c_void_p(st)),
               "fcc_dct_inverse_packed_host")
        return x_host

    def inverse_host(self, y_host, x_host):
        """End-to-end inverse with host tensors (see forward_host)."""
        import torch
        self._need_host(y_host, "fcc_dct_inverse_host", True)
        self._need_host(x_host, "fcc_dct_inverse_host", not self.real_input)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().fcc_dct_inverse_host(self.handle, ctypes.c_void_p(y_host.data_ptr()),
                                          ctypes.c_void_p(x_host.data_ptr()), ctypes.c_void_p(st)),
               "fcc_dct_inverse_host")
        return x_host

    def forward_host(self, x_host, y_host):
        """End-to-end call with host tensors (pinned for async copies); the
        caller synchronises the current stream before reading y_host."""
        import torch
        self._need_host(x_host, "fcc_dct_forward_host", not self.real_input)
        self._need_host(y_host, "fcc_dct_forward_host", True)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().fcc_dct_forward_host(self.handle, ctypes.c_void_p(x_host.data_ptr()),
                                          ctypes.c_void_p(y_host.data_ptr()), ctypes.c_void_p(st)),
               "fcc_dct_forward_host")
        return y_host
