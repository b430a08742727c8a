"""FP64 oracle for the FCC cosine transform (Seifert, Hueper, Uhl 2018).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product library never loads it and shares no code with it.

Contents (each function names the passage it follows):

* ``weyl_group``      -- closure of the printed generators s1, s2, s3 (Sec. 3).
* ``chebyshev``       -- T_k(theta) = (1/24) sum_w exp(2 pi i (w k).theta),
                         the power form of Sec. 3 / Def. 1.
* ``sample_points``   -- theta_{i,l,q} = ((r+i)/n, (s+l)/n, (t+q)/n)
                         (Lemma 1, Lemma 2, Def. 2).
* ``dct_matrix``      -- the explicit matrix form of Def. 2 (rows = points,
                         columns = basis polynomials, lexicographic).
* ``forward_rows`` / ``adjoint_rows`` -- y = D x and D^H g evaluated row by
                         row from the definition (C, exact integer phases).
* ``forward_dense`` / ``adjoint_dense`` / ``inverse_dense`` -- the same with
                         the dense matrix; the inverse is an LU solve.
* ``forward_sum_fft`` / ``adjoint_sum_fft`` -- the definition with the two
                         sums (over k and over w) exchanged and the inner
                         exponential sum over the grid done by a library FFT.
                         Pinned against ``dct_matrix`` in the tests.
* ``conjugate_partner`` / ``pack_hermitian`` / ``unpack_hermitian`` -- the
                         involution pi of the point grid under which the
                         values of a real input come in conjugate pairs
                         (-theta is a W-image of theta_pi(a) modulo Z^3,
                         Lemma 1 / Def. 2 with Prop. 1 (iii)), and the layout
                         that stores those n^3 complex values as n^3 reals.
* ``oracle.radix2``   -- the radix-2x2x2 factorisation of Sec. 4.B (eq.
                         FastAlgorithm) with the basis change B_n derived
                         from its definition; a second, recursive FP64
                         evaluation of the transform at n = 2^k.
* ``chebyshev_recurrence`` -- an independent second evaluator: T_k from the
                         values x = T_100, y = T_010, z = T_001 through the
                         mother recurrence (Prop. 1 (iv)) with l = e_j and
                         W-invariance (Prop. 1 (iii)).

Readings of the paper taken here: W acts on k from the left (the power form
is authoritative over the w^T of Prop. 1); the forward map sends
coefficients to point values (rows = points); no normalisation besides the
1/24 inside T_k; the skew parameter of DCT_{n x n x n} is (1/8, 0, 3/8).
"""
import ctypes
import functools
import os

import numpy as np

from .build import build_oracle

CANONICAL_SKEW = ((1, 0, 3), 8)   # (r, s, t) = (1/8, 0, 3/8), Def. 2

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.fcc_oracle_weyl_group.argtypes = [i32p, ctypes.c_int]
        L.fcc_oracle_weyl_group.restype = ctypes.c_int
        L.fcc_oracle_chebyshev.argtypes = [i32p, f64p, f64p, f64p]
        L.fcc_oracle_chebyshev.restype = None
        L.fcc_oracle_matrix.argtypes = [ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, ctypes.c_int]
        L.fcc_oracle_matrix.restype = ctypes.c_int
        for name in ("fcc_oracle_forward_rows", "fcc_oracle_adjoint_rows"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, i64p, ctypes.c_int64,
                          f64p, f64p, ctypes.c_int]
            f.restype = ctypes.c_int
        L.fcc_oracle_max_threads.argtypes = []
        L.fcc_oracle_max_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def max_threads():
    return lib().fcc_oracle_max_threads()


@functools.lru_cache(maxsize=None)
def _weyl_group_cached():
    out = np.zeros(24 * 9, dtype=np.int32)
    m = lib().fcc_oracle_weyl_group(_ptr(out, ctypes.c_int), 24)
    if m != 24:
        raise RuntimeError("generator closure has order %d, expected 24" % m)
    return out.reshape(24, 3, 3).astype(np.int64)


def weyl_group():
    """The 24 matrices of W generated by the printed s1, s2, s3 (Sec. 3)."""
    return _weyl_group_cached().copy()


def chebyshev(k, theta):
    """T_k(theta) for integer k (3,) and real theta (3,): orbit sum (Def. 1,
    power form of Sec. 3)."""
    kk = np.ascontiguousarray(np.asarray(k, dtype=np.int32).reshape(3))
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(3))
    re = ctypes.c_double()
    im = ctypes.c_double()
    lib().fcc_oracle_chebyshev(_ptr(kk, ctypes.c_int), _ptr(th, ctypes.c_double),
                               ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def sample_points(n, skew=CANONICAL_SKEW):
    """theta_{i,l,q} = ((r+i)/n, (s+l)/n, (t+q)/n), lexicographic (Lemma 2)."""
    a, d = skew
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    idx = idx.reshape(-1, 3).astype(np.float64)
    return (np.asarray(a, dtype=np.float64) / d + idx) / n


def dct_matrix(n, skew=CANONICAL_SKEW, nthreads=0):
    """Dense DCT_{n x n x n}(r,s,t) of Def. 2: D[point, coefficient]."""
    a, d = skew
    N = n ** 3
    if N > 4096:
        raise ValueError("dense matrix only for n^3 <= 4096")
    re = np.zeros((N, N))
    im = np.zeros((N, N))
    aa = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    rc = lib().fcc_oracle_matrix(n, _ptr(aa, ctypes.c_int), d, _ptr(re, ctypes.c_double),
                                 _ptr(im, ctypes.c_double), nthreads)
    if rc:
        raise RuntimeError("fcc_oracle_matrix failed")
    return re + 1j * im


def _rows_call(name, vol, n, rows, skew, nthreads):
    a, d = skew
    vol = np.asarray(vol).reshape(-1)
    if vol.size != n ** 3:
        raise ValueError("volume must hold n^3 values")
    re = np.ascontiguousarray(vol.real, dtype=np.float64)
    im = np.ascontiguousarray(vol.imag, dtype=np.float64) if np.iscomplexobj(vol) else None
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
    if rows.size and (rows.min() < 0 or rows.max() >= n ** 3):
        raise ValueError("row index out of range")
    ore = np.zeros(rows.size)
    oim = np.zeros(rows.size)
    aa = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    rc = getattr(lib(), name)(n, _ptr(aa, ctypes.c_int), d, _ptr(re, ctypes.c_double),
                              _ptr(im, ctypes.c_double) if im is not None else None,
                              _ptr(rows, ctypes.c_int64), rows.size,
                              _ptr(ore, ctypes.c_double), _ptr(oim, ctypes.c_double), nthreads)
    if rc:
        raise RuntimeError(name + " failed")
    return ore + 1j * oim


def forward_rows(x, n, rows, skew=CANONICAL_SKEW, nthreads=0):
    """(D x)[rows] for one volume x of n^3 coefficients (Def. 2, row by row)."""
    return _rows_call("fcc_oracle_forward_rows", x, n, rows, skew, nthreads)


def adjoint_rows(g, n, cols, skew=CANONICAL_SKEW, nthreads=0):
    """(D^H g)[cols] for one volume g of n^3 point values."""
    return _rows_call("fcc_oracle_adjoint_rows", g, n, cols, skew, nthreads)


def _flat_batch(v, n):
    v = np.asarray(v)
    return v.reshape(-1, n ** 3)


def forward_dense(x, n, skew=CANONICAL_SKEW):
    """y = D x with the dense matrix; x has shape (..., n, n, n)."""
    D = dct_matrix(n, skew)
    shape = np.asarray(x).shape
    return (_flat_batch(x, n) @ D.T).reshape(shape)


def adjoint_dense(g, n, skew=CANONICAL_SKEW):
    D = dct_matrix(n, skew)
    shape = np.asarray(g).shape
    return (_flat_batch(g, n) @ D.conj()).reshape(shape)


def inverse_dense(y, n, skew=CANONICAL_SKEW):
    """x = D^{-1} y by an LU solve (the CRT isomorphism of Lemma 2 is
    invertible because the n^3 zeros are distinct)."""
    D = dct_matrix(n, skew)
    shape = np.asarray(y).shape
    return np.linalg.solve(D, _flat_batch(y, n).T).T.reshape(shape)


def _orbit_maps(n, skew):
    """For every w: the flat index of (w k mod n) and the phase numerator
    (w k).a mod (d n) for all k in lexicographic order."""
    a, d = skew
    W = weyl_group()
    k = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    k = k.reshape(-1, 3)
    out = []
    for w in W:
        wk = k @ w.T
        kap = np.mod(wk, n)
        flat = (kap[:, 0] * n + kap[:, 1]) * n + kap[:, 2]
        num = np.mod(wk @ np.asarray(a), d * n)
        out.append((flat, np.exp(2j * np.pi * num / (d * n))))
    return out


def forward_sum_fft(x, n, skew=CANONICAL_SKEW):
    """y = D x with the sums exchanged:

        y[idx] = sum_kappa Z[kappa] exp(+2 pi i kappa.idx / n),
        Z[kappa] = (1/24) sum_{(k,w): w k = kappa mod n} x_k exp(2 pi i (w k).a/(d n)),

    i.e. the power form at theta_idx = (a/d + idx)/n split into its shift
    part and its grid part; the grid part is an unnormalised 3-D inverse DFT
    (numpy's ifftn times n^3).  x: (..., n, n, n)."""
    shape = np.asarray(x).shape
    xb = _flat_batch(x, n).astype(np.complex128)
    Z = np.zeros_like(xb)
    for flat, ph in _orbit_maps(n, skew):
        Z[:, flat] += xb * ph        # k -> w k mod n is a bijection per w
    Z /= 24.0
    y = np.fft.ifftn(Z.reshape(-1, n, n, n), axes=(1, 2, 3)) * (n ** 3)
    return y.reshape(shape)


def adjoint_sum_fft(g, n, skew=CANONICAL_SKEW):
    """D^H g with the same exchange of sums: x[k] = (1/24) sum_w
    conj(exp(2 pi i (w k).a/(d n))) G[w k mod n], G = unnormalised forward
    DFT of g."""
    shape = np.asarray(g).shape
    gb = _flat_batch(g, n).astype(np.complex128)
    G = np.fft.fftn(gb.reshape(-1, n, n, n), axes=(1, 2, 3)).reshape(gb.shape)
    x = np.zeros_like(G)
    for flat, ph in _orbit_maps(n, skew):
        x += G[:, flat] * np.conj(ph)
    x /= 24.0
    return x.reshape(shape)


# ---------------------------------------------------------------------------
# Independent second evaluator: the mother recurrence (Prop. 1 (iv)).
# ---------------------------------------------------------------------------

def dominant(k):
    """Move an integer weight into the dominant chamber (all coordinates >= 0)
    with the printed simple reflections s1, s2, s3 (Sec. 3)."""
    k = [int(v) for v in k]
    while True:
        if k[0] < 0:
            k = [-k[0], k[0] + k[1], k[2]]
        elif k[1] < 0:
            k = [k[0] + k[1], -k[1], k[1] + k[2]]
        elif k[2] < 0:
            k = [k[0], k[1] + k[2], -k[2]]
        else:
            return tuple(k)


def chebyshev_recurrence(kmax, x, y, z):
    """T_k for every k in [0, kmax)^3 from x = T_100, y = T_010, z = T_001.

    Uses only Prop. 1 (i)-(iv): T_0 = 1, T_{e_j} = x_j, T_{wk} = T_k and
    T_{e_j} T_m = (1/24) sum_w T_{m + w e_j}.  Solving that product for its
    leading term gives T_k from weights strictly lower in dominance order.
    x, y, z may be numpy arrays (evaluated point-wise).  Returns a dict
    {k: value}."""
    W = weyl_group()
    E = [np.eye(3, dtype=np.int64)[j] for j in range(3)]
    orbit = [[tuple(int(c) for c in (w @ E[j])) for w in W] for j in range(3)]
    gen = [np.asarray(x), np.asarray(y), np.asarray(z)]
    memo = {(0, 0, 0): np.ones_like(gen[0] * 1.0 + 0j)}

    def T(k):
        k = dominant(k)
        if k in memo:
            return memo[k]
        j = next(i for i in range(3) if k[i] >= 1)
        m = (k[0] - E[j][0], k[1] - E[j][1], k[2] - E[j][2])
        lhs = 24.0 * gen[j] * T(m)
        same = 0
        rest = 0
        for u in orbit[j]:
            t = dominant((m[0] + u[0], m[1] + u[1], m[2] + u[2]))
            if t == k:
                same += 1
            else:
                rest = rest + T(t)
        memo[k] = (lhs - rest) / same
        return memo[k]

    return {(a, b, c): T((a, b, c)) for a in range(kmax) for b in range(kmax) for c in range(kmax)}


# ---------------------------------------------------------------------------
# Conjugate pairs of point values of a real input, and the packed layout.
# ---------------------------------------------------------------------------

def conjugate_partner(n):
    """pi(i, l, q) = ((i - l) mod n, (-l) mod n, (q - l) mod n) as flat point
    indices.  With c = (1/8, 0, 3/8): -theta_{i,l,q} differs from
    theta_{pi(i,l,q)} by a W-image modulo Z^3, so for real x
    (D x)[pi(a)] = conj((D x)[a]) (T_k is W-invariant, Prop. 1 (iii))."""
    out = np.empty(n ** 3, dtype=np.int64)
    for i in range(n):
        for l in range(n):
            for q in range(n):
                out[(i * n + l) * n + q] = (((i - l) % n) * n + (-l) % n) * n + (q - l) % n
    return out


def packed_primary(n):
    """Points whose real part the packed layout stores: 2l < n, or 2l = n and
    2q < n (row l = 0, the fixed points of pi, included)."""
    i, l, q = np.indices((n, n, n)).reshape(3, -1)   # flat point index (i n + l) n + q
    return (2 * l < n) | ((2 * l == n) & (2 * q < n))


def pack_hermitian(y, n):
    """n^3 complex point values with y[pi(a)] = conj(y[a]) -> n^3 reals:
    Re y[a] at primary points, -Im y[a] (the imaginary part at the primary
    partner) elsewhere.  Works on the last axis of a batch [..., n^3]."""
    y = np.asarray(y).reshape(-1, n ** 3)
    prim = packed_primary(n)
    return np.where(prim[None, :], y.real, -y.imag)


def unpack_hermitian(pk, n):
    """Inverse of pack_hermitian: y[a] = pk[a] + i pk[pi(a)] at a primary point
    off the row l = 0, pk[a] on that row, pk[pi(a)] - i pk[a] elsewhere."""
    pk = np.asarray(pk, dtype=np.float64).reshape(-1, n ** 3)
    pi = conjugate_partner(n)
    prim = packed_primary(n)
    row0 = np.indices((n, n, n)).reshape(3, -1)[1] == 0
    y = np.empty(pk.shape, dtype=np.complex128)
    y[:, prim] = pk[:, prim] + 1j * np.where(row0[prim][None, :], 0.0, pk[:, pi[prim]])
    y[:, ~prim] = pk[:, pi[~prim]] - 1j * pk[:, ~prim]
    return y
