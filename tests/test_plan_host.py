"""Host logic of the CUDA library, checked on the CPU.

The library exports its orbit tables (fcc_dct_describe, no CUDA call).  Here
the per-orbit algorithm the kernels run is replayed in numpy from those
tables -- gather 24 slots, class core, row phase, scatter; then the 3-D DFT
-- and compared with the oracle's plain definition.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1807_10058_gb300 import binding

RNG = np.random.default_rng(5)
CANONICAL = ((1, 0, 3), 8)


def _tables(n, skew=CANONICAL):
    d = binding.describe(n, skew)
    d["W"] = binding.weyl_group()
    d["v"], d["d"] = np.array(skew[0]), skew[1]
    return d


def _slots(d, n, o):
    k = d["reps"][o]
    c = d["cls"][o]
    p = d["W"] @ k                           # (24, 3) unreduced slots
    kap = p - n * d["wrap"][c]
    assert kap.min() >= 0 and kap.max() < n
    idx = (kap[:, 0] * n + kap[:, 1]) * n + kap[:, 2]
    M = d["d"] * n
    R = np.exp(2j * np.pi * np.mod(p @ d["v"], M) / M)
    canon = d["canon"][c] == np.arange(24)
    return c, idx, R, canon


def emulate(d, n, vol, mode):
    N = n ** 3
    vol = np.asarray(vol, dtype=np.complex128).reshape(N)
    out = np.zeros(N, dtype=np.complex128)
    if mode == "fwd":
        src = vol
    elif mode == "inv":
        src = np.fft.fftn(vol.reshape(n, n, n)).reshape(N) / N
    else:
        src = np.fft.fftn(vol.reshape(n, n, n)).reshape(N)
    for o in range(len(d["reps"])):
        c, idx, R, canon = _slots(d, n, o)
        if mode == "fwd":
            z = R * (d["fwd"][c] @ src[idx])
            out[idx[canon]] = z[canon]
        else:
            t = np.where(canon, np.conj(R) * src[idx], 0)
            x = d[mode][c] @ t
            out[idx[canon]] = x[canon]
    if mode == "fwd":
        out = np.fft.ifftn(out.reshape(n, n, n)).reshape(N) * N
    return out.reshape(n, n, n)


def test_library_group_equals_oracle_group():
    a = {tuple(w.ravel()) for w in binding.weyl_group()}
    b = {tuple(w.ravel()) for w in oracle.weyl_group()}
    assert a == b and len(a) == 24


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 24])
def test_orbits_partition_the_grid(n):
    d = _tables(n)
    seen = np.zeros(n ** 3, dtype=int)
    for o in range(len(d["reps"])):
        k = d["reps"][o]
        assert k.min() >= 0 and k.sum() <= n            # closed alcove
        c, idx, R, canon = _slots(d, n, o)
        seen[idx[canon]] += 1
        assert len(set(idx[canon])) == canon.sum() == len(set(idx))
    assert (seen == 1).all()
    if n <= 4:
        # no free orbit: the open alcove is empty, or (n=4) its only point
        # (1,1,1) is fixed by the rotation of the extended diagram
        assert d["free_class"] == -1
    else:
        fc = d["free_class"]
        assert fc == 0
        core = d["fwd"][fc] * 24
        assert np.allclose(np.abs(core), 1)               # 8th roots of unity
        assert np.allclose(np.mod(np.angle(core) / (2 * np.pi / 8) + 0.5, 1), 0.5)
        frac = (d["cls"] == fc).sum() * 24 / n ** 3
        assert frac > (0.6 if n >= 16 else 0.1)


@pytest.mark.parametrize("n", [8, 16, 24, 32, 64, 128])
def test_tiles_partition_the_orbits(n):
    """The tiles the mixing kernels walk: at most 32 orbits of one class each,
    every orbit in exactly one tile, the free class first; each free tile is a
    whole 4 x 4 x 2 box of (a', b', c') = (k1+k2+k3, k1+k2, k1) or a full run
    of 32 orbits of cut boxes (the last one may be short), and no free tile
    could be merged with another: at most one short free tile, and the box
    tiles are exactly the boxes the alcove leaves whole."""
    d = binding.describe(n)
    off, nfree, tk = binding.describe_tiles(n)
    sizes = np.diff(off)
    assert off[0] == 0 and (sizes >= 1).all() and (sizes <= 32).all()
    key = lambda k: tuple(k.tolist())
    order_cls = {key(k): c for k, c in zip(d["reps"], d["cls"])}
    assert sorted(map(key, tk)) == sorted(map(key, d["reps"]))          # a partition of the orbits
    tcls = np.array([order_cls[key(k)] for k in tk])
    for t in range(len(sizes)):
        c = tcls[off[t]:off[t + 1]]
        assert (c == c[0]).all(), t                                     # class-pure
        assert (t < nfree) == (c[0] == d["free_class"]), t               # free tiles first
    if nfree == 0:
        return
    free = d["reps"][d["cls"] == d["free_class"]]
    box_of = lambda k: ((k[:, 0] + k[:, 1] + k[:, 2]) // 4, (k[:, 0] + k[:, 1]) // 4, k[:, 0] // 2)
    ba, bb, bc = box_of(free)
    _, counts = np.unique(np.stack([ba, bb, bc], 1), axis=0, return_counts=True)
    whole = (counts == 32).sum()
    short = 0
    box_tiles = 0
    for t in range(nfree):
        k = tk[off[t]:off[t + 1]]
        a, b, c = box_of(k)
        one_box = len(set(zip(a.tolist(), b.tolist(), c.tolist()))) == 1
        if len(k) == 32 and one_box:
            box_tiles += 1
        short += len(k) < 32
    assert short <= 1
    assert box_tiles == whole   # a merged tile of 32 cannot come from one cut box
    cut = len(free) - 32 * whole
    assert nfree == whole + (cut + 31) // 32, (nfree, whole, cut)


@pytest.mark.parametrize("n", [32, 64, 96, 128])
def test_slot_indices_stay_in_the_grid_at_large_orders(n):
    """The host-side bounds check of the tables the kernels index with, at the
    large orders: for every orbit and slot, the reduced image W_g k - n wrap
    lies in [0, n)^3 (so every gather and scatter address lies inside its
    volume), and the canonical slots cover each grid point exactly once."""
    d = _tables(n)
    reps, cls = d["reps"].astype(np.int64), d["cls"].astype(np.int64)
    assert reps.min() >= 0 and reps.sum(axis=1).max() <= n
    p = np.einsum("gij,oj->ogi", d["W"].astype(np.int64), reps)        # (orbits, 24, 3)
    kap = p - n * d["wrap"][cls].astype(np.int64)
    assert kap.min() >= 0 and kap.max() < n
    idx = (kap[..., 0] * n + kap[..., 1]) * n + kap[..., 2]
    canon = d["canon"][cls] == np.arange(24)[None, :]
    seen = np.bincount(idx[canon], minlength=n ** 3)
    assert seen.shape == (n ** 3,) and (seen == 1).all()
    # the free class's wraps are the ones the free-tile kernels build in at
    # compile time: -1 in row r of slot g exactly where that row of W_g sums
    # to a negative number (a negated positive form on the open alcove)
    fc = d["free_class"]
    fw = np.where(d["W"].sum(axis=2) < 0, -1, 0)
    assert (d["wrap"][fc] == fw).all()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 12])
def test_emulated_forward_inverse_adjoint_match_oracle(n):
    d = _tables(n)
    x = RNG.standard_normal((n, n, n)) + 1j * RNG.standard_normal((n, n, n))
    D = oracle.dct_matrix(n)
    y = (D @ x.reshape(-1)).reshape(n, n, n)
    assert np.abs(emulate(d, n, x, "fwd") - y).max() < 1e-11 * max(1, n ** 1.5)
    assert np.abs(emulate(d, n, y, "inv") - x).max() < 1e-11 * max(1, n ** 1.5)
    g = RNG.standard_normal((n, n, n)) + 1j * RNG.standard_normal((n, n, n))
    ah = (D.conj().T @ g.reshape(-1)).reshape(n, n, n)
    assert np.abs(emulate(d, n, g, "adj") - ah).max() < 1e-11 * max(1, n ** 1.5)


def test_emulated_forward_order_24_sampled_rows():
    n = 24
    d = _tables(n)
    x = RNG.standard_normal((n, n, n))
    y = emulate(d, n, x, "fwd").reshape(-1)
    rows = RNG.integers(0, n ** 3, size=12)
    assert np.abs(y[rows] - oracle.forward_rows(x, n, rows)).max() < 1e-10


# shifts of DCT_n(r,s,t): the halved shifts (c + a)/2 of the radix-2 step
# (invertible), c + e1 (the canonical points moved by one grid step), a shift
# with a denominator that is not a power of two, and two singular ones
SKEWS = [((1, 0, 11), 16), ((9, 8, 11), 16), ((1, 0, 3), 32), ((9, 0, 3), 8), ((5, 3, 1), 24), ((0, 0, 0), 1),
         ((1, 1, 1), 4)]


@pytest.mark.parametrize("skew", SKEWS)
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_emulated_skew_transforms_match_oracle(n, skew):
    d = _tables(n, skew)
    D = oracle.dct_matrix(n, skew)
    sv = np.linalg.svd(D, compute_uv=False)
    # the plan's block test agrees with the rank of the dense matrix
    assert d["invertible"] == (sv[-1] > 1e-9 * sv[0])
    x = RNG.standard_normal((n, n, n)) + 1j * RNG.standard_normal((n, n, n))
    y = (D @ x.reshape(-1)).reshape(n, n, n)
    tol = 1e-11 * max(1, n ** 1.5)
    assert np.abs(emulate(d, n, x, "fwd") - y).max() < tol
    g = RNG.standard_normal((n, n, n)) + 1j * RNG.standard_normal((n, n, n))
    ah = (D.conj().T @ g.reshape(-1)).reshape(n, n, n)
    assert np.abs(emulate(d, n, g, "adj") - ah).max() < tol
    if d["invertible"]:
        assert np.abs(emulate(d, n, y, "inv") - x).max() < tol * sv[0] / sv[-1]
    else:   # some class block is singular: its inverse core is left zero
        assert any(not np.any(m) for m in d["inv"])


def test_equal_shifts_give_equal_cores():
    a = binding.describe(12, CANONICAL)
    b = binding.describe(12, ((2, 0, 6), 16))
    assert np.array_equal(a["reps"], b["reps"]) and np.array_equal(a["cls"], b["cls"])
    for m in ("fwd", "inv", "adj"):
        assert np.abs(a[m] - b[m]).max() < 1e-15


@pytest.mark.parametrize("n", [8, 12, 16])
def test_phase_free_forward_factorisation(n):
    """The phase-free form of the tensor-core forward, replayed from the
    library's host tables: with W_g kO = kappa_g + n m_g the row phase is
    w_{8n}^{kappa_g . v} w_8^{m_g . v}; row g of each class core times
    w_8^{m_g . v}, the sums scattered without phase, then the separable
    modulation w_{8n}^{kappa_1} w_{8n}^{3 kappa_3} / 24 and the + sign DFT give
    D x of the oracle."""
    d = binding.describe(n)
    W = binding.weyl_group().reshape(24, 3, 3).astype(np.int64)
    v = np.array([1, 0, 3])
    M = 8 * n
    x = np.random.default_rng(n).standard_normal((n, n, n))
    Zf = np.zeros((n, n, n), complex)
    for o, k in enumerate(d["reps"]):
        c = d["cls"][o]
        wrap, canon = d["wrap"][c], d["canon"][c]
        kap = W @ k - n * wrap
        cg = np.exp(2j * np.pi * ((wrap @ v) % 8) / 8)
        vals = cg * ((24 * d["fwd"][c]) @ x[kap[:, 0], kap[:, 1], kap[:, 2]])
        for g in range(24):
            if canon[g] == g:
                Zf[tuple(kap[g])] = vals[g]
    idx = np.arange(n)
    Z = Zf * np.exp(2j * np.pi * idx / M)[:, None, None] * np.exp(2j * np.pi * 3 * idx / M)[None, None, :] / 24
    y = np.fft.ifftn(Z) * n ** 3
    ref = oracle.forward_sum_fft(x, n).reshape(n, n, n)
    assert np.abs(y - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n", [8, 16, 24, 40, 64, 88, 96, 128])
def test_pencil_pair_enumeration_writes_the_packed_layout(n):
    """Replay of the fused split pass's pencil enumeration: primary pencils
    (l, q) for l = 0 .. n/2 (row n/2: q < n/2) store Re y at their points,
    their partners (n - l, q - l) (none for l = 0) store -Im y.  Every point of
    the volume is written exactly once, Re exactly at the oracle's primary
    points, and the partner pencil holds pi of the primary pencil's points."""
    wrote = np.zeros((n, n, n), dtype=np.int8)     # +1 Re, -1 -Im
    count = np.zeros((n, n, n), dtype=np.int32)
    pi = oracle.conjugate_partner(n).reshape(n, n, n)
    k = np.arange(n)
    for l in range(n // 2 + 1):
        qlim = n // 2 if 2 * l == n else n
        for q in range(qlim):
            wrote[k, l, q] = 1
            count[k, l, q] += 1
            if l == 0:
                continue
            lp, qp = (n - l) % n, (q - l) % n
            wrote[k, lp, qp] = -1
            count[k, lp, qp] += 1
            # the counterpart of primary index k sits at k - l on the partner pencil
            assert (pi[k, l, q] == ((k - l) % n) * n * n + lp * n + qp).all()
    assert (count == 1).all()
    assert ((wrote.reshape(-1) == 1) == oracle.packed_primary(n)).all()
