"""Pins for the FP64 oracle against what the paper fixes (CPU only).

Every check compares the oracle with something other than itself: matrices,
monomials and zeros transcribed from the paper (tests/golden/), closed
forms, an independent recurrence evaluator, or brute force on tiny orders.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests import goldens

RNG = np.random.default_rng(1234)


def _T(k, theta):
    return oracle.chebyshev(k, theta)


# --- Weyl group (Sec. 3, generator matrices and relations) -----------------

def _order(m):
    p = np.eye(3, dtype=np.int64)
    for i in range(1, 50):
        p = p @ m
        if (p == np.eye(3)).all():
            return i
    return None


def test_weyl_group_is_generated_by_printed_matrices():
    gens, printed, corrected, order = goldens.generators()
    W = oracle.weyl_group()
    assert len(W) == order == 24
    keys = {tuple(w.ravel()) for w in W}
    assert len(keys) == 24
    for s in gens.values():
        assert tuple(s.ravel()) in keys
        assert (s @ s == np.eye(3)).all()
    for a in W:                                  # closed under products / inverses
        assert abs(round(np.linalg.det(a))) == 1
        for b in W:
            assert tuple((a @ b).ravel()) in keys
    s1, s2, s3 = gens["s1"], gens["s2"], gens["s3"]
    got = {"s1s2": _order(s1 @ s2), "s1s3": _order(s1 @ s3), "s2s3": _order(s2 @ s3)}
    assert got == corrected
    # The printed (s1 s2)^2 = 1 and (s1 s3)^3 = 1 do not hold (misprint).
    assert got["s1s2"] != printed["s1s2"] and got["s1s3"] != printed["s1s3"]
    assert got["s2s3"] == printed["s2s3"]


# --- Power form (Sec. 3) -----------------------------------------------------

@pytest.mark.parametrize("trial", range(5))
def test_orbit_exponents_equal_printed_power_form(trial):
    E = goldens.power_form()
    k = RNG.integers(-9, 10, size=3)
    printed = sorted(tuple(int(v) for v in e @ k) for e in E)
    W = oracle.weyl_group()
    left = sorted(tuple(int(v) for v in w @ k) for w in W)
    assert left == printed
    # The literal w^T k of Prop. 1 gives a different set (reading: left action).
    transposed = sorted(tuple(int(v) for v in w.T @ k) for w in W)
    if len(set(printed)) == 24:
        assert transposed != printed


def test_power_form_value_matches_printed_monomials():
    E = goldens.power_form()
    for _ in range(5):
        k = RNG.integers(-4, 5, size=3)
        th = RNG.random(3)
        uvw = np.exp(2j * np.pi * th)
        printed = np.mean([np.prod(uvw ** (e @ k)) for e in E])
        assert abs(_T(k, th) - printed) < 1e-13


# --- Prop. 1 and the parametrization ---------------------------------------

def test_generators_of_the_polynomial_ring_are_x_y_z():
    polys = goldens.polynomials()
    for _ in range(10):
        th = RNG.random(3)
        assert abs(_T((0, 0, 0), th) - 1) < 1e-15                   # Prop. 1 (i)
        assert abs(_T((1, 0, 0), th) - goldens.eval_poly(polys["x"], th)) < 1e-14
        assert abs(_T((0, 1, 0), th) - goldens.eval_poly(polys["y"], th)) < 1e-14
        assert abs(_T((0, 0, 1), th) - goldens.eval_poly(polys["z"], th)) < 1e-14
        # x and z are complex conjugates, y is real (Sec. 3).
        assert abs(np.conj(goldens.eval_poly(polys["x"], th)) - goldens.eval_poly(polys["z"], th)) < 1e-14
        assert abs(goldens.eval_poly(polys["y"], th).imag) < 1e-14


def test_conjugation_bounds_and_value_at_origin():
    for _ in range(20):
        k = RNG.integers(0, 7, size=3)
        th = RNG.random(3)
        t = _T(k, th)
        assert abs(np.conj(t) - _T(k[::-1], th)) < 1e-13            # x-bar = z
        assert abs(t) <= 1 + 1e-13
        assert abs(_T(k, np.zeros(3)) - 1) < 1e-14
        w = oracle.weyl_group()[RNG.integers(24)]
        assert abs(t - _T(w @ k, th)) < 1e-13                       # Prop. 1 (iii)


def test_independent_recurrence_evaluator_agrees():
    polys = goldens.polynomials()
    th = RNG.random((6, 3))
    x, y, z = (goldens.eval_poly(polys[c], th) for c in "xyz")
    table = oracle.chebyshev_recurrence(6, x, y, z)
    worst = 0.0
    for k, vals in table.items():
        for p in range(len(th)):
            worst = max(worst, abs(vals[p] - _T(k, th[p])))
    # the recurrence amplifies rounding (about 4e-11 at k = (5,5,5));
    # a dropped or mis-signed term gives errors of order one
    assert worst < 1e-9


def test_mother_recurrence():
    W = oracle.weyl_group()
    for _ in range(6):
        k = RNG.integers(-3, 4, size=3)
        l = RNG.integers(-3, 4, size=3)
        th = RNG.random(3)
        rhs = np.mean([_T(k + w @ l, th) for w in W])
        assert abs(_T(k, th) * _T(l, th) - rhs) < 1e-13


@pytest.mark.parametrize("ell", [2, 3])
def test_decomposition_property(ell):
    """Prop. 1 (vi): T_{k l e_j} = T_{k e_j} o (T_{l e1}, T_{l e2}, T_{l e3})."""
    th = RNG.random((4, 3))
    xl = [np.array([_T(ell * np.eye(3, dtype=int)[j], t) for t in th]) for j in range(3)]
    comp = oracle.chebyshev_recurrence(4, *xl)
    for j in range(3):
        for k in range(1, 4):
            e = np.zeros(3, dtype=int)
            e[j] = k
            direct = np.array([_T(ell * e, t) for t in th])
            assert np.abs(comp[tuple(e)] - direct).max() < 1e-11


# --- Lemma 1, Lemma 2, sigma / tau / rho ------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_lemma1_common_zeros(n):
    g = goldens.lemma1()
    th = oracle.sample_points(n)
    assert th.shape == (n ** 3, 3)
    idx = np.array(list(itertools.product(range(n), repeat=3)))
    # theta = ((1+8i)/(8n), 8j/(8n), (3+8k)/(8n)) as printed
    want = np.stack([(1 + 8 * idx[:, 0]) / (8 * n), (8 * idx[:, 1]) / (8 * n),
                     (3 + 8 * idx[:, 2]) / (8 * n)], 1)
    assert g["u"] == "1 + 8*i" and g["w"] == "3 + 8*k"
    assert np.abs(th - want).max() < 1e-15
    assert len({tuple(np.round(np.exp(2j * np.pi * t), 12)) for t in th}) == n ** 3
    for t in th:
        for e in np.eye(3, dtype=int):
            assert abs(_T(n * e, t)) < 1e-13
    if n == 8:
        assert len(th) == int(g["count_n8"])


def test_sigma_tau_rho_vanish_at_the_skew_zero():
    polys = goldens.polynomials()
    r = [float(eval(v)) for v in goldens.lemma1()["skew_zero"].split()]
    for c in ("sigma", "tau", "rho"):
        assert abs(goldens.eval_poly(polys[c], np.array(r))) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 4])
def test_lemma2_skew_zeros(n):
    """At theta = ((r+i)/n, (s+j)/n, (t+k)/n): T_{n00} = sigma, T_{0n0} = tau,
    T_{00n} = rho (the system of Sec. 4.A)."""
    polys = goldens.polynomials()
    for _ in range(3):
        rst = RNG.random(3)
        rhs = [goldens.eval_poly(polys[c], rst) for c in ("sigma", "tau", "rho")]
        for i, j, k in itertools.product(range(n), repeat=3):
            th = (rst + np.array([i, j, k])) / n
            for a, e in enumerate(np.eye(3, dtype=int)):
                assert abs(_T(n * e, th) - rhs[a]) < 1e-13


# --- The matrix of Def. 2 ----------------------------------------------------

def test_order_one_is_identity():
    D = oracle.dct_matrix(1)
    assert D.shape == (1, 1) and abs(D[0, 0] - 1) < 1e-15


@pytest.mark.parametrize("n", [2, 3])
def test_matrix_entries_are_chebyshev_at_points(n):
    D = oracle.dct_matrix(n)
    th = oracle.sample_points(n)
    ks = list(itertools.product(range(n), repeat=3))
    for r in range(n ** 3):
        for c, k in enumerate(ks):
            assert abs(D[r, c] - _T(k, th[r])) < 1e-13


def test_matrix_order2_from_recurrence():
    """DCT_{2x2x2}: every entry rebuilt by the independent recurrence."""
    polys = goldens.polynomials()
    th = oracle.sample_points(2)
    x, y, z = (goldens.eval_poly(polys[c], th) for c in "xyz")
    tab = oracle.chebyshev_recurrence(2, x, y, z)
    ks = list(itertools.product(range(2), repeat=3))
    R = np.stack([tab[k] for k in ks], 1)
    assert np.abs(R - oracle.dct_matrix(2)).max() < 1e-13


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_invertible_and_well_conditioned(n):
    D = oracle.dct_matrix(n)
    cond = np.linalg.cond(D)
    assert cond < 20.0
    y = RNG.standard_normal(n ** 3) + 1j * RNG.standard_normal(n ** 3)
    x = oracle.inverse_dense(y, n)
    assert np.linalg.norm(D @ x - y) / np.linalg.norm(y) < 1e-12


@pytest.mark.parametrize("n", [4, 6])
def test_shift_property(n):
    """ASP shift: D (T_100 * p mod I) = x(theta) . (D p) for p supported away
    from the box edges (Sec. 2, Sec. 4.A: T_100 is a shift)."""
    W = oracle.weyl_group()
    orbit_e1 = [tuple(int(v) for v in w @ np.array([1, 0, 0])) for w in W]
    p = np.zeros((n, n, n))
    p[1:n - 1, 1:n - 1, 1:n - 1] = RNG.standard_normal((n - 2,) * 3)
    q = np.zeros((n, n, n))
    for k in itertools.product(range(1, n - 1), repeat=3):
        for u in orbit_e1:
            q[k[0] + u[0], k[1] + u[1], k[2] + u[2]] += p[k] / 24.0
    D = oracle.dct_matrix(n)
    xs = np.array([_T((1, 0, 0), t) for t in oracle.sample_points(n)])
    lhs = D @ q.reshape(-1)
    rhs = xs * (D @ p.reshape(-1))
    assert np.abs(lhs - rhs).max() < 1e-12
    # The transposed reading (rows = coefficients) breaks it.
    assert np.abs(D.T @ q.reshape(-1) - xs * (D.T @ p.reshape(-1))).max() > 1e-3


# --- The row evaluators and the exchanged-sum form -------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8])
def test_sum_fft_form_matches_dense(n):
    x = RNG.standard_normal((2, n, n, n)) + 1j * RNG.standard_normal((2, n, n, n))
    ref = oracle.forward_dense(x, n)
    assert np.abs(oracle.forward_sum_fft(x, n) - ref).max() < 1e-12 * max(1, n ** 1.5)
    assert np.abs(oracle.adjoint_sum_fft(x, n) - oracle.adjoint_dense(x, n)).max() < 1e-12 * max(1, n ** 1.5)


def _orbit_size_mod_n(k, n):
    W = oracle.weyl_group()
    return len({tuple(int(c) for c in np.mod(w @ np.asarray(k), n)) for w in W})


def _special_indices(n, rng, want):
    """Flat indices of the grid that sit on the walls of the fundamental
    alcove {k >= 0, k1 + k2 + k3 <= n} modulo n, i.e. whose W-orbit in
    Z_n^3 has fewer than 24 members (the boundary classes of the orbit
    partition), plus the corners of the box."""
    out = [0, n ** 3 - 1]
    tries = 0
    while len(out) < want and tries < 20000:
        tries += 1
        k = rng.integers(0, n, size=3)
        c = rng.integers(0, 5)
        if c == 0:
            k[rng.integers(0, 3)] = 0
        elif c == 1:
            k[2] = (n - k[0] - k[1]) % n
        elif c == 2:
            k[1] = k[0]
        elif c == 3:
            k[:] = [k[0], 0, k[0]]
        else:
            k[:] = [(n // 2) * rng.integers(0, 2), (n // 2) * rng.integers(0, 2), (n // 2) * rng.integers(0, 2)]
        if _orbit_size_mod_n(k, n) < 24:
            out.append(int((k[0] * n + k[1]) * n + k[2]))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("n", [16, 24, 40, 64, 96, 128])
def test_sum_fft_form_matches_definition_rows_at_large_orders(n):
    """The exchanged-sum + FFT form (the full-volume comparator of the GPU
    tests) against the plain definition of Def. 2 evaluated row by row in C
    with exact integer phases: 48 uniform rows and 16 rows/columns on the
    alcove walls (non-free orbits, where the wrap of w k modulo n and the
    coinciding slots matter), forward and adjoint, complex input."""
    rng = np.random.default_rng(1000 + n)
    x = rng.standard_normal((1, n, n, n)) + 1j * rng.standard_normal((1, n, n, n))
    idx = np.concatenate([rng.integers(0, n ** 3, size=48), _special_indices(n, rng, 16)])
    sizes = [_orbit_size_mod_n(np.unravel_index(i, (n, n, n)), n) for i in idx[48:]]
    assert min(sizes) < 24 and len(idx) == 64
    y = oracle.forward_sum_fft(x, n).reshape(-1)
    ref = oracle.forward_rows(x[0], n, idx)
    scale = np.sqrt(np.mean(np.abs(y) ** 2))
    assert np.abs(y[idx] - ref).max() < 1e-13 * n * scale, np.abs(y[idx] - ref).max() / scale
    a = oracle.adjoint_sum_fft(x, n).reshape(-1)
    aref = oracle.adjoint_rows(x[0], n, idx)
    scale = np.sqrt(np.mean(np.abs(a) ** 2))
    assert np.abs(a[idx] - aref).max() < 1e-13 * n * scale, np.abs(a[idx] - aref).max() / scale


@pytest.mark.parametrize("n", [3, 5])
def test_row_evaluators_match_dense(n):
    x = RNG.standard_normal((n, n, n)) + 1j * RNG.standard_normal((n, n, n))
    rows = RNG.integers(0, n ** 3, size=20)
    assert np.abs(oracle.forward_rows(x, n, rows) - oracle.forward_dense(x, n).reshape(-1)[rows]).max() < 1e-12
    assert np.abs(oracle.adjoint_rows(x, n, rows) - oracle.adjoint_dense(x, n).reshape(-1)[rows]).max() < 1e-12
    xr = x.real.copy()
    assert np.abs(oracle.forward_rows(xr, n, rows) - oracle.forward_dense(xr, n).reshape(-1)[rows]).max() < 1e-12


def test_adjoint_identity():
    n = 6
    x = RNG.standard_normal(n ** 3) + 1j * RNG.standard_normal(n ** 3)
    g = RNG.standard_normal(n ** 3) + 1j * RNG.standard_normal(n ** 3)
    lhs = np.vdot(oracle.forward_sum_fft(x.reshape(n, n, n), n).reshape(-1), g)
    rhs = np.vdot(x, oracle.adjoint_sum_fft(g.reshape(n, n, n), n).reshape(-1))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


# --- Conjugate pairs of rows for real input (used to pair real volumes) ------

def _pi(n):
    """pi(i, l, q) = (i - l, -l, q - l) mod n on flat point indices."""
    idx = np.array(list(itertools.product(range(n), repeat=3)))
    p = np.stack([(idx[:, 0] - idx[:, 1]) % n, (-idx[:, 1]) % n, (idx[:, 2] - idx[:, 1]) % n], 1)
    return (p[:, 0] * n + p[:, 1]) * n + p[:, 2]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_rows_come_in_conjugate_pairs(n):
    """D[pi(r), :] = conj(D[r, :]): -theta_r is a W-image of theta_pi(r) modulo
    Z^3, and T_k is W-invariant with integer-periodic exponents (Prop. 1 (iii))."""
    D = oracle.dct_matrix(n)
    pi = _pi(n)
    assert (pi[pi] == np.arange(n ** 3)).all()
    assert np.abs(D[pi] - np.conj(D)).max() < 1e-13


@pytest.mark.parametrize("n", [3, 4, 5])
def test_pairing_identities(n):
    """One complex transform serves two real volumes; Re(D^-1 y) = D^-1 P(y) and
    Re(D^H y) = D^H P(y) with P(y) = (y + conj(y o pi)) / 2."""
    D = oracle.dct_matrix(n)
    pi = _pi(n)
    N = n ** 3
    x1, x2 = RNG.standard_normal(N), RNG.standard_normal(N)
    Y = D @ (x1 + 1j * x2)
    assert np.abs((Y + np.conj(Y[pi])) / 2 - D @ x1).max() < 1e-12
    assert np.abs((Y - np.conj(Y[pi])) / 2j - D @ x2).max() < 1e-12
    y = RNG.standard_normal(N) + 1j * RNG.standard_normal(N)
    P = (y + np.conj(y[pi])) / 2
    assert np.abs(np.linalg.solve(D, P) - np.linalg.solve(D, y).real).max() < 1e-12
    assert np.abs(D.conj().T @ P - (D.conj().T @ y).real).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_packed_layout_keeps_exactly_the_point_values(n):
    """The packed layout of real inputs: the oracle's pi pairs the rows of the
    dense matrix of Def. 2 into conjugates, every 2-cycle of pi has exactly one
    primary point and every fixed point (row l = 0, n^2 of them) is primary,
    unpack(pack(D x)) = D x, D^-1 unpack(pack(D x)) = x, and every real
    vector is the packing of exactly one conjugate-symmetric vector."""
    D = oracle.dct_matrix(n)
    pi = oracle.conjugate_partner(n)
    prim = oracle.packed_primary(n)
    assert np.abs(D[pi] - np.conj(D)).max() < 1e-13
    fixed = pi == np.arange(n ** 3)
    assert fixed.sum() == n * n
    assert prim[fixed].all()
    assert (prim[~fixed] != prim[pi[~fixed]]).all()
    x = RNG.standard_normal((3, n ** 3))
    y = (D @ x.T).T
    pk = oracle.pack_hermitian(y, n)
    assert pk.shape == (3, n ** 3) and pk.dtype == np.float64
    assert np.abs(oracle.unpack_hermitian(pk, n) - y).max() < 1e-13 * max(1.0, np.abs(y).max())
    assert np.abs(np.linalg.solve(D, oracle.unpack_hermitian(pk, n).T).T - x).max() < 1e-11
    r = RNG.standard_normal(n ** 3)
    u = oracle.unpack_hermitian(r, n)[0]
    assert np.abs(u[pi] - np.conj(u)).max() == 0
    assert np.abs(oracle.pack_hermitian(u, n)[0] - r).max() == 0
