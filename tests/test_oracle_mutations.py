"""Planted mistakes in the oracle must trip at least one pin (CPU only).

Each case swaps one ingredient of the oracle for a plausible wrong one and
checks that the corresponding pin predicate rejects it.
"""
import numpy as np

import oracle
from tests import goldens

RNG = np.random.default_rng(77)


def _power_form_ok(W):
    E = goldens.power_form()
    k = np.array([2, 5, 9])
    return sorted(tuple(e @ k) for e in E) == sorted(tuple(w @ k) for w in W)


def test_transposed_group_action_is_caught(monkeypatch):
    assert _power_form_ok(oracle.weyl_group())
    Wt = np.transpose(oracle.weyl_group(), (0, 2, 1)).copy()
    assert not _power_form_ok(Wt)
    # and the exchanged-sum form built on it leaves the dense definition
    monkeypatch.setattr(oracle, "weyl_group", lambda: Wt)
    n = 3
    x = RNG.standard_normal((n, n, n))
    monkeypatch.undo()
    ref = oracle.forward_dense(x, n)
    monkeypatch.setattr(oracle, "weyl_group", lambda: Wt)
    bad = oracle.forward_sum_fft(x, n)
    assert np.abs(bad - ref).max() > 1e-3


def test_wrong_skew_is_caught():
    n = 4
    good = oracle.sample_points(n)
    e = np.array([n, 0, 0])
    assert max(abs(oracle.chebyshev(e, t)) for t in good) < 1e-13
    # a dropped offset and a mistyped one (3/8 -> 1/8)
    for skew in (((0, 0, 0), 8), ((1, 0, 1), 8)):
        bad = oracle.sample_points(n, skew=skew)
        assert max(abs(oracle.chebyshev(e, t)) for t in bad) > 1e-3


def test_wrong_dft_sign_is_caught(monkeypatch):
    n = 4
    x = RNG.standard_normal((n, n, n)) + 1j * RNG.standard_normal((n, n, n))
    ref = oracle.forward_dense(x, n)
    monkeypatch.setattr(oracle.np.fft, "ifftn", lambda a, axes=None: np.fft.fftn(a, axes=axes) / n ** 3)
    assert np.abs(oracle.forward_sum_fft(x, n) - ref).max() > 1e-3


def test_dropped_normalisation_is_caught():
    th = RNG.random(3)
    t0 = oracle.chebyshev((0, 0, 0), th)
    assert abs(t0 - 1) < 1e-15 and abs(24 * t0 - 1) > 1


def test_wrong_packed_rule_is_caught(monkeypatch):
    """Row n/2 taken whole as primary (both points of its pairs) or the
    partner map with the wrong sign of the slow shift: the packed round trip
    of D x breaks."""
    n = 4
    D = oracle.dct_matrix(n)
    x = RNG.standard_normal(n ** 3)
    y = D @ x
    good = oracle.unpack_hermitian(oracle.pack_hermitian(y, n), n)[0]
    assert np.abs(good - y).max() < 1e-12
    keep = oracle.packed_primary
    monkeypatch.setattr(oracle, "packed_primary",
                        lambda m: np.array([2 * ((a // m) % m) <= m for a in range(m ** 3)]))
    assert np.abs(oracle.unpack_hermitian(oracle.pack_hermitian(y, n), n)[0] - y).max() > 1e-3
    monkeypatch.setattr(oracle, "packed_primary", keep)
    bad_pi = np.array([((((a // (n * n)) + (a // n) % n) % n) * n + (-(a // n)) % n) * n + (a % n - (a // n) % n) % n
                       for a in range(n ** 3)])
    monkeypatch.setattr(oracle, "conjugate_partner", lambda m: bad_pi)
    assert np.abs(oracle.unpack_hermitian(oracle.pack_hermitian(y, n), n)[0] - y).max() > 1e-3


def test_dropped_wrap_in_the_exchanged_sum_is_caught(monkeypatch):
    """The exchanged-sum form with the phase taken at the reduced member
    (w k mod n) instead of w k itself drops the 8th-root wrap factor of the
    power form at theta = (c + idx)/n; the row pin at a large order catches it."""
    n = 16
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, n, n, n))
    rows = rng.integers(0, n ** 3, size=16)
    ref = oracle.forward_rows(x[0], n, rows)
    assert np.abs(oracle.forward_sum_fft(x, n).reshape(-1)[rows] - ref).max() < 1e-10

    def bad_maps(m, skew):
        a, d = skew
        k = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
        out = []
        for w in oracle.weyl_group():
            kap = np.mod(k @ w.T, m)
            flat = (kap[:, 0] * m + kap[:, 1]) * m + kap[:, 2]
            out.append((flat, np.exp(2j * np.pi * np.mod(kap @ np.asarray(a), d * m) / (d * m))))
        return out

    monkeypatch.setattr(oracle, "_orbit_maps", bad_maps)
    assert np.abs(oracle.forward_sum_fft(x, n).reshape(-1)[rows] - ref).max() > 1e-3 * np.abs(ref).max()
