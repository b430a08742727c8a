"""The radix-2x2x2 factorisation of Sec. 4.B (eq. FastAlgorithm) in FP64, on
the CPU: a second evaluation of DCT_{n x n x n}(r,s,t) that shares with the
dense definition only the 2 x 2 x 2 transform.

B_n^{-1} is built symbolically (mother recurrence, W-invariance, reduction by
the ideal <T_{n e_j} - sigma_j>), so the identity
D_n B_n^{-1} = P_n (sum_i D_m((c+i)/2)) (D_2 (x) 1) checks the dense matrix of
Def. 2 at four families of shifts against the algebra it comes from.
"""
import numpy as np
import pytest

import oracle
from oracle import radix2

RNG = np.random.default_rng(1807)
SKEWS = [oracle.CANONICAL_SKEW, ((1, 0, 11), 16)]


@pytest.mark.parametrize("skew", SKEWS)
@pytest.mark.parametrize("n", [2, 4, 8])
def test_factorisation_identity(n, skew):
    Binv = radix2.basis_change_inverse(n, skew)
    lhs = oracle.dct_matrix(n, skew) @ Binv
    rhs = radix2.factor_product(n, skew)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_order_two_step_is_the_identity_basis_change():
    """m = 1: b~_2 = (T_{efg}(T_100, T_010, T_001)) = b_2, so B_2 = 1 and P_2 = 1."""
    for skew in SKEWS:
        assert np.abs(radix2.basis_change_inverse(2, skew) - np.eye(8)).max() < 1e-15
    assert (radix2.point_permutation(2) == np.arange(8)).all()


@pytest.mark.parametrize("m", [2, 3, 5])
def test_composition_property(m):
    """T_{efg}(T_{m00}, T_{0m0}, T_{00m}) = T_{m(e,f,g)}: T_{efg} as the
    polynomial in x, y, z of the recurrence evaluator, evaluated at the
    order-m generators, against the orbit sum at m (e,f,g)."""
    for _ in range(4):
        th = RNG.random(3)
        gens = [oracle.chebyshev(m * np.eye(3, dtype=np.int64)[j], th) for j in range(3)]
        T = oracle.chebyshev_recurrence(2, *gens)
        for k, val in T.items():
            assert abs(val - oracle.chebyshev(m * np.array(k), th)) < 1e-12, (k, th)


@pytest.mark.parametrize("skew", SKEWS)
@pytest.mark.parametrize("n", [4, 8])
def test_recursion_matches_dense_definition(n, skew):
    x = RNG.standard_normal((2, n ** 3)) + 1j * RNG.standard_normal((2, n ** 3))
    ref = x @ oracle.dct_matrix(n, skew).T
    y = radix2.forward_radix2(x, n, skew)
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


def test_ideal_constants_vanish_at_the_canonical_shift():
    """sigma, tau, rho are zero at (1/8, 0, 3/8) (Sec. 4.A), so the reduction
    of the canonical basis change has no constant term."""
    assert max(abs(v) for v in radix2.ideal_values(oracle.CANONICAL_SKEW)) < 1e-15
    assert min(abs(v) for v in radix2.ideal_values(((1, 0, 11), 16))) > 1e-3


def test_dropped_ideal_constant_is_caught(monkeypatch):
    """A planted mistake: the reduction with sigma = tau = rho = 0 at a skew
    shift breaks the identity."""
    skew = ((1, 0, 11), 16)
    monkeypatch.setattr(radix2, "ideal_values", lambda s: [0j, 0j, 0j])
    Binv = radix2.basis_change_inverse.__wrapped__(4, skew)
    assert np.abs(oracle.dct_matrix(4, skew) @ Binv - radix2.factor_product(4, skew)).max() > 1e-3


def test_wrong_point_permutation_is_caught(monkeypatch):
    """A planted mistake: P_n sending row (i, k) to 2i + k instead of i + 2k."""
    n = 4
    good = radix2.point_permutation

    def swapped(m2):
        m = m2 // 2
        perm = good(m2).copy()
        for row in range(m2 ** 3):
            i, k = divmod(row, m ** 3)
            i0, i1, i2 = (i >> 2) & 1, (i >> 1) & 1, i & 1
            k0, k1, k2 = k // (m * m), (k // m) % m, k % m
            perm[row] = ((2 * i0 + k0) * m2 + (2 * i1 + k1)) * m2 + (2 * i2 + k2)
        return perm

    monkeypatch.setattr(radix2, "point_permutation", swapped)
    lhs = oracle.dct_matrix(n) @ radix2.basis_change_inverse(n)
    assert np.abs(lhs - radix2.factor_product(n)).max() > 1e-3


def test_sub_shift_without_halving_is_caught(monkeypatch):
    """A planted mistake: the sub-transforms at c + i instead of (c + i)/2."""
    n = 4
    monkeypatch.setattr(radix2, "sub_shift", lambda skew, i: (tuple(int(skew[0][a]) + int(i[a]) * skew[1]
                                                                    for a in range(3)), skew[1]))
    lhs = oracle.dct_matrix(n) @ radix2.basis_change_inverse(n)
    assert np.abs(lhs - radix2.factor_product(n)).max() > 1e-3
