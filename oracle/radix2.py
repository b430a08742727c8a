"""The radix-2x2x2 factorisation of DCT_{n x n x n}(r,s,t) (Sec. 4.B, eq.
FastAlgorithm) in FP64: a second, recursive evaluation of the transform.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

For n = 2m the paper factors

    D_n(c) = P_n . (direct sum over i in {0,1}^3 of D_m((c + i)/2))
                 . (D_2(c) (x) 1_{m^3}) . B_n(c)

and leaves the basis change B_n to future work.  Here B_n follows from its
definition.  b_n = (T_{jkp}), 0 <= j,k,p < n, lexicographic, is the basis of
A = C[x,y,z] / <T_{n,0,0} - sigma, T_{0,n,0} - tau, T_{0,0,n} - rho> whose
coordinates the transform takes; the new basis is

    b~_n = (T_{abc} . T_{efg}(T_{m,0,0}, T_{0,m,0}, T_{0,0,m})),
           (e,f,g) in {0,1}^3 major, (a,b,c) in [0,m)^3 minor.

Column (efg, abc) of B_n^{-1} holds the b_n coordinates of that element:
  * T_{efg}(T_{m,0,0}, T_{0,m,0}, T_{0,0,m}) = T_{m(e,f,g)}: T_{efg} is a
    polynomial in T_{100}, T_{010}, T_{001} (Prop. 1) and T_k(m theta) =
    T_{mk}(theta) by the power form;
  * T_{abc} T_l = (1/24) sum_w T_{(a,b,c) + w l}       (Prop. 1 (iv));
  * T_{wk} = T_k moves every index to its dominant representative
                                                        (Prop. 1 (iii));
  * a dominant index k outside the box, k_j >= n, is reduced with the ideal:
    T_{n e_j} = sigma_j, the value of T_{e_j} at c (the grid points are its
    zeros, Lemma 2), so from T_{n e_j} T_{k - n e_j} = (1/|W e_j|) sum over
    u in W e_j of T_{k - n e_j + n u}
        T_k = (|W e_j| sigma_j T_{k - n e_j} - sum_{u: dom != k} T_{...}) / #{u: dom = k}.
    Every other index on the right lies strictly below k in dominance order
    (e_j is the highest weight of its orbit), so the reduction ends.

With B_n so defined, the factorisation is checked against the dense matrix
of Def. 2 (tests/test_oracle_radix2.py) and ``forward_radix2`` evaluates it
recursively down to D_2, the 2 x 2 x 2 transform from the definition.
``python -m oracle.radix2`` prints the non-zeros of B_n, the complex
multiply-adds per point of the whole recursion and its error evaluated in
FP64 and in FP32 against the FP64 dense matrix.
"""
import functools

import numpy as np

from . import CANONICAL_SKEW, chebyshev, dct_matrix, dominant, weyl_group


def _box_index(k, n):
    return (k[0] * n + k[1]) * n + k[2]


@functools.lru_cache(maxsize=None)
def _orbits():
    """Distinct images W e_j of the three unit weights, e_j first."""
    W = weyl_group()
    out = []
    for j in range(3):
        e = np.zeros(3, dtype=np.int64)
        e[j] = 1
        seen = [tuple(int(v) for v in e)]
        for w in W:
            u = tuple(int(v) for v in w @ e)
            if u not in seen:
                seen.append(u)
        out.append(seen)
    return out


def sub_shift(skew, i):
    """(c + i) / 2 for c = v / d and i in {0,1}^3, as (numerators, denominator)."""
    v, d = skew
    return (tuple(int(v[a]) + int(i[a]) * d for a in range(3)), 2 * d)


def ideal_values(skew):
    """sigma, tau, rho at c: T_{e_j}(c) for j = 1, 2, 3 (the constants that
    T_{n e_j} takes at every grid point of the shift, Lemma 2)."""
    v, d = skew
    c = np.asarray(v, dtype=np.float64) / d
    return [chebyshev(np.eye(3, dtype=np.int64)[j], c) for j in range(3)]


def _reducer(n, skew):
    """T_k (k dominant, any size) -> {box index: coefficient} in b_n."""
    sig = ideal_values(skew)
    orb = _orbits()
    memo = {}

    def red(k):
        if all(0 <= c < n for c in k):
            return {_box_index(k, n): 1.0 + 0j}
        if k in memo:
            return memo[k]
        j = next(a for a in range(3) if k[a] >= n)
        low = tuple(k[a] - (n if a == j else 0) for a in range(3))
        same = 0
        acc = {}
        for key, val in red(low).items():
            acc[key] = acc.get(key, 0) + len(orb[j]) * sig[j] * val
        for u in orb[j]:
            t = dominant(tuple(low[a] + n * u[a] for a in range(3)))
            if t == k:
                same += 1
                continue
            for key, val in red(t).items():
                acc[key] = acc.get(key, 0) - val
        out = {key: val / same for key, val in acc.items()}
        memo[k] = out
        return out

    return red


@functools.lru_cache(maxsize=None)
def basis_change_inverse(n, skew=CANONICAL_SKEW):
    """B_n^{-1} (dense, n^3 x n^3): column (efg, abc) = b_n coordinates of
    T_{abc} T_{m(e,f,g)}.  n even."""
    if n % 2:
        raise ValueError("the radix-2 step needs an even order")
    m = n // 2
    W = weyl_group()
    red = _reducer(n, skew)
    N = n ** 3
    out = np.zeros((N, N), dtype=np.complex128)
    for e in range(2):
        for f in range(2):
            for g in range(2):
                l = np.array([m * e, m * f, m * g], dtype=np.int64)
                for a in range(m):
                    for b in range(m):
                        for c in range(m):
                            col = (e * 4 + f * 2 + g) * m ** 3 + (a * m + b) * m + c
                            base = np.array([a, b, c], dtype=np.int64)
                            for w in W:
                                t = dominant(tuple(int(v) for v in base + w @ l))
                                for key, val in red(t).items():
                                    out[key, col] += val / 24.0
    return out


@functools.lru_cache(maxsize=None)
def basis_change(n, skew=CANONICAL_SKEW):
    """B_n(c) = (B_n^{-1})^{-1}: b_n coordinates -> b~_n coordinates."""
    return np.linalg.inv(basis_change_inverse(n, skew))


def point_permutation(n):
    """P_n as flat indices: row (i, k) of the stacked sub-transforms (i in
    {0,1}^3 major, k in [0,m)^3 minor) is grid point j = i + 2k."""
    m = n // 2
    perm = np.empty(n ** 3, dtype=np.int64)
    for i0 in range(2):
        for i1 in range(2):
            for i2 in range(2):
                for k0 in range(m):
                    for k1 in range(m):
                        for k2 in range(m):
                            row = (i0 * 4 + i1 * 2 + i2) * m ** 3 + (k0 * m + k1) * m + k2
                            perm[row] = _box_index((i0 + 2 * k0, i1 + 2 * k1, i2 + 2 * k2), n)
    return perm


_BITS = [(i0, i1, i2) for i0 in range(2) for i1 in range(2) for i2 in range(2)]


def factor_product(n, skew=CANONICAL_SKEW):
    """P_n . (sum_i D_m((c+i)/2)) . (D_2(c) (x) 1): the matrix that equals
    D_n(c) B_n^{-1} when the factorisation holds (dense, n <= 16)."""
    m = n // 2
    D2 = dct_matrix(2, skew)
    N, M = n ** 3, m ** 3
    out = np.zeros((N, N), dtype=np.complex128)
    perm = point_permutation(n)
    for ii, i in enumerate(_BITS):
        Dm = dct_matrix(m, sub_shift(skew, i))
        for ef in range(8):
            out[perm[ii * M:(ii + 1) * M], ef * M:(ef + 1) * M] = D2[ii, ef] * Dm
    return out


def forward_radix2(x, n, skew=CANONICAL_SKEW, dtype=np.complex128):
    """y = D_n(c) x by the recursion (n a power of 2), every product in
    `dtype` (complex128, or complex64 to measure the recursion in FP32).
    x: [..., n^3] coefficients; returns point values [..., n^3]."""
    x = np.asarray(x).astype(dtype)
    if n == 2:
        return x @ dct_matrix(2, skew).T.astype(dtype)
    m = n // 2
    M = m ** 3
    xt = x @ basis_change(n, skew).T.astype(dtype)               # b~ coordinates
    u = np.einsum("ie,...ek->...ik", dct_matrix(2, skew).astype(dtype), xt.reshape(x.shape[:-1] + (8, M)))
    y = np.empty(x.shape, dtype=dtype)
    perm = point_permutation(n)
    for ii, i in enumerate(_BITS):
        y[..., perm[ii * M:(ii + 1) * M]] = forward_radix2(u[..., ii, :], m, sub_shift(skew, i), dtype)
    return y


def nonzeros_per_row(A, rel=1e-12):
    A = np.abs(A)
    return float((A > rel * A.max()).sum()) / A.shape[0]


def recursion_macs(n, skew=CANONICAL_SKEW, rel=1e-12):
    """Complex multiply-adds of one transform by the recursion: the
    non-zeros of B_n, 8 x 8 per column block of D_2 (x) 1, and the eight
    sub-transforms (their shifts differ); D_2 itself dense (64)."""
    if n == 2:
        return 64
    m = n // 2
    B = np.abs(basis_change(n, skew))
    own = int((B > rel * B.max()).sum()) + 64 * m ** 3
    return own + sum(recursion_macs(m, sub_shift(skew, i), rel) for i in _BITS)


def main():
    rng = np.random.default_rng(0)
    print("n   nnz/row B_n   max|B_n|   MACs/pt   rel L2 of the recursion vs the dense matrix: FP64   FP32")
    for n in (4, 8, 16):
        B = basis_change(n)
        x = rng.standard_normal(n ** 3)
        ref = dct_matrix(n) @ x
        e64 = np.linalg.norm(forward_radix2(x, n) - ref) / np.linalg.norm(ref)
        e32 = np.linalg.norm(forward_radix2(x.astype(np.float32), n, dtype=np.complex64) - ref) / np.linalg.norm(ref)
        print("%-3d %-13.2f %-10.3g %-9.1f %-52.2e %.2e" % (n, nonzeros_per_row(B), np.abs(B).max(),
                                                           recursion_macs(n) / n ** 3, e64, e32))


if __name__ == "__main__":
    main()
