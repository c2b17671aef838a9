"""Pins for Steps 2-4 of Ozaki scheme II (Section 2.2) in the oracle, by brute force.

On tiny inputs every integer stage is recomputed with Python's exact integers directly from
the definitions (a' = trunc(mu a), A'B' as an exact integer product, no CRT at all), the
final doubles are checked against Python's correctly rounded int->float, and the emulated
product is checked against the exact rational product with a rigorous truncation bound.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic


def py_trunc_scaled(x: float, e: int) -> int:
    v = Fraction(float(x)) * Fraction(2) ** e
    return math.trunc(v)


def sym(x: int, p: int) -> int:
    r = x % p
    return r - p if 2 * r >= p else r


CASES = [(1, 1, 1), (3, 5, 7), (8, 6, 5), (5, 8, 9)]


@pytest.mark.parametrize("N", [2, 5, 8, 14, 17, 20])
@pytest.mark.parametrize("phi", [0.5, 2.0, 4.0])
@pytest.mark.parametrize("shape", CASES)
def test_integer_stages_brute_force(orc, N, phi, shape):
    m, n, k = shape
    seed = 7 * m + 11 * n + 13 * k + N
    A = synthetic.paper_matrix(m, k, phi, seed)
    B = synthetic.paper_matrix(k, n, phi, seed + 1)
    Am, Bm = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    p = orc.constants(N)["p"]
    e, _ = orc.shifts_a(A, m, k, N)
    f, _ = orc.shifts_b(B, k, n, N)
    Ap = [[py_trunc_scaled(Am[i, h], int(e[i])) for h in range(k)] for i in range(m)]
    Bp = [[py_trunc_scaled(Bm[h, j], int(f[j])) for j in range(n)] for h in range(k)]
    RA = orc.residues_a(A, m, k, e, N)
    RB = orc.residues_b(B, k, n, f, N)
    for l in range(N):
        for i in range(m):
            for h in range(k):
                assert RA[l, i, h] == sym(Ap[i][h], p[l])
        for j in range(n):
            for h in range(k):
                assert RB[l, j, h] == sym(Bp[h][j], p[l])
    c = orc.residue_products(RA, RB)
    for l in range(N):
        for i in range(m):
            for j in range(n):
                g = sum(int(RA[l, i, h]) * int(RB[l, j, h]) for h in range(k))
                assert c[l, i, j] == sym(g, p[l])
    Cpp = orc.crt_exact(c)
    P = orc.constants(N)["P"]
    C = synthetic.colmajor_view(orc.dgemm(A, B, m, n, k, N))
    for i in range(m):
        for j in range(n):
            exact = sum(Ap[i][h] * Bp[h][j] for h in range(k))
            assert 2 * sum(abs(Ap[i][h] * Bp[h][j]) for h in range(k)) < P   # eq. os2-condition
            assert int(Cpp[i, j]) == exact                                    # eq. os2-C''
            assert C[i, j] == math.ldexp(float(exact), -(int(e[i]) + int(f[j])))   # Step 4


@pytest.mark.parametrize("N", [8, 14, 20])
@pytest.mark.parametrize("phi", [0.5, 1.0, 4.0])
def test_error_within_truncation_bound(orc, N, phi):
    """|C - AB| <= sum_h (|a| 2^-f + |b| 2^-e + 2^-(e+f)) + |C| 2^-53, from a' = mu a - d_a with
    |d_a| < 1 (trunc) and one rounding of C'' to double."""
    m, n, k = 6, 5, 40
    A = synthetic.paper_matrix(m, k, phi, 50 + N)
    B = synthetic.paper_matrix(k, n, phi, 60 + N)
    Am, Bm = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    e, _ = orc.shifts_a(A, m, k, N)
    f, _ = orc.shifts_b(B, k, n, N)
    C = synthetic.colmajor_view(orc.dgemm(A, B, m, n, k, N))
    for i in range(m):
        for j in range(n):
            ex = sum(Fraction(float(Am[i, h])) * Fraction(float(Bm[h, j])) for h in range(k))
            ei, fj = Fraction(2) ** -int(e[i]), Fraction(2) ** -int(f[j])
            bound = sum(abs(Fraction(float(Am[i, h]))) * fj + abs(Fraction(float(Bm[h, j]))) * ei
                        + ei * fj for h in range(k))
            bound += abs(Fraction(float(C[i, j]))) * Fraction(1, 2**53)
            assert abs(Fraction(float(C[i, j])) - ex) <= bound


def test_alpha_beta_and_quick_cases(orc):
    m, n, k, N = 7, 6, 9, 14
    A = synthetic.paper_matrix(m, k, 1.0, 1)
    B = synthetic.paper_matrix(k, n, 1.0, 2)
    Cin = synthetic.paper_matrix(m, n, 1.0, 3)
    base = orc.dgemm(A, B, m, n, k, N)
    got = orc.dgemm(A, B, m, n, k, N, alpha=-2.5, beta=0.75, Cin=Cin)
    assert np.array_equal(got, (-2.5 * base) + 0.75 * Cin)
    nan_in = np.full_like(Cin, np.nan)
    assert np.array_equal(orc.dgemm(A, B, m, n, k, N, beta=0.0, Cin=nan_in), base)
    z = orc.dgemm(A[:0], B[:, :0], m, n, 0, N, alpha=3.0, beta=0.5, Cin=Cin, lda=m, ldb=1)
    assert np.array_equal(z, 0.5 * Cin)


def test_transposes_agree(orc):
    """op(A) = A^T stored k x m (lda = k) and op(B) = B^T stored n x k give the same bits."""
    m, n, k, N = 9, 7, 11, 14
    A = synthetic.paper_matrix(m, k, 1.0, 8)
    B = synthetic.paper_matrix(k, n, 1.0, 9)
    nn = orc.dgemm(A, B, m, n, k, N)
    tn = orc.dgemm(np.ascontiguousarray(synthetic.colmajor_view(A)), B, m, n, k, N, transA="T",
                   lda=k)
    nt = orc.dgemm(A, np.ascontiguousarray(synthetic.colmajor_view(B)), m, n, k, N, transB="T",
                   ldb=n)
    assert np.array_equal(nn, tn)
    assert np.array_equal(nn, nt)


def test_block_matches_full(orc):
    m, n, k, N = 40, 33, 50, 14
    A = synthetic.paper_matrix(m, k, 2.0, 12)
    B = synthetic.paper_matrix(k, n, 2.0, 13)
    full = synthetic.colmajor_view(orc.dgemm(A, B, m, n, k, N))
    I = [0, 5, 39, 17]
    J = [32, 0, 9]
    blk = synthetic.colmajor_view(orc.dgemm_block(A, B, m, n, k, N, I, J))
    assert np.array_equal(blk, full[np.ix_(I, J)])


def test_dd_reference_against_exact(orc):
    """The double-double reference is within 2^-100 sum|ab| of the exact product."""
    m, n, k = 5, 4, 64
    A = synthetic.paper_matrix(m, k, 3.0, 70)
    B = synthetic.paper_matrix(k, n, 3.0, 71)
    Am, Bm = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    hi, lo = orc.dd_block(A, B, k, list(range(m)), list(range(n)))
    for i in range(m):
        for j in range(n):
            ex = sum(Fraction(float(Am[i, h])) * Fraction(float(Bm[h, j])) for h in range(k))
            mag = sum(abs(Fraction(float(Am[i, h])) * Fraction(float(Bm[h, j]))) for h in range(k))
            got = Fraction(float(hi[j, i])) + Fraction(float(lo[j, i]))
            assert abs(got - ex) <= mag * Fraction(1, 2**100)


def test_error_decreases_with_moduli(orc):
    """Section 5.1 trend: the maximum relative error falls as N grows (values unpinned)."""
    m = n = k = 64
    A = synthetic.paper_matrix(m, k, 1.0, 90)
    B = synthetic.paper_matrix(k, n, 1.0, 91)
    I, J = list(range(m)), list(range(n))
    hi, lo = orc.dd_block(A, B, k, I, J)
    errs = {}
    for N in (8, 11, 14, 17, 20):
        C = orc.dgemm(A, B, m, n, k, N)
        errs[N] = orc.max_rel_error(C, hi, lo)[0]
    assert errs[20] < errs[14] < errs[8]
    assert errs[20] < 1e-15
