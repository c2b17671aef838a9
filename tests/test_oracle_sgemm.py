"""Pins for SGEMM through Ozaki scheme II in the oracle (FP32 inputs and output; Section 5
evaluates it for N = 3..12).  Every float is a double, so the scaling and the integer stages are
those of the pinned DGEMM pipeline; Step 4 rounds to single.  Checked against: brute-force exact
integers A'B' on tiny inputs with a correctly rounded 24-bit conversion written here (including
subnormal and overflowing outputs), the BLAS alpha/beta rules in single precision, and the
truncation error bound of the product."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic


def rn_bits(x: int, bits: int) -> Fraction:
    """The integer x rounded to `bits` significant bits, ties to even."""
    if x == 0:
        return Fraction(0)
    a = abs(x)
    sh = a.bit_length() - bits
    if sh > 0:
        q, r = divmod(a, 1 << sh)
        half = 1 << (sh - 1)
        if r > half or (r == half and q & 1):
            q += 1
        a = q << sh
    return Fraction(a if x > 0 else -a)


def to_f32(v: Fraction) -> np.float32:
    """A rational rounded once to single precision (ties to even, subnormals, overflow)."""
    if v == 0:
        return np.float32(0.0)
    sign = -1 if v < 0 else 1
    a = abs(v)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    lsb = max(e - 23, -149)                         # subnormals keep the 2^-149 grid
    q, r = divmod(a / Fraction(2) ** lsb, 1)
    q = int(q)
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q & 1):
        q += 1
    val = Fraction(q) * Fraction(2) ** lsb
    if val >= Fraction(2) ** 128:
        return np.float32(sign * np.inf)
    return np.float32(sign * float(val))


def brute_sgemm(orc, A, B, m, n, k, N, alpha=1.0, beta=0.0, Cin=None):
    """Exact A'B' with the oracle's (pinned) shifts of the widened inputs, then Step 4 in single."""
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    e, _ = orc.shifts_a(Ad, m, k, N)
    f, _ = orc.shifts_b(Bd, k, n, N)
    Am, Bm = synthetic.colmajor_view(Ad), synthetic.colmajor_view(Bd)
    Ap = [[math.trunc(Fraction(float(Am[i, h])) * Fraction(2) ** int(e[i])) for h in range(k)]
          for i in range(m)]
    Bp = [[math.trunc(Fraction(float(Bm[h, j])) * Fraction(2) ** int(f[j])) for j in range(n)]
          for h in range(k)]
    out = np.zeros((n, m), np.float32)
    for i in range(m):
        for j in range(n):
            c = sum(Ap[i][h] * Bp[h][j] for h in range(k))
            y = to_f32(rn_bits(c, 24) * Fraction(2) ** (-int(e[i]) - int(f[j])))
            v = np.float32(np.float32(alpha) * y)
            if beta != 0.0:
                v = np.float32(v + np.float32(np.float32(beta) * Cin[j, i]))
            out[j, i] = v
    return out


@pytest.mark.parametrize("N", [3, 7, 12])
def test_tiny_against_exact_integers(orc, N):
    rng = np.random.default_rng(N)
    m, n, k = 5, 4, 9
    A = synthetic.paper_matrix(m, k, 1.0, 100 + N).astype(np.float32)
    B = synthetic.paper_matrix(k, n, 1.0, 200 + N).astype(np.float32)
    Cin = rng.standard_normal((n, m)).astype(np.float32)
    got = orc.sgemm(A, B, m, n, k, N, alpha=-1.5, beta=0.25, Cin=Cin)
    ref = brute_sgemm(orc, A, B, m, n, k, N, -1.5, 0.25, Cin)
    assert np.array_equal(got.view(np.int32), ref.view(np.int32))


@pytest.mark.parametrize("scale,expect", [(2.0**-70, "subnormal"), (2.0**66, "overflow")])
def test_subnormal_and_overflow_outputs(orc, scale, expect):
    """Products around 2^-140 round onto the subnormal grid once; products beyond 2^128
    overflow to infinity."""
    m, n, k, N = 3, 3, 4, 10
    A = (synthetic.paper_matrix(m, k, 0.5, 7) * scale).astype(np.float32)
    B = (synthetic.paper_matrix(k, n, 0.5, 8) * scale).astype(np.float32)
    got = orc.sgemm(A, B, m, n, k, N)
    ref = brute_sgemm(orc, A, B, m, n, k, N)
    assert np.array_equal(got.view(np.int32), ref.view(np.int32))
    if expect == "subnormal":
        assert np.all(np.abs(got[got != 0]) < np.finfo(np.float32).tiny)
        assert np.any(got != 0)
    else:
        assert np.any(np.isinf(got))


def test_quick_returns_and_blas_rules(orc):
    m, n, k, N = 4, 3, 5, 8
    A = synthetic.paper_matrix(m, k, 1.0, 1).astype(np.float32)
    B = synthetic.paper_matrix(k, n, 1.0, 2).astype(np.float32)
    Cin = np.full((n, m), np.nan, np.float32)
    assert np.all(orc.sgemm(A, B, m, n, k, N, beta=0.0, Cin=Cin) ==
                  orc.sgemm(A, B, m, n, k, N))                 # beta = 0 never reads C
    C2 = np.arange(n * m, dtype=np.float32).reshape(n, m)
    got = orc.sgemm(A, B, m, n, k, N, alpha=0.0, beta=3.0, Cin=C2)
    assert np.array_equal(got, np.float32(3.0) * C2)           # alpha = 0: C = beta C
    got = orc.sgemm(A[:0], B[:, :0], m, n, 0, N, beta=0.5, Cin=C2)
    assert np.array_equal(got, np.float32(0.5) * C2)           # k = 0


@pytest.mark.parametrize("N", [6, 9, 12])
def test_error_within_truncation_bound(orc, N):
    """|C - AB| <= 2^-f_j sum|a_i.| + 2^-e_i sum|b_.j| + k 2^-(e_i+f_j) + |C| 2^-23 (truncation
    of a' and b', one rounding to 24 bits and one to single)."""
    m, n, k = 40, 30, 300
    A = synthetic.paper_matrix(m, k, 1.0, 31).astype(np.float32)
    B = synthetic.paper_matrix(k, n, 1.0, 32).astype(np.float32)
    C = orc.sgemm(A, B, m, n, k, N).astype(np.float64)
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    e, _ = orc.shifts_a(Ad, m, k, N)
    f, _ = orc.shifts_b(Bd, k, n, N)
    hi, lo = orc.dd_block(Ad, Bd, k, np.arange(m, dtype=np.int32), np.arange(n, dtype=np.int32))
    ra = np.abs(synthetic.colmajor_view(Ad)).sum(axis=1)
    cb = np.abs(synthetic.colmajor_view(Bd)).sum(axis=0)
    ei, fj = 2.0 ** -e.astype(np.float64), 2.0 ** -f.astype(np.float64)
    bound = (ra[None, :] * fj[:, None] + cb[:, None] * ei[None, :] + k * fj[:, None] * ei[None, :]
             + np.abs(C) * 2.0**-23) * 1.001
    assert np.all(np.abs((C - hi) - lo) <= bound)


def test_cpp_rounded_once_to_24_bits(orc):
    """Step 4 for FP32 rounds C'' to 24 bits directly.  Constructed case: one row (u, 2^-e) and one
    column (v, -2^-f) with u v odd in [2^24, 2^25) and u v = 3 (mod 4) give
    C'' = u v 2^(e+f) - 1, whose bits after the 24 leading ones start 0111...1: rounding first to
    53 bits would make a tie that rounds up, the single rounding goes down."""
    N = 12
    for u in range(4097, 8191, 2):
        v = next((w for w in range(4097, 8191, 2)
                  if 2**24 <= u * w < 2**25 and (u * w) % 4 == 3), None)
        if v is None:
            continue
        e0 = int(orc.shifts_a(np.array([[u], [0.0]]), 1, 2, N)[0][0])
        f0 = int(orc.shifts_b(np.array([[v, 0.0]]), 2, 1, N)[0][0])
        A = np.array([[u], [2.0**-e0]], np.float32)              # storage (k, m): row (u, 2^-e)
        B = np.array([[v, -(2.0**-f0)]], np.float32)             # storage (n, k): column (v, -2^-f)
        e = int(orc.shifts_a(A.astype(np.float64), 1, 2, N)[0][0])
        f = int(orc.shifts_b(B.astype(np.float64), 2, 1, N)[0][0])
        if (e, f) != (e0, f0):
            continue
        c = u * v * 2 ** (e + f) - 1
        assert rn_bits(c, 24) != rn_bits(int(rn_bits(c, 53)), 24)
        got = orc.sgemm(A, B, 1, 1, 2, N)
        want = to_f32(rn_bits(c, 24) * Fraction(2) ** (-e - f))
        assert got[0, 0] == want
        assert got[0, 0] < np.float32(u) * np.float32(v)         # rounded down, not to the tie
        return
    pytest.fail("no constructed case found")


def test_block_matches_whole_product(orc):
    m, n, k, N = 37, 29, 150, 9
    A = synthetic.paper_matrix(k, m, 2.0, 91).astype(np.float32)     # op(A) = A^T
    B = synthetic.paper_matrix(n, k, 2.0, 92).astype(np.float32)     # op(B) = B^T
    Cin = np.random.default_rng(3).standard_normal((n, m)).astype(np.float32)
    full = orc.sgemm(A, B, m, n, k, N, "T", "T", 0.5, -2.0, Cin)
    I = np.array([0, 5, 36], np.int32)
    J = np.array([1, 28], np.int32)
    blk = orc.sgemm_block(A, B, k, N, I, J, "T", "T", 0.5, -2.0, Cin[np.ix_(J, I)])
    assert np.array_equal(blk.view(np.int32), full[np.ix_(J, I)].view(np.int32))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_agrees_with_the_dgemm_modes(orc, mode):
    """SGEMM is the DGEMM pipeline on widened inputs up to the final rounding: every entry is
    the single rounding of C'' while DGEMM rounds it to 53 bits, so the two agree to within one
    unit in the last place of single (and exactly, apart from rare double-rounding cases)."""
    m, n, k, N = 50, 40, 400, 10
    A = synthetic.paper_matrix(m, k, 1.0, 71).astype(np.float32)
    B = synthetic.paper_matrix(k, n, 1.0, 72).astype(np.float32)
    S = orc.sgemm(A, B, m, n, k, N, mode=mode)
    D = orc.dgemm_mode(A.astype(np.float64), B.astype(np.float64), m, n, k, N, mode)
    Df = D.astype(np.float32)
    ulp = np.spacing(np.abs(Df))
    assert np.all(np.abs(S.astype(np.float64) - Df.astype(np.float64)) <= ulp)
    assert np.mean(S == Df) > 0.999
