"""Pins for the accurate mode of the oracle (Section 2.3: mu', a-bar, the auxiliary product
C-bar = A-bar B-bar, eq. (mu_accu)/(nu_accu) with the log2~ of eq. (flog2)).

Checked against: exact rational a-bar = ceil(mu' |a|), brute-force C-bar maxima, the CRT
condition (eq. os2-condition) on exact integers, near-maximality against a 50-digit decimal
optimum, exact invariance under alpha = 2^s (Fig. 2: constant accuracy across alpha), the
all-ones closed form (same a' as the proposed scaling), and the special lines."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import synthetic


def exact_ceil_bar(a: float, E: int) -> int:
    return math.ceil(abs(Fraction(a)) * Fraction(2) ** (5 - E)) if a != 0 else 0


def test_bar_is_exact_ceiling(orc):
    rng = np.random.default_rng(1)
    m, k = 12, 40
    A = synthetic.paper_matrix(m, k, 2.0, 9)
    Av = synthetic.colmajor_view(A)
    Av[2, :] = 0.0
    Av[3, 5] = 1e300
    Av[3, 6] = 1e-300          # mu' |a| underflows: the exact ceiling is 1
    Av[4, :] = rng.choice([0.0, 5e-324, -3e-310], size=k)
    Av[5, 7] = -2.0**40
    bar, E, kind = orc.accu_bar(A, m, k)
    for i in range(m):
        row = Av[i]
        mx = np.max(np.abs(row))
        if mx == 0:
            assert kind[i] == 0 and not bar[i].any()
            continue
        assert kind[i] == 1
        assert E[i] == math.frexp(mx)[1] - 1
        for h in range(k):
            assert bar[i, h] == exact_ceil_bar(row[h], int(E[i])), (i, h)
        assert bar[i].max() <= 64 and np.all((bar[i] > 0) == (row != 0))
    assert bar[3, 6] == 1


def test_cbar_maxima_brute_force(orc):
    m, n, k = 23, 17, 301
    A = synthetic.paper_matrix(m, k, 1.0, 3)
    B = synthetic.paper_matrix(k, n, 1.0, 4)
    e, f, rm, cm = orc.accurate_shifts(A, B, m, n, k, 14)
    Ab, _, _ = orc.accu_bar(A, m, k, side=0)
    Bb, _, _ = orc.accu_bar(B, n, k, side=1)
    Cbar = Ab.astype(np.int64) @ Bb.astype(np.int64).T
    assert np.array_equal(rm, Cbar.max(axis=1)) and np.array_equal(cm, Cbar.max(axis=0))


@pytest.mark.parametrize("N,phi", [(8, 1.0), (14, 0.5), (20, 2.0), (17, 1.0)])
def test_crt_condition_holds_exactly(orc, N, phi):
    """eq. (os2-condition): 2 sum_h |a'_ih| |b'_hj| < P for every (i, j)."""
    m, n, k = 14, 11, 120
    A = synthetic.paper_matrix(m, k, phi, 10 + N)
    B = synthetic.paper_matrix(k, n, phi, 20 + N)
    e, f, _, _ = orc.accurate_shifts(A, B, m, n, k, N)
    P = orc.constants(N)["P"]
    Am, Bm = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    Ap = [[abs(math.trunc(Fraction(float(Am[i, h])) * Fraction(2) ** int(e[i])))
           for h in range(k)] for i in range(m)]
    Bp = [[abs(math.trunc(Fraction(float(Bm[h, j])) * Fraction(2) ** int(f[j])))
           for j in range(n)] for h in range(k)]
    worst = 0
    for i in range(m):
        for j in range(n):
            s = sum(Ap[i][h] * Bp[h][j] for h in range(k))
            assert 2 * s < P, (i, j)
            worst = max(worst, Fraction(2 * s, P))
    assert worst > Fraction(1, 2**12)   # not trivially small: the bound is used


def test_shift_is_near_optimal(orc):
    """log2 mu_i = 5 - E_i + floor(P' - 0.5 log2 max_j c-bar_ij) up to the delta margin:
    equal to the exact decimal value except where its fractional part is within 1e-5 of an
    integer, and never above it."""
    getcontext().prec = 50
    N = 16
    pp = Decimal(float(np.float32(orc.constants(N)["pprime"])))
    rng = np.random.default_rng(7)
    near = 0
    for trial in range(2000):
        cmax = int(rng.integers(1, 2**31))
        E = int(rng.integers(-50, 50))
        e = orc.accu_shift(1, E, cmax, float(pp))
        exact = pp - Decimal(cmax).ln() / Decimal(2).ln() / 2
        opt = 5 - E + int(exact.to_integral_value(rounding="ROUND_FLOOR"))
        assert e <= opt
        frac = exact - exact.to_integral_value(rounding="ROUND_FLOOR")
        if frac > Decimal("1e-5"):
            assert e == opt, (cmax, E)
        else:
            near += 1
    assert near < 20


def test_scale_invariance_power_of_two(orc):
    """Fig. 2: accurate mode keeps its accuracy for every alpha = 2^s: A' and B' are identical
    (e + s constant per line) and so is the result up to the factor alpha^2."""
    m, n, k, N = 20, 13, 200, 18
    A0 = synthetic.paper_matrix(m, k, 1.0, 5)
    B0 = synthetic.paper_matrix(k, n, 1.0, 6)
    e0, f0, _, _ = orc.accurate_shifts(A0, B0, m, n, k, N)
    C0 = orc.dgemm_mode(A0, B0, m, n, k, N, orc.ACCURATE_MODE)
    for s in (-40, -7, 3, 25):
        e, f, _, _ = orc.accurate_shifts(A0 * 2.0**s, B0 * 2.0**s, m, n, k, N)
        assert np.array_equal(e + s, e0) and np.array_equal(f + s, f0)
        C = orc.dgemm_mode(A0 * 2.0**s, B0 * 2.0**s, m, n, k, N, orc.ACCURATE_MODE)
        assert np.array_equal(C, C0 * 4.0**s)


@pytest.mark.parametrize("k,expect", [(1024, 72), (16384, 70)])
def test_all_ones_closed_form(orc, k, expect):
    """All-ones, N = 20: a-bar = 32, C-bar = 1024 k, so e + s = 5 + floor(P' - delta
    (log2 k + 10)), which is 72 for k = 1024 and 70 for k = 16384 (the proposed scaling's values);
    A'B' = k 2^(2(e+s)) < P/2 and the product is exact for every s."""
    N = 20
    P = orc.constants(N)["P"]
    for s in (-10, -2, 0, 7):
        A = synthetic.ones_matrix(2, k, 2.0**s)
        B = synthetic.ones_matrix(k, 3, 2.0**s)
        e, f, rm, cm = orc.accurate_shifts(A, B, 2, 3, k, N)
        assert np.all(rm == 1024 * k) and np.all(cm == 1024 * k)
        assert np.all(e + s == expect) and np.all(f + s == expect)
        assert 2 * k * 2 ** (2 * expect) < P
    A = synthetic.ones_matrix(3, 1024, 0.25)
    B = synthetic.ones_matrix(1024, 2, 0.25)
    C = orc.dgemm_mode(A, B, 3, 2, 1024, N, orc.ACCURATE_MODE)
    assert np.all(C == 1024 / 16)


def test_wider_than_fast_mode(orc):
    """Section 2.3: the accurate estimate allows at least the fast mode's bit width."""
    m, n, k, N = 40, 30, 500, 14
    for phi in (0.5, 1.0, 2.0):
        A = synthetic.paper_matrix(m, k, phi, 61)
        B = synthetic.paper_matrix(k, n, phi, 62)
        e, f, _, _ = orc.accurate_shifts(A, B, m, n, k, N)
        assert np.all(e >= orc.shifts_mode(A, m, k, N, orc.FAST_MODE))
        assert np.all(f >= orc.shifts_mode(B, n, k, N, orc.FAST_MODE, side=1))


def test_special_lines(orc):
    """Zero line -> 0; non-finite line -> SHIFT_NONFINITE (and NaN outputs); a nonzero line whose
    products all vanish -> SHIFT_VANISH (a' = 0, output exactly 0)."""
    m, n, k, N = 5, 4, 16, 14
    A = synthetic.paper_matrix(m, k, 1.0, 1)
    B = synthetic.paper_matrix(k, n, 1.0, 2)
    Av, Bv = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    Av[0, :] = 0.0
    Av[1, 3] = np.inf
    Av[2, :] = 0.0
    Av[2, 4] = 3.0             # only h = 4 is nonzero in row 2 ...
    Bv[4, :] = 0.0             # ... and row 4 of B is zero: row 2 of C-bar vanishes
    e, f, rm, cm = orc.accurate_shifts(A, B, m, n, k, N)
    assert e[0] == 0 and e[1] == orc.SHIFT_NONFINITE and e[2] == orc.SHIFT_VANISH
    assert rm[2] == 0
    C = orc.dgemm_mode(A, B, m, n, k, N, orc.ACCURATE_MODE)
    Cv = synthetic.colmajor_view(C)
    assert np.all(Cv[0] == 0) and np.all(np.isnan(Cv[1])) and np.all(Cv[2] == 0)
    hi, lo = orc.dd_block(A, B, k, np.arange(3, 5, dtype=np.int32), np.arange(n, dtype=np.int32))
    err, _ = orc.max_rel_error(C[:, 3:5], hi, lo)
    assert err < 1e-10


def _ru_f32(x: Fraction) -> Fraction:
    f = np.float32(float(x))
    if Fraction(float(f)) < x:
        f = np.nextafter(f, np.float32(np.inf))
    return Fraction(float(f))


def test_delta_decides_the_floor(orc):
    """The shift uses delta (eq. delta), not 0.5: over lines where the two floors differ, the
    oracle takes the delta one.  log2~ is evaluated as eq. (flog2) on the oracle's pinned log2."""
    N = 14
    pp = Fraction(float(np.float32(orc.constants(N)["pprime"])))
    delta = Fraction(orc.fast_delta())
    hits = 0
    # the floors differ when 0.5 log2~ <= P' - j < delta log2~: scan integers around 2^(2(P'-j))
    for j in range(int(pp) - 15, int(pp) - 2):
        centre = int(round(2 ** (2 * float(pp - j))))
        for cmax in range(max(1, centre - 300), centre + 300):
            s = cmax.bit_length() - 1
            xf = _ru_f32(Fraction(cmax, 2**s))
            lg = _ru_f32(Fraction(float(orc.log2_ru(float(xf)))) + s)
            with_delta = math.floor(pp - delta * lg)
            if with_delta == math.floor(pp - lg / 2):
                continue
            hits += 1
            assert orc.accu_shift(1, 0, cmax, float(pp)) == 5 + with_delta, cmax
    assert hits > 0
