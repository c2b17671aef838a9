"""Pins for the scaling step (Algorithm 2, Section 4) in the oracle.

Checked against: the exact rational squared norm (rounding-up must give an upper bound), the
CRT condition of eq. (proposed-condition) in exact rational arithmetic, near-maximality of
each shift against a 60-digit decimal optimum, the exact scale-invariance argument of
Section 4 for alpha = 2^s, the effective-bit-width formula of Section 3.1 for non-power-of-two
alpha, and the all-ones worked example of Section 3.1 in closed form.
"""
import math
import struct
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import synthetic


def exact_sq_norms_rows(Acm):
    """Exact sum of squares of each row of the column-major matrix (storage (k, m))."""
    M = synthetic.colmajor_view(Acm)
    return [sum(Fraction(float(v)) ** 2 for v in M[i]) for i in range(M.shape[0])]


def optimum_shift(P, S):
    """E = floor(log2(sqrt((P-1)/2) / sqrt(S))) and its fractional part, 60 digits."""
    getcontext().prec = 60
    S = Fraction(S)
    x = (Decimal(P - 1).ln() - Decimal(2).ln() - (Decimal(S.numerator).ln()
         - Decimal(S.denominator).ln())) / (2 * Decimal(2).ln())
    E = math.floor(x)
    return E, float(x - E)


@pytest.mark.parametrize("phi", [0.5, 1.0, 2.0, 4.0])
def test_norms_round_up_and_are_tight(orc, phi):
    m, k = 24, 300
    A = synthetic.paper_matrix(m, k, phi, 11)
    _, nr = orc.shifts_a(A, m, k, 14)
    for i, S in enumerate(exact_sq_norms_rows(A)):
        assert Fraction(float(nr[i])) >= S
        # single-precision terms and sums, each rounded up: at most 2k + 4 relative steps of
        # 2^-23 in one block (a conversion and an addition per term, the rescalings)
        assert Fraction(float(nr[i])) <= S * (1 + Fraction(2 * k + 4, 2**23))


@pytest.mark.parametrize("N", [2, 8, 14, 17, 20])
@pytest.mark.parametrize("phi", [0.5, 1.0, 4.0])
def test_shift_satisfies_crt_bound_and_is_near_optimal(orc, N, phi):
    """2 mu_i^2 ||a_i||^2 <= P - 1 exactly (eq. proposed-condition as used by eq. proposed-mu),
    and e_i is the optimum E_i or E_i - 1, equal to E_i away from a boundary."""
    m, k = 32, 200
    A = synthetic.paper_matrix(m, k, phi, 100 + N)
    P = orc.constants(N)["P"]
    e, _ = orc.shifts_a(A, m, k, N)
    for i, S in enumerate(exact_sq_norms_rows(A)):
        mu2 = Fraction(2) ** (2 * int(e[i]))
        assert 2 * mu2 * S <= P - 1
        E, frac = optimum_shift(P, S)
        assert E - 1 <= e[i] <= E
        if frac > 2**-10:
            assert e[i] == E


def test_alg2_on_extreme_norms(orc):
    """Algorithm 2 on norms spread over the whole double range, including subnormals."""
    rng = np.random.default_rng(5)
    vals = [5e-324, 1e-310, 2.2250738585072014e-308, 1e-200, 0.5, 1.0, 1.5, 2.0, 3.0,
            1e100, 1.7976931348623157e308]
    vals += list(np.exp(rng.uniform(-700, 700, 200)))
    for N in (2, 14, 20):
        c = orc.constants(N)
        for v in vals:
            e = orc.alg2_shift(v, c["pprime"])
            assert 2 * Fraction(2) ** (2 * e) * Fraction(float(v)) <= c["P"] - 1
            E, frac = optimum_shift(c["P"], Fraction(float(v)))
            assert E - 1 <= e <= E
            if frac > 2**-10:
                assert e == E


def test_zero_and_nonfinite_lines(orc):
    k = 16
    A = synthetic.paper_matrix(3, k, 1.0, 4)
    A[:, 1] = 0.0            # row 1 all zero
    A[5, 2] = np.inf         # row 2 has an infinity
    e, _ = orc.shifts_a(A, 3, k, 14)
    assert e[1] == 0
    assert e[2] == orc.SHIFT_NONFINITE
    B = synthetic.paper_matrix(k, 2, 1.0, 5)
    C = synthetic.colmajor_view(orc.dgemm(A, B, 3, 2, k, 14))
    assert np.all(C[1] == 0.0)
    assert np.all(np.isnan(C[2]))
    assert np.all(np.isfinite(C[0]))


@pytest.mark.parametrize("s", [40, -40])
@pytest.mark.parametrize("N", [8, 14, 20])
def test_scale_invariance_power_of_two(orc, s, N):
    """Section 4: with alpha = 2^s, log2(alpha) cancels, so mu shifts by -s and A' is identical."""
    m, k, n = 20, 64, 18
    A = synthetic.paper_matrix(m, k, 1.0, 21)
    B = synthetic.paper_matrix(k, n, 2.0, 22)
    e0, _ = orc.shifts_a(A, m, k, N)
    e1, _ = orc.shifts_a(A * 2.0**s, m, k, N)
    f0, _ = orc.shifts_b(B, k, n, N)
    f1, _ = orc.shifts_b(B * 2.0**s, k, n, N)
    assert np.array_equal(e1, e0 - s)
    assert np.array_equal(f1, f0 - s)
    R0 = orc.residues_a(A, m, k, e0, N)
    R1 = orc.residues_a(A * 2.0**s, m, k, e1, N)
    assert np.array_equal(R0, R1)
    C0 = orc.dgemm(A, B, m, n, k, N)
    C1 = orc.dgemm(A * 2.0**s, B * 2.0**s, m, n, k, N)
    assert np.array_equal(C1, C0 * 2.0 ** (2 * s))


def effective_bits(Acm, e):
    """Section 3.1: log2(mu_i) + floor(log2 max_h |a_ih|) + 1, per row."""
    M = np.abs(synthetic.colmajor_view(Acm))
    mx = M.max(axis=1)
    return np.array([int(e[i]) + math.floor(math.log2(mx[i])) + 1 for i in range(len(e))])


@pytest.mark.parametrize("alpha", [3.7e20, 3.7e-20, 2.0**40, 2.0**-40])
def test_effective_bits_invariant(orc, alpha):
    """The effective bit width of A' does not depend on alpha (exact for 2^s; for other alpha
    the two floors can each move by one, so the width moves by at most one)."""
    m, k = 64, 128
    for phi in (0.5, 1.0, 2.0):
        A = synthetic.paper_matrix(m, k, phi, 31)
        e0, _ = orc.shifts_a(A, m, k, 14)
        e1, _ = orc.shifts_a(A * alpha, m, k, 14)
        d = effective_bits(A * alpha, e1) - effective_bits(A, e0)
        if math.log2(alpha).is_integer():
            assert np.all(d == 0)
        else:
            assert np.all(np.abs(d) <= 1)


@pytest.mark.parametrize("k", [1024, 16384])
@pytest.mark.parametrize("s", [-10, -5, -2, 0, 3, 10])
def test_all_ones_closed_form(orc, k, s):
    """All-ones example of Section 3.1 with the proposed scaling, N = 20: the squared norm is
    k 2^{2s} (a power of two), so Algorithm 2 gives e = floor(P' - (log2 k)/2 - s - 2^-23);
    A'B' = k 2^{2(e+s)} stays below P/2, and the emulated product is exactly k alpha^2."""
    N, m, n = 20, 2, 3
    c = orc.constants(N)
    alpha = 2.0**s
    A = synthetic.ones_matrix(m, k, alpha)
    B = synthetic.ones_matrix(k, n, alpha)
    e, _ = orc.shifts_a(A, m, k, N)
    lg = int(math.log2(k))
    expect = math.floor(Fraction(c["pprime"]) - Fraction(lg, 2) - s - Fraction(1, 2**23))
    assert np.all(e == expect)
    assert expect + s == (72 if k == 1024 else 70)
    assert k * 2 ** (2 * (expect + s)) < c["P"] / 2
    C = synthetic.colmajor_view(orc.dgemm(A, B, m, n, k, N))
    assert np.all(C == k * alpha * alpha)


@pytest.mark.parametrize("N", [8, 14, 20])
def test_log2_margin_of_proposed_mu(orc, N):
    """eq. (proposed-mu) keeps a 4u_32 margin on log2: e <= floor(P' - 0.5 (log2 a_norm + 4u_32))
    with the exact log2.  Norms are scanned float by float across the point where the margin
    decides the floor, so dropping the margin (or rounding t the wrong way) fails here."""
    getcontext().prec = 60
    c = orc.constants(N)
    pp = Fraction(c["pprime"])
    ln2 = Decimal(2).ln()
    hit = 0
    for s in range(-40, 41):
        w = pp - Fraction(s, 2)
        frac = w - math.floor(w)
        if not (Fraction(1, 64) < frac < Fraction(1, 2)):
            continue
        x0 = np.float32(2.0 ** (2 * float(frac)))
        for step in range(-48, 49):
            xf = float(np.float32(x0) + np.float32(step) * np.spacing(np.float32(x0)))
            a_norm = math.ldexp(xf, s)
            e = orc.alg2_shift(a_norm, c["pprime"])
            lg = Decimal(xf).ln() / ln2 + s
            limit = math.floor(Decimal(c["pprime"]) - Decimal("0.5") * (lg + Decimal(2) ** -22))
            assert e <= limit
            assert e >= limit - 1
            hit += math.floor(Decimal(c["pprime"]) - Decimal("0.5") * lg) != limit
    assert hit > 0      # the scan reached points where only the margin moves the floor


def _ru(x: Fraction) -> float:
    """The smallest double >= x (rounding upward), from exact rational arithmetic."""
    try:
        d = float(x)
    except OverflowError:
        return math.inf
    return d if Fraction(d) >= x else math.nextafter(d, math.inf)


def _ru32(x: Fraction) -> float:
    """The smallest single >= x >= 0 (rounding upward), from exact rational arithmetic."""
    if x == 0:
        return 0.0
    f = np.float32(float(x)) if x < 2**120 else np.float32(2.0**120)
    while Fraction(float(f)) < x:
        f = np.nextafter(f, np.float32(np.inf))
    while f > 0 and Fraction(float(np.nextafter(f, np.float32(0)))) >= x:
        f = np.nextafter(f, np.float32(0))
    return float(f)


def _exp_field(a: float) -> int:
    """Biased exponent field of a finite nonzero double, a subnormal counting as 1."""
    e = (struct.unpack("<Q", struct.pack("<d", a))[0] >> 52) & 0x7FF
    return max(int(e), 1)


def blocked_norm_ru(line, block=256, group=16):
    """The squared norm of Section 4 in single precision with rounding up, as the reading
    defines it, from exact rational arithmetic: blocks of `block` terms in groups of `group`;
    before a group, E becomes the largest of E, 1 and the group's exponent fields and a rise of E
    by d rescales f to single-up(f 2^(-2d)); each term then adds x = single-up(|a| 2^(1023 - E))
    as f = single-up(x^2 + f); the block value is double-up(double-up(f 2^(E - 1023))
    2^(E - 1023)), and the block values are added in order, rounded up."""
    total = 0.0
    for b0 in range(0, len(line), block):
        blk = [abs(float(a)) for a in line[b0:b0 + block]]
        E, f = 0, 0.0
        has_nan = any(math.isnan(a) for a in blk)
        has_inf = any(math.isinf(a) for a in blk)
        if not (has_nan or has_inf):
            for g0 in range(0, len(blk), group):
                grp = blk[g0:g0 + group]
                En = max([E, 1] + [_exp_field(a) for a in grp if a != 0.0])
                if En > E and f:
                    f = _ru32(Fraction(f) / Fraction(2) ** (2 * (En - E)))
                E = En
                for a in grp:
                    if a != 0.0:
                        x = _ru32(Fraction(a) * Fraction(2) ** (1023 - E))
                        f = _ru32(Fraction(x) ** 2 + Fraction(f))
        if has_nan:
            v = math.nan
        elif has_inf:
            v = math.inf
        elif E == 0:
            v = 0.0
        else:
            p = Fraction(2) ** (E - 1023)
            v = _ru(Fraction(_ru(Fraction(f) * p)) * p)
        if math.isnan(v) or math.isnan(total):
            total = math.nan
        elif math.isinf(v) or math.isinf(total):
            total = math.inf
        else:
            total = _ru(Fraction(total) + Fraction(v))
    return total


def _same(a: float, b: float) -> bool:
    return (math.isnan(a) and math.isnan(b)) or a == b


@pytest.mark.parametrize("k", [255, 256, 257, 700, 2048])
def test_blocked_norm_order_and_bound(orc, k):
    """The squared norm of Section 4 rounds every operation up, in single or double precision;
    the reading takes single precision on terms rescaled exactly by a power of two that follows
    the largest term seen, in blocks of 256 terms taken 16 at a time.  The oracle matches that sequence of upward roundings bit for
    bit (against exact rationals), bounds the exact sum from above and stays within
    (2k + 4 blocks) 2^-23 of it."""
    m = 6
    A = synthetic.paper_matrix(m, k, 2.0, 40 + k)
    _, nr = orc.shifts_a(A, m, k, 14)
    M = synthetic.colmajor_view(A)
    blocks = -(-k // 256)
    for i, S in enumerate(exact_sq_norms_rows(A)):
        assert float(nr[i]) == blocked_norm_ru(M[i]), i
        assert Fraction(float(nr[i])) >= S
        assert Fraction(float(nr[i])) <= S * (1 + Fraction(2 * k + 4 * blocks, 2**23))


def _wide_lines():
    """Lines that reach every branch of the reading: wide magnitude ranges (the block maximum
    rising late, terms 2^-140 below it that round to subnormal singles), subnormal doubles, zeros,
    huge terms whose block value overflows, and non-finite terms."""
    g = np.random.Generator(np.random.PCG64(77))
    lines = []
    lines.append(np.sort(np.abs(g.standard_normal(300))) * 2.0 ** g.integers(-60, 60, 300))
    lines.append(g.standard_normal(600) * np.exp(16.0 * g.standard_normal(600)))
    lines.append(np.concatenate([g.random(100) * 2.0**-140, [1.5], g.random(100) * 2.0**-75]))
    lines.append(g.random(300) * 5e-310)                        # subnormal doubles only
    lines.append(np.concatenate([g.random(50) * 5e-310, g.random(50) * 1e-300, [0.0] * 20]))
    z = g.standard_normal(513)
    z[::7] = 0.0
    lines.append(z)
    lines.append(np.concatenate([g.random(10), [1e200], g.random(10)]))   # overflows: +Inf
    lines.append(np.concatenate([g.random(10), [np.inf], g.random(10)]))
    lines.append(np.concatenate([g.random(300), [np.nan], g.random(10)]))
    lines.append(np.concatenate([[2.0**-1000], g.random(5) * 2.0**1000]))  # rises by 2000 binades
    lines.append(g.random(400) * 2.0**-1060)                    # deep subnormals
    return lines


def test_blocked_norm_wide_ranges_match_definition(orc):
    """The oracle's norms equal the exact-rational restatement of the reading on lines that reach
    its rescalings, subnormal singles and doubles, zeros, overflow and non-finite terms; finite
    ones bound the exact sum from above."""
    for idx, line in enumerate(_wide_lines()):
        k = len(line)
        A = np.ascontiguousarray(line.reshape(k, 1))   # column-major 1 x k, lda = 1
        _, nr = orc.shifts_a(A, 1, k, 14)
        want = blocked_norm_ru(line)
        assert _same(float(nr[0]), want), (idx, float(nr[0]), want)
        if math.isfinite(want):
            S = sum(Fraction(float(v)) ** 2 for v in line)
            assert Fraction(want) >= S, idx


def test_blocked_norm_differs_from_sequential_where_it_should():
    """The blocked and the one-block upward sums are different readings of the same definition:
    on a line whose first block ends on a large partial sum they differ, which the order pin
    above can tell apart."""
    line = [1.0] * 256 + [2.0**-20] * 300
    assert blocked_norm_ru(line) != blocked_norm_ru(line, block=len(line))
