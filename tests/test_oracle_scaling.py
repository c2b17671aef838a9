"""Pins for the scaling step (Algorithm 2, Section 4) in the oracle.

Checked against: the exact rational squared norm (rounding-up must give an upper bound), the
CRT condition of eq. (proposed-condition) in exact rational arithmetic, near-maximality of
each shift against a 60-digit decimal optimum, the exact scale-invariance argument of
Section 4 for alpha = 2^s, the effective-bit-width formula of Section 3.1 for non-power-of-two
alpha, and the all-ones worked example of Section 3.1 in closed form.
"""
import math
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
        assert Fraction(float(nr[i])) <= S * (1 + Fraction(k + 2, 2**52))


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
    d = float(x)
    return d if Fraction(d) >= x else math.nextafter(d, math.inf)


def blocked_norm_ru(line, block=256):
    """Upward-rounded squared norm in the blocked order, every operation rounded upward from its
    exact rational value: fma per term within each block of `block` terms, then the block sums
    added in order."""
    total = 0.0
    for b0 in range(0, len(line), block):
        s = 0.0
        for a in line[b0:b0 + block]:
            s = _ru(Fraction(float(a)) ** 2 + Fraction(s))
        total = _ru(Fraction(total) + Fraction(s))
    return total


@pytest.mark.parametrize("k", [255, 256, 257, 700, 2048])
def test_blocked_norm_order_and_bound(orc, k):
    """The squared norm of Section 4 rounds every operation up; with no order given by the paper,
    the reading sums blocks of 256 terms in order, then the block sums in order.  The oracle
    matches that sequence of upward roundings bit for bit (against exact rationals), bounds the
    exact sum from above and stays within (k + blocks + 2) 2^-52 of it."""
    m = 6
    A = synthetic.paper_matrix(m, k, 2.0, 40 + k)
    _, nr = orc.shifts_a(A, m, k, 14)
    M = synthetic.colmajor_view(A)
    blocks = -(-k // 256)
    for i, S in enumerate(exact_sq_norms_rows(A)):
        assert float(nr[i]) == blocked_norm_ru(M[i]), i
        assert Fraction(float(nr[i])) >= S
        assert Fraction(float(nr[i])) <= S * (1 + Fraction(k + blocks + 2, 2**52))


def test_blocked_norm_differs_from_sequential_where_it_should():
    """The blocked and the sequential upward sums are different readings of the same definition:
    on a line whose first block ends on a large partial sum they differ in the last bit, which the
    order pin above can tell apart."""
    line = [1.0] * 256 + [2.0**-30] * 300
    seq = 0.0
    for a in line:
        seq = _ru(Fraction(a) ** 2 + Fraction(seq))
    assert blocked_norm_ru(line) != seq
