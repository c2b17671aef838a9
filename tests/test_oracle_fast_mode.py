"""Pins for the original fast mode (Section 2.3, eq. fast-mode-mu, Algorithm 1) in the oracle.

Checked against: the exact rational definition of delta (eq. delta), a 60-digit decimal value of
P'_fast, the paper's statement about the all-ones example of Section 3.1 (golden fixture: CRT
recovery fails exactly for alpha <= 2^-2 at N = 20), the breakdown that Fig. 3 reports for that
region, and the effective-precision formula of Section 3.1 (bit width falling as alpha grows).
"""
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fixture_claims():
    out = {}
    with open(os.path.join(GOLDEN, "all_ones_fast_mode_claim.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, s = line.split()
            out[int(k)] = int(s)
    return out


def test_delta_is_single_up(orc):
    d = orc.fast_delta()
    exact = Fraction(1, 2) / (1 - Fraction(4, 2**24))
    assert Fraction(d) >= exact
    below = float(np.nextafter(np.float32(d), np.float32(0)))
    assert Fraction(below) < exact


@pytest.mark.parametrize("N", [8, 14, 20])
def test_pprime_fast_is_single_down(orc, N):
    getcontext().prec = 60
    P = orc.constants(N)["P"]
    exact = Decimal(P - 1).ln() / Decimal(2).ln() / 2 - Decimal("1.5")
    f = np.float32(orc.pprime_fast(N))
    assert Decimal(float(f)) <= exact < Decimal(float(np.nextafter(f, np.float32(np.inf))))
    assert orc.pprime_fast(N) == pytest.approx(orc.constants(N)["pprime"] - 1.0, abs=1e-5)


@pytest.mark.parametrize("k", sorted(fixture_claims()))
def test_all_ones_crt_failure_region(orc, k):
    """Section 3.1: with all-ones A = B = alpha 1 and N = 20, fast mode makes
    (A'B')_ij = k 2^{2(e+s)} exceed P/2 exactly in the region alpha = 2^s <= 2^-2."""
    fails_up_to = fixture_claims()[k]
    N = 20
    P = orc.constants(N)["P"]
    for s in range(-10, 11):
        A = synthetic.ones_matrix(2, k, 2.0**s)
        e = orc.shifts_mode(A, 2, k, N, orc.FAST_MODE)
        assert e[0] == e[1]
        entry = 2 ** (int(e[0]) + s)            # every a' = trunc(2^e 2^s) = 2^(e+s)
        fails = 2 * k * entry * entry >= P      # |A'B'| >= P/2: CRT recovery cannot succeed
        assert fails == (s <= fails_up_to), (k, s)
        e_prop = orc.shifts_mode(A, 2, k, N, orc.PROPOSED_MODE)
        entry = 2 ** (int(e_prop[0]) + s)
        assert 2 * k * entry * entry < P        # the proposed scaling never fails


@pytest.mark.parametrize("s", [-3, -6])
def test_fast_mode_breakdown_on_all_ones(orc, s):
    """Fig. 3: in the failure region the fast-mode product is wrong (relative error ~1),
    while the proposed scaling returns k alpha^2 exactly."""
    k, m, n, N = 1024, 3, 2, 20
    alpha = 2.0**s
    A = synthetic.ones_matrix(m, k, alpha)
    B = synthetic.ones_matrix(k, n, alpha)
    exact = k * alpha * alpha
    Cf = orc.dgemm_mode(A, B, m, n, k, N, orc.FAST_MODE)
    Cp = orc.dgemm_mode(A, B, m, n, k, N, orc.PROPOSED_MODE)
    assert np.all(Cp == exact)
    assert np.all(np.abs(Cf - exact) / exact > 0.5)


def test_fast_mode_bits_fall_with_alpha(orc):
    """eq. (effective-precision-fast): when delta (log2~(sum a^2) + 2 log2 alpha) > 1 the bit
    width floor(P'_fast - max(1, ...)) + 1 decreases as alpha grows; the proposed one does not."""
    m, k, N = 16, 256, 20
    A = synthetic.paper_matrix(m, k, 1.0, 42)
    M = np.abs(synthetic.colmajor_view(A))
    def bits(mode, s):
        e = orc.shifts_mode(A * 2.0**s, m, k, N, mode)
        return e + np.floor(np.log2(M.max(axis=1) * 2.0**s)).astype(int) + 1
    assert np.all(bits(orc.FAST_MODE, 10) < bits(orc.FAST_MODE, 0))
    assert np.all(bits(orc.FAST_MODE, 20) < bits(orc.FAST_MODE, 10))
    assert np.array_equal(bits(orc.PROPOSED_MODE, 10), bits(orc.PROPOSED_MODE, 0))


def test_fast_mode_still_satisfies_its_own_bound_on_random_data(orc):
    """For ordinary data (alpha = 1) fast mode keeps sum |a'||b'| < P/2 (eq. os2-condition)."""
    m, n, k, N = 20, 16, 300, 14
    A = synthetic.paper_matrix(m, k, 1.0, 3)
    B = synthetic.paper_matrix(k, n, 1.0, 4)
    e = orc.shifts_mode(A, m, k, N, orc.FAST_MODE)
    f = orc.shifts_mode(B, n, k, N, orc.FAST_MODE, side=1)
    Am, Bm = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    P = orc.constants(N)["P"]
    Ap = [[math.trunc(Fraction(float(Am[i, h])) * Fraction(2) ** int(e[i])) for h in range(k)]
          for i in range(m)]
    Bp = [[math.trunc(Fraction(float(Bm[h, j])) * Fraction(2) ** int(f[j])) for j in range(n)]
          for h in range(k)]
    for i in range(m):
        for j in range(n):
            assert 2 * sum(abs(Ap[i][h] * Bp[h][j]) for h in range(k)) < P


@pytest.mark.parametrize("s", [-3, -2])
def test_fast_mode_breakdown_on_random_phi_half(orc, s):
    """Section 3.2, Fig. 2: with phi = 0.5 and m = n = k = 1024 (N = 20) the fast mode breaks
    down (relative error ~1 on some entries) for alpha <= 2^-3 and not above; the proposed
    scaling stays at the level of one rounding."""
    m = n = k = 1024
    N = 20
    A = synthetic.paper_matrix(m, k, 0.5, 11) * 2.0**s
    B = synthetic.paper_matrix(k, n, 0.5, 12) * 2.0**s
    Cf = orc.dgemm_mode(A, B, m, n, k, N, orc.FAST_MODE)
    Cp = orc.dgemm_mode(A, B, m, n, k, N, orc.PROPOSED_MODE)
    diff = np.abs(Cf - Cp)
    J = np.sort(np.argsort(diff.max(axis=1))[-4:]).astype(np.int32)
    I = np.sort(np.argsort(diff.max(axis=0))[-4:]).astype(np.int32)
    hi, lo = orc.dd_block(A, B, k, I, J)
    err_f, _ = orc.max_rel_error(Cf[np.ix_(J, I)], hi, lo)
    err_p, _ = orc.max_rel_error(Cp[np.ix_(J, I)], hi, lo)
    assert err_p < 2e-16
    assert (err_f > 0.5) == (s <= -3)
    if s > -3:
        assert np.all(diff <= 1e-13 * np.abs(Cp))
