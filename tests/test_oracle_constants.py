"""Pins for Step 1 of Ozaki scheme II (Section 2.2) and P'_prop (Section 4) in the oracle.

Each check uses something other than the oracle's own arithmetic: the moduli list printed in
the paper (eq. moduli), number theory (coprimality, the CRT identity P_i q_i = 1 mod p_i),
Python's exact integers, and a 60-digit decimal logarithm for P'_prop.
"""
import math
import os
import random
from decimal import Decimal, getcontext

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_moduli():
    vals = []
    with open(os.path.join(GOLDEN, "moduli.txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            vals += [int(t) for t in line.split()]
    return vals


def test_moduli_are_the_papers_list(orc):
    mod = paper_moduli()
    assert len(mod) == 20
    for N in range(2, 21):
        assert orc.constants(N)["p"] == mod[:N]


def test_moduli_pairwise_coprime_and_int8_sized():
    mod = paper_moduli()
    for a in range(20):
        assert 2 <= mod[a] <= 256
        for b in range(a + 1, 20):
            assert math.gcd(mod[a], mod[b]) == 1


@pytest.mark.parametrize("N", range(2, 21))
def test_P_and_crt_weights(orc, N):
    c = orc.constants(N)
    P = math.prod(c["p"])
    assert c["P"] == P
    for l, (p, q) in enumerate(zip(c["p"], c["q"])):
        Pl = P // p
        assert 0 <= q < p
        assert (Pl * q) % p == 1            # q_l is the inverse of P_l modulo p_l
        assert c["Pq"][l] == Pl * q
        for j, pj in enumerate(c["p"]):     # P_l q_l vanishes modulo every other modulus
            if j != l:
                assert c["Pq"][l] % pj == 0


@pytest.mark.parametrize("N", range(2, 21))
def test_pprime_is_single_down_of_log_bound(orc, N):
    """P'_prop = single-down(log2(P - 1)/2 - 0.5) (Section 4), checked with 60-digit decimals."""
    getcontext().prec = 60
    c = orc.constants(N)
    Pm1 = Decimal(c["P"] - 1)
    exact = Pm1.ln() / Decimal(2).ln() / 2 - Decimal("0.5")
    f = np.float32(c["pprime"])
    up = np.nextafter(f, np.float32(np.inf))
    assert Decimal(float(f)) <= exact < Decimal(float(up))


def test_crt_round_trip_on_symmetric_range(orc):
    """CRT theorem (Section 2.2): residues of any x with |x| < P/2 reconstruct x exactly."""
    rng = random.Random(7)
    for N in (2, 3, 8, 14, 16, 17, 20):
        P = math.prod(paper_moduli()[:N])
        half = (P - 1) // 2
        xs = [0, 1, -1, half, -half, half - 1, -(half - 1), P // 2 - 1]
        xs += [rng.randrange(-half, half + 1) for _ in range(60)]
        res = orc.int_residues(xs, N)
        for x, r in zip(xs, res):
            for l, p in enumerate(paper_moduli()[:N]):
                assert (x - int(r[l])) % p == 0
                assert -(p // 2) <= int(r[l]) <= (p - 1) // 2
        # feed the residues through the oracle's Step 3 as an m x 1 "product" array
        c = np.ascontiguousarray(res.T.reshape(N, len(xs), 1).astype(np.int8))
        back = orc.crt_exact(c)[:, 0]
        assert [int(v) for v in back] == xs


def test_residue_tie_for_256_maps_to_minus_128(orc):
    """Reading of rmod for the even modulus 256: the tie goes to -128 (INT8 range)."""
    xs = [128, -128, 384, -384, 128 + 256 * 7]
    res = orc.int_residues(xs, 2)
    assert all(int(r[0]) == -128 for r in res)


def test_bigint_to_double_is_correctly_rounded(orc):
    """Rounded conversion of 256-bit integers equals Python's correctly rounded int->float."""
    rng = random.Random(3)
    xs = [0, 1, -1, 2**53 + 1, 2**54 + 2, (2**53 + 1) * 2**10 + 2**9, (2**53 + 3) * 2**10 + 2**9,
          -((2**53 + 1) * 2**40 + 2**39), 2**155 - 1, -(2**155 - 1), 2**200 + 2**147]
    for _ in range(300):
        b = rng.randrange(1, 200)
        xs.append(rng.randrange(-(2**b), 2**b))
    got = orc.words_to_double(xs)
    for x, g in zip(xs, got):
        assert g == float(x), x
