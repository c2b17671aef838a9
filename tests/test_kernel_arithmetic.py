"""Exactness arguments of the GPU kernels' integer arithmetic, checked with exact Python integers
(no GPU, and independent of both the CUDA sources and the oracle).

Conversion (Step 2): for every modulus and limb count, the limb combination t stays below 2^31,
the 2^39 magic quotient of x = t + h is exact for every such x, and y - q p with y = 1.5 2^23 + t
is the float 1.5 2^23 + s with s the symmetric residue.  Reconstruction (eq. os2-C''): with the
moduli in pairs and K_l = (prod_g / p_l) q_l mod prod_g, the biased pair sums stay in [0, 2^25),
X = sum_g (P / prod_g) v_g is congruent to sum_l P_l q_l c_l modulo P, and the 48-bit fixed-point
estimate of X / P is within 2^-20."""
import math
import random
from fractions import Fraction

import pytest

# eq. (moduli): the twenty moduli, largest first
MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 191,
          181, 179, 173]
FLOAT_B = 0x4B400000          # bits of 1.5 2^23
MAGIC_SHIFT = 39


@pytest.mark.parametrize("p", MODULI[1:])
def test_convert_quotient_and_offset_exact(p):
    h = (p - 1) // 2
    m = -(-(1 << MAGIC_SHIFT) // p)                      # ceil(2^39 / p)
    e = m * p - (1 << MAGIC_SHIFT)
    assert 0 <= e < p
    for limbs in (1, 2, 3, 4):
        t_max = ((1 << 21) - 1) * (1 + (limbs - 1) * (p - 1))   # limb sum with 2^(21j) mod p < p
        x_max = t_max + h
        assert x_max < 1 << 31
        # floor(x m / 2^39) = floor(x / p) for every x with x e < 2^39 (the error term stays
        # below 1/p), which holds up to x_max:
        assert x_max * e < 1 << MAGIC_SHIFT
    rng = random.Random(p)
    t_max = ((1 << 21) - 1) * (1 + 3 * (p - 1))
    bias = FLOAT_B - h
    for t in [0, 1, p - 1, p, t_max - 1, t_max] + [rng.randrange(t_max + 1) for _ in range(2000)]:
        y = (FLOAT_B + t) & 0xFFFFFFFF
        x = (y - bias) & 0xFFFFFFFF
        assert x == t + h
        xm = (y * m + ((-bias * m) & ((1 << 64) - 1))) & ((1 << 64) - 1)   # one 64-bit multiply-add
        q = xm >> MAGIC_SHIFT
        assert q == x // p
        fb = (y - q * p) & 0xFFFFFFFF
        s = fb - FLOAT_B
        assert -h <= s <= h and (s - t) % p == 0          # the symmetric residue of t
        assert abs(s) < 1 << 22                            # bits FLOAT_B + s are the float B + s


def pair_tables(N):
    ps = MODULI[:N]
    P = math.prod(ps)
    q = [pow(P // p, -1, p) for p in ps]
    groups = [list(range(2 * g, min(2 * g + 2, N))) for g in range((N + 1) // 2)]
    K = [0] * N
    tab = []
    for ls in groups:
        prod = math.prod(ps[l] for l in ls)
        for l in ls:
            K[l] = (prod // ps[l]) * q[l] % prod
        tab.append(dict(ls=ls, prod=prod, bias=256 * prod, PG=P // prod,
                        R46=((1 << 46) + prod // 2) // prod))
    return ps, P, q, K, tab


@pytest.mark.parametrize("N", range(2, 21))
def test_crt_pair_groups_exact(N):
    ps, P, q, K, tab = pair_tables(N)
    rng = random.Random(N)
    cases = [[-128] * N, [127] * N, [0] * N]
    cases += [[rng.randint(-128, 127) for _ in range(N)] for _ in range(400)]
    for c in cases:
        S = X = 0
        for g in tab:
            v = (g["bias"] + sum(c[l] * K[l] for l in g["ls"])) & 0xFFFFFFFF  # wraps mod 2^32
            assert 0 <= v < 1 << 25                        # so the wrapped value is exact
            if len(g["ls"]) == 2:                          # a pair: a 32-bit constant
                assert g["R46"] < 1 << 32
            S += v * g["R46"]
            X += g["PG"] * v
        assert S < 1 << 64
        assert (X - sum(c[l] * (P // ps[l]) * q[l] for l in range(N))) % P == 0
        assert abs(Fraction(S, 1 << 46) - Fraction(X, P)) < Fraction(1, 1 << 18)
        Q = (S + (1 << 45)) >> 46
        Y = X - Q * P
        frac = S & ((1 << 46) - 1)
        if abs(frac - (1 << 45)) >= 1 << 36:               # away from a tie: already reduced
            assert -P // 2 <= Y < P // 2
        else:                                              # near a tie: one correction at most
            assert -P <= Y < P


def _byte_perm(x, y, s):
    """The byte permute of the CUDA ISA: result byte i is byte (nibble i of s) of y:x."""
    src = [(x >> (8 * b)) & 0xFF for b in range(4)] + [(y >> (8 * b)) & 0xFF for b in range(4)]
    return sum(src[(s >> (4 * i)) & 7] << (8 * i) for i in range(4))


def _dp2a(a, b, c, hi):
    """dp2a.{lo,hi}.u32.s32: c + a.h0 * b.byte(0 or 2) + a.h1 * b.byte(1 or 3), modulo 2^32, with
    the halves of a unsigned and the bytes of b signed."""
    sb = [((b >> (8 * i)) & 0xFF) - (256 if (b >> (8 * i)) & 0x80 else 0) for i in range(4)]
    h0, h1 = a & 0xFFFF, a >> 16
    k = 2 if hi else 0
    return (c + h0 * sb[k] + h1 * sb[k + 1]) & 0xFFFFFFFF


@pytest.mark.parametrize("N", range(2, 21))
def test_crt_pair_sums_by_byte_permute_and_dot_product(N):
    """The reconstruction reads four entries' residues per plane in one 32-bit word, interleaves
    the words of the two planes of a pair with byte permutes (0x5140: entries 0 and 1, 0x7362:
    entries 2 and 3) and forms each pair sum with one two-way dot product of the packed
    constants K_2g | K_2g+1 << 16: the same v_g as the residue-by-residue sum."""
    ps, P, q, K, tab = pair_tables(N)
    rng = random.Random(100 + N)
    for _ in range(200):
        c = [[rng.randint(-128, 127) for _ in range(4)] for _ in range(N)]  # c[l][entry]
        words = [sum((c[l][e] & 0xFF) << (8 * e) for e in range(4)) for l in range(N)]
        for g in tab:
            ls = g["ls"]
            assert all(0 <= K[l] < 1 << 16 for l in ls)
            kpair = K[ls[0]] | ((K[ls[1]] << 16) if len(ls) > 1 else 0)
            w0 = words[ls[0]]
            w1 = words[ls[1]] if len(ls) > 1 else 0
            lo, hi = _byte_perm(w0, w1, 0x5140), _byte_perm(w0, w1, 0x7362)
            for e in range(4):
                want = (g["bias"] + sum(c[l][e] * K[l] for l in ls)) & 0xFFFFFFFF
                got = _dp2a(kpair, lo if e < 2 else hi, g["bias"], e & 1)
                assert got == want
