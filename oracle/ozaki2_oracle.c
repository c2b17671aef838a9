/*
 * ozaki2_oracle.c -- CPU oracle for Ozaki scheme II DGEMM emulation, fast mode with the
 * scale-invariant scaling of Algorithm 2 (Kawakami & Takahashi, "Improved Scaling for Fast
 * Mode of Ozaki Scheme II").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * and reference legs may load it.  It shares no code, header, table or constant generator with the CUDA
 * library; it takes matrices as arguments and never calls the GPU.
 *
 * Every step follows the paper's definitions in the paper's order:
 *   Section 2.1  notation: mod, rmod (round half to even), trunc, single-up / single-down.
 *   Section 2.2  Theorem (CRT) and Steps 1-4 of Ozaki scheme II.
 *   Section 4    proposed scaling: eq. (proposed-mu) / (proposed-nu), P'_prop, Algorithm 2.
 *   Section 3.2  eq. (moduli): the 20 moduli, of which the first N are used.
 * Readings where the paper is silent are marked "reading:" in the comments.
 *
 * Arithmetic: int64 for residue dot products (exact for any k < 2^48), a 256-bit two's
 * complement integer for a', P, P_i q_i, C' and C'' (P reaches 2^156 at N = 20, beyond
 * __int128), FP64 for the scaling.  The row/column norms are evaluated with the FPU in
 * round-upward mode; compile with -frounding-math -ffp-contract=off.
 *
 * Parity pins (see tests/test_oracle_*.py): number-theoretic identities of the constants,
 * an exact-decimal check of P'_prop, exact-rational checks of the CRT bound and of
 * near-maximality of every shift, exact scale invariance for alpha = 2^s, the all-ones
 * closed form of Section 3.1, brute-force big-integer A'B' on tiny inputs, correctly rounded
 * conversion, and a rigorous truncation-error bound against the exact rational product.
 */
#include <fenv.h>
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FENV_ACCESS ON

#define ORC_MAX_MODULI 20
/* Accurate mode: a line whose products with every line of the other operand vanish
 * (max of its row/column of C-bar is 0) gets this shift, which makes every a' zero. */
#define ORC_SHIFT_VANISH (-1100)
/* A line whose squared norm is not finite gets this shift; its outputs become NaN. */
#define ORC_SHIFT_NONFINITE INT32_MIN

/* eq. (moduli), Section 3.2: the GEMMul8 moduli.  Reading: for N < 20 the first N are used. */
static const int MODULI[ORC_MAX_MODULI] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227,
                                           223, 217, 211, 199, 197, 193, 191, 181, 179, 173};

/* ------------------------------------------------------------------------------------ */
/* 256-bit two's complement integer, w[0] least significant.                             */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t w[4];
} i256;

static i256 i256_from_i64(int64_t v) {
    i256 r;
    uint64_t ext = v < 0 ? ~0ull : 0ull;
    r.w[0] = (uint64_t)v;
    r.w[1] = r.w[2] = r.w[3] = ext;
    return r;
}
static i256 i256_from_u64(uint64_t v) {
    i256 r = {{v, 0, 0, 0}};
    return r;
}
static int i256_is_neg(i256 a) { return (int)(a.w[3] >> 63); }
static int i256_is_zero(i256 a) { return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) == 0; }

static i256 i256_add(i256 a, i256 b) {
    i256 r;
    uint64_t carry = 0;
    for (int i = 0; i < 4; ++i) {
        unsigned __int128 s = (unsigned __int128)a.w[i] + b.w[i] + carry;
        r.w[i] = (uint64_t)s;
        carry = (uint64_t)(s >> 64);
    }
    return r;
}
static i256 i256_neg(i256 a) {
    i256 r;
    for (int i = 0; i < 4; ++i) r.w[i] = ~a.w[i];
    return i256_add(r, i256_from_u64(1));
}
static i256 i256_sub(i256 a, i256 b) { return i256_add(a, i256_neg(b)); }
static i256 i256_abs(i256 a) { return i256_is_neg(a) ? i256_neg(a) : a; }

/* Unsigned comparison of two non-negative values. */
static int u256_cmp(i256 a, i256 b) {
    for (int i = 3; i >= 0; --i) {
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    }
    return 0;
}
/* Non-negative value times a 64-bit unsigned factor (caller keeps the product below 2^255). */
static i256 u256_mul_u64(i256 a, uint64_t m) {
    i256 r;
    uint64_t carry = 0;
    for (int i = 0; i < 4; ++i) {
        unsigned __int128 p = (unsigned __int128)a.w[i] * m + carry;
        r.w[i] = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
    }
    return r;
}
/* Signed value times a signed 64-bit factor. */
static i256 i256_mul_i64(i256 a, int64_t m) {
    int neg = i256_is_neg(a) ^ (m < 0);
    uint64_t um = m < 0 ? (uint64_t)(-(m + 1)) + 1u : (uint64_t)m;
    i256 r = u256_mul_u64(i256_abs(a), um);
    return neg ? i256_neg(r) : r;
}
static int u256_bit(i256 a, int i) { return (int)((a.w[i >> 6] >> (i & 63)) & 1u); }
static i256 u256_shl(i256 a, int n) { /* 0 <= n < 256 */
    i256 r = {{0, 0, 0, 0}};
    int ws = n / 64, bs = n % 64;
    for (int i = 3; i >= ws; --i) {
        uint64_t v = a.w[i - ws] << bs;
        if (bs && i - ws - 1 >= 0) v |= a.w[i - ws - 1] >> (64 - bs);
        r.w[i] = v;
    }
    return r;
}
static i256 u256_shr(i256 a, int n) { /* 0 <= n < 256, logical */
    i256 r = {{0, 0, 0, 0}};
    int ws = n / 64, bs = n % 64;
    for (int i = 0; i + ws <= 3; ++i) {
        uint64_t v = a.w[i + ws] >> bs;
        if (bs && i + ws + 1 <= 3) v |= a.w[i + ws + 1] << (64 - bs);
        r.w[i] = v;
    }
    return r;
}
/* Index of the highest set bit of a non-negative value, -1 for zero. */
static int u256_msb(i256 a) {
    for (int i = 3; i >= 0; --i)
        if (a.w[i]) return 64 * i + 63 - __builtin_clzll(a.w[i]);
    return -1;
}
/* Shift-and-subtract long division of non-negative a by positive d, one quotient bit per
 * step from the highest possible one down. */
static void u256_divmod(i256 a, i256 d, i256* q, i256* r) {
    i256 Q = {{0, 0, 0, 0}};
    int s = u256_msb(a) - u256_msb(d);
    for (; s >= 0; --s) {
        i256 ds = u256_shl(d, s);
        if (u256_cmp(a, ds) >= 0) {
            a = i256_sub(a, ds);
            Q.w[s >> 6] |= 1ull << (s & 63);
        }
    }
    *q = Q;
    *r = a;
}
/* Non-negative value modulo a small positive integer. */
static uint32_t u256_mod_small(i256 a, uint32_t p) {
    unsigned __int128 rem = 0;
    for (int i = 3; i >= 0; --i) rem = ((rem << 64) | a.w[i]) % p;
    return (uint32_t)rem;
}

/* x mod p (Section 2.1: x - p*floor(x/p)), a value in [0, p). */
static int64_t i256_mod(i256 x, int p) {
    if (!i256_is_neg(x)) return (int64_t)u256_mod_small(x, (uint32_t)p);
    int64_t m = (int64_t)u256_mod_small(i256_neg(x), (uint32_t)p);
    return m ? p - m : 0;
}
static int64_t i64_mod(int64_t x, int p) {
    int64_t m = x % p;
    return m < 0 ? m + p : m;
}
/* rmod(x, p) of Section 2.1 from m = x mod p: the representative nearest to zero.  For odd p
 * this is exactly rmod, range [-(p-1)/2, (p-1)/2].  Reading (p even, i.e. p = 256): the tie
 * x/p = j + 1/2 maps to -p/2, so residues lie in [-128, 127] and fit INT8; only the
 * congruence class matters to the CRT. */
static int sym_from_mod(int64_t m, int p) { return (int)(2 * m >= p ? m - p : m); }

/* rmod(x, P) of Section 2.1 for a 256-bit x: x - P*round(x/P), round half to even. */
static i256 i256_rmod(i256 x, i256 P) {
    i256 q, r;
    if (!i256_is_neg(x)) {
        u256_divmod(x, P, &q, &r);
    } else {
        i256 q1, r1;
        u256_divmod(i256_neg(x), P, &q1, &r1);
        if (i256_is_zero(r1)) {
            q = i256_neg(q1);
            r = r1;
        } else {
            q = i256_sub(i256_neg(q1), i256_from_u64(1));
            r = i256_sub(P, r1);
        }
    }
    /* x/P = q + r/P with 0 <= r < P; round(x/P) is q or q+1. */
    i256 twice_r = u256_shl(r, 1);
    int c = u256_cmp(twice_r, P);
    int round_up = c > 0 || (c == 0 && (q.w[0] & 1u));
    return round_up ? i256_sub(r, P) : r;
}

/* Round a 256-bit integer to the nearest double, ties to even. */
/* x rounded to `bits` significant bits (ties to even), returned as a double (bits <= 53; the
 * exponent is unbounded here, |x| < 2^255). */
static double i256_round_bits(i256 x, int bits) {
    int neg = i256_is_neg(x);
    i256 a = i256_abs(x);
    int msb = u256_msb(a);
    double v;
    if (msb < 0) return 0.0;
    if (msb <= bits - 1) {
        v = (double)a.w[0];
    } else {
        int shift = msb - (bits - 1);
        i256 top = u256_shr(a, shift);
        uint64_t mant = top.w[0]; /* `bits` bits */
        int half = u256_bit(a, shift - 1);
        int sticky = 0;
        for (int i = 0; i < shift - 1; ++i) sticky |= u256_bit(a, i);
        if (half && (sticky || (mant & 1u))) {
            mant += 1;
            if (mant == (1ull << bits)) {
                mant >>= 1;
                shift += 1;
            }
        }
        v = ldexp((double)mant, shift);
    }
    return neg ? -v : v;
}

static double i256_to_double(i256 x) { return i256_round_bits(x, 53); }

/* An integral double (|x| < 2^255) as a 256-bit integer. */
static i256 i256_from_integral_double(double x) {
    double a = fabs(x);
    if (a < 1.0) return i256_from_u64(0);
    int e;
    double f = frexp(a, &e);                    /* a = f * 2^e, f in [0.5, 1) */
    uint64_t mant = (uint64_t)ldexp(f, 53);     /* exact integer below 2^53 */
    int shift = e - 53;                         /* a = mant * 2^shift */
    i256 r = i256_from_u64(mant);
    r = shift >= 0 ? u256_shl(r, shift) : u256_shr(r, -shift);
    return x < 0 ? i256_neg(r) : r;
}

/* ------------------------------------------------------------------------------------ */
/* Rounding helpers (Section 2.1: single, single-up, single-down)                         */
/* ------------------------------------------------------------------------------------ */
static float ru_float(double v) { /* single-up of a double value */
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}
static float rd_float(double v) { /* single-down of a double value */
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}
static double sub_rd(double a, double b) { /* a - b rounded toward -inf */
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    volatile double r = a - b;
    fesetround(old);
    return r;
}

/* ------------------------------------------------------------------------------------ */
/* Step 1 (Section 2.2): moduli, P, P_i, q_i; and P'_prop (Section 4)                    */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int N;
    int p[ORC_MAX_MODULI];
    int q[ORC_MAX_MODULI];     /* q_i = P_i^{-1} mod p_i */
    i256 P;                    /* product of the moduli */
    i256 Pq[ORC_MAX_MODULI];   /* P_i * q_i */
    float pprime;              /* P'_prop */
    float pprime_fast;         /* P'_fast (original fast mode) */
} orc_consts;

static int mod_inverse(int a, int m) { /* extended Euclid; a and m coprime */
    int old_r = a, r = m, old_s = 1, s = 0;
    while (r != 0) {
        int quo = old_r / r, t;
        t = old_r - quo * r; old_r = r; r = t;
        t = old_s - quo * s; old_s = s; s = t;
    }
    int inv = old_s % m;
    return inv < 0 ? inv + m : inv;
}

/* log2 of a positive 256-bit integer, to double accuracy: bit length plus log2 of the top bits. */
static double u256_log2(i256 a) {
    int msb = u256_msb(a);
    if (msb < 64) return log2((double)a.w[0]);
    i256 top = u256_shr(a, msb - 63);
    return (double)(msb - 63) + log2((double)top.w[0]);
}

static int make_consts(int N, orc_consts* c) {
    if (N < 2 || N > ORC_MAX_MODULI) return -1;
    c->N = N;
    c->P = i256_from_u64(1);
    for (int l = 0; l < N; ++l) {
        c->p[l] = MODULI[l];
        c->P = u256_mul_u64(c->P, (uint64_t)MODULI[l]);
    }
    for (int l = 0; l < N; ++l) {
        i256 Pl = i256_from_u64(1);
        for (int j = 0; j < N; ++j)
            if (j != l) Pl = u256_mul_u64(Pl, (uint64_t)MODULI[j]);
        c->q[l] = mod_inverse((int)u256_mod_small(Pl, (uint32_t)MODULI[l]), MODULI[l]);
        c->Pq[l] = u256_mul_u64(Pl, (uint64_t)c->q[l]);
    }
    /* P'_prop := single-down(log2(P - 1)/2 - 0.5), Section 4 (eq. P-prime-proposed). */
    double lg = u256_log2(i256_sub(c->P, i256_from_u64(1)));
    c->pprime = rd_float(lg / 2.0 - 0.5);
    /* P'_fast := single-down(log2(P - 1)/2 - 1.5), Section 2.3 (original fast mode). */
    c->pprime_fast = rd_float(lg / 2.0 - 1.5);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Step 2 scaling: row/column squared norms and Algorithm 2                              */
/* ------------------------------------------------------------------------------------ */

/* a_norm := sum_h a_h^2 "computed with rounding-up" (the input of Algorithm 2); Section 4 lets the
 * sums be evaluated in single or double precision, each with rounding up.  Reading: single
 * precision on exactly rescaled terms, in blocks of ORC_NORM_BLOCK consecutive h (the paper
 * gives no order), each block taken in groups of ORC_NORM_GROUP consecutive terms (the last
 * group of a line may be shorter).  Before a group is added, E, the block's scale, becomes the
 * largest of E, 1 and the exponent fields of the group's terms (E = 0 at the start of a block);
 * a rise of E by d rescales the block's single-precision sum to f = single-up(f 2^(-2d)).  Each
 * term of the group then enters as x = single-up(|a| 2^(1023 - E)), a value in [0, 2), and
 * f = single-up(x x + f), from f = 0 in the order h.  The block's value is
 * double-up(double-up(f 2^(E - 1023)) 2^(E - 1023)), which is f 2^(2 (E - 1023)) whenever that is
 * a normal double; the block values are added in block order, each addition rounded upward.
 * Every operation rounds up and every rescaling is by a power of two, so a_norm bounds the exact
 * sum from above.  A block with an infinite term has value +Inf, one with a NaN term NaN (as an
 * FP64 sum of the squares would have). */
#define ORC_NORM_BLOCK 256
#define ORC_NORM_GROUP 16

/* single-up(v 2^k) for a finite v > 0 (v a double, k any integer).  Below 2^-200 the value is
 * under the least positive single, which single-up gives; otherwise the scaled value is a
 * normal double (>= 2^-252), computed exactly, then rounded up to single. */
static float ru_float_pow2(double v, int k) {
    if (ilogb(v) + k < -200) return 0x1p-149f;
    return ru_float(ldexp(v, k));
}

/* The biased exponent field of a finite nonzero double, a subnormal counting as 1. */
static int exp_field(double v) {
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    int e = (int)((b >> 52) & 0x7FF);
    return e ? e : 1;
}

static double line_norm_ru(const double* x, int64_t stride, int64_t len) {
    int old = fegetround();
    fesetround(FE_UPWARD);
    double total = 0.0;
    for (int64_t b0 = 0; b0 < len; b0 += ORC_NORM_BLOCK) {
        const int64_t b1 = b0 + ORC_NORM_BLOCK < len ? b0 + ORC_NORM_BLOCK : len;
        int E = 0;
        float f = 0.0f;
        int has_inf = 0, has_nan = 0;
        for (int64_t g0 = b0; g0 < b1; g0 += ORC_NORM_GROUP) {
            const int64_t g1 = g0 + ORC_NORM_GROUP < b1 ? g0 + ORC_NORM_GROUP : b1;
            int En = E > 1 ? E : 1;
            for (int64_t h = g0; h < g1; ++h) {
                const double a = fabs(x[h * stride]);
                if (isnan(a)) has_nan = 1;
                else if (isinf(a)) has_inf = 1;
                else if (a != 0.0 && exp_field(a) > En) En = exp_field(a);
            }
            if (has_nan || has_inf) continue;   /* the block's value is settled */
            if (En > E && f != 0.0f) f = ru_float_pow2((double)f, -2 * (En - E));
            E = En;
            for (int64_t h = g0; h < g1; ++h) {
                const double a = fabs(x[h * stride]);
                if (a == 0.0) continue;        /* x = 0 leaves f unchanged */
                const float xf = ru_float_pow2(a, 1023 - E);
                /* x x is exact in double (24-bit operands); the sum rounds up in double, then
                 * up to single: rounding up twice is rounding up once (every single is a double) */
                const double sum = (double)xf * (double)xf + (double)f;
                f = ru_float(sum);
            }
        }
        double v;
        if (has_nan) {
            v = NAN;
        } else if (has_inf) {
            v = INFINITY;
        } else if (E == 0) {
            v = 0.0;
        } else {
            const double p = ldexp(1.0, E - 1023);   /* exact: E in [1, 2046] */
            volatile double t = (double)f * p;        /* rounded up */
            v = t * p;                                /* rounded up */
        }
        total = total + v;
    }
    fesetround(old);
    return total;
}

/* Stand-in for __log2f on x in [1, 2] (eqs. flog2 and logf-bound).  Reading: libm's double
 * log2 of the float argument, rounded up to single.  Its error is far inside the 4u_32 that
 * Algorithm 2's +2u_32 margin assumes, so the bound of eq. (proposed-condition) still holds. */
float orc_log2_ru(float x) { return ru_float(log2((double)x)); }

/* Algorithm 2: log2(mu_i) from a_norm.
 *   s := floor(log2 a_norm)
 *   t := single-up(0.5 * log2f(a_norm / 2^s) + 2u_32)
 *   w := single-down(P'_prop - 0.5 s)
 *   return floor(w - t)
 * Readings: a_norm / 2^s is rounded up to single before the logarithm (the argument of
 * __log2f is single); w - t is floored exactly (subtraction rounded toward -inf, which
 * preserves the floor); a zero line gets shift 0; a non-finite a_norm is flagged. */
int orc_alg2_shift(double a_norm, float pprime) {
    if (a_norm == 0.0) return 0;
    if (!isfinite(a_norm)) return ORC_SHIFT_NONFINITE;
    int s = ilogb(a_norm);
    double xprime = scalbn(a_norm, -s);          /* in [1, 2), exact */
    float xf = ru_float(xprime);
    float lg = orc_log2_ru(xf);
    float t = ru_float(0.5 * (double)lg + 0x1p-23); /* 2u_32 = 2^-23; the sum is exact */
    float w = rd_float((double)pprime - 0.5 * (double)s);
    return (int)floor(sub_rd((double)w, (double)t));
}

static double mul_ru(double a, double b) { /* a * b rounded toward +inf */
    int old = fegetround();
    fesetround(FE_UPWARD);
    volatile double r = a * b;
    fesetround(old);
    return r;
}

/* delta := single-up(0.5 / (1 - 4u_32)), eq. (delta), Section 2.3. */
float orc_fast_delta(void) {
    int old = fegetround();
    fesetround(FE_UPWARD);
    volatile double den = 1.0 - 4.0 * 0x1p-24;   /* exact */
    volatile double q = 0.5 / den;
    fesetround(old);
    return ru_float(q);
}

/* Algorithm 1 (original fast mode), log2(mu_i) from a_norm and a_max:
 *   s := floor(log2 a_norm)
 *   t := single-up(delta * (log2f(a_norm / 2^s) + s))
 *   return floor(P'_fast - max(1, t)) - floor(log2 a_max)
 * with the same log2 stand-in and readings as Algorithm 2 (argument rounded up to single,
 * floors taken exactly).  A zero line gets shift 0; a non-finite a_norm is flagged. */
int orc_alg1_shift(double a_norm, double a_max, float pprime_fast) {
    if (a_norm == 0.0 || a_max == 0.0) return 0;
    if (!isfinite(a_norm) || !isfinite(a_max)) return ORC_SHIFT_NONFINITE;
    int s = ilogb(a_norm);
    double xprime = scalbn(a_norm, -s);
    float lg = orc_log2_ru(ru_float(xprime));
    float delta = orc_fast_delta();
    float t = ru_float(mul_ru((double)delta, (double)lg + (double)s)); /* lg + s is exact */
    double mx = t > 1.0f ? (double)t : 1.0;
    return (int)floor(sub_rd((double)pprime_fast, mx)) - ilogb(a_max);
}

/* Line accessors.  Matrices are column-major (BLAS).  Row i of op(A) and column j of op(B). */
static void row_of_opA(char trans, const double* A, int64_t lda, int i, const double** base,
                       int64_t* stride) {
    if (trans == 'N' || trans == 'n') { *base = A + i; *stride = lda; }
    else { *base = A + (int64_t)i * lda; *stride = 1; }
}
static void col_of_opB(char trans, const double* B, int64_t ldb, int j, const double** base,
                       int64_t* stride) {
    if (trans == 'N' || trans == 'n') { *base = B + (int64_t)j * ldb; *stride = 1; }
    else { *base = B + j; *stride = ldb; }
}

/* Residues of one line: a'_h = trunc(2^e a_h) (Step 2), r_l = rmod(a'_h, p_l) (eq. os2-C').
 * Output layout out[l * lstride + h]. */
static void line_residues(const double* x, int64_t stride, int64_t len, int e,
                          const orc_consts* c, int8_t* out, int64_t lstride) {
    for (int64_t h = 0; h < len; ++h) {
        if (e == ORC_SHIFT_NONFINITE) {
            for (int l = 0; l < c->N; ++l) out[l * lstride + h] = 0;
            continue;
        }
        double v = trunc(ldexp(x[h * stride], e));
        i256 ai = i256_from_integral_double(v);
        for (int l = 0; l < c->N; ++l)
            out[l * lstride + h] = (int8_t)sym_from_mod(i256_mod(ai, c->p[l]), c->p[l]);
    }
}

/* Step 3 for one entry: C' = sum_l P_l q_l c_l (eq. os2-C'), C'' = rmod(C', P) (eq. os2-C'').
 * c_l is any representative of the l-th product residue. */
static i256 entry_crt(const int* cl, const orc_consts* c) {
    i256 acc = i256_from_u64(0);
    for (int l = 0; l < c->N; ++l) acc = i256_add(acc, i256_mul_i64(c->Pq[l], cl[l]));
    return i256_rmod(acc, c->P);
}

/* Step 4 and the BLAS update for one entry.  Reading: x = RN(C''), y = x * 2^-(e_i + f_j)
 * (ldexp), then alpha*y and, when beta != 0, + beta*C_in, each rounded to nearest. */
static double entry_output(i256 cpp, int e, int f, double alpha, double beta, double cin) {
    if (e == ORC_SHIFT_NONFINITE || f == ORC_SHIFT_NONFINITE) return NAN;
    double x = i256_to_double(cpp);
    double y = ldexp(x, -(e + f));
    double out = alpha * y;
    if (beta != 0.0) out = out + beta * cin;
    return out;
}

/* SGEMM output (reading of Step 4 for FP32, as R11 for FP64): x = C'' rounded to 24 bits,
 * y = x 2^-(e+f) rounded once to single (the double carrier holds x and the product exactly,
 * so the conversion to float is that one rounding, subnormal and overflow included), then
 * alpha y (+ beta C) in single precision. */
static float entry_output_float(i256 cpp, int e, int f, float alpha, float beta, float cin) {
    if (e == ORC_SHIFT_NONFINITE || f == ORC_SHIFT_NONFINITE) return NAN;
    double x = i256_round_bits(cpp, 24);
    float y = (float)ldexp(x, -(e + f));
    float out = alpha * y;
    if (beta != 0.0f) {
        float t = beta * cin;
        out = out + t;
    }
    return out;
}

/* ------------------------------------------------------------------------------------ */
/* Exported entry points (plain pointers; matrices column-major)                          */
/* ------------------------------------------------------------------------------------ */

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Constants of Step 1 for N moduli.  P and P_i q_i are returned as 4 little-endian 64-bit
 * words each (two's complement). */
int orc_constants(int N, int* p, int* q, float* pprime, uint64_t* P_words, uint64_t* Pq_words) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
    for (int l = 0; l < N; ++l) {
        p[l] = c.p[l];
        q[l] = c.q[l];
        for (int w = 0; w < 4; ++w) Pq_words[4 * l + w] = c.Pq[l].w[w];
    }
    for (int w = 0; w < 4; ++w) P_words[w] = c.P.w[w];
    *pprime = c.pprime;
    return 0;
}

static double line_max_abs(const double* x, int64_t stride, int64_t len) {
    double mx = 0.0;
    for (int64_t h = 0; h < len; ++h) {
        double a = fabs(x[h * stride]);
        if (!(a <= mx)) mx = a;   /* NaN propagates */
    }
    return mx;
}

/* Shifts of the rows of op(A) (side 0) or the columns of op(B) (side 1) under a scaling mode:
 * mode 0 = the proposed scaling (Algorithm 2), mode 1 = the original fast mode (Algorithm 1). */
int orc_shifts_mode(int side, char trans, int lines, int len, const double* X, int64_t ld, int N,
                    int mode, int* shifts) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < lines; ++i) {
        const double* base; int64_t st;
        if (side == 0) row_of_opA(trans, X, ld, i, &base, &st);
        else col_of_opB(trans, X, ld, i, &base, &st);
        double nr = line_norm_ru(base, st, len);
        shifts[i] = mode == 1 ? orc_alg1_shift(nr, line_max_abs(base, st, len), c.pprime_fast)
                              : orc_alg2_shift(nr, c.pprime);
    }
    return 0;
}

int orc_residues_a(char transA, int m, int k, const double* A, int64_t lda, const int* e, int N,
                   int8_t* R);
int orc_residues_b(char transB, int k, int n, const double* B, int64_t ldb, const int* f, int N,
                   int8_t* R);
int orc_residue_products(int N, int m, int n, int k, const int8_t* RA, const int8_t* RB,
                         int8_t* cout);
int orc_crt(int N, int m, int n, const int8_t* cres, const int* e, const int* f, double alpha,
            double beta, double* C, int64_t ldc);

/* ---------------------------------------------------------------- accurate mode
 * Section 2.3: mu'_i = 2^(5 - floor(log2 max_h |a_ih|)),  a-bar_ih = ceil(mu'_i |a_ih|) <= 64,
 * C-bar = A-bar B-bar (exact integers), and
 *   log2 mu_i = log2 mu'_i + floor(P'_accu - delta * log2~(max_j c-bar_ij))
 * with P'_accu = single-down(log2(P - 1)/2 - 0.5) and log2~ of eq. (flog2).
 * Reading: the paper prints mu'^(-1)_i in eq. (mu_accu), but its own bound chain
 * 2 mu_i mu'^(-1)_i c-bar_ij nu'^(-1)_j nu_j < P only holds with mu_i = mu'_i 2^(...), which is
 * the reading taken.  The floor is of the exact value (the double product delta * log2~ of two
 * singles is exact, and so is the difference).  A line whose max c-bar is 0 contributes
 * nothing to any product and gets ORC_SHIFT_VANISH; a zero line gets 0; a line with a
 * non-finite entry gets ORC_SHIFT_NONFINITE and a zero a-bar line. */

/* Exponent E = floor(log2 max |x_h|) of a line and its a-bar entries; returns 0 (zero line),
 * 1 (finite, nonzero) or -1 (non-finite). */
static int accu_bar_line(const double* x, int64_t stride, int64_t len, int* E, uint8_t* bar) {
    double mx = line_max_abs(x, stride, len);
    if (!(mx <= DBL_MAX)) {
        for (int64_t h = 0; h < len; ++h) bar[h] = 0;
        return -1;
    }
    if (mx == 0.0) {
        for (int64_t h = 0; h < len; ++h) bar[h] = 0;
        *E = 0;
        return 0;
    }
    *E = ilogb(mx);
    for (int64_t h = 0; h < len; ++h) {
        double a = fabs(x[h * stride]);
        if (a == 0.0) { bar[h] = 0; continue; }
        /* mu' |a| <= 2^5 * 2 = 64; ldexp is exact unless it underflows, and then the exact value
         * is below 1, whose ceiling is 1 */
        double v = ceil(ldexp(a, 5 - *E));
        bar[h] = (uint8_t)(v < 1.0 ? 1.0 : v);
    }
    return 1;
}

/* log2 mu_i from E_i and the maximum of row i of C-bar. */
int orc_accu_shift(int kind, int E, int64_t cmax, float pprime_accu) {
    if (kind < 0) return ORC_SHIFT_NONFINITE;
    if (kind == 0) return 0;
    if (cmax == 0) return ORC_SHIFT_VANISH;
    /* eq. (flog2): s = floor(log2 x), x' = x / 2^s in [1, 2) (exact: x < 2^53) */
    int s = 63 - __builtin_clzll((unsigned long long)cmax);
    double xprime = ldexp((double)cmax, -s);
    float lg = ru_float((double)orc_log2_ru(ru_float(xprime)) + (double)s);
    float delta = orc_fast_delta();
    double u = (double)delta * (double)lg;             /* exact: 24 x 24 bits */
    return 5 - E + (int)floor(sub_rd((double)pprime_accu, u));
}

/* a-bar of the rows of op(A) (side 0) or the columns of op(B) (side 1): bar[i * len + h],
 * exps[i] = E_i, kinds[i] as accu_bar_line. */
int orc_accu_bar(int side, char trans, int lines, int len, const double* X, int64_t ld,
                 uint8_t* bar, int* exps, int* kinds) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < lines; ++i) {
        const double* base; int64_t st;
        if (side == 0) row_of_opA(trans, X, ld, i, &base, &st);
        else col_of_opB(trans, X, ld, i, &base, &st);
        exps[i] = 0;
        kinds[i] = accu_bar_line(base, st, len, &exps[i], bar + (int64_t)i * len);
    }
    return 0;
}

/* Shifts of accurate mode for both operands, with the row and column maxima of C-bar. */
int orc_accurate_shifts(char transA, char transB, int m, int n, int k, const double* A,
                        int64_t lda, const double* B, int64_t ldb, int N, int* e, int* f,
                        int64_t* rowmax, int64_t* colmax) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
    size_t kk = (size_t)(k ? k : 1);
    uint8_t* Abar = (uint8_t*)malloc((size_t)(m ? m : 1) * kk);
    uint8_t* Bbar = (uint8_t*)malloc((size_t)(n ? n : 1) * kk);
    int* EA = (int*)malloc(sizeof(int) * (size_t)(m ? m : 1));
    int* EB = (int*)malloc(sizeof(int) * (size_t)(n ? n : 1));
    int* KA = (int*)malloc(sizeof(int) * (size_t)(m ? m : 1));
    int* KB = (int*)malloc(sizeof(int) * (size_t)(n ? n : 1));
    if (!Abar || !Bbar || !EA || !EB || !KA || !KB) {
        free(Abar); free(Bbar); free(EA); free(EB); free(KA); free(KB);
        return -2;
    }
    orc_accu_bar(0, transA, m, k, A, lda, Abar, EA, KA);
    orc_accu_bar(1, transB, n, k, B, ldb, Bbar, EB, KB);
    int64_t* Cbar = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m ? m : 1) * (n ? n : 1));
    if (!Cbar) {
        free(Abar); free(Bbar); free(EA); free(EB); free(KA); free(KB);
        return -2;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < m; ++i) {                   /* C-bar = A-bar B-bar, exact */
        const uint8_t* ar = Abar + (size_t)i * kk;
        for (int j = 0; j < n; ++j) {
            const uint8_t* bc = Bbar + (size_t)j * kk;
            int64_t cbar = 0;
            for (int h = 0; h < k; ++h) cbar += (int64_t)ar[h] * bc[h];
            Cbar[(size_t)i * n + j] = cbar;
        }
    }
    for (int i = 0; i < m; ++i) {
        int64_t r = 0;
        for (int j = 0; j < n; ++j) r = Cbar[(size_t)i * n + j] > r ? Cbar[(size_t)i * n + j] : r;
        rowmax[i] = r;
    }
    for (int j = 0; j < n; ++j) {
        int64_t r = 0;
        for (int i = 0; i < m; ++i) r = Cbar[(size_t)i * n + j] > r ? Cbar[(size_t)i * n + j] : r;
        colmax[j] = r;
    }
    free(Cbar);
    for (int i = 0; i < m; ++i) e[i] = orc_accu_shift(KA[i], EA[i], rowmax[i], c.pprime);
    for (int j = 0; j < n; ++j) f[j] = orc_accu_shift(KB[j], EB[j], colmax[j], c.pprime);
    free(Abar); free(Bbar); free(EA); free(EB); free(KA); free(KB);
    return 0;
}

/* The whole emulated DGEMM under a scaling mode (0 proposed, 1 original fast mode,
 * 2 accurate mode). */
int orc_dgemm_mode(char transA, char transB, int m, int n, int k, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                   int64_t ldc, int N, int mode) {
    if (N < 2 || N > ORC_MAX_MODULI || m < 0 || n < 0 || k < 0) return -1;
    if (m == 0 || n == 0) return 0;
    int* e = (int*)malloc(sizeof(int) * (size_t)m);
    int* f = (int*)malloc(sizeof(int) * (size_t)n);
    int8_t* RA = (int8_t*)malloc((size_t)N * m * (k ? k : 1));
    int8_t* RB = (int8_t*)malloc((size_t)N * n * (k ? k : 1));
    int8_t* cr = (int8_t*)malloc((size_t)N * m * n);
    int rc = -2;
    if (e && f && RA && RB && cr) {
        if (mode == 2) {
            int64_t* rmx = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
            int64_t* cmx = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
            if (rmx && cmx)
                orc_accurate_shifts(transA, transB, m, n, k, A, lda, B, ldb, N, e, f, rmx, cmx);
            free(rmx); free(cmx);
        } else {
            orc_shifts_mode(0, transA, m, k, A, lda, N, mode, e);
            orc_shifts_mode(1, transB, n, k, B, ldb, N, mode, f);
        }
        orc_residues_a(transA, m, k, A, lda, e, N, RA);
        orc_residues_b(transB, k, n, B, ldb, f, N, RB);
        orc_residue_products(N, m, n, k, RA, RB, cr);
        rc = orc_crt(N, m, n, cr, e, f, alpha, beta, C, ldc);
    }
    free(e); free(f); free(RA); free(RB); free(cr);
    return rc;
}

int orc_pprime_fast(int N, float* out) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
    *out = c.pprime_fast;
    return 0;
}

/* Row shifts e_i = log2(mu_i) of op(A) (m x k) and their squared norms. */
int orc_shifts_a(char transA, int m, int k, const double* A, int64_t lda, int N, int* e,
                 double* norms) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < m; ++i) {
        const double* base; int64_t st;
        row_of_opA(transA, A, lda, i, &base, &st);
        double nr = line_norm_ru(base, st, k);
        if (norms) norms[i] = nr;
        e[i] = orc_alg2_shift(nr, c.pprime);
    }
    return 0;
}

/* Column shifts f_j = log2(nu_j) of op(B) (k x n) and their squared norms. */
int orc_shifts_b(char transB, int k, int n, const double* B, int64_t ldb, int N, int* f,
                 double* norms) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < n; ++j) {
        const double* base; int64_t st;
        col_of_opB(transB, B, ldb, j, &base, &st);
        double nr = line_norm_ru(base, st, k);
        if (norms) norms[j] = nr;
        f[j] = orc_alg2_shift(nr, c.pprime);
    }
    return 0;
}

/* Residues of op(A) rows: R[l][i][h], layout l*m*k + i*k + h. */
int orc_residues_a(char transA, int m, int k, const double* A, int64_t lda, const int* e, int N,
                   int8_t* R) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < m; ++i) {
        const double* base; int64_t st;
        row_of_opA(transA, A, lda, i, &base, &st);
        line_residues(base, st, k, e[i], &c, R + (int64_t)i * k, (int64_t)m * k);
    }
    return 0;
}

/* Residues of op(B) columns: R[l][j][h], layout l*n*k + j*k + h (k contiguous). */
int orc_residues_b(char transB, int k, int n, const double* B, int64_t ldb, const int* f, int N,
                   int8_t* R) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < n; ++j) {
        const double* base; int64_t st;
        col_of_opB(transB, B, ldb, j, &base, &st);
        line_residues(base, st, k, f[j], &c, R + (int64_t)j * k, (int64_t)n * k);
    }
    return 0;
}

/* Residue products of eq. (os2-C'): G_l = rmod(A', p_l) rmod(B', p_l) exactly (int64), then
 * c_l = rmod(G_l, p_l).  Output layout c[l][i][j] = l*m*n + i*n + j. */
int orc_residue_products(int N, int m, int n, int k, const int8_t* RA, const int8_t* RB,
                         int8_t* cout) {
    if (N < 2 || N > ORC_MAX_MODULI) return -1;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int l = 0; l < N; ++l) {
        for (int i = 0; i < m; ++i) {
            const int8_t* ra = RA + (int64_t)l * m * k + (int64_t)i * k;
            for (int j = 0; j < n; ++j) {
                const int8_t* rb = RB + (int64_t)l * n * k + (int64_t)j * k;
                int64_t g = 0;
                for (int h = 0; h < k; ++h) g += (int64_t)ra[h] * rb[h];
                cout[(int64_t)l * m * n + (int64_t)i * n + j] =
                    (int8_t)sym_from_mod(i64_mod(g, MODULI[l]), MODULI[l]);
            }
        }
    }
    return 0;
}

/* Step 3 + Step 4 from product residues c[l][i][j] (layout of orc_residue_products).
 * C is column-major m x n with leading dimension ldc; it is read only when beta != 0. */
int orc_crt(int N, int m, int n, const int8_t* cres, const int* e, const int* f, double alpha,
            double beta, double* C, int64_t ldc) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
            int cl[ORC_MAX_MODULI];
            for (int l = 0; l < N; ++l) cl[l] = cres[(int64_t)l * m * n + (int64_t)i * n + j];
            i256 cpp = entry_crt(cl, &c);
            double cin = beta != 0.0 ? C[i + (int64_t)j * ldc] : 0.0;
            C[i + (int64_t)j * ldc] = entry_output(cpp, e[i], f[j], alpha, beta, cin);
        }
    }
    return 0;
}

int orc_crt_float(int N, int m, int n, const int8_t* cres, const int* e, const int* f,
                  float alpha, float beta, float* C, int64_t ldc) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
            int cl[ORC_MAX_MODULI];
            for (int l = 0; l < N; ++l) cl[l] = cres[(int64_t)l * m * n + (int64_t)i * n + j];
            i256 cpp = entry_crt(cl, &c);
            float cin = beta != 0.0f ? C[i + (int64_t)j * ldc] : 0.0f;
            C[i + (int64_t)j * ldc] = entry_output_float(cpp, e[i], f[j], alpha, beta, cin);
        }
    }
    return 0;
}

/* SGEMM through Ozaki scheme II: every float is exactly a double, so Steps 1-3 and the
 * scaling are those of the DGEMM on the widened inputs (the squared norms are the same upward
 * rounded FP64 sums); only Step 4 rounds to single (entry_output_float). */
int orc_sgemm_mode(char transA, char transB, int m, int n, int k, float alpha, const float* A,
                   int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                   int N, int mode) {
    if (N < 2 || N > ORC_MAX_MODULI || m < 0 || n < 0 || k < 0) return -1;
    if (m == 0 || n == 0) return 0;
    const int arows = (transA == 'N' || transA == 'n') ? m : k;
    const int acols = (transA == 'N' || transA == 'n') ? k : m;
    const int brows = (transB == 'N' || transB == 'n') ? k : n;
    const int bcols = (transB == 'N' || transB == 'n') ? n : k;
    double* Ad = (double*)malloc(sizeof(double) * (size_t)(lda * (acols ? acols : 1)));
    double* Bd = (double*)malloc(sizeof(double) * (size_t)(ldb * (bcols ? bcols : 1)));
    int* e = (int*)malloc(sizeof(int) * (size_t)m);
    int* f = (int*)malloc(sizeof(int) * (size_t)n);
    int8_t* RA = (int8_t*)malloc((size_t)N * m * (k ? k : 1));
    int8_t* RB = (int8_t*)malloc((size_t)N * n * (k ? k : 1));
    int8_t* cr = (int8_t*)malloc((size_t)N * m * n);
    int rc = -2;
    if (Ad && Bd && e && f && RA && RB && cr) {
        for (int64_t c2 = 0; c2 < acols; ++c2)
            for (int64_t r = 0; r < arows; ++r) Ad[r + c2 * lda] = (double)A[r + c2 * lda];
        for (int64_t c2 = 0; c2 < bcols; ++c2)
            for (int64_t r = 0; r < brows; ++r) Bd[r + c2 * ldb] = (double)B[r + c2 * ldb];
        if (mode == 2) {
            int64_t* rmx = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
            int64_t* cmx = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
            if (rmx && cmx)
                orc_accurate_shifts(transA, transB, m, n, k, Ad, lda, Bd, ldb, N, e, f, rmx, cmx);
            free(rmx); free(cmx);
        } else {
            orc_shifts_mode(0, transA, m, k, Ad, lda, N, mode, e);
            orc_shifts_mode(1, transB, n, k, Bd, ldb, N, mode, f);
        }
        orc_residues_a(transA, m, k, Ad, lda, e, N, RA);
        orc_residues_b(transB, k, n, Bd, ldb, f, N, RB);
        orc_residue_products(N, m, n, k, RA, RB, cr);
        if (k == 0 || alpha == 0.0f) {
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < m; ++i) {
                    float* p = &C[i + (int64_t)j * ldc];
                    *p = beta == 0.0f ? 0.0f : beta * *p;
                }
            rc = 0;
        } else {
            rc = orc_crt_float(N, m, n, cr, e, f, alpha, beta, C, ldc);
        }
    }
    free(Ad); free(Bd); free(e); free(f); free(RA); free(RB); free(cr);
    return rc;
}

int orc_sgemm(char transA, char transB, int m, int n, int k, float alpha, const float* A,
              int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
              int N) {
    return orc_sgemm_mode(transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, N, 0);
}

/* C'' = rmod(C', P) as 4 little-endian 64-bit words per entry, entry order i*n + j. */
int orc_crt_exact(int N, int m, int n, const int8_t* cres, uint64_t* words) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
            int cl[ORC_MAX_MODULI];
            for (int l = 0; l < N; ++l) cl[l] = cres[(int64_t)l * m * n + (int64_t)i * n + j];
            i256 cpp = entry_crt(cl, &c);
            for (int w = 0; w < 4; ++w) words[((int64_t)i * n + j) * 4 + w] = cpp.w[w];
        }
    }
    return 0;
}

/* Rounded conversion of 256-bit integers given as words (for pinning against Python). */
int orc_words_to_double(int count, const uint64_t* words, double* out) {
    for (int t = 0; t < count; ++t) {
        i256 a;
        for (int w = 0; w < 4; ++w) a.w[w] = words[4 * t + w];
        out[t] = i256_to_double(a);
    }
    return 0;
}

/* Symmetric residues of 256-bit integers given as words: out[t*N + l]. */
int orc_words_residues(int count, const uint64_t* words, int N, int* out) {
    if (N < 1 || N > ORC_MAX_MODULI) return -1;
    for (int t = 0; t < count; ++t) {
        i256 a;
        for (int w = 0; w < 4; ++w) a.w[w] = words[4 * t + w];
        for (int l = 0; l < N; ++l) out[t * N + l] = sym_from_mod(i256_mod(a, MODULI[l]), MODULI[l]);
    }
    return 0;
}

/* The whole emulated DGEMM, C = alpha op(A) op(B) + beta C, all four steps in order. */
int orc_dgemm(char transA, char transB, int m, int n, int k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
              int N) {
    if (N < 2 || N > ORC_MAX_MODULI || m < 0 || n < 0 || k < 0) return -1;
    if (m == 0 || n == 0) return 0;
    int* e = (int*)malloc(sizeof(int) * (size_t)m);
    int* f = (int*)malloc(sizeof(int) * (size_t)n);
    int8_t* RA = (int8_t*)malloc((size_t)N * m * (k ? k : 1));
    int8_t* RB = (int8_t*)malloc((size_t)N * n * (k ? k : 1));
    int8_t* cr = (int8_t*)malloc((size_t)N * m * n);
    int rc = -2;
    if (e && f && RA && RB && cr) {
        orc_shifts_a(transA, m, k, A, lda, N, e, NULL);
        orc_shifts_b(transB, k, n, B, ldb, N, f, NULL);
        orc_residues_a(transA, m, k, A, lda, e, N, RA);
        orc_residues_b(transB, k, n, B, ldb, f, N, RB);
        orc_residue_products(N, m, n, k, RA, RB, cr);
        rc = orc_crt(N, m, n, cr, e, f, alpha, beta, C, ldc);
    }
    free(e); free(f); free(RA); free(RB); free(cr);
    return rc;
}

/* A block of the emulated DGEMM: out[a + b*nI] = C(I[a], J[b]) for rows I and columns J.
 * Shifts come from e_in / f_in when given (indexed by row / column number), else they are
 * computed for the needed lines only.  Cin (same layout as out) is read when beta != 0. */
int orc_dgemm_block(char transA, char transB, int m, int n, int k, double alpha, const double* A,
                    int64_t lda, const double* B, int64_t ldb, double beta, const double* Cin,
                    int N, int nI, const int* I, int nJ, const int* J, const int* e_in,
                    const int* f_in, double* out) {
    orc_consts c;
    (void)m; (void)n;
    if (make_consts(N, &c)) return -1;
    int* e = (int*)malloc(sizeof(int) * (size_t)(nI ? nI : 1));
    int* f = (int*)malloc(sizeof(int) * (size_t)(nJ ? nJ : 1));
    int8_t* RA = (int8_t*)malloc((size_t)N * (nI ? nI : 1) * (k ? k : 1));
    int8_t* RB = (int8_t*)malloc((size_t)N * (nJ ? nJ : 1) * (k ? k : 1));
    if (!e || !f || !RA || !RB) { free(e); free(f); free(RA); free(RB); return -2; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < nI; ++a) {
        const double* base; int64_t st;
        row_of_opA(transA, A, lda, I[a], &base, &st);
        e[a] = e_in ? e_in[I[a]] : orc_alg2_shift(line_norm_ru(base, st, k), c.pprime);
        line_residues(base, st, k, e[a], &c, RA + (int64_t)a * k, (int64_t)nI * k);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nJ; ++b) {
        const double* base; int64_t st;
        col_of_opB(transB, B, ldb, J[b], &base, &st);
        f[b] = f_in ? f_in[J[b]] : orc_alg2_shift(line_norm_ru(base, st, k), c.pprime);
        line_residues(base, st, k, f[b], &c, RB + (int64_t)b * k, (int64_t)nJ * k);
    }
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
    for (int b = 0; b < nJ; ++b) {
        for (int a = 0; a < nI; ++a) {
            int cl[ORC_MAX_MODULI];
            for (int l = 0; l < N; ++l) {
                const int8_t* ra = RA + (int64_t)l * nI * k + (int64_t)a * k;
                const int8_t* rb = RB + (int64_t)l * nJ * k + (int64_t)b * k;
                int64_t g = 0;
                for (int h = 0; h < k; ++h) g += (int64_t)ra[h] * rb[h];
                cl[l] = sym_from_mod(i64_mod(g, c.p[l]), c.p[l]);
            }
            i256 cpp = entry_crt(cl, &c);
            double cin = beta != 0.0 ? Cin[a + (int64_t)b * nI] : 0.0;
            out[a + (int64_t)b * nI] = entry_output(cpp, e[a], f[b], alpha, beta, cin);
        }
    }
    free(e); free(f); free(RA); free(RB);
    return 0;
}

/* A block of the emulated SGEMM (proposed scaling): out[a + b*nI] = C(I[a], J[b]) in single
 * precision.  The needed lines are widened to double (exactly); shifts come from e_in / f_in
 * when given, else from the widened lines.  Cin (same layout as out) is read when beta != 0. */
int orc_sgemm_block(char transA, char transB, int k, float alpha, const float* A, int64_t lda,
                    const float* B, int64_t ldb, float beta, const float* Cin, int N, int nI,
                    const int* I, int nJ, const int* J, const int* e_in, const int* f_in,
                    float* out) {
    orc_consts c;
    if (make_consts(N, &c)) return -1;
    int64_t kk = k ? k : 1;
    int* e = (int*)malloc(sizeof(int) * (size_t)(nI ? nI : 1));
    int* f = (int*)malloc(sizeof(int) * (size_t)(nJ ? nJ : 1));
    double* la = (double*)malloc(sizeof(double) * (size_t)(nI ? nI : 1) * kk);
    double* lb = (double*)malloc(sizeof(double) * (size_t)(nJ ? nJ : 1) * kk);
    int8_t* RA = (int8_t*)malloc((size_t)N * (nI ? nI : 1) * kk);
    int8_t* RB = (int8_t*)malloc((size_t)N * (nJ ? nJ : 1) * kk);
    if (!e || !f || !la || !lb || !RA || !RB) {
        free(e); free(f); free(la); free(lb); free(RA); free(RB);
        return -2;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < nI; ++a) {
        const int notrans = transA == 'N' || transA == 'n';
        double* x = la + (int64_t)a * kk;
        for (int64_t h = 0; h < k; ++h)
            x[h] = (double)(notrans ? A[I[a] + h * lda] : A[h + (int64_t)I[a] * lda]);
        e[a] = e_in ? e_in[I[a]] : orc_alg2_shift(line_norm_ru(x, 1, k), c.pprime);
        line_residues(x, 1, k, e[a], &c, RA + (int64_t)a * k, (int64_t)nI * k);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nJ; ++b) {
        const int notrans = transB == 'N' || transB == 'n';
        double* x = lb + (int64_t)b * kk;
        for (int64_t h = 0; h < k; ++h)
            x[h] = (double)(notrans ? B[h + (int64_t)J[b] * ldb] : B[J[b] + h * ldb]);
        f[b] = f_in ? f_in[J[b]] : orc_alg2_shift(line_norm_ru(x, 1, k), c.pprime);
        line_residues(x, 1, k, f[b], &c, RB + (int64_t)b * k, (int64_t)nJ * k);
    }
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
    for (int b = 0; b < nJ; ++b) {
        for (int a = 0; a < nI; ++a) {
            int cl[ORC_MAX_MODULI];
            for (int l = 0; l < N; ++l) {
                const int8_t* ra = RA + (int64_t)l * nI * k + (int64_t)a * k;
                const int8_t* rb = RB + (int64_t)l * nJ * k + (int64_t)b * k;
                int64_t g = 0;
                for (int h = 0; h < k; ++h) g += (int64_t)ra[h] * rb[h];
                cl[l] = sym_from_mod(i64_mod(g, c.p[l]), c.p[l]);
            }
            i256 cpp = entry_crt(cl, &c);
            float cin = beta != 0.0f ? Cin[a + (int64_t)b * nI] : 0.0f;
            out[a + (int64_t)b * nI] = entry_output_float(cpp, e[a], f[b], alpha, beta, cin);
        }
    }
    free(e); free(f); free(la); free(lb); free(RA); free(RB);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Double-double reference product (the "double-double precision" reference of Section 3.2) */
/* ------------------------------------------------------------------------------------ */
/* Reading: sequential accumulation with the error-free transformations TwoSum (Knuth) and
 * TwoProd via fma (Dekker's product with a fused multiply-add). */
static void two_sum(double a, double b, double* s, double* err) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *err = (a - av) + (b - bv);
    *s = x;
}
static void fast_two_sum(double a, double b, double* s, double* err) {
    double x = a + b;
    *err = b - (x - a);
    *s = x;
}

/* hi/lo[a + b*nI] = (op(A) op(B))(I[a], J[b]) in double-double. */
int orc_dd_block(char transA, char transB, int k, const double* A, int64_t lda, const double* B,
                 int64_t ldb, int nI, const int* I, int nJ, const int* J, double* hi, double* lo) {
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
    for (int b = 0; b < nJ; ++b) {
        for (int a = 0; a < nI; ++a) {
            const double *ra, *cb; int64_t sa, sb;
            row_of_opA(transA, A, lda, I[a], &ra, &sa);
            col_of_opB(transB, B, ldb, J[b], &cb, &sb);
            double sh = 0.0, sl = 0.0;
            for (int h = 0; h < k; ++h) {
                double x = ra[h * sa], y = cb[h * sb];
                double p = x * y;
                double pe = fma(x, y, -p);
                double s1, s2;
                two_sum(sh, p, &s1, &s2);
                s2 += sl + pe;
                fast_two_sum(s1, s2, &sh, &sl);
            }
            hi[a + (int64_t)b * nI] = sh;
            lo[a + (int64_t)b * nI] = sl;
        }
    }
    return 0;
}
