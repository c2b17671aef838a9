// crt.cu -- Steps 3-4 of Ozaki scheme II: CRT reconstruction (eqs. os2-C', os2-C'') and the
// rescaling C = diag(mu)^-1 C'' diag(nu)^-1, then C = alpha C (+ beta C_in).
//
// GB300 design: FP64 throughput is a small fraction of the integer rate on this part, so the
// reconstruction is exact multi-word integer arithmetic instead of split FP64 constants:
//   X    = sum_l P_l q_l c_l modulo P, as sum_g PG_g v_g over pairs of moduli (below)
//          (W 32-bit words, 64-bit column sums)
//   Q    = round(X / P)                          (46-bit fixed-point estimate of sum_g v_g/prod_g)
//   C''  = X - Q P                               (exact; corrected by +-P if the estimate sat
//                                                 within 2^-10 of a half-integer)
// X and Q P are formed modulo 2^(32 W) with W just large enough for Y (see crt_words).
// The moduli are taken in pairs: with prod_g the pair's product and K_l = (prod_g / p_l) q_l mod
// prod_g, v_g = bias_g + sum_{l in g} c_l K_l is congruent modulo prod_g to the pair's share of
// X / PG_g, so each residue costs one multiply-add and X one 64-bit multiply-add per pair and
// word; the kernel is instantiated per N so every table entry is a constant-bank operand.
// Since X == sum_l P_l q_l c_l (mod P), C'' = rmod(sum_l P_l q_l c_l, P) of eq. (os2-C'').
// C'' is rounded to the nearest double (ties to even) with the unscaling 2^-(e_i + f_j) folded
// into the exponent; results outside the normal range take a two-multiply path that rounds once.
//
// Memory: reads N bytes of product residues per entry, writes 8 bytes (reads 8 more if beta != 0).
#include "ozaki2_internal.h"

namespace ozaki2 {
namespace {

// Tiles of the output, 256 threads each: 32 rows x 64 columns on the padded layout (VEC), where
// a thread reconstructs eight consecutive entries of one row; 32 x 32 otherwise.
constexpr int TI = 32, TJ = 32, TJV = 64;
template <bool VEC>
__host__ __device__ constexpr int tile_cols() { return VEC ? TJV : TJ; }

// y * 2^s rounded to nearest once, for any s (x is a normal double).  Only results outside the
// normal range come here; kept out of line so that none of its FP64 multiplies is if-converted
// into the common path.
__device__ __noinline__ double scale_pow2_rn(double x, int s) {
    if (s > 0) {
        while (s > 1000) { x = __dmul_rn(x, 0x1p1000); s -= 1000; }
        return __dmul_rn(x, __longlong_as_double((long long)(s + 1023) << 52));
    }
    // bring x to [1, 2) exactly, then one rounding multiply by 2^(e + s) split as 2^(t) 2^-600
    int e = ilogb(x);
    double m = __dmul_rn(x, __longlong_as_double((long long)(1023 - e) << 52));
    int t = e + s;  // final exponent
    if (t >= -1022) return __dmul_rn(m, __longlong_as_double((long long)(t + 1023) << 52));
    if (t < -1022 - 600) return __dmul_rn(m, 0.0);  // far below the smallest subnormal: +-0
    double m2 = __dmul_rn(m, __longlong_as_double((long long)(t + 600 + 1023) << 52));  // exact
    return __dmul_rn(m2, 0x1p-600);
}

// The double with these bits rounded to single (the out-of-range single results only).
__device__ __noinline__ float double_bits_to_float(uint64_t bits) {
    return __double2float_rn(__longlong_as_double((long long)bits));
}

// 32-bit words of the working integers.  X and Q P are only needed modulo 2^(32 W): the result
// Y = X - Q P satisfies |Y| < P (Q is round(X/P) or one off near a tie), so W words holding
// bits(P) + 2 bits carry Y exactly in two's complement.
__host__ __device__ constexpr int crt_pbits(int N) {
    // bits(P) for N = 2..20: 16 24 32 40 48 56 64 72 80 88 95 103 111 118 126 133 141 148 156
    constexpr int b[21] = {0, 8, 16, 24, 32, 40, 48, 56, 64, 72, 80,
                           88, 95, 103, 111, 118, 126, 133, 141, 148, 156};
    return b[N];
}
__host__ __device__ constexpr int crt_words(int N) { return (crt_pbits(N) + 2 + 31) / 32; }
// The word that holds the leading bit of a large |C''| (< P/2 < 2^(bits(P) - 1)): the top word
// of the W, except where bits(P) is a multiple of 32 (N = 4, 8, 12), whose extra sign word stays
// zero for every |C''| < P.
__host__ __device__ constexpr int crt_top(int N) { return (crt_pbits(N) - 2) / 32; }
// Where |C''| < P/2 reaches fewer than 12 bits into word TOP (N = 5, 9, 13, 17), an ordinary entry
// (some bits below the bound) often starts in the word below: the straight-line path then also
// takes its window one word lower.
__host__ __device__ constexpr bool crt_window_drops(int N) {
    return crt_top(N) >= 1 && (crt_pbits(N) - 2) % 32 < 12;
}

// ---- multi-word integer steps with the carry flag: each chain is one asm statement, so nothing
// the compiler schedules can come between an instruction that sets the carry and the one that
// reads it.  Words are little-endian; every result is modulo 2^(32 W), W = 1 .. 5.

// X = sum_j acc[j] 2^(32 j): word j is lo(acc[j]) + hi(acc[j-1]) + carry.
template <int W>
__device__ __forceinline__ void fold_columns(const uint64_t (&acc)[W], uint32_t (&X)[W]) {
    uint32_t lo[W], hi[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        lo[j] = (uint32_t)acc[j];
        hi[j] = (uint32_t)(acc[j] >> 32);
    }
    X[0] = lo[0];
    if constexpr (W == 2) {
        X[1] = lo[1] + hi[0];
    } else if constexpr (W == 3) {
        asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;"
            : "=&r"(X[1]), "=&r"(X[2])
            : "r"(lo[1]), "r"(hi[0]), "r"(lo[2]), "r"(hi[1]));
    } else if constexpr (W == 4) {
        asm("add.cc.u32 %0, %3, %4;\n\taddc.cc.u32 %1, %5, %6;\n\taddc.u32 %2, %7, %8;"
            : "=&r"(X[1]), "=&r"(X[2]), "=&r"(X[3])
            : "r"(lo[1]), "r"(hi[0]), "r"(lo[2]), "r"(hi[1]), "r"(lo[3]), "r"(hi[2]));
    } else if constexpr (W == 5) {
        asm("add.cc.u32 %0, %4, %5;\n\taddc.cc.u32 %1, %6, %7;\n\taddc.cc.u32 %2, %8, %9;\n\t"
            "addc.u32 %3, %10, %11;"
            : "=&r"(X[1]), "=&r"(X[2]), "=&r"(X[3]), "=&r"(X[4])
            : "r"(lo[1]), "r"(hi[0]), "r"(lo[2]), "r"(hi[1]), "r"(lo[3]), "r"(hi[2]),
              "r"(lo[4]), "r"(hi[3]));
    }
}

// Y = X + Q M for a one-word Q: the low halves of the products in one carry chain, the high
// halves (shifted one word up) in a second.
template <int W>
__device__ __forceinline__ void add_word_times(const uint32_t (&X)[W], uint32_t Q,
                                               const uint32_t* M, uint32_t (&Y)[W]) {
    if constexpr (W == 1) {
        Y[0] = X[0] + Q * M[0];
    } else if constexpr (W == 2) {
        asm("mad.lo.cc.u32 %0, %2, %3, %5;\n\tmadc.lo.u32 %1, %2, %4, %6;\n\t"
            "mad.hi.u32 %1, %2, %3, %1;"
            : "=&r"(Y[0]), "=&r"(Y[1])
            : "r"(Q), "r"(M[0]), "r"(M[1]), "r"(X[0]), "r"(X[1]));
    } else if constexpr (W == 3) {
        asm("mad.lo.cc.u32 %0, %3, %4, %7;\n\tmadc.lo.cc.u32 %1, %3, %5, %8;\n\t"
            "madc.lo.u32 %2, %3, %6, %9;\n\t"
            "mad.hi.cc.u32 %1, %3, %4, %1;\n\tmadc.hi.u32 %2, %3, %5, %2;"
            : "=&r"(Y[0]), "=&r"(Y[1]), "=&r"(Y[2])
            : "r"(Q), "r"(M[0]), "r"(M[1]), "r"(M[2]), "r"(X[0]), "r"(X[1]), "r"(X[2]));
    } else if constexpr (W == 4) {
        asm("mad.lo.cc.u32 %0, %4, %5, %9;\n\tmadc.lo.cc.u32 %1, %4, %6, %10;\n\t"
            "madc.lo.cc.u32 %2, %4, %7, %11;\n\tmadc.lo.u32 %3, %4, %8, %12;\n\t"
            "mad.hi.cc.u32 %1, %4, %5, %1;\n\tmadc.hi.cc.u32 %2, %4, %6, %2;\n\t"
            "madc.hi.u32 %3, %4, %7, %3;"
            : "=&r"(Y[0]), "=&r"(Y[1]), "=&r"(Y[2]), "=&r"(Y[3])
            : "r"(Q), "r"(M[0]), "r"(M[1]), "r"(M[2]), "r"(M[3]), "r"(X[0]), "r"(X[1]),
              "r"(X[2]), "r"(X[3]));
    } else if constexpr (W == 5) {
        asm("mad.lo.cc.u32 %0, %5, %6, %11;\n\tmadc.lo.cc.u32 %1, %5, %7, %12;\n\t"
            "madc.lo.cc.u32 %2, %5, %8, %13;\n\tmadc.lo.cc.u32 %3, %5, %9, %14;\n\t"
            "madc.lo.u32 %4, %5, %10, %15;\n\t"
            "mad.hi.cc.u32 %1, %5, %6, %1;\n\tmadc.hi.cc.u32 %2, %5, %7, %2;\n\t"
            "madc.hi.cc.u32 %3, %5, %8, %3;\n\tmadc.hi.u32 %4, %5, %9, %4;"
            : "=&r"(Y[0]), "=&r"(Y[1]), "=&r"(Y[2]), "=&r"(Y[3]), "=&r"(Y[4])
            : "r"(Q), "r"(M[0]), "r"(M[1]), "r"(M[2]), "r"(M[3]), "r"(M[4]), "r"(X[0]),
              "r"(X[1]), "r"(X[2]), "r"(X[3]), "r"(X[4]));
    }
}

// |Y| in place (two's complement): complement every word when negative, then add 1 through a
// carry chain.  Returns the sign.
template <int W>
__device__ __forceinline__ bool abs_words(uint32_t (&Y)[W]) {
    const uint32_t m = (uint32_t)((int32_t)Y[W - 1] >> 31);
    const uint32_t one = m & 1u;
#pragma unroll
    for (int j = 0; j < W; ++j) Y[j] ^= m;
    if constexpr (W == 1) {
        Y[0] += one;
    } else if constexpr (W == 2) {
        asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(Y[0]), "+r"(Y[1]) : "r"(one));
    } else if constexpr (W == 3) {
        asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, %2, 0;"
            : "+r"(Y[0]), "+r"(Y[1]), "+r"(Y[2])
            : "r"(one));
    } else if constexpr (W == 4) {
        asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\t"
            "addc.u32 %3, %3, 0;"
            : "+r"(Y[0]), "+r"(Y[1]), "+r"(Y[2]), "+r"(Y[3])
            : "r"(one));
    } else if constexpr (W == 5) {
        asm("add.cc.u32 %0, %0, %5;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\t"
            "addc.cc.u32 %3, %3, 0;\n\taddc.u32 %4, %4, 0;"
            : "+r"(Y[0]), "+r"(Y[1]), "+r"(Y[2]), "+r"(Y[3]), "+r"(Y[4])
            : "r"(one));
    }
    return m != 0;
}

// Pair sums v_g = bias_g + sum_{l in g} c_l K_l from the residues of one entry: one multiply-add
// per residue (the signed product wraps modulo 2^32 to the exact value, in [0, 2^25)).
template <int N>
__device__ __forceinline__ void pair_sums(const int (&cres)[N], const CrtTables& t,
                                          uint32_t (&v)[(N + 1) / 2]) {
#pragma unroll
    for (int g = 0; g < (N + 1) / 2; ++g) {
        v[g] = t.grp_bias[g];
#pragma unroll
        for (int l = 2 * g; l < 2 * g + 2 && l < N; ++l) v[g] += (uint32_t)cres[l] * t.K[l];
    }
}

// c + K_lo b_lo + K_hi b_hi with K_lo, K_hi the unsigned 16-bit halves of `kpair` and b_lo, b_hi
// the signed bytes 0, 1 (HI = false) or 2, 3 (HI = true) of `b`: the same pair sum in one
// instruction (exact: the true value lies in [0, 2^25)).
template <bool HI>
__device__ __forceinline__ uint32_t dot2(uint32_t kpair, uint32_t b, uint32_t c) {
    uint32_t d;
    if constexpr (HI)
        asm("dp2a.hi.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(kpair), "r"(b), "r"(c));
    else
        asm("dp2a.lo.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(kpair), "r"(b), "r"(c));
    return d;
}

// The W words of Y = X - Q P, passed by value to the out-of-line path.
template <int W>
struct Words {
    uint32_t w[W];
};

// Rounding of C'' = Y (two's complement, |Y| < P) to OutT, scaled by 2^-(ea + fb), for every
// case the straight-line path of crt_value leaves: an estimate near a half-integer (Y may be off
// by P), a leading word below the top one, a result outside the normal range.  Out of line, so
// the common path carries none of it.
template <int N, typename OutT>
__device__ __noinline__ OutT crt_value_rare(Words<crt_words(N)> Yw, bool near_half, int ea,
                                            int fb, const CrtTables& t) {
    constexpr int W = crt_words(N);
    uint32_t (&Y)[W] = Yw.w;
    if (near_half) {
        // make -P/2 <= Y < P/2 exactly
        const bool neg = (Y[W - 1] >> 31) != 0;
        uint32_t mag[W];
        uint32_t cb = 1;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint32_t v = neg ? ~Y[j] : Y[j];
            const uint64_t s = (uint64_t)v + (neg ? cb : 0u);
            mag[j] = (uint32_t)s;
            cb = (uint32_t)(s >> 32);
        }
        int cmp = 0;  // sign of |Y| - P/2
#pragma unroll
        for (int j = W - 1; j >= 0; --j)
            if (cmp == 0 && mag[j] != t.halfP[j]) cmp = mag[j] > t.halfP[j] ? 1 : -1;
        const bool too_high = !neg && cmp >= 0;  // Y >= P/2
        const bool too_low = neg && cmp > 0;     // Y < -P/2
        if (too_high || too_low) {
            uint64_t c2 = 0;
            int64_t b2 = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                if (too_high) {
                    const int64_t d = (int64_t)Y[j] - (int64_t)t.P[j] - b2;
                    Y[j] = (uint32_t)d;
                    b2 = d < 0 ? 1 : 0;
                } else {
                    const uint64_t s = (uint64_t)Y[j] + t.P[j] + c2;
                    Y[j] = (uint32_t)s;
                    c2 = s >> 32;
                }
            }
        }
    }
    const bool neg = abs_words<W>(Y);
    int top = -1;
#pragma unroll
    for (int j = W - 1; j >= 0; --j)
        if (top < 0 && Y[j] != 0) top = j;
    if (top < 0) return (OutT)0;
    uint32_t w0 = 0, w1 = 0, w2 = 0, low_or = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (j == top) w0 = Y[j];
        if (j == top - 1) w1 = Y[j];
        if (j == top - 2) w2 = Y[j];
        if (j < top - 2) low_or |= Y[j];
    }
    const int lz = __clz(w0);
    const int msb = 32 * top + 31 - lz;
    const uint32_t hi = __funnelshift_l(w1, w0, lz), lo = __funnelshift_l(w2, w1, lz);
    const uint32_t sticky = ((w2 << lz) | low_or) != 0 ? 1u : 0u;
    const uint64_t win = ((uint64_t)hi << 32) | lo | sticky;
    const int E = msb - (ea + fb);
    if constexpr (sizeof(OutT) == 4) {
        const uint32_t m24 = (uint32_t)(win >> 40);
        const uint64_t rem = win & ((1ull << 40) - 1);
        const uint32_t m = m24 + (uint32_t)((rem + ((1ull << 39) - 1) + (m24 & 1u)) >> 40);
        const uint32_t sign = neg ? 0x80000000u : 0u;
        if (E >= -126 && E <= 126)
            return __uint_as_float(sign | (((uint32_t)(E + 126) << 23) + m));
        // outside the normal single range: x 2^-(e+f) (24 bits, exponent within +-500 for
        // single inputs) is exact in double and its conversion to float is the one rounding
        const uint32_t mr = m >> 24 ? m >> 1 : m;
        const int Er = m >> 24 ? E + 1 : E;
        return double_bits_to_float(((uint64_t)sign << 32) | ((uint64_t)(Er + 1023) << 52) |
                                    ((uint64_t)(mr & 0x7FFFFFu) << 29));
    } else {
        const uint64_t m53 = win >> 11;
        const uint32_t rem = (uint32_t)win & 0x7FFu;
        const uint64_t m = m53 + ((rem + 0x3FFu + ((uint32_t)m53 & 1u)) >> 11);
        const uint64_t sign = neg ? (1ull << 63) : 0ull;
        if (E >= -1022 && E <= 1022)
            return __longlong_as_double(
                (long long)(sign | (((uint64_t)(E + 1022) << 52) + m)));
        const uint64_t mr = m >> 53 ? m >> 1 : m;
        const int msbr = m >> 53 ? msb + 1 : msb;
        const double x = __longlong_as_double(
            (long long)(sign | ((uint64_t)(msbr + 1023) << 52) | (mr & ((1ull << 52) - 1))));
        return scale_pow2_rn(x, -(ea + fb));
    }
}

// OutT = double (DGEMM) or float (SGEMM): C'' is rounded to 53 or 24 bits, then scaled by
// 2^-(ea + fb).  v: the pair sums of the entry (pair_sums or dot2).  The shifts must be finite
// (the caller substitutes 0 for OZAKI2_SHIFT_NONFINITE and selects NaN afterwards).
template <int N, typename OutT>
__device__ __forceinline__ OutT crt_value(const uint32_t (&v)[(N + 1) / 2], int ea, int fb,
                                          const CrtTables& t) {
    constexpr int W = crt_words(N);
    constexpr int G = (N + 1) / 2;
    // X = sum_g PG_g v_g (64-bit column sums) and S ~ 2^46 X / P (fixed point).  A pair's
    // constant round(2^46 / prod_g) is below 2^32, so its term is one 32 x 32 -> 64-bit
    // multiply-add; a single modulus (odd N) keeps a 64-bit constant.
    uint64_t acc[W];
#pragma unroll
    for (int j = 0; j < W; ++j) acc[j] = 0;
    uint64_t S = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (2 * g + 1 < N) S += (uint64_t)v[g] * (uint32_t)t.R46[g];
        else S += (uint64_t)v[g] * t.R46[g];
#pragma unroll
        for (int j = 0; j < W; ++j) acc[j] += (uint64_t)t.PG[g][j] * v[g];
    }
    uint32_t X[W];
    fold_columns<W>(acc, X);
    // Q = round(X / P) from the fixed-point estimate (|S/2^46 - X/P| < 2^-18, S < 2^60): adding
    // 2^45 touches only the high word.  The estimate is within 2^-10 of a half-integer when
    // (S - 2^45 + 2^36) mod 2^46 < 2^37, i.e. bits 37..45 of that difference are clear; Q may
    // then be one off, which crt_value_rare settles exactly.
    const uint32_t s_hi = (uint32_t)(S >> 32);
    const uint32_t Q = (s_hi + (1u << 13)) >> 14;
    const bool near_half =
        ((uint32_t)((S - ((1ull << 45) - (1ull << 36))) >> 32) & 0x3FE0u) == 0;
    Words<W> Yw;
    add_word_times<W>(X, Q, t.negP, Yw.w);  // Y = X - Q P (mod 2^(32 W))
    // The common case, straight-line: |Y| with its leading bit in word TOP (the shifts make |C''|
    // large against P) and a result in the normal range.  The 64 bits from the leading one down
    // come by funnel shifts (a shift of 0 keeps the words), every lower bit folded into bit 0 as
    // a sticky bit (it lies below every rounding position); rounding to nearest even adds the
    // remainder, half an ulp less one and the kept part's last bit, and a rounded-up 2^53 (2^24)
    // carries into the exponent field.
    uint32_t A[W];
#pragma unroll
    for (int j = 0; j < W; ++j) A[j] = Yw.w[j];
    const bool neg = abs_words<W>(A);
    constexpr int TOP = crt_top(N);
    uint32_t w0 = A[TOP], w1 = TOP > 0 ? A[TOP - 1] : 0u, w2 = TOP > 1 ? A[TOP - 2] : 0u;
    uint32_t low_or = 0, high_or = 0;
#pragma unroll
    for (int j = 0; j < TOP - 3; ++j) low_or |= A[j];    // words below TOP - 3
    const uint32_t w3 = TOP > 2 ? A[TOP - 3] : 0u;
#pragma unroll
    for (int j = TOP + 1; j < W; ++j) high_or |= A[j];  // zero unless Q was one off
    int top = TOP;
    if constexpr (crt_window_drops(N)) {
        // a zero word TOP: the window one word lower, word TOP - 3 in it rather than sticky
        const bool down = w0 == 0u;
        w0 = down ? w1 : w0;
        w1 = down ? w2 : w1;
        w2 = down ? w3 : w2;
        low_or |= down ? 0u : w3;
        top = down ? TOP - 1 : TOP;
    } else {
        low_or |= w3;
    }
    const int lz = __clz(w0);  // 32 when that word is zero: the rare path then
    const uint32_t hi = __funnelshift_l(w1, w0, lz), lo = __funnelshift_l(w2, w1, lz);
    const uint32_t sticky = ((w2 << lz) | low_or) != 0 ? 1u : 0u;
    const uint64_t win = ((uint64_t)hi << 32) | lo | sticky;
    const int E = 32 * top + 31 - lz - (ea + fb);
    OutT y;
    bool normal;
    if constexpr (sizeof(OutT) == 4) {
        const uint32_t m24 = (uint32_t)(win >> 40);
        const uint64_t rem = win & ((1ull << 40) - 1);
        const uint32_t m = m24 + (uint32_t)((rem + ((1ull << 39) - 1) + (m24 & 1u)) >> 40);
        y = __uint_as_float((neg ? 0x80000000u : 0u) | (((uint32_t)(E + 126) << 23) + m));
        normal = E >= -126 && E <= 126;
    } else {
        const uint64_t m53 = win >> 11;
        const uint32_t rem = (uint32_t)win & 0x7FFu;
        const uint64_t m = m53 + ((rem + 0x3FFu + ((uint32_t)m53 & 1u)) >> 11);
        y = __longlong_as_double(
            (long long)((neg ? (1ull << 63) : 0ull) | (((uint64_t)(E + 1022) << 52) + m)));
        normal = E >= -1022 && E <= 1022;
    }
    if (near_half || w0 == 0 || high_or != 0 || !normal)
        y = crt_value_rare<N, OutT>(Yw, near_half, ea, fb, t);
    return y;
}

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// ab: bit 0 set when alpha != 1 (multiply by alpha), bit 1 when beta != 0 (add beta C); the
// host decides, so the kernel makes no floating-point comparisons.
__host__ __device__ inline int ab_flags(double alpha, double beta) {
    return (alpha != 1.0 ? 1 : 0) | (beta != 0.0 ? 2 : 0);
}

template <typename OutT>
__device__ __forceinline__ OutT quiet_nan() {
    if constexpr (sizeof(OutT) == 4) return __uint_as_float(0x7FC00000u);
    else return __longlong_as_double(0x7FF8000000000000ll);
}

// C'' scaled for one entry, NaN when either line is non-finite (the value is computed with
// zero shifts then, and replaced).
template <int N, typename OutT>
__device__ __forceinline__ OutT crt_entry(const uint32_t (&v)[(N + 1) / 2], int ea, int fb,
                                          const CrtTables& t) {
    const bool bad = ea == OZAKI2_SHIFT_NONFINITE || fb == OZAKI2_SHIFT_NONFINITE;
    const OutT y = crt_value<N, OutT>(v, bad ? 0 : ea, bad ? 0 : fb, t);
    return bad ? quiet_nan<OutT>() : y;
}

// One tile of C (rows i0.., columns j0..; 32 x 64 for VEC, 32 x 32 otherwise); all 256 threads
// take part.  VEC: the residue planes are padded to whole 32 x 64 tiles and 8-byte aligned (the
// library's own layout), so thread t reconstructs the eight consecutive entries of row t/8 from
// column 8 (t % 8), reading them with one 64-bit load per plane (half the loads and address
// arithmetic per entry of four-entry threads); entries outside C are computed from zero shifts
// like the others and only their stores are skipped.  A non-finite shift of the row or of a
// column replaces the entries it touches by NaN after the fact, so the common path computes
// every entry the same way.  Otherwise each residue is read on its own.
template <int N, typename OutT, bool VEC, bool AB = true>
__device__ __forceinline__ void crt_tile(const int8_t* __restrict__ res, int64_t ldr,
                                         int64_t plane, int m, int n, const int* __restrict__ sa,
                                         const int* __restrict__ sb, OutT alpha, OutT beta,
                                         int ab, OutT* __restrict__ C, int64_t ldc,
                                         const CrtTables& t, int i0, int j0,
                                         OutT (*tile)[TI + 1]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int COLS = tile_cols<VEC>();
    if constexpr (VEC) {
        const int il = threadIdx.x >> 3, jq = (threadIdx.x & 7) * 8;
        const int i = i0 + il;
        const int ea = i < m ? sa[i] : 0;
        int fb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) fb[q] = j0 + jq + q < n ? sb[j0 + jq + q] : 0;
        bool bad = ea == OZAKI2_SHIFT_NONFINITE;
#pragma unroll
        for (int q = 0; q < 8; ++q) bad |= fb[q] == OZAKI2_SHIFT_NONFINITE;
        const int ea_u = ea == OZAKI2_SHIFT_NONFINITE ? 0 : ea;
        const int8_t* base = res + (int64_t)i * ldr + j0 + jq;
        constexpr int G = (N + 1) / 2;
        // per pair of planes, the residues of the eight entries interleaved two entries to a
        // word: w[g][h] holds entries 2h and 2h + 1 (bytes c_2g, c_2g+1 of each)
        uint32_t w[G][4];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint2 a = __ldg(reinterpret_cast<const uint2*>(base + (int64_t)(2 * g) * plane));
            const uint2 b = 2 * g + 1 < N ? __ldg(reinterpret_cast<const uint2*>(
                                                base + (int64_t)(2 * g + 1) * plane))
                                          : make_uint2(0u, 0u);
            w[g][0] = __byte_perm(a.x, b.x, 0x5140);
            w[g][1] = __byte_perm(a.x, b.x, 0x7362);
            w[g][2] = __byte_perm(a.y, b.y, 0x5140);
            w[g][3] = __byte_perm(a.y, b.y, 0x7362);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t v[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t b = w[g][q >> 1];
                v[g] = (q & 1) ? dot2<true>(t.Kpair[g], b, t.grp_bias[g])
                               : dot2<false>(t.Kpair[g], b, t.grp_bias[g]);
            }
            const int fbu = fb[q] == OZAKI2_SHIFT_NONFINITE ? 0 : fb[q];
            tile[jq + q][il] = crt_value<N, OutT>(v, ea_u, fbu, t);
        }
        if (bad) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (ea == OZAKI2_SHIFT_NONFINITE || fb[q] == OZAKI2_SHIFT_NONFINITE)
                    tile[jq + q][il] = quiet_nan<OutT>();
        }
    } else {
        const int j = j0 + lane;
        const int fb = j < n ? sb[j] : 0;
#pragma unroll
        for (int r = 0; r < TI / 8; ++r) {
            const int il = warp + 8 * r;
            const int i = i0 + il;
            OutT y = 0;
            if (i < m && j < n) {
                const int8_t* p = res + (int64_t)i * ldr + j;
                int c[N];
#pragma unroll
                for (int l = 0; l < N; ++l) c[l] = p[(int64_t)l * plane];
                uint32_t v[(N + 1) / 2];
                pair_sums<N>(c, t, v);
                y = crt_entry<N, OutT>(v, sa[i], fb, t);
            }
            tile[lane][il] = y;
        }
    }
    __syncthreads();
    // Two loops rather than one with selects: a select between the product and the plain value
    // still issues the (predicated-off) floating-point multiply, which for doubles occupies the
    // narrow FP64 pipe.  AB = false (alpha = 1, beta = 0, decided on the host) compiles only the
    // plain stores.
    if (!AB || ab == 0) {
#pragma unroll
        for (int r = 0; r < COLS / 8; ++r) {
            const int jl = warp + 8 * r;
            const int jj = j0 + jl, ii = i0 + lane;
            if (ii < m && jj < n) C[ii + (int64_t)jj * ldc] = tile[jl][lane];
        }
    } else if constexpr (AB) {
#pragma unroll 1
        for (int r = 0; r < COLS / 8; ++r) {
            const int jl = warp + 8 * r;
            const int jj = j0 + jl, ii = i0 + lane;
            if (ii < m && jj < n) {
                OutT* out = C + ii + (int64_t)jj * ldc;
                const OutT y = tile[jl][lane];
                OutT v = (ab & 1) ? mul_rn(alpha, y) : y;
                if (ab & 2) v = add_rn(v, mul_rn(beta, *out));
                *out = v;
            }
        }
    }
}

// Blocks per SM the register budget is cut for: four (64 registers a thread) where that spills
// nothing, measured faster at N = 16 than the three that the compiler's own choice leaves room
// for; three for the five-word N >= 17 and for the grouped kernel from N = 12 on, where four
// would spill.
__host__ __device__ constexpr int crt_min_blocks(int N, bool grouped) {
    return (grouped ? N <= 11 : N <= 16) ? 4 : 3;
}

// AB = false: alpha = 1 and beta = 0 (the kernel has no alpha/beta code at all).
template <int N, typename OutT, bool VEC, bool AB>
__global__ void __launch_bounds__(256, crt_min_blocks(N, false)) crt_kernel(const int8_t* __restrict__ res, int64_t ldr,
                                                  int64_t plane, int m, int n,
                                                  const int* __restrict__ sa,
                                                  const int* __restrict__ sb, OutT alpha,
                                                  OutT beta, int ab, OutT* __restrict__ C,
                                                  int64_t ldc, const CrtTables t) {
    // tiles of C in row-band order, blocks striding over them (one tile per block when
    // the grid covers them all; fewer blocks leave room on each SM for another kernel).  The
    // (band, column) position advances by the stride's quotient and remainder, so the loop
    // divides nothing.
    constexpr int COLS = tile_cols<VEC>();
    __shared__ OutT tile[COLS][TI + 1];
    const unsigned tiles_j = (unsigned)(n + COLS - 1) / COLS, tiles_i = (unsigned)(m + TI - 1) / TI;
    const unsigned step_i = gridDim.x / tiles_j, step_j = gridDim.x % tiles_j;
    unsigned ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
    while (ti < tiles_i) {
        crt_tile<N, OutT, VEC, AB>(res, ldr, plane, m, n, sa, sb, alpha, beta, ab, C, ldc, t,
                               (int)(ti * TI), (int)(tj * COLS), tile);
        __syncthreads();  // the tile buffer is written again by the next tile
        ti += step_i;
        tj += step_j;
        if (tj >= tiles_j) {
            tj -= tiles_j;
            ++ti;
        }
    }
}

// Grouped: each block reconstructs one 32 x 64 tile of one problem's C (the work list holds
// their corners; every problem's product residues are padded to whole tiles).
template <int N>
__global__ void __launch_bounds__(256, crt_min_blocks(N, true)) crt_grouped_kernel(const GroupProblem* __restrict__ probs,
                                                          const CrtWork* __restrict__ work,
                                                          const CrtTables t) {
    __shared__ double tile[TJV][TI + 1];
    const CrtWork w = work[blockIdx.x];
    const GroupProblem& P = probs[w.problem];
    crt_tile<N, double, true>(P.res, P.n_pad, (int64_t)P.m_pad * P.n_pad, P.m, P.n, P.e, P.f,
                              P.alpha, P.beta, P.ab,
                P.C, P.ldc, t, w.i0, w.j0, tile);
}

template <typename T>
__global__ void scale_c_kernel(int m, int n, T beta, T* C, int64_t ldc) {
    const int64_t total = (int64_t)m * n;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = g / m, i = g - j * m;
        T* p = C + i + j * ldc;
        *p = beta == (T)0 ? (T)0 : mul_rn(beta, *p);
    }
}

}  // namespace

namespace {
template <typename OutT, bool VEC>
cudaError_t launch_crt_typed(const int8_t* res, int64_t ldr, int64_t plane, int m, int n,
                             const int* sa, const int* sb, OutT alpha, OutT beta, OutT* C,
                             int64_t ldc, const ModTables& t, cudaStream_t stream,
                             int max_blocks) {
    const int64_t tiles = (int64_t)((n + tile_cols<VEC>() - 1) / tile_cols<VEC>()) * ((m + TI - 1) / TI);
    const int64_t cap = max_blocks > 0 ? max_blocks : (int64_t)INT32_MAX;
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    const int ab = ab_flags(alpha, beta);
#define OZAKI2_CRT_CASE(NN)                                                                   \
    case NN:                                                                                  \
        if (ab)                                                                               \
            crt_kernel<NN, OutT, VEC, true><<<grid, 256, 0, stream>>>(                         \
                res, ldr, plane, m, n, sa, sb, alpha, beta, ab, C, ldc, t.crt);                \
        else                                                                                  \
            crt_kernel<NN, OutT, VEC, false><<<grid, 256, 0, stream>>>(                        \
                res, ldr, plane, m, n, sa, sb, alpha, beta, ab, C, ldc, t.crt);                \
        break;
    switch (t.N) {
        OZAKI2_CRT_CASE(2) OZAKI2_CRT_CASE(3) OZAKI2_CRT_CASE(4) OZAKI2_CRT_CASE(5)
        OZAKI2_CRT_CASE(6) OZAKI2_CRT_CASE(7) OZAKI2_CRT_CASE(8) OZAKI2_CRT_CASE(9)
        OZAKI2_CRT_CASE(10) OZAKI2_CRT_CASE(11) OZAKI2_CRT_CASE(12) OZAKI2_CRT_CASE(13)
        OZAKI2_CRT_CASE(14) OZAKI2_CRT_CASE(15) OZAKI2_CRT_CASE(16) OZAKI2_CRT_CASE(17)
        OZAKI2_CRT_CASE(18) OZAKI2_CRT_CASE(19) OZAKI2_CRT_CASE(20)
        default: return cudaErrorInvalidValue;
    }
#undef OZAKI2_CRT_CASE
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_crt(const int8_t* res, int64_t ldr, int64_t plane, int m, int n,
                       const int* sa, const int* sb, double alpha, double beta, void* C,
                       int64_t ldc, const ModTables& t, unsigned* status, cudaStream_t stream,
                       bool f32, bool padded, int max_blocks) {
    (void)status;
    if (m <= 0 || n <= 0) return cudaSuccess;
    // the 64-bit residue loads need 8-byte alignment and planes padded to whole 32 x 64 tiles
    const bool vec = padded && (reinterpret_cast<uintptr_t>(res) & 7u) == 0 && ldr % 8 == 0 &&
                     plane % 8 == 0 && ldr >= (int64_t)(n + TJV - 1) / TJV * TJV &&
                     plane >= (int64_t)(m + TI - 1) / TI * TI * ldr;
    if (f32) {
        auto* c = static_cast<float*>(C);
        return vec ? launch_crt_typed<float, true>(res, ldr, plane, m, n, sa, sb, (float)alpha,
                                                   (float)beta, c, ldc, t, stream, max_blocks)
                   : launch_crt_typed<float, false>(res, ldr, plane, m, n, sa, sb, (float)alpha,
                                                    (float)beta, c, ldc, t, stream, max_blocks);
    }
    auto* c = static_cast<double*>(C);
    return vec ? launch_crt_typed<double, true>(res, ldr, plane, m, n, sa, sb, alpha, beta, c, ldc,
                                                t, stream, max_blocks)
               : launch_crt_typed<double, false>(res, ldr, plane, m, n, sa, sb, alpha, beta, c,
                                                 ldc, t, stream, max_blocks);
}

cudaError_t launch_crt_grouped(int N, const GroupProblem* probs, const CrtWork* work, int blocks,
                               const CrtTables& t, cudaStream_t stream) {
    if (blocks <= 0) return cudaSuccess;
    switch (N) {
#define OZAKI2_CRT_GROUPED_CASE(NN)                                                    \
    case NN:                                                                           \
        crt_grouped_kernel<NN><<<blocks, 256, 0, stream>>>(probs, work, t);            \
        break;
        OZAKI2_CRT_GROUPED_CASE(2) OZAKI2_CRT_GROUPED_CASE(3) OZAKI2_CRT_GROUPED_CASE(4)
        OZAKI2_CRT_GROUPED_CASE(5) OZAKI2_CRT_GROUPED_CASE(6) OZAKI2_CRT_GROUPED_CASE(7)
        OZAKI2_CRT_GROUPED_CASE(8) OZAKI2_CRT_GROUPED_CASE(9) OZAKI2_CRT_GROUPED_CASE(10)
        OZAKI2_CRT_GROUPED_CASE(11) OZAKI2_CRT_GROUPED_CASE(12) OZAKI2_CRT_GROUPED_CASE(13)
        OZAKI2_CRT_GROUPED_CASE(14) OZAKI2_CRT_GROUPED_CASE(15) OZAKI2_CRT_GROUPED_CASE(16)
        OZAKI2_CRT_GROUPED_CASE(17) OZAKI2_CRT_GROUPED_CASE(18) OZAKI2_CRT_GROUPED_CASE(19)
        OZAKI2_CRT_GROUPED_CASE(20)
#undef OZAKI2_CRT_GROUPED_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_scale_c(int m, int n, double beta, void* C, int64_t ldc,
                           cudaStream_t stream, bool f32) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int64_t total = (int64_t)m * n;
    const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (f32)
        scale_c_kernel<float><<<grid, 256, 0, stream>>>(m, n, (float)beta, static_cast<float*>(C),
                                                        ldc);
    else
        scale_c_kernel<double><<<grid, 256, 0, stream>>>(m, n, beta, static_cast<double*>(C),
                                                         ldc);
    return cudaGetLastError();
}

}  // namespace ozaki2
