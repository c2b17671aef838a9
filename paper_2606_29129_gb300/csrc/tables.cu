// tables.cu -- Step 1 of Ozaki scheme II (Section 2.2) on the host: the moduli of eq. (moduli),
// P, P_l = P/p_l, q_l = P_l^{-1} mod p_l, P'_prop (Section 4), and the derived per-kernel
// tables.  Multi-word arithmetic uses little-endian 32-bit words.
#include <math.h>

#include <mutex>
#include <vector>

#include "ozaki2_internal.h"

namespace ozaki2 {
namespace {

// eq. (moduli): the twenty pairwise coprime moduli, largest first; N moduli = the first N.
const int kModuli[kMaxModuli] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227,
                                 223, 217, 211, 199, 197, 193, 191, 181, 179, 173};

using Words = std::vector<uint32_t>;

void mul_small(Words& a, uint32_t f) {
    uint64_t carry = 0;
    for (auto& w : a) {
        uint64_t t = (uint64_t)w * f + carry;
        w = (uint32_t)t;
        carry = t >> 32;
    }
    if (carry) a.push_back((uint32_t)carry);
}

uint32_t mod_small(const Words& a, uint32_t p) {
    uint64_t r = 0;
    for (size_t i = a.size(); i-- > 0;) r = ((r << 32) | a[i]) % p;
    return (uint32_t)r;
}

int bit_length(const Words& a) {
    for (size_t i = a.size(); i-- > 0;)
        if (a[i]) return 32 * (int)i + 32 - __builtin_clz(a[i]);
    return 0;
}

// log2 of a positive multi-word integer from its leading 64 bits.
double log2_words(const Words& a) {
    int b = bit_length(a);
    if (b <= 64) {
        uint64_t v = 0;
        for (size_t i = a.size(); i-- > 0;) v = (v << 32) | a[i];
        return log2((double)v);
    }
    int shift = b - 64;
    uint64_t top = 0;
    for (int bit = b - 1; bit >= shift; --bit)
        top = (top << 1) | ((a[bit / 32] >> (bit % 32)) & 1u);
    return (double)shift + log2((double)top);
}

uint32_t inverse_mod(uint32_t a, uint32_t p) {  // p is small: search is exact and obvious
    for (uint32_t x = 1; x < p; ++x)
        if ((uint64_t)a * x % p == 1) return x;
    return 0;
}

float round_down_to_float(double v) {
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}

void build(int N, ModTables& t) {
    t.N = N;
    Words P{1};
    for (int l = 0; l < N; ++l) mul_small(P, (uint32_t)kModuli[l]);
    Words Pm1 = P;
    Pm1[0] -= 1;  // P is a multiple of 256, so no borrow
    t.pprime = round_down_to_float(log2_words(Pm1) / 2.0 - 0.5);
    t.pprime_fast = round_down_to_float(log2_words(Pm1) / 2.0 - 1.5);
    {   // delta = single-up(0.5 / (1 - 4u_32)) = 0.5 + 2^-23 + 2^-45 + ... -> 0.5 + 3 * 2^-24
        const double q = 0.5 / (1.0 - 4.0 * 0x1p-24);
        float d = (float)q;
        if ((double)d < q) d = nextafterf(d, INFINITY);
        t.delta = d;
    }

    t.conv.N = t.crt.N = t.epi.N = N;
    for (int l = 0; l < N; ++l) {
        const uint32_t p = (uint32_t)kModuli[l];
        Words Pl{1};
        for (int j = 0; j < N; ++j)
            if (j != l) mul_small(Pl, (uint32_t)kModuli[j]);
        const uint32_t q = inverse_mod(mod_small(Pl, p), p);
        t.moduli[l] = (int)p;
        t.inverses[l] = (int)q;

        t.conv.p[l] = p;
        for (int j = 0; j < 4; ++j) {
            uint64_t v = 1;
            for (int b = 0; b < 21 * j; ++b) v = (v * 2) % p;
            t.conv.pow21[l][j] = (uint32_t)v;
        }
        const uint32_t h = (p - 1) / 2;
        t.conv.bias[l] = 0x4B400000u - h;
        t.conv.magic39[l] = (uint32_t)(((1ull << 39) + p - 1) / p);
        t.conv.neg_bias_magic[l] =
            (unsigned long long)(0ull - (uint64_t)t.conv.bias[l] * t.conv.magic39[l]);

        t.epi.p[l] = (float)p;
        t.epi.inv_p[l] = 1.0f / (float)p;
        t.epi.hi[l] = (p % 2) ? (float)((p - 1) / 2) : (float)(p / 2 - 1);
        t.epi.lo[l] = (p % 2) ? -(float)((p - 1) / 2) : -(float)(p / 2);
    }
    for (int g = 0; 2 * g < N; ++g) {
        const int l0 = 2 * g, l1 = (2 * g + 2 < N) ? 2 * g + 2 : N;
        uint64_t prod = 1;
        for (int l = l0; l < l1; ++l) prod *= (uint64_t)kModuli[l];
        for (int l = l0; l < l1; ++l) {
            const uint64_t cf = prod / (uint64_t)kModuli[l];
            t.crt.K[l] = (uint32_t)(cf * (uint64_t)t.inverses[l] % prod);
        }
        t.crt.Kpair[g] = t.crt.K[l0] | (l1 - l0 > 1 ? t.crt.K[l0 + 1] << 16 : 0u);
        t.crt.grp_bias[g] = (uint32_t)(256 * prod);  // >= 128 sum K_l: the group sum stays >= 0
        Words PG{1};
        for (int j = 0; j < N; ++j)
            if (j < l0 || j >= l1) mul_small(PG, (uint32_t)kModuli[j]);
        for (int w = 0; w < kMaxWords; ++w) t.crt.PG[g][w] = w < (int)PG.size() ? PG[w] : 0u;
        t.crt.R46[g] = (unsigned long long)(((unsigned __int128)1 << 46) / prod +
                                            ((((unsigned __int128)1 << 46) % prod) * 2 >= prod));
    }
    {   // two's complement of P over kMaxWords words
        uint64_t borrow = 0;
        for (int w = 0; w < kMaxWords; ++w) {
            const uint64_t pw = w < (int)P.size() ? P[w] : 0u;
            const uint64_t d = (uint64_t)0 - pw - borrow;
            t.crt.negP[w] = (uint32_t)d;
            borrow = (pw + borrow) != 0 ? 1 : 0;
        }
    }
    for (int w = 0; w < kMaxWords; ++w) {
        t.crt.P[w] = w < (int)P.size() ? P[w] : 0u;
        uint32_t hi_bit = (w + 1 < (int)P.size()) ? (P[w + 1] & 1u) : 0u;
        t.crt.halfP[w] = (w < (int)P.size() ? (P[w] >> 1) : 0u) | (hi_bit << 31);
    }
}

ModTables g_tables[kMaxModuli + 1];
std::once_flag g_once;

}  // namespace

const ModTables* mod_tables(int N) {
    if (N < OZAKI2_MIN_MODULI || N > OZAKI2_MAX_MODULI) return nullptr;
    std::call_once(g_once, [] {
        for (int n = OZAKI2_MIN_MODULI; n <= OZAKI2_MAX_MODULI; ++n) build(n, g_tables[n]);
    });
    return &g_tables[N];
}

}  // namespace ozaki2
