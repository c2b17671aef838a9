// scale.cu -- Step 2 scaling of Ozaki scheme II with the scale-invariant formula of Section 4
// (eq. (proposed-mu)/(proposed-nu), Algorithm 2).
//
// Each line (row of op(A) or column of op(B)) gets a_norm = sum_h a_h^2 rounded upward (Section
// 4, which allows single or double precision), in a fixed order: blocks of kNormBlock = 256
// consecutive terms, each summed in single precision on terms rescaled exactly by a power of two
// (LineAcc), then the block values added in block order with upward rounding.  Every partial sum
// is an upper bound, as Algorithm 2 requires, and the fixed order keeps the shifts bit-identical
// to a sequential reference.  Then log2(mu) = floor(w - t) from Algorithm 2.
//
// The kernels are bound by HBM reads of the matrix (8 bytes per element): the per-term work is
// integer and single-precision arithmetic, with only a few FP64 operations per block of 256
// terms.  Lines of at most one block run one thread per line; longer lines, when the
// caller gives scratch for the block sums, run two kernels: one warp per norm block of 32 lines
// (scale_partials_kernel), then one thread per line adding its block sums in order
// (scale_fold_kernel).
#include <float.h>

#include <algorithm>

#include "ozaki2_internal.h"
#include "sm103_ptx.cuh"

namespace ozaki2 {
namespace {

// Algorithm 2 for one line.
//   s := floor(log2 a_norm);  t := single-up(0.5 * log2(a_norm / 2^s) + 2u_32);
//   w := single-down(P'_prop - 0.5 s);  return floor(w - t).
// The single-precision log2 of Algorithm 2 (__log2f, error <= 4u_32 on [1,2]) is replaced by the
// double-precision log2 of the argument rounded up to single and then rounded up to single:
// a tighter bound, inside the margin that the 2u_32 term provides.  The argument a_norm/2^s is
// rounded up to single first.  floor(w - t) is taken exactly (subtraction rounded down).
__device__ int alg2_shift(double a_norm, float pprime, unsigned* status) {
    if (a_norm == 0.0) return 0;
    if (!(a_norm <= DBL_MAX)) {  // +Inf or NaN
        atomicOr(status, OZAKI2_STATUS_NONFINITE);
        return OZAKI2_SHIFT_NONFINITE;
    }
    const int s = ilogb(a_norm);
    const double xprime = scalbn(a_norm, -s);               // [1, 2), exact
    const float xf = __double2float_ru(xprime);
    const float lg = __double2float_ru(log2((double)xf));
    const float t = __double2float_ru(0.5 * (double)lg + 0x1p-23);   // exact sum, then up
    const float w = __double2float_rd((double)pprime - 0.5 * (double)s);
    return (int)floor(__dsub_rd((double)w, (double)t));
}

// Algorithm 1 (original fast mode, Section 2.3) for one line.
//   s := floor(log2 a_norm);  t := single-up(delta * (log2(a_norm / 2^s) + s));
//   return floor(P'_fast - max(1, t)) - floor(log2 a_max)
// with the same logarithm stand-in and exact floors as alg2_shift.
__device__ int alg1_shift(double a_norm, double a_max, float pprime_fast, float delta,
                          unsigned* status) {
    if (a_norm == 0.0 || a_max == 0.0) return 0;
    if (!(a_norm <= DBL_MAX) || !(a_max <= DBL_MAX)) {
        atomicOr(status, OZAKI2_STATUS_NONFINITE);
        return OZAKI2_SHIFT_NONFINITE;
    }
    const int s = ilogb(a_norm);
    const double xprime = scalbn(a_norm, -s);
    const float lg = __double2float_ru(log2((double)__double2float_ru(xprime)));
    const float t = __double2float_ru(__dmul_ru((double)delta, (double)lg + (double)s));
    const double mx = t > 1.0f ? (double)t : 1.0;
    return (int)floor(__dsub_rd((double)pprime_fast, mx)) - ilogb(a_max);
}

// Accurate mode, first pass (Section 2.3): E = floor(log2 max_h |a_h|) of the line, from which
// mu' = 2^(5 - E).  Returns E, kAccuZeroLine for a zero line, or OZAKI2_SHIFT_NONFINITE (and
// raises the status flag) for a line with an Inf or NaN.  `mb` is the largest |a_h| as bits:
// for nonnegative doubles the integer order is the value order, and NaN/Inf bits exceed every
// finite value.
__device__ __forceinline__ int accu_line_exponent(uint64_t mb, unsigned* status) {
    if (mb >= 0x7FF0000000000000ull) {
        atomicOr(status, OZAKI2_STATUS_NONFINITE);
        return OZAKI2_SHIFT_NONFINITE;
    }
    if (mb == 0) return kAccuZeroLine;
    return ilogb(__longlong_as_double((long long)mb));
}

constexpr int kNormBlock = 256;  // terms per block of the squared-norm sum

// single-up(f 2^-s) for a single f >= 0 and s >= 1, from the bits: a normal result is f with its
// exponent lowered; a subnormal one is the mantissa shifted right, rounded up on any lost bit
// (the least positive single when nothing is left).  Taken only when a block's largest exponent
// rises.
__device__ __forceinline__ float scale_down_ru(float f, int s) {
    const uint32_t b = __float_as_uint(f);
    if (b == 0u) return 0.0f;
    const int ef = (int)(b >> 23);
    if (ef > s) return __uint_as_float(b - ((uint32_t)s << 23));
    const uint32_t m = ef ? ((b & 0x7FFFFFu) | 0x800000u) : b;
    const int r = s + 1 - (ef ? ef : 1);  // >= 1
    if (r >= 25) return __uint_as_float(1u);
    const uint32_t q = m >> r;
    return __uint_as_float(q + ((m & ((1u << r) - 1u)) != 0u ? 1u : 0u));
}

// single-up(|v| 2^(1023 - E)) for the bits b of |v| (finite, nonzero) whose exponent field is at
// most E, when |v| is a subnormal double or the result may be a subnormal single.  With M the
// integer mantissa, the value is M 2^-sh in units of 2^-149 (the least positive single); a
// normal single keeps the 24 bits from M's leading one and rounds up on any lower one, a
// subnormal single is the unit count rounded up (the least positive single when M 2^-sh < 1).
__device__ __forceinline__ float single_up_rare(uint64_t b, int E) {
    const int ef = (int)(b >> 52);
    uint64_t M = b & ((1ull << 52) - 1);
    int e2 = ef;                              // |v| = M 2^(e2 - 1075)
    if (ef) M |= 1ull << 52; else e2 = 1;
    const int sh = E - e2 - 97;               // value = M 2^(e2 - E - 52) = M 2^-sh units
    const int p = 63 - __clzll((long long)M); // M's leading bit
    if (p - sh >= 23) {                       // a normal single, exponent p - sh - 149
        const int ex = p - sh - 149;
        const uint64_t frac = M ^ (1ull << p);
        const int drop = p - 23;
        uint32_t mant;
        bool lost = false;
        if (drop >= 0) {
            mant = (uint32_t)(frac >> drop);
            lost = (frac & ((1ull << drop) - 1)) != 0;
        } else {
            mant = (uint32_t)(frac << -drop);
        }
        return __uint_as_float((((uint32_t)(ex + 127)) << 23) + mant + (lost ? 1u : 0u));
    }
    if (sh <= 0) return __uint_as_float((uint32_t)(M << -sh));  // exact, below 2^23 units
    if (sh >= 64) return __uint_as_float(1u);
    const bool lost = (M & ((1ull << sh) - 1)) != 0;
    return __uint_as_float((uint32_t)(M >> sh) + (lost ? 1u : 0u));
}

// Running state of one line.  The squared norm (proposed and fast modes) is summed in single
// precision with every operation rounded upward (Section 4 allows single or double precision),
// on terms rescaled exactly: blocks of kNormBlock consecutive terms, taken in groups of
// kNormGroup.  Before a group, E (0 at a block's start) becomes the largest of E, 1 and the
// group's exponent fields, and a rise of E by d rescales the block sum to f = single-up(f 2^(-2d));
// each term then enters as x = single-up(|a| 2^(1023 - E)) in [0, 2) and f = single-up(x x + f).
// Closing a block adds its value double-up(double-up(f 2^(E - 1023)) 2^(E - 1023)) to `total`,
// rounded upward.  Every step rounds up and every rescaling is by a power of two, so the norm
// bounds the exact sum from above; the per-term work is integer and single-precision arithmetic,
// none on the FP64 pipe that GB300 keeps narrow.  The largest |a| (fast and accurate modes) is
// kept as bits: for nonnegative doubles the integer order is the value order, and NaN and Inf
// bits exceed every finite value.
// T = double (DGEMM) or float (SGEMM: every float is exactly a double, so the sums and the
// shifts are those of the widened values).
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return widen_exact(x); }
constexpr int kNormGroup = 16;
static_assert(kNormBlock % kNormGroup == 0, "groups must not straddle a norm block");

template <int SCALING>
struct LineAcc {
    float f = 0.0f;
    int E = 0;       // the open block's scale (0: no group yet)
    int nf = 0;      // bit 0: an infinite term, bit 1: a NaN term in the open block
    double total = 0.0;
    uint64_t mb = 0;
    __device__ __forceinline__ double block_value() const {
        if (nf) return (nf & 2) ? __longlong_as_double(0x7FF8000000000000ll)
                                : __longlong_as_double(0x7FF0000000000000ll);
        if (E == 0) return 0.0;
        const double pw = __longlong_as_double((long long)E << 52);  // 2^(E - 1023), exact
        return __dmul_ru(__dmul_ru(widen_exact(f), pw), pw);
    }
    // closes the open block: total += its value, rounded upward
    __device__ __forceinline__ void end_block() {
        if (SCALING != OZAKI2_SCALING_ACCURATE) {
            total = __dadd_ru(total, block_value());
            f = 0.0f;
            E = 0;
            nf = 0;
        }
    }
    // One group: the first `cnt` of the G values v[] (G <= kNormGroup), the next terms of the
    // line in order.  The common case runs straight through; a non-finite term (which settles
    // the block's value), a zero or subnormal term, a term more than 126 binades below E (a
    // subnormal x) and a rescale into the subnormal range take branches.
    // v: the group's terms in order, absent ones (past the end of a line) as zeros.
    template <int G, typename T>
    __device__ __forceinline__ void add_group(const T (&v)[G]) {
        static_assert(G == kNormGroup, "one group at a time");
        constexpr int cnt = G;
        if constexpr (sizeof(T) == 4 && SCALING == OZAKI2_SCALING_PROPOSED) {
            // Single-precision inputs whose group holds only normal nonzero singles: a single's
            // exponent field plus 896 is its double's, and its 23 fraction bits are the top ones
            // of the double's, so x is built from the single's bits with nothing rounded off.
            uint32_t wmax = 0u, wmin = 0xFFFFFFFFu;
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const uint32_t w = u < cnt ? __float_as_uint(v[u]) & 0x7FFFFFFFu : 0u;
                wmax = max(wmax, w);
                wmin = min(wmin, w);
            }
            const int fmax = (int)(wmax >> 23), fmin = (int)(wmin >> 23);
            if (fmin != 0 && fmax != 0xFF && !nf) {
                const int gmax = fmax + 896;
                if (gmax > E) {
                    if (E) f = scale_down_ru(f, 2 * (gmax - E));
                    E = gmax;
                }
                if (E - (fmin + 896) <= 126) {
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        const uint32_t w = __float_as_uint(v[u]) & 0x7FFFFFFFu;
                        const int t = E - ((int)(w >> 23) + 896);
                        const float x = __uint_as_float(((uint32_t)(127 - t) << 23) +
                                                        (w & 0x7FFFFFu));
                        f = __fmaf_ru(x, x, f);
                    }
                    return;
                }
                // a term more than 126 binades below the group's largest: the general path
                // below, whose E is already the group's
            }
        }
        // the upper words of |a| (sign cleared): their extremes give the group's largest and
        // smallest exponent fields; absent terms count as zeros
        auto word = [&](int u) -> uint32_t {
            return u < cnt ? (uint32_t)((uint64_t)__double_as_longlong(to_double(v[u])) >> 32) &
                                 0x7FFFFFFFu
                           : 0u;
        };
        uint32_t wmax = 0u, wmin = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const uint32_t w = word(u);
            wmax = max(wmax, w);
            wmin = min(wmin, w);
            if (SCALING != OZAKI2_SCALING_PROPOSED) {
                const uint64_t b = u < cnt ? (uint64_t)__double_as_longlong(to_double(v[u])) &
                                                 0x7FFFFFFFFFFFFFFFull
                                           : 0ull;
                mb = b > mb ? b : mb;
            }
        }
        if (SCALING == OZAKI2_SCALING_ACCURATE) return;
        const int gmax = max((int)(wmax >> 20), 1), gmin = (int)(wmin >> 20);
        if (gmax == 0x7FF || nf) {  // an Inf or NaN: the block's value is settled
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const uint64_t b = u < cnt ? (uint64_t)__double_as_longlong(to_double(v[u])) &
                                                 0x7FFFFFFFFFFFFFFFull
                                           : 0ull;
                if ((b >> 52) == 0x7FF) nf |= (b & ((1ull << 52) - 1)) ? 2 : 1;
            }
            return;
        }
        if (gmax > E) {
            if (E) f = scale_down_ru(f, 2 * (gmax - E));
            E = gmax;
        }
        if (gmin != 0 && E - gmin <= 126) {
            // every term a normal double whose x is a normal single: (1 + M/2^52) 2^-t with
            // exponent -t, the top 23 fraction bits, plus one for any lower bit
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const uint64_t b = (uint64_t)__double_as_longlong(to_double(v[u]));
                const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
                const int t = E - (int)((hi >> 20) & 0x7FFu);
                const uint32_t top = __funnelshift_l(lo, hi & 0xFFFFFu, 3);
                const uint32_t lost = min(lo & 0x1FFFFFFFu, 1u);
                const float x = __uint_as_float(((uint32_t)(127 - t) << 23) + top + lost);
                f = __fmaf_ru(x, x, f);
            }
        } else {
            // zeros, subnormal doubles, subnormal singles or a short group: term by term
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const uint64_t b = (uint64_t)__double_as_longlong(to_double(v[u])) &
                                   0x7FFFFFFFFFFFFFFFull;
                const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
                const int ef = (int)(hi >> 20);
                const int t = E - ef;
                uint32_t xb;
                if (ef != 0 && t <= 126) {
                    const uint32_t top = __funnelshift_l(lo, hi & 0xFFFFFu, 3);
                    const uint32_t lost = min(lo & 0x1FFFFFFFu, 1u);
                    xb = ((uint32_t)(127 - t) << 23) + top + lost;
                } else {
                    xb = b == 0 ? 0u : __float_as_uint(single_up_rare(b, E));
                }
                const float x = __uint_as_float(xb);
                f = __fmaf_ru(x, x, f);
            }
        }
    }
    __device__ __forceinline__ int result(float pprime, float delta, unsigned* status) {
        if (SCALING == OZAKI2_SCALING_ACCURATE) return accu_line_exponent(mb, status);
        end_block();
        if (SCALING == OZAKI2_SCALING_FAST)
            return alg1_shift(total, __longlong_as_double((long long)mb), pprime, delta, status);
        return alg2_shift(total, pprime, status);
    }
};

// Lines adjacent in memory (line_stride == 1): thread i walks line i in order; a warp reads 32
// consecutive elements per step, so every load is coalesced.  The loads of the next group of 16
// are issued before the current group is summed, so that two groups are in flight per thread.
// Every group is a register array handed over by reference (a pointer into it had put the
// arrays in local memory).

// T = double (DGEMM) or float (SGEMM: every float is exactly a double, so the sums and the
// shifts are those of the widened values).
template <int SCALING, typename T = double>
__device__ __forceinline__ void scale_adjacent_line(const T* __restrict__ X, int64_t ld,
                                                    int i, int len, float pprime, float delta,
                                                    int* shifts, unsigned* status,
                                                    double* norms = nullptr) {
    constexpr int kB = kNormGroup;  // a group per batch, two batches in flight
    const T* p = X + i;
    LineAcc<SCALING> acc;
    const int full = len / kB * kB;
    T a[kB], b[kB];
    if (full > 0) {
#pragma unroll
        for (int u = 0; u < kB; ++u) a[u] = __ldg(p + (int64_t)u * ld);
    }
    for (int h = 0; h < full; h += 2 * kB) {
        const bool has_b = h + kB < full;
        if (has_b) {
#pragma unroll
            for (int u = 0; u < kB; ++u) b[u] = __ldg(p + (int64_t)(h + kB + u) * ld);
        }
        acc.add_group(a);
        if (((h + kB) & (kNormBlock - 1)) == 0) acc.end_block();
        if (!has_b) break;
        if (h + 2 * kB < full) {
#pragma unroll
            for (int u = 0; u < kB; ++u)
                a[u] = __ldg(p + (int64_t)(h + 2 * kB + u) * ld);
        }
        acc.add_group(b);
        if (((h + 2 * kB) & (kNormBlock - 1)) == 0) acc.end_block();
    }
    for (int h = full; h < len; h += kNormGroup) {  // the rest, a group at a time
        const int cnt = min(kNormGroup, len - h);
        T r[kNormGroup];
#pragma unroll
        for (int u = 0; u < kNormGroup; ++u) r[u] = u < cnt ? __ldg(p + (int64_t)(h + u) * ld) : (T)0;
        acc.add_group(r);
        if (((h + cnt) & (kNormBlock - 1)) == 0) acc.end_block();
    }
    shifts[i] = acc.result(pprime, delta, status);
    if (norms) norms[i] = acc.total;
}

template <int SCALING>
__global__ void __launch_bounds__(32) scale_adjacent_kernel(const double* __restrict__ X,
                                                            int64_t ld, int lines, int len,
                                                            float pprime, float delta,
                                                            int* shifts, unsigned* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < lines) scale_adjacent_line<SCALING>(X, ld, i, len, pprime, delta, shifts, status);
}

// Contiguous lines (elem_stride == 1): each warp owns 32 lines.  Tiles of 32 elements per line
// are read with one coalesced 256-byte load per line, the next tile is held in registers while
// the current one (in shared memory) is summed, each lane walking its own line in order.
constexpr int kWarpsPerBlock = 4;
constexpr int kTileLen = 32;

// Elements per line and tile: 32 doubles or 64 floats (256 bytes), loaded as W = 8 / sizeof(T)
// coalesced 128- or 256-byte rows per line.
template <typename T>
__host__ __device__ constexpr int tile_len() { return kTileLen * (8 / (int)sizeof(T)); }

// Lines line0 .. line0 + 31 of a contiguous-line matrix, summed by one warp (t: its smem tile).
template <int SCALING, typename T = double>
__device__ __forceinline__ void scale_contiguous_warp(const T* __restrict__ X, int64_t ld,
                                                      int lines, int len, int line0,
                                                      float pprime, float delta, int* shifts,
                                                      unsigned* status,
                                                      T (*t)[tile_len<T>() + 1],
                                                      double* norms = nullptr) {
    constexpr int W = 8 / (int)sizeof(T), TL = tile_len<T>();
    const int lane = threadIdx.x & 31;
    const int nl = min(32, lines - line0);
    T reg[32][W];
    auto load = [&](int h0) {
#pragma unroll
        for (int r = 0; r < 32; ++r)
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int h = h0 + 32 * w + lane;
                reg[r][w] = (r < nl && h < len) ? __ldg(X + (int64_t)(line0 + r) * ld + h) : (T)0;
            }
    };
    LineAcc<SCALING> acc;
    if (len > 0) load(0);
    for (int h0 = 0; h0 < len; h0 += TL) {
        const int cnt = min(TL, len - h0);
#pragma unroll
        for (int r = 0; r < 32; ++r)
#pragma unroll
            for (int w = 0; w < W; ++w) t[r][32 * w + lane] = reg[r][w];
        __syncwarp();
        if (h0 + TL < len) load(h0 + TL);
        if (lane < nl) {
#pragma unroll
            for (int g = 0; g < TL; g += kNormGroup) {
                if (g < cnt) {
                    T r[kNormGroup];
#pragma unroll
                    for (int u = 0; u < kNormGroup; ++u) r[u] = g + u < cnt ? t[lane][g + u] : (T)0;
                    acc.add_group(r);
                }
            }
            // tiles start at multiples of TL, which divides kNormBlock
            if (((h0 + cnt) & (kNormBlock - 1)) == 0) acc.end_block();
        }
        __syncwarp();
    }
    if (lane < nl) {
        shifts[line0 + lane] = acc.result(pprime, delta, status);
        if (norms) norms[line0 + lane] = acc.total;
    }
}

template <int SCALING>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) scale_contiguous_kernel(
    const double* __restrict__ X, int64_t ld, int lines, int len, float pprime, float delta,
    int* shifts, unsigned* status) {
    __shared__ double tile[kWarpsPerBlock][32][kTileLen + 1];
    const int warp = threadIdx.x >> 5;
    const int line0 = (blockIdx.x * kWarpsPerBlock + warp) * 32;
    if (line0 < lines)
        scale_contiguous_warp<SCALING>(X, ld, lines, len, line0, pprime, delta, shifts, status,
                                       tile[warp]);
}

// LAYOUT: kLayoutAny decides per work item; kLayoutAdjacent / kLayoutContiguous compile one
// layout only (the host has sorted the work list by layout), which keeps the other's registers
// out of the kernel.
template <int SCALING, int LAYOUT>
__device__ __forceinline__ void scale_grouped_lines(const GroupProblem& P, const ScaleWork& w,
                                                    const double* X, int64_t ls, int64_t es,
                                                    int lines, int* shifts, unsigned* status,
                                                    double (*tile)[32][kTileLen + 1]) {
    const bool adjacent = LAYOUT == kLayoutAny ? scale_lines_adjacent(ls, es)
                                               : LAYOUT == kLayoutAdjacent;
    if (adjacent) {
        const int i = w.line0 + (int)threadIdx.x;
        if (i < lines)
            scale_adjacent_line<SCALING>(X, es, i, P.k, P.pprime, P.delta, shifts, status);
    } else {
        const int warp = threadIdx.x >> 5;
        const int line0 = w.line0 + 32 * warp;
        if (line0 < lines)
            scale_contiguous_warp<SCALING>(X, ls, lines, P.k, line0, P.pprime, P.delta, shifts,
                                           status, tile[warp]);
    }
}

// Both operands of one product in one launch: blocks [0, blocks_a) take 128 rows of op(A) each,
// the rest 128 columns of op(B), so the two matrices stream from HBM at the same time.
struct ScaleSide {
    const void* X;
    int64_t ls, es;
    int lines;
    int* shifts;
    double* norms = nullptr;  // optional: the squared norms the shifts come from
};

// ---- lines longer than one block: the blocks of 32 lines split across the 8 warps of a block
constexpr int kSplitWarps = 8;

// Elements per tile row of the split kernel's transposes: 128 bytes.
template <typename T>
__host__ __device__ constexpr int split_tile() { return 128 / (int)sizeof(T); }

// One block [hb, he) of the adjacent line i, summed in order into acc.  The loads of the next
// group are issued before the current one is summed, so each thread keeps a group in flight
// while it computes.
template <int SCALING, typename T>
__device__ __forceinline__ void adjacent_block(const T* __restrict__ X, int64_t ld, int i, int hb,
                                               int he, LineAcc<SCALING>& acc) {
    constexpr int G = kNormGroup;
    const T* p = X + i;
    const int full = hb + (he - hb) / G * G;
    T a[G], b[G];
    auto load = [&](T (&r)[G], int h) {
#pragma unroll
        for (int u = 0; u < G; ++u) r[u] = __ldg(p + (int64_t)(h + u) * ld);
    };
    int h = hb;
    if (h < full) load(a, h);
    for (; h < full; h += 2 * G) {
        const bool more = h + G < full;
        if (more) load(b, h + G);
        acc.add_group(a);
        if (!more) {
            h += G;
            break;
        }
        if (h + 2 * G < full) load(a, h + 2 * G);
        acc.add_group(b);
    }
    if (h < he) {  // the last, shorter group
        const int cnt = he - h;
#pragma unroll
        for (int u = 0; u < G; ++u) a[u] = u < cnt ? __ldg(p + (int64_t)(h + u) * ld) : (T)0;
        acc.add_group(a);
    }
}

// One block [hb, he) of the contiguous lines line0 .. line0 + nl - 1, one line per lane, read in
// coalesced 128-byte rows and transposed through the warp's tile t; the next tile is loaded into
// registers while the current one is summed.
template <int SCALING, typename T>
__device__ __forceinline__ void contiguous_block(const T* __restrict__ X, int64_t ld, int nl,
                                                 int line0, int hb, int he,
                                                 T (*t)[split_tile<T>() + 1],
                                                 LineAcc<SCALING>& acc) {
    constexpr int TL = split_tile<T>();
    static_assert(TL == 16 || TL == 32, "tile of 128 bytes");
    constexpr int RPS = 32 / TL;  // rows copied per step of the warp: lane -> (row, column)
    constexpr int STEPS = 32 / RPS;
    const int lane = threadIdx.x & 31;
    const int rc = lane % TL, rr = lane / TL;
    T reg[STEPS];
    auto load = [&](int h0) {
#pragma unroll
        for (int r = 0; r < STEPS; ++r) {
            const int row = RPS * r + rr, h = h0 + rc;
            reg[r] = (row < nl && h < he) ? __ldg(X + (int64_t)(line0 + row) * ld + h) : (T)0;
        }
    };
    if (hb < he) load(hb);
    for (int h0 = hb; h0 < he; h0 += TL) {
        const int cnt = min(TL, he - h0);
#pragma unroll
        for (int r = 0; r < STEPS; ++r) t[RPS * r + rr][rc] = reg[r];
        __syncwarp();
        if (h0 + TL < he) load(h0 + TL);
        if (lane < nl) {
#pragma unroll
            for (int g = 0; g < TL; g += kNormGroup) {
                if (g < cnt) {
                    T r[kNormGroup];
#pragma unroll
                    for (int u = 0; u < kNormGroup; ++u) r[u] = g + u < cnt ? t[lane][g + u] : (T)0;
                    acc.add_group(r);
                }
            }
        }
        __syncwarp();
    }
}

// Norm-block sums: block (g, c) of the grid takes the 32 lines of group g and warp w sums their
// norm block c * 8 + w.  part: [nblocks][lines] block sums, then (fast mode) [nblocks][lines]
// block maxima, per side.
template <int SCALING, typename T>
__global__ void __launch_bounds__(32 * kSplitWarps) scale_partials_kernel(
    ScaleSide a, ScaleSide b, int groups_a, int chunks, int len, double* part_a,
    double* part_b) {
    static_assert(SCALING != OZAKI2_SCALING_ACCURATE, "accurate mode takes no squared norm");
    __shared__ T tile[kSplitWarps][32][split_tile<T>() + 1];
    const int group = (int)blockIdx.x / chunks, chunk = (int)blockIdx.x % chunks;
    const bool side_b = group >= groups_a;
    const ScaleSide& S = side_b ? b : a;
    double* part = side_b ? part_b : part_a;
    const T* X = static_cast<const T*>(S.X);
    const int line0 = (group - (side_b ? groups_a : 0)) * 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nl = min(32, S.lines - line0);
    const int nblocks = (len + kNormBlock - 1) / kNormBlock;
    const int blk = chunk * kSplitWarps + warp;
    if (blk >= nblocks) return;  // the whole warp: no block barrier follows
    const int hb = blk * kNormBlock, he = min(hb + kNormBlock, len);
    LineAcc<SCALING> acc;
    if (S.es != 1 || S.ls == 1) {
        if (lane < nl) adjacent_block<SCALING, T>(X, S.es, line0 + lane, hb, he, acc);
    } else {
        contiguous_block<SCALING, T>(X, S.ls, nl, line0, hb, he, tile[warp], acc);
    }
    if (lane < nl) {
        part[(int64_t)blk * S.lines + line0 + lane] = acc.block_value();
        if (SCALING == OZAKI2_SCALING_FAST)
            part[(int64_t)(nblocks + blk) * S.lines + line0 + lane] =
                __longlong_as_double((long long)acc.mb);
    }
}

// One thread per line: the block sums added in block order, rounded upward (the blocked sum of
// LineAcc, bit for bit), the maximum of the block maxima, then the shift.
template <int SCALING>
__global__ void __launch_bounds__(256) scale_fold_kernel(ScaleSide a, ScaleSide b, int len,
                                                        const double* __restrict__ part_a,
                                                        const double* __restrict__ part_b,
                                                        float pprime, float delta,
                                                        unsigned* status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool side_b = t >= a.lines;
    const ScaleSide& S = side_b ? b : a;
    const int i = side_b ? t - a.lines : t;
    if (i >= S.lines) return;
    const double* part = side_b ? part_b : part_a;
    const int nblocks = (len + kNormBlock - 1) / kNormBlock;
    LineAcc<SCALING> acc;
    for (int blk = 0; blk < nblocks; ++blk) {
        acc.total = __dadd_ru(acc.total, part[(int64_t)blk * S.lines + i]);
        if (SCALING == OZAKI2_SCALING_FAST) {
            const uint64_t b = (uint64_t)__double_as_longlong(
                part[(int64_t)(nblocks + blk) * S.lines + i]);
            acc.mb = b > acc.mb ? b : acc.mb;
        }
    }
    S.shifts[i] = acc.result(pprime, delta, status);
    if (S.norms) S.norms[i] = acc.total;
}

template <int SCALING, typename T>
__global__ void __launch_bounds__(128) scale_pair_kernel(ScaleSide a, ScaleSide b, int blocks_a,
                                                         int len, float pprime, float delta,
                                                         unsigned* status) {
    __shared__ T tile[kWarpsPerBlock][32][tile_len<T>() + 1];
    const bool side_b = (int)blockIdx.x >= blocks_a;
    const ScaleSide& S = side_b ? b : a;
    const T* X = static_cast<const T*>(S.X);
    const int line0 = ((int)blockIdx.x - (side_b ? blocks_a : 0)) * 128;
    if (S.es != 1 || S.ls == 1) {
        const int i = line0 + (int)threadIdx.x;
        if (i < S.lines)
            scale_adjacent_line<SCALING, T>(X, S.es, i, len, pprime, delta, S.shifts, status,
                                            S.norms);
    } else {
        const int warp = threadIdx.x >> 5;
        const int l0 = line0 + 32 * warp;
        if (l0 < S.lines)
            scale_contiguous_warp<SCALING, T>(X, S.ls, S.lines, len, l0, pprime, delta, S.shifts,
                                              status, tile[warp], S.norms);
    }
}

// Grouped: each block takes 128 lines of one side of one problem (one thread per line for
// adjacent lines, one warp per 32 lines for contiguous lines).
// The scaling mode is a template parameter (every problem of a call shares it), and so is the
// memory layout of the lines when the host has sorted the work list by layout, so each
// instantiation carries one mode's and one layout's registers only.
template <int SCALING, int LAYOUT>
__global__ void __launch_bounds__(128) scale_grouped_kernel(const GroupProblem* __restrict__ probs,
                                                            const ScaleWork* __restrict__ work,
                                                            unsigned* status) {
    __shared__ double tile[kWarpsPerBlock][32][kTileLen + 1];
    const ScaleWork w = work[blockIdx.x];
    const GroupProblem& P = probs[w.problem];
    const double* X = w.side ? P.B : P.A;
    const int64_t ls = w.side ? P.b_ls : P.a_ls, es = w.side ? P.b_es : P.a_es;
    const int lines = w.side ? P.n : P.m;
    int* shifts = w.side ? P.f : P.e;
    if (SCALING == OZAKI2_SCALING_ACCURATE) {
        // clear this block's entries of the C-bar maxima (they live in the product residues)
        uint32_t* cmax = reinterpret_cast<uint32_t*>(P.res);
        const int i = w.line0 + (int)threadIdx.x;
        if (i < lines) cmax[(w.side ? P.m_pad : 0) + i] = 0u;
    }
    scale_grouped_lines<SCALING, LAYOUT>(P, w, X, ls, es, lines, shifts, status, tile);
}

}  // namespace

template <int LAYOUT>
static void launch_scale_grouped_l(const GroupProblem* probs, const ScaleWork* work, int blocks,
                                   unsigned* status, cudaStream_t stream, int scaling) {
    if (scaling == OZAKI2_SCALING_FAST)
        scale_grouped_kernel<OZAKI2_SCALING_FAST, LAYOUT><<<blocks, 128, 0, stream>>>(probs, work,
                                                                                     status);
    else if (scaling == OZAKI2_SCALING_ACCURATE)
        scale_grouped_kernel<OZAKI2_SCALING_ACCURATE, LAYOUT><<<blocks, 128, 0, stream>>>(
            probs, work, status);
    else
        scale_grouped_kernel<OZAKI2_SCALING_PROPOSED, LAYOUT><<<blocks, 128, 0, stream>>>(
            probs, work, status);
}

cudaError_t launch_scale_grouped(const GroupProblem* probs, const ScaleWork* work, int blocks,
                                 unsigned* status, cudaStream_t stream, int scaling,
                                 int adjacent_blocks) {
    if (blocks <= 0) return cudaSuccess;
    if (adjacent_blocks < 0) {
        launch_scale_grouped_l<kLayoutAny>(probs, work, blocks, status, stream, scaling);
    } else {
        if (adjacent_blocks > 0)
            launch_scale_grouped_l<kLayoutAdjacent>(probs, work, adjacent_blocks, status, stream,
                                                    scaling);
        if (blocks > adjacent_blocks)
            launch_scale_grouped_l<kLayoutContiguous>(probs, work + adjacent_blocks,
                                                      blocks - adjacent_blocks, status, stream,
                                                      scaling);
    }
    return cudaGetLastError();
}

// Lines longer than one norm block, with scratch for the block sums: the partial sums of every
// (32 lines, block), then the ordered fold per line.  Side b may have no lines.
template <int SCALING, typename T>
static void launch_split(const ScaleSide& sa, const ScaleSide& sb, int len, float pprime,
                         float delta, double* partials, unsigned* status, cudaStream_t stream) {
    const int nblocks = (len + kNormBlock - 1) / kNormBlock;
    const int chunks = (nblocks + kSplitWarps - 1) / kSplitWarps;
    const int ga = (sa.lines + 31) / 32, gb = (sb.lines + 31) / 32;
    double* pa = partials;
    double* pb = partials + 2 * (int64_t)nblocks * sa.lines;
    scale_partials_kernel<SCALING, T><<<(ga + gb) * chunks, 32 * kSplitWarps, 0, stream>>>(
        sa, sb, ga, chunks, len, pa, pb);
    const int lines = sa.lines + sb.lines;
    scale_fold_kernel<SCALING><<<(lines + 255) / 256, 256, 0, stream>>>(sa, sb, len, pa, pb,
                                                                       pprime, delta, status);
}

template <int SCALING>
static void launch_scale_t(const double* X, int64_t line_stride, int64_t elem_stride, int lines,
                           int len, float pprime, float delta, int* shifts, unsigned* status,
                           cudaStream_t stream, double* partials) {
    if constexpr (SCALING != OZAKI2_SCALING_ACCURATE) {
        if (partials && len > kNormBlock) {  // long lines: split across warps
            const ScaleSide side{X, line_stride, elem_stride, lines, shifts};
            const ScaleSide none{X, line_stride, elem_stride, 0, shifts};
            launch_split<SCALING, double>(side, none, len, pprime, delta, partials, status,
                                          stream);
            return;
        }
    }
    if (elem_stride != 1 || line_stride == 1) {  // lines adjacent
        scale_adjacent_kernel<SCALING><<<(lines + 31) / 32, 32, 0, stream>>>(
            X, elem_stride, lines, len, pprime, delta, shifts, status);
    } else {
        const int per_block = 32 * kWarpsPerBlock;
        scale_contiguous_kernel<SCALING><<<(lines + per_block - 1) / per_block, per_block, 0,
                                           stream>>>(X, line_stride, lines, len, pprime, delta,
                                                     shifts, status);
    }
}

cudaError_t launch_scale(const double* X, int64_t line_stride, int64_t elem_stride, int lines,
                         int len, float pprime, int* shifts, unsigned* status,
                         cudaStream_t stream, int scaling, float delta, double* partials) {
    if (lines <= 0) return cudaSuccess;
    if (scaling == OZAKI2_SCALING_FAST)
        launch_scale_t<OZAKI2_SCALING_FAST>(X, line_stride, elem_stride, lines, len, pprime,
                                            delta, shifts, status, stream, partials);
    else if (scaling == OZAKI2_SCALING_ACCURATE)
        launch_scale_t<OZAKI2_SCALING_ACCURATE>(X, line_stride, elem_stride, lines, len, pprime,
                                                delta, shifts, status, stream, partials);
    else
        launch_scale_t<OZAKI2_SCALING_PROPOSED>(X, line_stride, elem_stride, lines, len, pprime,
                                                delta, shifts, status, stream, partials);
    return cudaGetLastError();
}

template <typename T>
static void launch_scale_pair_t(const ScaleSide& sa, const ScaleSide& sb, int blocks_a, int grid,
                                int len, float pprime, float delta, unsigned* status,
                                cudaStream_t stream, int scaling, double* partials) {
    if (partials && scaling != OZAKI2_SCALING_ACCURATE && len > kNormBlock) {  // long lines
        if (scaling == OZAKI2_SCALING_FAST)
            launch_split<OZAKI2_SCALING_FAST, T>(sa, sb, len, pprime, delta, partials, status,
                                                 stream);
        else
            launch_split<OZAKI2_SCALING_PROPOSED, T>(sa, sb, len, pprime, delta, partials,
                                                     status, stream);
        return;
    }
    if (scaling == OZAKI2_SCALING_FAST)
        scale_pair_kernel<OZAKI2_SCALING_FAST, T><<<grid, 128, 0, stream>>>(
            sa, sb, blocks_a, len, pprime, delta, status);
    else if (scaling == OZAKI2_SCALING_ACCURATE)
        scale_pair_kernel<OZAKI2_SCALING_ACCURATE, T><<<grid, 128, 0, stream>>>(
            sa, sb, blocks_a, len, pprime, delta, status);
    else
        scale_pair_kernel<OZAKI2_SCALING_PROPOSED, T><<<grid, 128, 0, stream>>>(
            sa, sb, blocks_a, len, pprime, delta, status);
}

cudaError_t launch_scale_pair(const void* A, int64_t a_ls, int64_t a_es, int m, const void* B,
                              int64_t b_ls, int64_t b_es, int n, int len, float pprime,
                              float delta, int* e, int* f, unsigned* status, cudaStream_t stream,
                              int scaling, bool f32, double* partials, double* norms_a,
                              double* norms_b) {
    const int blocks_a = (m + 127) / 128, blocks_b = (n + 127) / 128;
    if (blocks_a + blocks_b == 0) return cudaSuccess;
    const ScaleSide sa{A, a_ls, a_es, m, e, norms_a}, sb{B, b_ls, b_es, n, f, norms_b};
    const int grid = blocks_a + blocks_b;
    if (f32)
        launch_scale_pair_t<float>(sa, sb, blocks_a, grid, len, pprime, delta, status, stream,
                                   scaling, partials);
    else
        launch_scale_pair_t<double>(sa, sb, blocks_a, grid, len, pprime, delta, status, stream,
                                    scaling, partials);
    return cudaGetLastError();
}

// ---- accurate mode, last pass: the shifts from E and the maxima of C-bar
namespace {

// log2 mu_i = 5 - E_i + floor(P'_accu - delta log2~(max_j c-bar_ij)) (eq. (mu_accu) with the
// reading mu_i = mu'_i 2^floor(...)), log2~ of eq. (flog2) with the logarithm stand-in of
// alg2_shift; the floor is of the exact value (delta * log2~ is exact in double, and so is the
// difference).  A line whose c-bar maximum is 0 meets no nonzero product: OZAKI2_SHIFT_VANISH.
__device__ __forceinline__ int accu_shift(int code, uint32_t cmax, float pprime, float delta) {
    if (code == OZAKI2_SHIFT_NONFINITE) return code;
    if (code == kAccuZeroLine) return 0;
    if (cmax == 0) return OZAKI2_SHIFT_VANISH;
    const int s = 31 - __clz(cmax);
    const double xprime = scalbn((double)cmax, -s);           // [1, 2), exact
    const float lg0 = __double2float_ru(log2((double)__double2float_ru(xprime)));
    const float lg = __double2float_ru((double)lg0 + (double)s);
    const double u = (double)delta * (double)lg;
    return 5 - code + (int)floor(__dsub_rd((double)pprime, u));
}

__global__ void accu_shift_kernel(int* e, int m, int* f, int n, const uint32_t* __restrict__ cmax,
                                  int m_pad, float pprime, float delta) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) e[t] = accu_shift(e[t], cmax[t], pprime, delta);
    else if (t < m + n) f[t - m] = accu_shift(f[t - m], cmax[m_pad + (t - m)], pprime, delta);
}

__global__ void accu_shift_grouped_kernel(const GroupProblem* __restrict__ probs,
                                          const ScaleWork* __restrict__ work) {
    const ScaleWork w = work[blockIdx.x];
    const GroupProblem& P = probs[w.problem];
    if (P.scaling != OZAKI2_SCALING_ACCURATE) return;
    const int i = w.line0 + (int)threadIdx.x;
    const uint32_t* cmax = reinterpret_cast<const uint32_t*>(P.res);
    if (w.side == 0) {
        if (i < P.m) P.e[i] = accu_shift(P.e[i], cmax[i], P.pprime, P.delta);
    } else {
        if (i < P.n) P.f[i] = accu_shift(P.f[i], cmax[P.m_pad + i], P.pprime, P.delta);
    }
}

// Copy of `count` words of W bytes from host memory the device can address into device memory.
// Each thread keeps four loads in flight: the link to host memory has a long latency.
template <typename Word>
__global__ void __launch_bounds__(256) stage_in_kernel(Word* __restrict__ dst,
                                                       const Word* __restrict__ src,
                                                       int64_t count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < count; i += 4 * stride) {
        Word w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[i + u * stride] = w[u];
    }
    for (; i < count; i += stride) dst[i] = src[i];
}

// 2-D copies: copy c moves c.height rows of c.width bytes (c.width / W words), row r from
// c.src + r c.spitch to c.dst + r c.dpitch.  Blocks [0, blocks0) take copy 0, the others copy 1;
// a block copies rows b, b + (its copy's blocks), ..., each thread keeping four words in flight,
// so one block per SM already covers the host link's latency.  Launched to overlap the grid
// before it (programmatic serialization), the kernel waits for that grid at its end, so that
// work launched after the copy also runs after that grid.
template <typename Word>
__global__ void __launch_bounds__(256) copy_2d_kernel(const Copy2D c0, const Copy2D c1,
                                                      int blocks0) {
    const bool second = (int)blockIdx.x >= blocks0;
    const Copy2D& c = second ? c1 : c0;
    const int64_t b = second ? blockIdx.x - blocks0 : blockIdx.x;
    const int64_t nb = second ? gridDim.x - blocks0 : blocks0;
    const int64_t words = (int64_t)(c.width / sizeof(Word));
    for (int64_t r = b; r < (int64_t)c.height; r += nb) {
        const Word* s = reinterpret_cast<const Word*>(static_cast<const char*>(c.src) +
                                                      r * (int64_t)c.spitch);
        Word* d = reinterpret_cast<Word*>(static_cast<char*>(c.dst) + r * (int64_t)c.dpitch);
        int64_t i = threadIdx.x;
        for (; i + 3 * 256 < words; i += 4 * 256) {
            Word w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = s[i + u * 256];
#pragma unroll
            for (int u = 0; u < 4; ++u) d[i + u * 256] = w[u];
        }
        for (; i < words; i += 256) d[i] = s[i];
    }
    pdl_wait_prerequisites();
}

template <typename Word>
cudaError_t launch_copy_2d_w(const Copy2D& c0, const Copy2D& c1, int blocks0, int blocks1,
                             bool overlap_previous, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)(blocks0 + blocks1));
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = overlap_previous ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, copy_2d_kernel<Word>, c0, c1, blocks0);
}

}  // namespace

cudaError_t launch_copies_2d(const Copy2D* copies, int count, int blocks, bool overlap_previous,
                             cudaStream_t stream) {
    Copy2D c[2] = {};
    int nb[2] = {0, 0}, used = 0;
    uintptr_t a = 0;
    for (int i = 0; i < count && i < 2; ++i) {
        const Copy2D& x = copies[i];
        if (x.width == 0 || x.height == 0) continue;
        if (x.dpitch < x.width || x.spitch < x.width) return cudaErrorInvalidValue;
        a |= reinterpret_cast<uintptr_t>(x.dst) | reinterpret_cast<uintptr_t>(x.src) |
             (uintptr_t)x.dpitch | (uintptr_t)x.spitch | (uintptr_t)x.width;
        c[used] = x;
        nb[used] = (int)std::min<int64_t>(blocks > 0 ? blocks : 1, (int64_t)x.height);
        ++used;
    }
    if (count > 2) return cudaErrorInvalidValue;
    if (used == 0) return cudaSuccess;
    if ((a & 15) == 0)
        return launch_copy_2d_w<uint4>(c[0], c[1], nb[0], nb[1], overlap_previous, stream);
    if ((a & 7) == 0)
        return launch_copy_2d_w<uint2>(c[0], c[1], nb[0], nb[1], overlap_previous, stream);
    if ((a & 3) == 0)
        return launch_copy_2d_w<unsigned>(c[0], c[1], nb[0], nb[1], overlap_previous, stream);
    return launch_copy_2d_w<unsigned char>(c[0], c[1], nb[0], nb[1], overlap_previous, stream);
}

cudaError_t launch_stage_in(void* dst, const void* src, size_t bytes, int num_sms,
                            cudaStream_t stream, int blocks_per_sm) {
    if (bytes == 0) return cudaSuccess;
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) |
                        (uintptr_t)bytes;
    const int grid = (blocks_per_sm > 0 ? blocks_per_sm : 1) * (num_sms > 0 ? num_sms : 1);
    if ((a & 15) == 0)
        stage_in_kernel<<<grid, 256, 0, stream>>>(static_cast<uint4*>(dst),
                                                  static_cast<const uint4*>(src),
                                                  (int64_t)(bytes / 16));
    else if ((a & 7) == 0)
        stage_in_kernel<<<grid, 256, 0, stream>>>(static_cast<uint2*>(dst),
                                                  static_cast<const uint2*>(src),
                                                  (int64_t)(bytes / 8));
    else if ((a & 3) == 0)
        stage_in_kernel<<<grid, 256, 0, stream>>>(static_cast<unsigned*>(dst),
                                                  static_cast<const unsigned*>(src),
                                                  (int64_t)(bytes / 4));
    else
        stage_in_kernel<<<grid, 256, 0, stream>>>(static_cast<unsigned char*>(dst),
                                                  static_cast<const unsigned char*>(src),
                                                  (int64_t)bytes);
    return cudaGetLastError();
}

cudaError_t launch_accu_shift(int* e, int m, int* f, int n, const uint32_t* cmax, int m_pad,
                              float pprime, float delta, cudaStream_t stream) {
    if (m + n <= 0) return cudaSuccess;
    accu_shift_kernel<<<(m + n + 255) / 256, 256, 0, stream>>>(e, m, f, n, cmax, m_pad, pprime,
                                                              delta);
    return cudaGetLastError();
}

cudaError_t launch_accu_shift_grouped(const GroupProblem* probs, const ScaleWork* work,
                                      int blocks, cudaStream_t stream) {
    if (blocks <= 0) return cudaSuccess;
    accu_shift_grouped_kernel<<<blocks, 128, 0, stream>>>(probs, work);
    return cudaGetLastError();
}

}  // namespace ozaki2
