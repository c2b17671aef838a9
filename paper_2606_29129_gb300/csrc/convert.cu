// convert.cu -- Step 2 conversion of Ozaki scheme II: a'_ih = trunc(2^{e_i} a_ih), and the
// residues rmod(a', p_l) of eq. (os2-C') for every modulus, written as bf16 residue planes with
// K contiguous (the operand layout of the residue GEMM).
//
// Integer-only arithmetic.  The double's 53-bit mantissa M and its exponent give
// |a'| = floor(M 2^sh), held as L 21-bit limbs d_j (L = 1 for N <= 3, 2 up to N = 9, 3 up to
// N = 14, 4 up to N = 20).  For an odd modulus, t = sum_j d_j (2^(21 j) mod p) < 2^31 and one
// exact quotient gives the symmetric residue of |a'|, negated for negative a'.  For p = 256 the
// residue is the low byte of +-|a'| read as a signed byte ([-128, 127]).  Each small integer is
// exact in bf16.  Kernels are instantiated per N so every per-modulus constant is an immediate
// operand.
//
// Traffic per element: 8 bytes read, 2N bytes written.
#include <cuda_bf16.h>

#include "ozaki2_internal.h"

namespace ozaki2 {
namespace {

constexpr uint32_t kMask21 = (1u << 21) - 1;

// bits(P) for N moduli, N = 2..20 (P = product of the first N moduli of eq. (moduli)).
__host__ __device__ constexpr int p_bits(int N) {
    constexpr int b[21] = {0, 8, 16, 24, 32, 40, 48, 56, 64, 72, 80,
                           88, 95, 103, 111, 118, 126, 133, 141, 148, 156};
    return b[N];
}
// 21-bit limbs covering |a'|.  The proposed and fast scalings keep |a'| <= sqrt((P-1)/2) <
// 2^(bits(P)/2); accurate mode allows up to 2^6 times more (|a| < 2^(E+1), mu' = 2^(5-E), and
// the second factor is at most 2^P'), so floor(bits(P)/2) + 6 bits are provided.
__host__ __device__ constexpr int limbs_for(int N) { return (p_bits(N) / 2 + 6 + 20) / 21; }
// The proposed and fast scalings keep |a'| < 2^(log2(P-1)/2 - 0.5), i.e. at most
// floor(bits(P)/2 - 0.5) + 1 bits: one limb fewer for N = 4, 5, 10, 15 and 16.
__host__ __device__ constexpr int limbs_scaled(int N) {
    return ((p_bits(N) * 2 - 1) / 4 + 1 + 20) / 21;
}

// The float 1.5 * 2^23 (bits 0x4B400000): for |s| < 2^22 the bits B + s are the float B + s.
constexpr uint32_t kFloatB = 0x4B400000u;

// |a'| as limbs.  d[0] carries kFloatB in its unused upper bits (d[0] = limb 0 | kFloatB, the
// two never overlap), so a residue sum started from d[0] is offset by kFloatB at no cost.
struct Scaled {
    uint32_t d[4];
    uint32_t low;  // low 32 bits of |a'|
    float sgn;     // +1 or -1: the sign of a'
    bool neg;
};

// |trunc(M 2^sh)| (M of mbits bits) as 21-bit limbs.  Flags OZAKI2_STATUS_RANGE when the value
// needs more than 21*L bits (only possible with shifts that break the bound of
// eq. (proposed-condition)).
template <int L>
__device__ __forceinline__ Scaled split_mantissa(uint64_t M, int mbits, int sh, bool neg,
                                                 unsigned* status) {
    Scaled r;
    r.neg = neg;
    uint64_t lo = 0, hi = 0;
    if (M != 0 && sh > 21 * L - mbits) {
        // bits of |a'| = (64 - clz(M)) + sh must fit in 21 L
        if (sh > 21 * L - (64 - __clzll((long long)M))) atomicOr(status, OZAKI2_STATUS_RANGE);
        sh = min(sh, min(21 * L - mbits + 11, 63));
    }
    if (sh >= 0) {
        lo = M << sh;
        hi = sh ? (M >> (64 - sh)) : 0;
    } else if (sh > -64) {
        lo = M >> (-sh);
    }
    r.low = (uint32_t)lo;
    r.sgn = neg ? -1.0f : 1.0f;
    r.d[0] = ((uint32_t)lo & kMask21) | kFloatB;
    r.d[1] = (uint32_t)(lo >> 21) & kMask21;
    r.d[2] = (uint32_t)(lo >> 42) & kMask21;
    r.d[3] = (uint32_t)((lo >> 63) | (hi << 1)) & kMask21;
    return r;
}

// |trunc(a 2^e)| of a double (53-bit mantissa) or a float (24-bit mantissa), from the bits.
template <int L>
__device__ __forceinline__ Scaled split_scaled(double a, int e, unsigned* status) {
    const uint64_t bits = (uint64_t)__double_as_longlong(a);
    int E = (int)((bits >> 52) & 0x7FF);
    uint64_t M = bits & ((1ull << 52) - 1);
    if (E) M |= 1ull << 52; else E = 1;
    return split_mantissa<L>(M, 53, E - 1075 + e, (bits >> 63) != 0, status);
}
template <int L>
__device__ __forceinline__ Scaled split_scaled(float a, int e, unsigned* status) {
    const uint32_t bits = __float_as_uint(a);
    int E = (int)((bits >> 23) & 0xFF);
    uint64_t M = bits & 0x7FFFFFu;
    if (E) M |= 1ull << 23; else E = 1;
    return split_mantissa<L>(M, 24, E - 150 + e, (bits >> 31) != 0, status);
}

// bf16 bits (in the upper half of a float) of the small integer s.
__device__ __forceinline__ uint32_t small_int_bits(int s) {
    return __float_as_uint(__int_as_float((int)kFloatB + s) - 12582912.0f);
}

// Symmetric residue of +-|a'| modulo the l-th modulus, as bf16 bits.
template <int L>
__device__ __forceinline__ uint32_t residue_bits(const Scaled& v, const ConvertTables& t, int l) {
    if (l == 0) {  // p = 256: the low byte of a' in two's complement
        const uint32_t b = (v.neg ? 0u - v.low : v.low) & 0xFFu;
        return small_int_bits((int)(int8_t)(uint8_t)b);
    }
    // Odd p, h = (p - 1)/2: t == |a'| (mod p) with t <= (2^21 - 1)(1 + 3(p - 1)) < 2^31, summed
    // from d[0] so y = kFloatB + t.  With q = floor((t + h)/p), s = t - q p lies in [-h, h] and is
    // the symmetric residue of |a'|; y - q p = kFloatB + s is the float 1.5 2^23 + s, and one
    // exact FMA gives sgn s.  x = t + h < 2^31 is y - (kFloatB - h) (table `bias`), and its
    // quotient by p is exact with the 2^39 magic m (x (ceil(2^39/p) p - 2^39) < 2^39 for every
    // such x and modulus); x m comes from y m plus the table's -(bias m) modulo 2^64.
    const uint32_t p = t.p[l];
    uint32_t y = v.d[0];
#pragma unroll
    for (int j = 1; j < L; ++j) y += v.d[j] * t.pow21[l][j];
    // x m = y m - bias m exactly (x < 2^31, so x m < 2^63): one 64-bit multiply-add
    const uint64_t xm = (uint64_t)y * t.magic39[l] + t.neg_bias_magic[l];
    const uint32_t fb = y - (uint32_t)(xm >> 39) * p;
    return __float_as_uint(fmaf(v.sgn, __uint_as_float(fb), v.sgn * -12582912.0f));
}

// Accurate mode (Section 2.3): a-bar = ceil(2^(5 - E) |a|) <= 64 with E = floor(log2 max |a|) of
// the line, in integer arithmetic: |a| = M 2^(Ex - 1075) with the mantissa M (hidden bit
// included for normal numbers), so 2^(5 - E) |a| = M 2^-rs with rs = 1070 + E - Ex, and the
// ceiling is (M + 2^rs - 1) >> rs.  rs >= 47 for a normal a (a <= 2^(E+1)); a subnormal a in a
// line of subnormals can give rs down to -5, a left shift of a small M.  For rs >= 64 the value
// lies in (0, 1) and its ceiling is 1.
__device__ __forceinline__ uint32_t bar_bits(double a, int E) {
    const uint64_t bits = (uint64_t)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
    if (bits == 0) return small_int_bits(0);
    int Ex = (int)(bits >> 52);
    uint64_t M = bits & ((1ull << 52) - 1);
    if (Ex) M |= 1ull << 52; else Ex = 1;
    const int rs = 1070 + E - Ex;
    uint32_t c;
    if (rs >= 64) c = 1u;
    else if (rs > 0) c = (uint32_t)((M + ((1ull << rs) - 1)) >> rs);
    else c = (uint32_t)(M << -rs);
    return small_int_bits((int)c);
}

__device__ __forceinline__ uint32_t bar_bits(float a, int E) {
    // as above with |a| = M 2^(Ex - 150): rs = 145 + E - Ex (>= 18 for a normal a)
    const uint32_t bits = __float_as_uint(a) & 0x7FFFFFFFu;
    if (bits == 0) return small_int_bits(0);
    int Ex = (int)(bits >> 23);
    uint64_t M = bits & 0x7FFFFFu;
    if (Ex) M |= 1ull << 23; else Ex = 1;
    const int rs = 145 + E - Ex;
    uint32_t c;
    if (rs >= 64) c = 1u;
    else if (rs > 0) c = (uint32_t)((M + ((1ull << rs) - 1)) >> rs);
    else c = (uint32_t)(M << -rs);
    return small_int_bits((int)c);
}

// Writes the residues of 8 consecutive elements of one line into the N planes.  N = 1 is the
// a-bar plane of accurate mode instead, with e the line's exponent code.
template <int N, int L, typename V>
__device__ __forceinline__ void store_residues8(const V (&v)[8], int e, bool live,
                                                const ConvertTables& t, __nv_bfloat16* planes,
                                                int64_t plane_elems, int64_t offset,
                                                unsigned* status) {
    if constexpr (N == 1) {
        const bool zero = !live || e == OZAKI2_SHIFT_NONFINITE || e == kAccuZeroLine;
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t a = zero ? 0u : bar_bits(v[2 * u], e);
            const uint32_t b = zero ? 0u : bar_bits(v[2 * u + 1], e);
            w[u] = __byte_perm(a, b, 0x7632);
        }
        *reinterpret_cast<uint4*>(planes + offset) = make_uint4(w[0], w[1], w[2], w[3]);
        return;
    }
    Scaled sc[8];
    const bool zero = (e == OZAKI2_SHIFT_NONFINITE) || !live;
#pragma unroll
    for (int u = 0; u < 8; ++u)
        sc[u] = zero ? Scaled{{kFloatB, 0, 0, 0}, 0, 1.0f, false}
                     : split_scaled<L>(v[u], e, status);
#pragma unroll
    for (int l = 0; l < N; ++l) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t a = residue_bits<L>(sc[2 * u], t, l);
            const uint32_t b = residue_bits<L>(sc[2 * u + 1], t, l);
            w[u] = __byte_perm(a, b, 0x7632);  // upper halves: a -> bits 0..15, b -> 16..31
        }
        *reinterpret_cast<uint4*>(planes + (int64_t)l * plane_elems + offset) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Lines contiguous (elem_stride == 1): thread = (line, group of 8 elements); a warp covers 256
// consecutive elements of one line, so loads and stores are both contiguous.
// Eight consecutive elements of one line as doubles (a float widens exactly); 16-byte vector
// loads when the line start allows them.
__device__ __forceinline__ void load8(const double* src, bool vec, double (&v)[8]) {
    if (vec) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 d = __ldg(reinterpret_cast<const double2*>(src) + u);
            v[2 * u] = d.x;
            v[2 * u + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(src + u);
    }
}
__device__ __forceinline__ void load8(const float* src, bool vec, float (&v)[8]) {
    if (vec) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float4 d = __ldg(reinterpret_cast<const float4*>(src) + u);
            v[4 * u] = d.x;
            v[4 * u + 1] = d.y;
            v[4 * u + 2] = d.z;
            v[4 * u + 3] = d.w;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(src + u);
    }
}

// T = double (DGEMM) or float (SGEMM).
template <int N, int L, typename T>
__device__ __forceinline__ void convert_contiguous_item(
    const T* __restrict__ X, int64_t ld, int lines, int len, const int* __restrict__ shifts,
    const ConvertTables& t, __nv_bfloat16* __restrict__ planes, int64_t plane_elems, int k_pad,
    int64_t g, unsigned* status) {
    const int groups = k_pad / 8;
    constexpr int per16 = 16 / (int)sizeof(T);  // elements per 16 bytes
    const bool vec = (ld % per16 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
    {
        const int i = (int)(g / groups);
        const int h0 = (int)(g - (int64_t)i * groups) * 8;
        const bool row_live = i < lines;
        T v[8];
        const T* src = X + (int64_t)i * ld + h0;
        if (row_live && h0 + 8 <= len) {
            load8(src, vec, v);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (row_live && h0 + u < len) ? __ldg(src + u) : (T)0;
        }
        const int e = row_live ? shifts[i] : 0;
        store_residues8<N, L>(v, e, row_live, t, planes, plane_elems, (int64_t)i * k_pad + h0,
                           status);
    }
}

// One item per thread (a grid-stride loop here made the compiler keep two items' limbs live and
// halved the occupancy).
template <int N, int L, typename T>
__global__ void __launch_bounds__(256) convert_contiguous_kernel(
    const T* __restrict__ X, int64_t ld, int lines, int len, const int* __restrict__ shifts,
    const ConvertTables t, __nv_bfloat16* __restrict__ planes, int rows_pad, int k_pad,
    int64_t plane_elems, unsigned* status) {
    const int64_t total = (int64_t)rows_pad * (k_pad / 8);
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < total)
        convert_contiguous_item<N, L, T>(X, ld, lines, len, shifts, t, planes, plane_elems,
                                         k_pad, g, status);
}

// Lines adjacent (line_stride == 1): a block converts a tile of 64 lines x 64 elements.  The tile
// is read with coalesced loads along the lines (a warp reads 32 consecutive doubles), transposed
// through shared memory, and each group of 8 lanes writes one line's 64 elements (128 bytes per
// plane) as 8 contiguous 16-byte stores.
constexpr int kTileLines = 64;
constexpr int kTileK = 64;

// Tile tt (64 lines x 64 elements) of an adjacent-line matrix; all 256 threads take part.
template <int N, int L, typename T>
__device__ __forceinline__ void convert_adjacent_tile(
    const T* __restrict__ X, int64_t ld, int lines, int len, const int* __restrict__ shifts,
    const ConvertTables& t, __nv_bfloat16* __restrict__ planes, int rows_pad, int k_pad,
    int64_t plane_elems, int64_t tt, T (*tile)[kTileLines + 1], unsigned* status) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_l = (rows_pad + kTileLines - 1) / kTileLines;
    {
        const int tl = (int)(tt % tiles_l);
        const int tk = (int)(tt / tiles_l);
        const int line0 = tl * kTileLines, h0 = tk * kTileK;
        // load: warp w reads rows h = w, w+8, ... of the tile, two 32-line halves each
#pragma unroll
        for (int r = 0; r < kTileK / 8; ++r) {
            const int hh = warp + 8 * r;
            const int h = h0 + hh;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int line = line0 + 32 * half + lane;
                tile[hh][32 * half + lane] =
                    (line < lines && h < len) ? __ldg(X + line + (int64_t)h * ld) : (T)0;
            }
        }
        __syncthreads();
        // convert: 256 threads x 2 = 64 lines x 8 groups of 8 elements
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int item = threadIdx.x + 256 * rep;
            const int ll = item >> 3, hg = item & 7;
            const int line = line0 + ll;
            if (line < rows_pad && h0 + 8 * hg < k_pad) {
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = tile[8 * hg + u][ll];
                const bool live = line < lines;
                const int e = live ? shifts[line] : 0;
                store_residues8<N, L>(v, e, live, t, planes, plane_elems,
                                   (int64_t)line * k_pad + h0 + 8 * hg, status);
            }
        }
        __syncthreads();
    }
}

template <int N, int L, typename T>
__global__ void __launch_bounds__(256) convert_adjacent_kernel(
    const T* __restrict__ X, int64_t ld, int lines, int len, const int* __restrict__ shifts,
    const ConvertTables t, __nv_bfloat16* __restrict__ planes, int rows_pad, int k_pad,
    int64_t plane_elems, unsigned* status) {
    __shared__ T tile[kTileK][kTileLines + 1];
    convert_adjacent_tile<N, L, T>(X, ld, lines, len, shifts, t, planes, rows_pad, k_pad,
                                   plane_elems, blockIdx.x, tile, status);  // one tile per block
}

// Grouped: each block converts one tile (adjacent lines) or 256 groups of 8 elements
// (contiguous lines) of one side of one problem.
template <int N, int L>
__global__ void __launch_bounds__(256) convert_grouped_kernel(
    const GroupProblem* __restrict__ probs, const ConvertWork* __restrict__ work,
    const ConvertTables t, unsigned* status) {
    __shared__ double tile[kTileK][kTileLines + 1];
    const ConvertWork w = work[blockIdx.x];
    const GroupProblem& P = probs[w.problem];
    const double* X = w.side ? P.B : P.A;
    const int64_t ls = w.side ? P.b_ls : P.a_ls, es = w.side ? P.b_es : P.a_es;
    const int lines = w.side ? P.n : P.m;
    const int rows = w.side ? P.geo.rows_b : P.geo.rows_a;
    const int* shifts = w.side ? P.f : P.e;
    auto* planes = static_cast<__nv_bfloat16*>(w.side ? P.pb : P.pa);
    if (es != 1) {
        convert_adjacent_tile<N, L, double>(X, es, lines, P.k, shifts, t, planes, rows,
                                            P.geo.ld, (int64_t)rows * P.geo.ld, w.block, tile,
                                            status);
    } else {
        const int64_t g = (int64_t)w.block * 256 + threadIdx.x;
        if (g < (int64_t)rows * (P.geo.ld / 8))
            convert_contiguous_item<N, L, double>(X, ls, lines, P.k, shifts, t, planes,
                                                  (int64_t)rows * P.geo.ld, P.geo.ld, g, status);
    }
}

template <int N, int L, typename T>
cudaError_t launch_convert_nl(const T* X, int64_t line_stride, int64_t elem_stride,
                              int lines, int len, const int* shifts, const ConvertTables& t,
                              __nv_bfloat16* out, int rows_pad, int k_pad, int64_t plane_elems,
                              unsigned* status, cudaStream_t stream) {
    if (elem_stride != 1) {  // then line_stride == 1: lines adjacent
        const int grid = (int)((int64_t)((rows_pad + kTileLines - 1) / kTileLines) *
                               ((k_pad + kTileK - 1) / kTileK));
        convert_adjacent_kernel<N, L, T><<<grid, 256, 0, stream>>>(X, elem_stride, lines, len,
                                                                shifts, t, out, rows_pad, k_pad,
                                                                plane_elems, status);
    } else {
        const int64_t total = (int64_t)rows_pad * (k_pad / 8);
        const int grid = (int)((total + 255) / 256);
        convert_contiguous_kernel<N, L, T><<<grid, 256, 0, stream>>>(X, line_stride, lines, len,
                                                                  shifts, t, out, rows_pad,
                                                                  k_pad, plane_elems, status);
    }
    return cudaGetLastError();
}

// Accurate mode's a' can take six more bits than the proposed and fast scalings allow.
template <int N, typename T>
cudaError_t launch_convert_n(const T* X, int64_t line_stride, int64_t elem_stride,
                             int lines, int len, const int* shifts, const ConvertTables& t,
                             __nv_bfloat16* out, int rows_pad, int k_pad, int64_t plane_elems,
                             unsigned* status, cudaStream_t stream, bool accurate = false) {
    if constexpr (limbs_scaled(N) != limbs_for(N)) {
        if (!accurate)
            return launch_convert_nl<N, limbs_scaled(N), T>(X, line_stride, elem_stride, lines,
                                                            len, shifts, t, out, rows_pad, k_pad,
                                                            plane_elems, status, stream);
    }
    return launch_convert_nl<N, limbs_for(N), T>(X, line_stride, elem_stride, lines, len, shifts,
                                                 t, out, rows_pad, k_pad, plane_elems, status,
                                                 stream);
}

}  // namespace

int convert_blocks(int lines, int64_t elem_stride, int rows, int ld) {
    (void)lines;
    if (elem_stride != 1)
        return ((rows + kTileLines - 1) / kTileLines) * ((ld + kTileK - 1) / kTileK);
    return (int)(((int64_t)rows * (ld / 8) + 255) / 256);
}

cudaError_t launch_convert_bar(const void* X, int64_t line_stride, int64_t elem_stride,
                               int lines, int len, const int* codes, void* plane, int rows_pad,
                               int k_pad, unsigned* status, cudaStream_t stream, bool f32) {
    if (rows_pad <= 0 || k_pad <= 0) return cudaSuccess;
    ConvertTables t = {};
    t.N = 1;
    auto* out = static_cast<__nv_bfloat16*>(plane);
    if (f32)
        return launch_convert_n<1>(static_cast<const float*>(X), line_stride, elem_stride, lines,
                                   len, codes, t, out, rows_pad, k_pad,
                                   (int64_t)rows_pad * k_pad, status, stream);
    return launch_convert_n<1>(static_cast<const double*>(X), line_stride, elem_stride, lines,
                               len, codes, t, out, rows_pad, k_pad, (int64_t)rows_pad * k_pad,
                               status, stream);
}

namespace {
template <int N>
void launch_convert_grouped_n(const GroupProblem* probs, const ConvertWork* work, int blocks,
                              const ConvertTables& t, unsigned* status, cudaStream_t stream,
                              bool accurate) {
    if constexpr (limbs_scaled(N) != limbs_for(N)) {
        if (!accurate) {
            convert_grouped_kernel<N, limbs_scaled(N)><<<blocks, 256, 0, stream>>>(probs, work, t,
                                                                                   status);
            return;
        }
    }
    convert_grouped_kernel<N, limbs_for(N)><<<blocks, 256, 0, stream>>>(probs, work, t, status);
}
}  // namespace

cudaError_t launch_convert_grouped(int N, const GroupProblem* probs, const ConvertWork* work,
                                   int blocks, const ConvertTables& t, unsigned* status,
                                   cudaStream_t stream, bool accurate) {
    if (blocks <= 0) return cudaSuccess;
    switch (N) {
#define OZAKI2_CONVERT_GROUPED_CASE(NN)                                                      \
    case NN:                                                                                 \
        launch_convert_grouped_n<NN>(probs, work, blocks, t, status, stream, accurate);      \
        break;
        OZAKI2_CONVERT_GROUPED_CASE(1)  // the A-bar / B-bar planes of accurate mode
        OZAKI2_CONVERT_GROUPED_CASE(2) OZAKI2_CONVERT_GROUPED_CASE(3)
        OZAKI2_CONVERT_GROUPED_CASE(4) OZAKI2_CONVERT_GROUPED_CASE(5)
        OZAKI2_CONVERT_GROUPED_CASE(6) OZAKI2_CONVERT_GROUPED_CASE(7)
        OZAKI2_CONVERT_GROUPED_CASE(8) OZAKI2_CONVERT_GROUPED_CASE(9)
        OZAKI2_CONVERT_GROUPED_CASE(10) OZAKI2_CONVERT_GROUPED_CASE(11)
        OZAKI2_CONVERT_GROUPED_CASE(12) OZAKI2_CONVERT_GROUPED_CASE(13)
        OZAKI2_CONVERT_GROUPED_CASE(14) OZAKI2_CONVERT_GROUPED_CASE(15)
        OZAKI2_CONVERT_GROUPED_CASE(16) OZAKI2_CONVERT_GROUPED_CASE(17)
        OZAKI2_CONVERT_GROUPED_CASE(18) OZAKI2_CONVERT_GROUPED_CASE(19)
        OZAKI2_CONVERT_GROUPED_CASE(20)
#undef OZAKI2_CONVERT_GROUPED_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

namespace {
template <typename T>
cudaError_t launch_convert_typed(const T* X, int64_t line_stride, int64_t elem_stride, int lines,
                                 int len, const int* shifts, const ConvertTables& t,
                                 __nv_bfloat16* out, int rows_pad, int k_pad,
                                 int64_t plane_elems, unsigned* status, cudaStream_t stream,
                                 bool accurate) {
    switch (t.N) {
#define OZAKI2_CONVERT_CASE(NN)                                                              \
    case NN:                                                                                 \
        return launch_convert_n<NN>(X, line_stride, elem_stride, lines, len, shifts, t, out, \
                                    rows_pad, k_pad, plane_elems, status, stream, accurate);
        OZAKI2_CONVERT_CASE(2) OZAKI2_CONVERT_CASE(3) OZAKI2_CONVERT_CASE(4)
        OZAKI2_CONVERT_CASE(5) OZAKI2_CONVERT_CASE(6) OZAKI2_CONVERT_CASE(7)
        OZAKI2_CONVERT_CASE(8) OZAKI2_CONVERT_CASE(9) OZAKI2_CONVERT_CASE(10)
        OZAKI2_CONVERT_CASE(11) OZAKI2_CONVERT_CASE(12) OZAKI2_CONVERT_CASE(13)
        OZAKI2_CONVERT_CASE(14) OZAKI2_CONVERT_CASE(15) OZAKI2_CONVERT_CASE(16)
        OZAKI2_CONVERT_CASE(17) OZAKI2_CONVERT_CASE(18) OZAKI2_CONVERT_CASE(19)
        OZAKI2_CONVERT_CASE(20)
#undef OZAKI2_CONVERT_CASE
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_convert(const void* X, int64_t line_stride, int64_t elem_stride, int lines,
                           int len, const int* shifts, const ConvertTables& t, void* planes,
                           int rows_pad, int k_pad, unsigned* status, cudaStream_t stream,
                           bool f32, bool accurate, int plane_rows) {
    if (rows_pad <= 0 || k_pad <= 0) return cudaSuccess;
    if (plane_rows <= 0) plane_rows = rows_pad;
    if (plane_rows < rows_pad) return cudaErrorInvalidValue;
    const int64_t plane_elems = (int64_t)plane_rows * k_pad;
    auto* out = static_cast<__nv_bfloat16*>(planes);
    if (f32)
        return launch_convert_typed(static_cast<const float*>(X), line_stride, elem_stride, lines,
                                    len, shifts, t, out, rows_pad, k_pad, plane_elems, status,
                                    stream, accurate);
    return launch_convert_typed(static_cast<const double*>(X), line_stride, elem_stride, lines,
                                len, shifts, t, out, rows_pad, k_pad, plane_elems, status, stream,
                                accurate);
}

}  // namespace ozaki2
