// convert.cu -- Step 2 conversion of Ozaki scheme II: a'_ih = trunc(2^{e_i} a_ih), and the
// residues rmod(a', p_l) of eq. (os2-C') for every modulus, written as bf16 residue planes with
// K contiguous (the operand layout of the residue GEMM).
//
// Integer-only arithmetic: the double's mantissa M (53 bits) and the exponent give
// |a'| = floor(M 2^sh), held as up to five 18-bit limbs d_j (|a'| < 2^(P'_prop+1) <= 2^79).
// For each modulus, x = sum_j d_j (2^(18 j) mod p) < 2^28 and one Barrett step gives |a'| mod p.
// The sign is applied and the symmetric representative taken ((p-1)/2 bound for odd p,
// [-128, 127] for 256); the small integer is exact in bf16.
//
// Traffic per element: 8 bytes read, 2N bytes written; HBM-bound for N <= ~14, ALU-heavy above.
#include <cuda_bf16.h>

#include "ozaki2_internal.h"

namespace ozaki2 {
namespace {

constexpr uint32_t kMask18 = (1u << 18) - 1;

struct Scaled {
    uint32_t d[5];
    bool neg;
};

// |trunc(a 2^e)| as 18-bit limbs.  Flags OZAKI2_STATUS_RANGE when the value needs more than
// 18*limbs bits (only possible with shifts that break the bound of eq. (proposed-condition)).
__device__ __forceinline__ Scaled split_scaled(double a, int e, int limbs, unsigned* status) {
    Scaled r;
    const uint64_t bits = (uint64_t)__double_as_longlong(a);
    r.neg = (bits >> 63) != 0;
    int E = (int)((bits >> 52) & 0x7FF);
    uint64_t M = bits & ((1ull << 52) - 1);
    if (E) M |= 1ull << 52; else E = 1;
    int sh = E - 1075 + e;
    uint64_t lo = 0, hi = 0;
    const int max_sh = 18 * limbs - 53;
    if (M != 0 && sh > max_sh) {
        // bits of |a'| = (64 - clz(M)) + sh must fit in 18*limbs
        if (sh > 18 * limbs - (64 - __clzll((long long)M))) atomicOr(status, OZAKI2_STATUS_RANGE);
        sh = min(sh, 37);
    }
    if (sh >= 0) {
        lo = M << sh;
        hi = sh ? (M >> (64 - sh)) : 0;
    } else if (sh > -64) {
        lo = M >> (-sh);
    }
    r.d[0] = (uint32_t)lo & kMask18;
    r.d[1] = (uint32_t)(lo >> 18) & kMask18;
    r.d[2] = (uint32_t)(lo >> 36) & kMask18;
    r.d[3] = (uint32_t)((lo >> 54) | (hi << 10)) & kMask18;
    r.d[4] = (uint32_t)(hi >> 8) & kMask18;
    return r;
}

// Symmetric residue of +-|a'| modulo p as a bf16 bit pattern in the upper 16 bits of a float.
__device__ __forceinline__ uint32_t residue_bits(const Scaled& v, const ConvertTables& t, int l) {
    const uint32_t p = t.p[l];
    uint32_t x = v.d[0];
#pragma unroll
    for (int j = 1; j < 5; ++j)
        if (j < t.limbs) x += v.d[j] * t.pow18[l][j];
    const uint32_t q = __umulhi(x, t.barrett[l]);
    uint32_t r = x - q * p;
    if (r >= p) r -= p;
    if (v.neg && r) r = p - r;
    const int s = (2 * r >= p) ? (int)r - (int)p : (int)r;
    // exact float of a small integer: 1.5*2^23 + s, minus 1.5*2^23
    const float f = __int_as_float(0x4B400000 + s) - 12582912.0f;
    return __float_as_uint(f);
}

// Writes the residues of 8 consecutive elements of one line into the N planes.
__device__ __forceinline__ void store_residues8(const double (&v)[8], int e, bool live,
                                                const ConvertTables& t, __nv_bfloat16* planes,
                                                int64_t plane_elems, int64_t offset,
                                                unsigned* status) {
    Scaled sc[8];
    const bool nonfinite = (e == OZAKI2_SHIFT_NONFINITE) || !live;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        sc[u] = nonfinite ? Scaled{{0, 0, 0, 0, 0}, false} : split_scaled(v[u], e, t.limbs, status);
    }
    for (int l = 0; l < t.N; ++l) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t a = residue_bits(sc[2 * u], t, l);
            const uint32_t b = residue_bits(sc[2 * u + 1], t, l);
            w[u] = __byte_perm(a, b, 0x7632);  // upper halves: a -> bits 0..15, b -> 16..31
        }
        *reinterpret_cast<uint4*>(planes + (int64_t)l * plane_elems + offset) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Lines contiguous (elem_stride == 1): thread = (line, group of 8 elements).
__global__ void __launch_bounds__(256) convert_contiguous_kernel(
    const double* __restrict__ X, int64_t ld, int lines, int len, const int* __restrict__ shifts,
    const ConvertTables t, __nv_bfloat16* __restrict__ planes, int rows_pad, int k_pad,
    unsigned* status) {
    const int groups = k_pad / 8;
    const int64_t total = (int64_t)rows_pad * groups;
    const int64_t plane_elems = (int64_t)rows_pad * k_pad;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / groups);
        const int h0 = (int)(g - (int64_t)i * groups) * 8;
        const bool row_live = i < lines;
        double v[8];
        const double* src = X + (int64_t)i * ld + h0;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (row_live && h0 + u < len) ? __ldg(src + u) : 0.0;
        const int e = row_live ? shifts[i] : 0;
        store_residues8(v, e, row_live, t, planes, plane_elems, (int64_t)i * k_pad + h0, status);
    }
}

// Lines adjacent (line_stride == 1): a block converts a tile of 32 lines x 64 elements.  The tile
// is read with coalesced loads along the lines (32 consecutive doubles per warp and element),
// transposed through shared memory, and each thread writes 8 consecutive elements of one line.
constexpr int kTileLines = 32;
constexpr int kTileK = 64;

__global__ void __launch_bounds__(256) convert_adjacent_kernel(
    const double* __restrict__ X, int64_t ld, int lines, int len, const int* __restrict__ shifts,
    const ConvertTables t, __nv_bfloat16* __restrict__ planes, int rows_pad, int k_pad,
    unsigned* status) {
    __shared__ double tile[kTileK][kTileLines + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t plane_elems = (int64_t)rows_pad * k_pad;
    const int tiles_l = rows_pad / kTileLines;
    const int tiles_k = k_pad / kTileK;
    const int64_t ntiles = (int64_t)tiles_l * tiles_k;
    for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const int tl = (int)(tt % tiles_l);
        const int tk = (int)(tt / tiles_l);
        const int line0 = tl * kTileLines, h0 = tk * kTileK;
        const int line = line0 + lane;
#pragma unroll
        for (int r = 0; r < kTileK / 8; ++r) {
            const int hh = warp + 8 * r;
            const int h = h0 + hh;
            tile[hh][lane] = (line < lines && h < len) ? __ldg(X + line + (int64_t)h * ld) : 0.0;
        }
        __syncthreads();
        // warp w converts elements h0 + 8w .. h0 + 8w + 7 of line line0 + lane
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = tile[8 * warp + u][lane];
        const bool live = line < lines;
        const int e = live ? shifts[line] : 0;
        store_residues8(v, e, live, t, planes, plane_elems, (int64_t)line * k_pad + h0 + 8 * warp,
                        status);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_convert(const double* X, int64_t line_stride, int64_t elem_stride, int lines,
                           int len, const int* shifts, const ConvertTables& t, void* planes,
                           int rows_pad, int k_pad, unsigned* status, cudaStream_t stream) {
    if (rows_pad <= 0 || k_pad <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto* out = static_cast<__nv_bfloat16*>(planes);
    if (elem_stride != 1) {  // then line_stride == 1: lines adjacent
        const int64_t ntiles = (int64_t)(rows_pad / kTileLines) * (k_pad / kTileK);
        const int grid = (int)(ntiles < (int64_t)sms * 8 ? ntiles : (int64_t)sms * 8);
        convert_adjacent_kernel<<<grid, 256, 0, stream>>>(X, elem_stride, lines, len, shifts, t,
                                                          out, rows_pad, k_pad, status);
    } else {
        const int64_t total = (int64_t)rows_pad * (k_pad / 8);
        const int grid = (int)((total + 255) / 256 < (int64_t)sms * 8 ? (total + 255) / 256 : (int64_t)sms * 8);
        convert_contiguous_kernel<<<grid, 256, 0, stream>>>(X, line_stride, lines, len, shifts,
                                                            t, out, rows_pad, k_pad, status);
    }
    return cudaGetLastError();
}

}  // namespace ozaki2
