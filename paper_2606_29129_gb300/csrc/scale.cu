// scale.cu -- Step 2 scaling of Ozaki scheme II with the scale-invariant formula of Section 4
// (eq. (proposed-mu)/(proposed-nu), Algorithm 2).
//
// Each line (row of op(A) or column of op(B)) gets a_norm = sum_h a_h^2 accumulated in the order
// h = 0..len-1, one fused multiply-add rounded upward per term (every partial sum is an upper
// bound, as Algorithm 2 requires), then log2(mu) = floor(w - t) from Algorithm 2.
//
// The kernel is bound by HBM reads of the matrix (8 bytes per element) and, on GB300, by the
// FP64 FMA rate; the fixed summation order keeps the shifts bit-identical to a sequential
// reference.
#include <float.h>

#include "ozaki2_internal.h"

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

// Lines adjacent in memory (line_stride == 1): thread i walks line i; a warp reads 32
// consecutive doubles per step, so every load is coalesced.
__global__ void __launch_bounds__(128) scale_adjacent_kernel(const double* __restrict__ X,
                                                             int64_t ld, int lines, int len,
                                                             float pprime, int* shifts,
                                                             unsigned* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lines) return;
    const double* p = X + i;
    double s = 0.0;
    int h = 0;
    for (; h + 8 <= len; h += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(p + (int64_t)(h + u) * ld);
#pragma unroll
        for (int u = 0; u < 8; ++u) s = __fma_ru(v[u], v[u], s);
    }
    for (; h < len; ++h) {
        const double v = __ldg(p + (int64_t)h * ld);
        s = __fma_ru(v, v, s);
    }
    shifts[i] = alg2_shift(s, pprime, status);
}

// Contiguous lines (elem_stride == 1): a block of 64 threads owns 64 lines.  Tiles of 32
// elements per line are staged through shared memory with coalesced loads (one warp reads one
// line's 32 consecutive doubles), then each thread sums its own line in order.
constexpr int kLinesPerBlock = 64;
constexpr int kTileLen = 32;

__global__ void __launch_bounds__(kLinesPerBlock) scale_contiguous_kernel(
    const double* __restrict__ X, int64_t ld, int lines, int len, float pprime, int* shifts,
    unsigned* status) {
    __shared__ double tile[kLinesPerBlock][kTileLen + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line0 = blockIdx.x * kLinesPerBlock;
    const int nlines = min(kLinesPerBlock, lines - line0);
    double s = 0.0;
    for (int h0 = 0; h0 < len; h0 += kTileLen) {
        const int cnt = min(kTileLen, len - h0);
        for (int r = warp; r < nlines; r += kLinesPerBlock / 32) {
            if (lane < cnt) tile[r][lane] = __ldg(X + (int64_t)(line0 + r) * ld + h0 + lane);
        }
        __syncthreads();
        if (threadIdx.x < nlines) {
            for (int u = 0; u < cnt; ++u) {
                const double v = tile[threadIdx.x][u];
                s = __fma_ru(v, v, s);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < nlines) shifts[line0 + threadIdx.x] = alg2_shift(s, pprime, status);
}

}  // namespace

cudaError_t launch_scale(const double* X, int64_t line_stride, int64_t elem_stride, int lines,
                         int len, float pprime, int* shifts, unsigned* status,
                         cudaStream_t stream) {
    if (lines <= 0) return cudaSuccess;
    if (elem_stride != 1 || line_stride == 1) {  // lines adjacent
        const int threads = 128;
        scale_adjacent_kernel<<<(lines + threads - 1) / threads, threads, 0, stream>>>(
            X, elem_stride, lines, len, pprime, shifts, status);
    } else {
        scale_contiguous_kernel<<<(lines + kLinesPerBlock - 1) / kLinesPerBlock, kLinesPerBlock,
                                  0, stream>>>(X, line_stride, lines, len, pprime, shifts,
                                               status);
    }
    return cudaGetLastError();
}

}  // namespace ozaki2
