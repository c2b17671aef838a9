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

template <int SCALING>
__device__ __forceinline__ int line_shift(double s, double mx, float pprime, float delta,
                                          unsigned* status) {
    if (SCALING == OZAKI2_SCALING_FAST) return alg1_shift(s, mx, pprime, delta, status);
    return alg2_shift(s, pprime, status);
}

// Lines adjacent in memory (line_stride == 1): thread i walks line i in order; a warp reads 32
// consecutive doubles per step, so every load is coalesced.  Loads run two batches of 16 ahead
// of the dependent FMA chain so that enough bytes are in flight with one thread per line.
constexpr int kBatch = 16;

template <int SCALING>
__device__ __forceinline__ void scale_adjacent_line(const double* __restrict__ X, int64_t ld,
                                                    int i, int len, float pprime, float delta,
                                                    int* shifts, unsigned* status) {
    const double* p = X + i;
    double s = 0.0, mx = 0.0;
    const int full = len / kBatch * kBatch;
    double a[kBatch], b[kBatch];
    if (full > 0) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) a[u] = __ldg(p + (int64_t)u * ld);
    }
    for (int h = 0; h < full; h += 2 * kBatch) {
        const bool has_b = h + kBatch < full;
        if (has_b) {
#pragma unroll
            for (int u = 0; u < kBatch; ++u) b[u] = __ldg(p + (int64_t)(h + kBatch + u) * ld);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            s = __fma_ru(a[u], a[u], s);
            if (SCALING == OZAKI2_SCALING_FAST) mx = fmax(mx, fabs(a[u]));
        }
        if (!has_b) break;
        if (h + 2 * kBatch < full) {
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                a[u] = __ldg(p + (int64_t)(h + 2 * kBatch + u) * ld);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            s = __fma_ru(b[u], b[u], s);
            if (SCALING == OZAKI2_SCALING_FAST) mx = fmax(mx, fabs(b[u]));
        }
    }
    for (int h = full; h < len; ++h) {
        const double v = __ldg(p + (int64_t)h * ld);
        s = __fma_ru(v, v, s);
        if (SCALING == OZAKI2_SCALING_FAST) mx = fmax(mx, fabs(v));
    }
    if (SCALING == OZAKI2_SCALING_FAST && isnan(s)) mx = s;
    shifts[i] = line_shift<SCALING>(s, mx, pprime, delta, status);
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

// Lines line0 .. line0 + 31 of a contiguous-line matrix, summed by one warp (t: its smem tile).
template <int SCALING>
__device__ __forceinline__ void scale_contiguous_warp(const double* __restrict__ X, int64_t ld,
                                                      int lines, int len, int line0,
                                                      float pprime, float delta, int* shifts,
                                                      unsigned* status,
                                                      double (*t)[kTileLen + 1]) {
    const int lane = threadIdx.x & 31;
    const int nl = min(32, lines - line0);
    double reg[32];
    auto load = [&](int h0) {
        const int cnt = min(kTileLen, len - h0);
#pragma unroll
        for (int r = 0; r < 32; ++r)
            reg[r] = (r < nl && lane < cnt) ? __ldg(X + (int64_t)(line0 + r) * ld + h0 + lane)
                                            : 0.0;
    };
    double s = 0.0, mx = 0.0;
    if (len > 0) load(0);
    for (int h0 = 0; h0 < len; h0 += kTileLen) {
        const int cnt = min(kTileLen, len - h0);
#pragma unroll
        for (int r = 0; r < 32; ++r) t[r][lane] = reg[r];
        __syncwarp();
        if (h0 + kTileLen < len) load(h0 + kTileLen);
        if (lane < nl) {
            for (int u = 0; u < cnt; ++u) {
                const double v = t[lane][u];
                s = __fma_ru(v, v, s);
                if (SCALING == OZAKI2_SCALING_FAST) mx = fmax(mx, fabs(v));
            }
        }
        __syncwarp();
    }
    if (SCALING == OZAKI2_SCALING_FAST && isnan(s)) mx = s;
    if (lane < nl) shifts[line0 + lane] = line_shift<SCALING>(s, mx, pprime, delta, status);
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

// Grouped: each block takes 128 lines of one side of one problem (one thread per line for
// adjacent lines, one warp per 32 lines for contiguous lines).
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
    const bool fast = P.scaling == OZAKI2_SCALING_FAST;
    if (es != 1 || ls == 1) {
        const int i = w.line0 + (int)threadIdx.x;
        if (i < lines) {
            if (fast)
                scale_adjacent_line<OZAKI2_SCALING_FAST>(X, es, i, P.k, P.pprime, P.delta, shifts,
                                                         status);
            else
                scale_adjacent_line<OZAKI2_SCALING_PROPOSED>(X, es, i, P.k, P.pprime, P.delta,
                                                             shifts, status);
        }
    } else {
        const int warp = threadIdx.x >> 5;
        const int line0 = w.line0 + 32 * warp;
        if (line0 < lines) {
            if (fast)
                scale_contiguous_warp<OZAKI2_SCALING_FAST>(X, ls, lines, P.k, line0, P.pprime,
                                                           P.delta, shifts, status, tile[warp]);
            else
                scale_contiguous_warp<OZAKI2_SCALING_PROPOSED>(X, ls, lines, P.k, line0,
                                                               P.pprime, P.delta, shifts, status,
                                                               tile[warp]);
        }
    }
}

}  // namespace

cudaError_t launch_scale_grouped(const GroupProblem* probs, const ScaleWork* work, int blocks,
                                 unsigned* status, cudaStream_t stream) {
    if (blocks <= 0) return cudaSuccess;
    scale_grouped_kernel<<<blocks, 128, 0, stream>>>(probs, work, status);
    return cudaGetLastError();
}

template <int SCALING>
static void launch_scale_t(const double* X, int64_t line_stride, int64_t elem_stride, int lines,
                           int len, float pprime, float delta, int* shifts, unsigned* status,
                           cudaStream_t stream) {
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
                         cudaStream_t stream, int scaling, float delta) {
    if (lines <= 0) return cudaSuccess;
    if (scaling == OZAKI2_SCALING_FAST)
        launch_scale_t<OZAKI2_SCALING_FAST>(X, line_stride, elem_stride, lines, len, pprime,
                                            delta, shifts, status, stream);
    else
        launch_scale_t<OZAKI2_SCALING_PROPOSED>(X, line_stride, elem_stride, lines, len, pprime,
                                                delta, shifts, status, stream);
    return cudaGetLastError();
}

}  // namespace ozaki2
