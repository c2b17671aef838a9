// noalloc.cu -- ozaki2_dgemm_noalloc: the emulated DGEMM for callers that may not allocate
// device memory when they call it.
//
// All intermediates of one call (row and column shifts, the bf16 residue planes of A and B, the
// int8 product residues and a status word) live in one file-scope device array of
// OZAKI2_NOALLOC_SCRATCH_BYTES bytes.  The array exists on every GPU that loads this library
// and stays there until the process exits.  The kernels are the same ones ozaki2_dgemm runs.
//
// In host code the array's name is only a host-side stand-in, so its device address is looked
// up with cudaGetSymbolAddress once per device (on the first call made with that device
// current) and kept.  Every call shares the array: calls that overlap on the GPU (different
// streams, or another thread) race on it and must be serialised by the caller.
#include <mutex>

#include "ozaki2_internal.h"

namespace {

using namespace ozaki2;

static __device__ __align__(256) unsigned char g_noalloc_scratch[OZAKI2_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices];   // device address of g_noalloc_scratch, per device
int g_scratch_sms[kMaxDevices];
bool g_pageable[kMaxDevices];       // the device can address ordinary (pageable) host memory
std::mutex g_scratch_mu;

// Device address of the scratch array for the current device; sets it up on first use.
int scratch_for_current_device(unsigned char** ptr, int* num_sms, bool* pageable) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return OZAKI2_ERROR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            major != 10 || minor != 3)
            return OZAKI2_ERROR_NO_DEVICE;
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return OZAKI2_ERROR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        int pg = 0;
        if (cudaDeviceGetAttribute(&pg, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
            cudaGetLastError();
            pg = 0;
        }
        g_pageable[dev] = pg != 0;
        g_scratch_sms[dev] = sms;
        g_scratch_dev[dev] = p;
    }
    *ptr = static_cast<unsigned char*>(g_scratch_dev[dev]);
    *num_sms = g_scratch_sms[dev];
    *pageable = g_pageable[dev];
    return OZAKI2_SUCCESS;
}

// True if the device can address p: device or managed memory, page-locked host memory, or any
// host memory on a device with pageable-memory access.  Looks only at the pointer's attributes
// (no allocation).
bool addressable(const void* p, bool pageable) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return pageable;
    }
    return a.type != cudaMemoryTypeUnregistered || pageable;
}

// After the reconstruction: if a bounded wait in the residue GEMM expired during this call (the
// status word is cleared at the start of each call), C holds no valid result, and every entry
// is set to NaN so that the caller, who gets no status from this entry point, can see it.
__global__ void nan_on_timeout_kernel(const unsigned* __restrict__ status, double* C, int m,
                                      int n, int64_t ldc) {
    if (!(__ldg(status) & OZAKI2_STATUS_TIMEOUT)) return;
    const int64_t total = (int64_t)m * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / m, i = t - j * m;
        C[i + j * ldc] = __longlong_as_double(0x7FF8000000000000ll);
    }
}

int64_t up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
bool trans_ok(char c) {
    return c == 'N' || c == 'n' || c == 'T' || c == 't' || c == 'C' || c == 'c';
}
bool notrans(char c) { return c == 'N' || c == 'n'; }

}  // namespace

extern "C" int ozaki2_dgemm_noalloc(char transA, char transB, int m, int n, int k, double alpha,
                                    const double* A, int lda, const double* B, int ldb,
                                    double beta, double* C, int ldc, int num_moduli,
                                    void* stream) {
    if (!trans_ok(transA)) return -1;
    if (!trans_ok(transB)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    const int arows = notrans(transA) ? m : k;
    const int brows = notrans(transB) ? k : n;
    if (lda < (arows > 1 ? arows : 1)) return -8;
    if (ldb < (brows > 1 ? brows : 1)) return -10;
    if (ldc < (m > 1 ? m : 1)) return -13;
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -14;
    if (m > 0 && k > 0 && !A) return -7;
    if (k > 0 && n > 0 && !B) return -9;
    if (m > 0 && n > 0 && !C) return -12;
    if (m == 0 || n == 0) return OZAKI2_SUCCESS;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    unsigned char* s = nullptr;
    int sms = 0;
    bool pageable = false;
    int rc = scratch_for_current_device(&s, &sms, &pageable);
    if (rc) return rc;
    // operands are read (and C written) in place, wherever they live
    if (k > 0 && !addressable(A, pageable)) return -7;
    if (k > 0 && !addressable(B, pageable)) return -9;
    if (!addressable(C, pageable)) return -12;
    if (k == 0 || alpha == 0.0)  // C = beta C: no scratch needed
        return launch_scale_c(m, n, beta, C, ldc, st) == cudaSuccess ? OZAKI2_SUCCESS
                                                                     : OZAKI2_ERROR_CUDA;

    // Scratch layout: status word, shifts e and f, planes of A and B, product residues.
    const int64_t m_pad = up(m, OZAKI2_ROWS_ALIGN_A), n_pad = up(n, OZAKI2_ROWS_ALIGN_B);
    const int64_t k_pad = up(k > 0 ? k : 1, OZAKI2_K_ALIGN);
    const PlaneGeom geo = compact_planes(m, n, k);  // as ozaki2_dgemm's workspace
    const int64_t off_e = 256;
    const int64_t off_f = off_e + up(4 * m_pad, 256);
    const int64_t off_pa = off_f + up(4 * n_pad, 256);
    const int64_t off_pb = off_pa + up(2 * num_moduli * (int64_t)geo.rows_a * geo.ld, 256);
    const int64_t off_res = off_pb + up(2 * num_moduli * (int64_t)geo.rows_b * geo.ld, 256);
    const int64_t off_part = off_res + up(num_moduli * m_pad * n_pad, 256);
    const int64_t total = off_part + up((int64_t)scale_partials_bytes(m + n, k), 256);
    if (total > (int64_t)OZAKI2_NOALLOC_SCRATCH_BYTES) return OZAKI2_ERROR_TOO_LARGE;

    unsigned* status = reinterpret_cast<unsigned*>(s);
    int* e = reinterpret_cast<int*>(s + off_e);
    int* f = reinterpret_cast<int*>(s + off_f);
    void* pa = s + off_pa;
    void* pb = s + off_pb;
    int8_t* res = reinterpret_cast<int8_t*>(s + off_res);
    // The kernels OR their flags into the status word; start it at zero.
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return OZAKI2_ERROR_CUDA;

    const int64_t als = notrans(transA) ? 1 : lda, aes = notrans(transA) ? lda : 1;
    const int64_t bls = notrans(transB) ? ldb : 1, bes = notrans(transB) ? 1 : ldb;
    // norm-block sums of long lines: A's, then B's
    double* part_a = reinterpret_cast<double*>(s + off_part);
    double* part_b = part_a + scale_partials_bytes(m, k) / sizeof(double);
    if (launch_scale(A, als, aes, m, k, T->pprime, e, status, st, OZAKI2_SCALING_PROPOSED, 0.0f,
                     part_a) != cudaSuccess ||
        launch_scale(B, bls, bes, n, k, T->pprime, f, status, st, OZAKI2_SCALING_PROPOSED, 0.0f,
                     part_b) != cudaSuccess ||
        launch_convert(A, als, aes, m, k, e, T->conv, pa, geo.rows_a, geo.ld, status, st) !=
            cudaSuccess ||
        launch_convert(B, bls, bes, n, k, f, T->conv, pb, geo.rows_b, geo.ld, status, st) !=
            cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    rc = launch_residue_gemm(num_moduli, (int)m_pad, (int)n_pad, (int)k_pad, geo, pa, pb, res,
                             T->epi,
                             status, sms, 960, OZAKI2_GEMM_AUTO, st);
    if (rc) return rc;
    if (launch_crt(res, n_pad, m_pad * n_pad, m, n, e, f, alpha, beta, C, ldc, *T, status, st,
                   false, true) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    const int64_t entries = (int64_t)m * n;
    const int blocks = (int)((entries + 255) / 256 < sms ? (entries + 255) / 256 : sms);
    nan_on_timeout_kernel<<<blocks, 256, 0, st>>>(status, C, m, n, ldc);
    return cudaGetLastError() == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
}
