/*
 * ozaki2.h -- C ABI of the GB300 (sm_103a) Ozaki scheme II DGEMM emulation.
 *
 * Method: Ozaki scheme II (Section 2.2 of Kawakami & Takahashi, "Improved Scaling for Fast Mode
 * of Ozaki Scheme II") in fast mode with the paper's scale-invariant scaling (Section 4,
 * eq. (proposed-mu)/(proposed-nu), Algorithm 2).  C = alpha op(A) op(B) + beta C is computed as
 *   Step 1  moduli p_1..p_N (the first N of eq. (moduli)), P, P_i, q_i;
 *   Step 2  shifts e_i = log2 mu_i, f_j = log2 nu_j (Algorithm 2), a' = trunc(2^e a);
 *   Step 3  N exact residue GEMMs rmod(A',p_l) rmod(B',p_l), CRT (eqs. os2-C', os2-C'');
 *   Step 4  C = diag(mu)^-1 C'' diag(nu)^-1.
 *
 * Conventions shared by every entry point:
 *  - Matrices are column-major (BLAS).  op(X) = X for trans 'N'/'n', X^T for 'T'/'t'/'C'/'c'.
 *  - All matrix, shift, plane and residue pointers are DEVICE pointers owned by the caller.  The
 *    library never frees them and never keeps them after the queued work has run.  Every GPU
 *    entry point is asynchronous on the handle's stream: keep buffers alive until that stream
 *    is synchronised.  A and B are only read.  C is read only when beta != 0.
 *  - handle == NULL selects a process-wide default handle (created on first use, stream 0).
 *  - Return value: OZAKI2_SUCCESS (0); -i when argument i (1-based, as in BLAS xerbla) is
 *    invalid; a positive OZAKI2_ERROR_* code otherwise.  Errors raised inside kernels are
 *    reported as flags by ozaki2_get_status.
 *  - There is no CPU fallback: without an sm_103 device every GPU entry point returns
 *    OZAKI2_ERROR_NO_DEVICE.
 */
#ifndef OZAKI2_H
#define OZAKI2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------------- */
#define OZAKI2_SUCCESS 0
#define OZAKI2_ERROR_CUDA 1       /* a CUDA runtime call or a kernel launch failed */
#define OZAKI2_ERROR_ALLOC 2      /* the handle could not allocate its workspace */
#define OZAKI2_ERROR_WORKSPACE 3  /* a workspace set with ozaki2_set_workspace is too small */
#define OZAKI2_ERROR_NO_DEVICE 4  /* the current device is not an sm_103 GPU */
#define OZAKI2_ERROR_DRIVER 5     /* the driver's tensor-map encoder is unavailable or failed */
#define OZAKI2_ERROR_TOO_LARGE 6  /* the problem does not fit ozaki2_dgemm_noalloc's scratch, or
                                     k > OZAKI2_ACCURATE_MAX_K in accurate mode */
#define OZAKI2_ERROR_MODE 7       /* the entry point does not apply in the handle's scaling mode */

/* ---- device status flags (ozaki2_get_status) ------------------------------------------- */
#define OZAKI2_STATUS_NONFINITE 1u /* a row of op(A) or column of op(B) had a non-finite squared
                                      norm (Inf/NaN input or overflow); its outputs are NaN */
#define OZAKI2_STATUS_TIMEOUT 2u   /* a bounded wait inside the residue GEMM expired; the
                                      outputs of that call are undefined */
#define OZAKI2_STATUS_RANGE 4u     /* a scaled entry trunc(2^e a) exceeded the range the shifts
                                      allow (only reachable with caller-supplied shifts) */

/* Layout constants of the residue planes (see ozaki2_convert_a / ozaki2_residue_gemm). */
#define OZAKI2_ROWS_ALIGN_A 128   /* rows_pad of A planes must be a multiple of this */
#define OZAKI2_ROWS_ALIGN_B 256   /* rows_pad of B planes must be a multiple of this */
#define OZAKI2_K_ALIGN 64         /* k_pad must be a multiple of this */
#define OZAKI2_MAX_MODULI 20
#define OZAKI2_MIN_MODULI 2
#define OZAKI2_SHIFT_NONFINITE INT32_MIN /* shift written for a line with a non-finite norm */
#define OZAKI2_SHIFT_VANISH (-1100)      /* accurate mode: shift of a nonzero line whose products
                                            with every line of the other operand vanish (its row
                                            or column of C-bar is 0); it makes every a' zero */
#define OZAKI2_ACCURATE_MAX_K 1048575    /* accurate mode: largest k (C-bar < 2^32) */

/* Options (ozaki2_set_option). */
#define OZAKI2_OPT_GEMM_VARIANT 1 /* residue-GEMM kernel: one of OZAKI2_GEMM_* (default AUTO) */
#define OZAKI2_OPT_CHUNK_K 2      /* most products accumulated between modular reductions in the
                                     residue GEMM: a multiple of 64 in [64, 960] (default 960); the
                                     K blocks are spread evenly over the chunks this gives */
#define OZAKI2_OPT_GRAPH 3        /* 1: ozaki2_dgemm_grouped captures each distinct problem list
                                     once into a CUDA graph and replays it on later calls with
                                     the same list (same pointers and sizes); 0 (default): off.
                                     A graph's table buffer is kept until the handle is destroyed,
                                     the option is turned off, or the workspace is reallocated. */
#define OZAKI2_OPT_SCALING 4      /* scaling step: OZAKI2_SCALING_PROPOSED (default) or
                                     OZAKI2_SCALING_FAST */
#define OZAKI2_OPT_WAIT_LIMIT_NS 5 /* bound, in nanoseconds, of every wait inside the residue-GEMM
                                     kernels (default 2000000000 = 2 s; any value >= 0).  A wait
                                     that runs out raises OZAKI2_STATUS_TIMEOUT: the kernel stops,
                                     lets its copies and tensor-core work finish, frees its
                                     tensor memory and returns, and the call's outputs are
                                     undefined.  A bound shorter than the kernel needs makes every
                                     call time out; tests use it to exercise that path.  Graphs
                                     of grouped calls are keyed on it. */
#define OZAKI2_OPT_GROUP_M 6      /* tile order of the single-problem residue GEMM: the number of
                                     m-tiles that sweep the n-tiles together (so that the CTAs
                                     running at the same time share A and B panels in L2); 0
                                     (default) = 32 for OZAKI2_GEMM_SINGLE and 4 for
                                     OZAKI2_GEMM_PAIR (fastest measured on GB300), else 1..1024.
                                     Results do not depend on it. */
#define OZAKI2_OPT_L2_HINTS 7     /* L2 eviction priority of the tile loads of the one-SM
                                     residue-GEMM kernel (OZAKI2_GEMM_SINGLE): bits 0-1 for the
                                     A tiles, bits 2-3 for the B tiles, each 0 (the default
                                     policy), 1 (evict last) or 2 (evict first).  Default 1: the
                                     A tiles, reused by the waves of tiles that sweep the n-tiles
                                     of a raster group, evict last (measured 0-2% faster at
                                     16384^3 on GB300).  The SM-pair kernel takes no hints
                                     (evict-last A measured 5% slower there at 8192^3).  Results
                                     do not depend on it. */
#define OZAKI2_OPT_HOST_COPIES 8  /* how ozaki2_dgemm / ozaki2_sgemm move host-resident
                                     operands when the call pipelines over blocks of C (host
                                     operands, n >= 4096, op(B) = B): 0 (default) = kernels:
                                     each next operand block is uploaded by a copy kernel beside
                                     the residue GEMMs, and the reconstruction writes host C
                                     directly; 1 = copy engines (when every host operand is
                                     page-locked; else as 0): the uploads run on a copy stream
                                     from the start, and C's blocks are reconstructed in device
                                     memory and downloaded while the next blocks compute.  On
                                     GB300 at 16384^3, 1 finished some calls in 88 ms against a
                                     steady 100 ms for 0, but its copy engines' rate is erratic
                                     (other calls took 115-270 ms).  Results do not depend on
                                     it. */
#define OZAKI2_SCALING_PROPOSED 0 /* Algorithm 2 (Section 4): scale-invariant, CRT bound by
                                     construction */
#define OZAKI2_SCALING_FAST 1     /* Algorithm 1 (Section 2.3): the original fast mode, kept for
                                     comparison; its shifts depend on the scale of the input and
                                     can break the CRT bound (Section 3.1) */
#define OZAKI2_SCALING_ACCURATE 2 /* accurate mode (Section 2.3, eq. (mu_accu)/(nu_accu)): shifts
                                     from the row/column maxima of an auxiliary product
                                     C-bar = A-bar B-bar of integers <= 64; k <= 2^20 - 1 */
#define OZAKI2_GEMM_AUTO 0        /* by size, as measured fastest on GB300: PAIR when the padded m
                                   * and n both lie in [2048, 8192], SINGLE otherwise */
#define OZAKI2_GEMM_SINGLE 1      /* 128 x 256 tiles, one CTA per SM (tcgen05 cta_group::1) */
#define OZAKI2_GEMM_PAIR 2        /* 256 x 256 tiles on SM pairs (tcgen05 cta_group::2) */

typedef struct ozaki2_context* ozaki2_handle_t;

/* ---- handle ------------------------------------------------------------------------------ */
/* Create a handle bound to the current CUDA device (stream 0, internal workspace).
 * Allocates a few bytes of device memory for status flags.  Errors: OZAKI2_ERROR_NO_DEVICE,
 * OZAKI2_ERROR_CUDA; -1 if handle is NULL. */
int ozaki2_create(ozaki2_handle_t* handle);

/* Destroy a handle; synchronises its stream, frees its internal workspace (never a workspace
 * given with ozaki2_set_workspace). */
int ozaki2_destroy(ozaki2_handle_t handle);

/* Set the cudaStream_t (passed as void*) on which the handle queues work. */
int ozaki2_set_stream(ozaki2_handle_t handle, void* stream);

/* Give the handle a caller-owned device workspace of `bytes` bytes (256-byte aligned), or
 * NULL/0 to return to the internal, growable workspace.  The caller keeps it alive while work
 * that uses it is queued. */
int ozaki2_set_workspace(ozaki2_handle_t handle, void* workspace, size_t bytes);

/* Set an OZAKI2_OPT_* option of the handle.  Returns -2 for an unknown option, -3 for a value
 * out of range.  Results do not depend on the options, except OZAKI2_OPT_SCALING, which selects
 * the scaling algorithm (and so the shifts and the result) of ozaki2_dgemm, ozaki2_dgemm_h,
 * ozaki2_dgemm_grouped, ozaki2_scale_a and ozaki2_scale_b on this handle. */
int ozaki2_set_option(ozaki2_handle_t handle, int option, int value);

/* Workspace bytes that ozaki2_dgemm needs for op(A) m x k, op(B) k x n and N moduli:
 * shifts, bf16 residue planes of A and B, and int8 product residues.  0 on invalid sizes. */
size_t ozaki2_workspace_size(int m, int n, int k, int num_moduli);

/* Synchronise the handle's stream, then return and clear the OR of the status flags raised by
 * the kernels queued since the last call.  *flags receives OZAKI2_STATUS_* bits. */
int ozaki2_get_status(ozaki2_handle_t handle, unsigned* flags);

/* Stage timing: with on = 1 the handle records CUDA events on its stream around the stages of
 * each later ozaki2_dgemm_h / ozaki2_dgemm / ozaki2_sgemm_h call (scaling of A and B, conversion of A and B,
 * residue GEMMs, CRT); on = 0 stops.  Costs four event records per call. */
int ozaki2_set_timing(ozaki2_handle_t handle, int on);

/* Milliseconds of each stage of the most recent timed ozaki2_dgemm call on this handle:
 * ms[0] scaling, ms[1] conversion, ms[2] residue GEMMs, ms[3] CRT (host array of 4 floats).
 * Waits for that call's events.  Returns OZAKI2_ERROR_CUDA if no timed call was made. */
int ozaki2_get_timing(ozaki2_handle_t handle, float* ms);

/* Human-readable text of a return code. */
const char* ozaki2_error_string(int code);

/* ---- Step 1: constants (host only) -------------------------------------------------------- */
/* Step 1 (Section 2.2) and P'_prop (Section 4): writes the first num_moduli moduli of
 * eq. (moduli), q_l = (P/p_l)^{-1} mod p_l, and P'_prop = single-down(log2(P-1)/2 - 0.5).
 * moduli and inverses are host arrays of num_moduli ints; pprime a host float. */
int ozaki2_constants(int num_moduli, int* moduli, int* inverses, float* pprime);

/* ---- the whole path ----------------------------------------------------------------------- */
/* Emulated DGEMM: C = alpha op(A) op(B) + beta C through Steps 1-4 with N = num_moduli moduli
 * (2..20).  op(A) is m x k, op(B) k x n, C is m x n with ldc >= max(1, m).  A, B and C may be
 * device memory or page-locked host memory (on a device with pageable-memory access any host
 * memory); a pointer the device cannot address is an argument error.  Host-resident A and B are
 * first copied into a device buffer that the handle allocates and keeps (a kernel reads them over
 * the CPU-GPU link); with a workspace set by ozaki2_set_workspace nothing is allocated and they
 * are read in place.  A host-resident C is written (and, for beta != 0, read) in place by the
 * reconstruction kernel.  Quick returns:
 * m = 0 or n = 0 does nothing; k = 0 or alpha = 0 computes C = beta C (C = 0 when beta = 0).
 * Uses the default handle.  Argument numbers for errors: transA 1, transB 2, m 3, n 4, k 5,
 * alpha 6, A 7, lda 8, B 9, ldb 10, beta 11, C 12, ldc 13, num_moduli 14. */
int ozaki2_dgemm(char transA, char transB, int m, int n, int k, double alpha, const double* A,
                 int lda, const double* B, int ldb, double beta, double* C, int ldc,
                 int num_moduli);

/* Same as ozaki2_dgemm on an explicit handle (argument numbers shift by one). */
int ozaki2_dgemm_h(ozaki2_handle_t handle, char transA, char transB, int m, int n, int k,
                   double alpha, const double* A, int lda, const double* B, int ldb,
                   double beta, double* C, int ldc, int num_moduli);

/* Emulated SGEMM (the single-precision case of Section 5): the same steps on FP32 operands and
 * result.  Every float is exactly a double, so the scaling and the integer stages are those of
 * ozaki2_dgemm on the widened inputs; Step 4 rounds C'' once to 24 bits, scales it by
 * 2^-(e_i + f_j) with one rounding to single (subnormal results and overflow to infinity
 * included), and applies alpha and beta in single precision.  Same conventions, quick returns,
 * options (OZAKI2_OPT_SCALING included) and argument numbers as ozaki2_dgemm; the workspace is
 * that of ozaki2_dgemm for the same sizes. */
int ozaki2_sgemm(char transA, char transB, int m, int n, int k, float alpha, const float* A,
                 int lda, const float* B, int ldb, float beta, float* C, int ldc,
                 int num_moduli);

/* Same as ozaki2_sgemm on an explicit handle (argument numbers shift by one). */
int ozaki2_sgemm_h(ozaki2_handle_t handle, char transA, char transB, int m, int n, int k,
                   float alpha, const float* A, int lda, const float* B, int ldb, float beta,
                   float* C, int ldc, int num_moduli);

/* ---- many independent problems at once ---------------------------------------------------- */
/* One problem of a grouped call: the arguments of ozaki2_dgemm. */
typedef struct ozaki2_problem {
    char transA, transB;
    int m, n, k;
    double alpha;
    const double* A;
    int lda;
    const double* B;
    int ldb;
    double beta;
    double* C;
    int ldc;
    int num_moduli;
} ozaki2_problem;

/* Residue-GEMM tile configuration of grouped calls, by size class.  Rule i (i < count) matches
 * a problem with n <= n_max[i] and k <= k_max[i]; the first matching rule gives that problem's
 * tile width tile_n[i] (256, 128 or 64 columns of C per tile; the tiles are 128 rows high) and
 * K chunk chunk_k[i] (products accumulated between modular reductions: a multiple of 64 in
 * [64, 960], or 0 for the handle's OZAKI2_OPT_CHUNK_K).  A problem that no rule matches gets an
 * automatic width (64 for n <= 64, 128 for n <= 128, else 256) and the handle's chunk.  count = 0
 * clears the rules.  Results never depend on the configuration, only the time does.  Setting
 * rules drops the handle's captured graphs of grouped calls.  Arrays are host memory of count
 * ints, read during the call.  Errors: -2 count < 0 or > OZAKI2_MAX_TILE_RULES, -3/-4/-5/-6 an
 * array is NULL (count > 0), -5 a tile width not in {64, 128, 256}, -6 an invalid chunk. */
#define OZAKI2_MAX_TILE_RULES 16
int ozaki2_set_grouped_tiles(ozaki2_handle_t handle, int count, const int* n_max,
                             const int* k_max, const int* tile_n, const int* chunk_k);

/* Workspace bytes ozaki2_dgemm_grouped needs for these problems (0 if one is invalid). */
size_t ozaki2_grouped_workspace_size(int count, const ozaki2_problem* problems);

/* `count` independent emulated DGEMMs (each exactly as ozaki2_dgemm computes it, bit for bit)
 * in a handful of launches: one grouped scaling launch, one grouped conversion launch per
 * distinct moduli count, ONE persistent residue-GEMM launch over the tiles of all problems, and
 * one grouped CRT launch per distinct moduli count.  Sizes, transposes, moduli counts and
 * alpha/beta may differ between problems; outputs must not overlap.  A, B and C may be device
 * or page-locked host memory, as for ozaki2_dgemm.  `problems` is a host array
 * that is read during the call only.  The per-problem tables are staged in pinned host memory
 * owned by the handle and copied with one cudaMemcpyAsync.  Errors: -2 count < 0, -3 problems
 * NULL; -(100 (i+1) + a) when argument a (numbered as for ozaki2_dgemm) of problem i is
 * invalid. */
int ozaki2_dgemm_grouped(ozaki2_handle_t handle, int count, const ozaki2_problem* problems);

/* ---- device-resident encoded operands ------------------------------------------------------ */
/* An operand of the emulated product kept in device memory after Step 2: the shifts of its
 * lines and its bf16 residue planes.  Under the proposed scaling (Section 4, eq. (proposed-mu),
 * (proposed-nu)) and the original fast mode, the shift of a row of op(A) depends on that row
 * only, and the shift of a column of op(B) on that column only, so the encoding of an operand
 * is a function of the operand and N alone and can be reused by every product it takes part in
 * (a server's residue cache).  Accurate mode's shifts depend on both operands: it has no
 * encoded operands (OZAKI2_ERROR_MODE).
 *
 * side 'A' encodes the rows of op(A) (lines = m), side 'B' the columns of op(B) (lines = n),
 * each of length k; trans, X and ld are as transA, A, lda (or transB, B, ldb) of ozaki2_dgemm
 * (device memory, or host memory the device can address: like ozaki2_dgemm, the handle first
 * copies a host-resident X into a device buffer it allocates and keeps, or reads it in place
 * when a workspace was set with ozaki2_set_workspace).  `data` is a
 * caller-owned device buffer of ozaki2_operand_bytes(side, lines, k, num_moduli) bytes, 256-byte
 * aligned; ozaki2_encode_operands writes it and sets `scaling` to the handle's scaling mode. */
typedef struct ozaki2_operand {
    char side, trans;
    int lines, k;
    const double* X;
    int ld;
    int num_moduli;
    void* data;
    int scaling;
} ozaki2_operand;

/* Bytes of the encoding of one operand (0 for invalid arguments). */
size_t ozaki2_operand_bytes(char side, int lines, int k, int num_moduli);

/* Encodes `count` operands (Step 2: Algorithm 2 shifts, or Algorithm 1 in the original fast
 * mode, and the residue planes) in one grouped scaling launch and one grouped conversion launch
 * per distinct moduli count, asynchronously on the handle's stream.  `ops` is a host array; its
 * `scaling` fields are written during the call.  Errors: -2 count < 0, -3 ops NULL;
 * -(100 (i+1) + a) for operand i with a = 1 side, 2 trans, 3 lines, 4 k, 5 X, 6 ld,
 * 7 num_moduli, 8 data (NULL or not 256-byte aligned, or not device memory);
 * OZAKI2_ERROR_MODE in accurate mode. */
int ozaki2_encode_operands(ozaki2_handle_t handle, int count, ozaki2_operand* ops);

/* ozaki2_dgemm_grouped with encoded operands: for problem i, enc_a[i] (when enc_a and enc_a[i]
 * are not NULL) replaces transA, A and lda, and enc_b[i] replaces transB, B and ldb; those sides
 * skip the scaling and the conversion, and the problem runs the residue GEMMs and the
 * reconstruction on the encoded planes.  The result is bit-identical to ozaki2_dgemm on the
 * operands that were encoded.  An encoded operand must match its problem (side 'A' with
 * lines = m, side 'B' with lines = n, the same k and num_moduli) and the handle's scaling mode,
 * else -(100 (i+1) + 7) (A) or -(100 (i+1) + 9) (B).  Its data must stay alive and unchanged
 * until the call's work has run.  OZAKI2_ERROR_MODE in accurate mode. */
int ozaki2_dgemm_grouped_encoded(ozaki2_handle_t handle, int count,
                                 const ozaki2_problem* problems,
                                 const ozaki2_operand* const* enc_a,
                                 const ozaki2_operand* const* enc_b);

/* Workspace bytes ozaki2_dgemm_grouped_encoded needs (the planes of encoded sides are not part
 * of it); 0 if a problem is invalid. */
size_t ozaki2_grouped_encoded_workspace_size(int count, const ozaki2_problem* problems,
                                             const ozaki2_operand* const* enc_a,
                                             const ozaki2_operand* const* enc_b);

/* ---- the stages, one entry point each ------------------------------------------------------ */
/* Step 2 scaling (Algorithm 2, eq. (proposed-mu)): shifts[i] = log2(mu_i) for the m rows of
 * op(A) (m x k, lda).  The squared norm (Section 4: single or double precision, rounded upward)
 * is summed in single precision with every operation rounded upward, on terms rescaled exactly
 * by powers of two: in blocks of 256 consecutive terms, with E the largest exponent field of
 * the block's terms so far, each term enters as x = single-up(|a| 2^(1023 - E)) and the
 * block's sum as f = single-up(x x + f) (a rise of E by d first rescales f to
 * single-up(f 2^(-2d))); the block values double-up(double-up(f 2^(E-1023)) 2^(E-1023)) are
 * added in block order, rounded upward.  The result bounds the exact sum from above.  A zero
 * row gets 0; a row with a non-finite squared norm (an Inf or NaN entry, or a norm beyond the
 * double range) gets OZAKI2_SHIFT_NONFINITE and raises OZAKI2_STATUS_NONFINITE.
 * shifts: device int[m].
 * With OZAKI2_OPT_SCALING = OZAKI2_SCALING_FAST the shifts are those of Algorithm 1 instead
 * (eq. (fast-mode-mu): the same norm, plus the row maximum max_h |a_ih|); a row whose norm or
 * maximum is zero gets 0.  In OZAKI2_SCALING_ACCURATE mode the shifts depend on both operands:
 * this entry returns OZAKI2_ERROR_MODE (use ozaki2_scale_accurate).
 * Arguments: handle 1, transA 2, m 3, k 4, A 5, lda 6, num_moduli 7, shifts 8. */
int ozaki2_scale_a(ozaki2_handle_t handle, char transA, int m, int k, const double* A, int lda,
                   int num_moduli, int* shifts);

/* Step 2 scaling for the n columns of op(B) (k x n, ldb): shifts[j] = log2(nu_j)
 * (eq. (proposed-nu)).  Same conventions as ozaki2_scale_a. */
int ozaki2_scale_b(ozaki2_handle_t handle, char transB, int k, int n, const double* B, int ldb,
                   int num_moduli, int* shifts);

/* The shifts of ozaki2_scale_a (side 'A': the rows of op(A), lines x k, X = A, ld = lda) or
 * ozaki2_scale_b (side 'B': the columns of op(B), k x lines, X = B, ld = ldb), computed by the
 * kernels ozaki2_dgemm runs, together with the squared norms they come from: norms[i] receives
 * a_norm of line i exactly as Algorithm 2 takes it (a double; +Inf or NaN for a non-finite
 * line).  Not in OZAKI2_SCALING_ACCURATE mode (OZAKI2_ERROR_MODE), which takes no norm.
 * shifts: device int[lines]; norms: device double[lines].
 * Arguments: handle 1, side 2, trans 3, lines 4, k 5, X 6, ld 7, num_moduli 8, shifts 9,
 * norms 10. */
int ozaki2_scale_norms(ozaki2_handle_t handle, char side, char trans, int lines, int k,
                       const double* X, int ld, int num_moduli, int* shifts, double* norms);

/* Both scalings of accurate mode (Section 2.3), which need A and B together: line maxima,
 * A-bar = ceil(mu' |A|) and B-bar as bf16 planes in the handle's workspace, the auxiliary
 * product C-bar = A-bar B-bar on the tensor cores (exact), and
 *   e[i] = log2 mu_i = 5 - E_i + floor(P'_accu - delta log2~(max_j c-bar_ij)),
 *   f[j] likewise from the column maxima,
 * with E_i = floor(log2 max_h |a_ih|) and the reading mu_i = mu'_i 2^floor(...) of eq. (mu_accu).
 * A zero line gets 0, a line with an Inf or NaN gets OZAKI2_SHIFT_NONFINITE (and raises
 * OZAKI2_STATUS_NONFINITE), a nonzero line whose C-bar row/column is 0 gets OZAKI2_SHIFT_VANISH.
 * e: device int[m], f: device int[n]; cmax: NULL or device uint32[m + n] that receives the row
 * maxima of C-bar then the column maxima.  Works in any scaling mode of the handle.
 * Errors: -2/-3 trans, -4/-5/-6 m/n/k < 0, -7 A NULL, -8 lda, -9 B NULL, -10 ldb, -11 N,
 * -12 e NULL, -13 f NULL, OZAKI2_ERROR_TOO_LARGE for k > OZAKI2_ACCURATE_MAX_K. */
int ozaki2_scale_accurate(ozaki2_handle_t handle, char transA, char transB, int m, int n, int k,
                          const double* A, int lda, const double* B, int ldb, int num_moduli,
                          int* e, int* f, unsigned* cmax);

/* Step 2 conversion (a' = trunc(2^{e_i} a_ih)) and the residues of eq. (os2-C'):
 * planes[l][i][h] = rmod(a'_ih, p_l) stored as bfloat16 (every residue is an integer in
 * [-128, 127], exact in bf16), layout l*rows_pad*k_pad + i*k_pad + h (K contiguous).  Rows
 * i >= m and columns h >= k of each plane are written as zero.  rows_pad >= m must be a
 * multiple of OZAKI2_ROWS_ALIGN_A, k_pad >= k a multiple of OZAKI2_K_ALIGN.  The residue of
 * the even modulus 256 uses the representative in [-128, 127].  A line with shift
 * OZAKI2_SHIFT_NONFINITE gets zero residues.  Arguments: handle 1, transA 2, m 3, k 4, A 5,
 * lda 6, shifts 7, num_moduli 8, planes 9, rows_pad 10, k_pad 11. */
int ozaki2_convert_a(ozaki2_handle_t handle, char transA, int m, int k, const double* A, int lda,
                     const int* shifts, int num_moduli, void* planes, int rows_pad, int k_pad);

/* Same for the columns of op(B): planes[l][j][h] = rmod(trunc(2^{f_j} b_hj), p_l), layout
 * l*rows_pad*k_pad + j*k_pad + h; rows_pad >= n a multiple of OZAKI2_ROWS_ALIGN_B. */
int ozaki2_convert_b(ozaki2_handle_t handle, char transB, int k, int n, const double* B, int ldb,
                     const int* shifts, int num_moduli, void* planes, int rows_pad, int k_pad);

/* Step 3 residue GEMMs (eq. (os2-C')): for every modulus l,
 *   residues[l][i][j] = rmod(sum_h A_l[i][h] B_l[j][h], p_l)
 * exactly, for all i < m_pad, j < n_pad (layout l*m_pad*n_pad + i*n_pad + j, int8, values in
 * [-128, 127]).  planes_a / planes_b are bf16 planes as written by ozaki2_convert_a/_b with
 * rows_pad = m_pad / n_pad and the same k_pad; their entries must be integers in
 * [-128, 127].  Runs on tcgen05 tensor cores (bf16 operands, FP32 accumulation kept exact by
 * reducing modulo p_l every <= 960 products).  Pointers 16-byte aligned.  Arguments: handle 1,
 * num_moduli 2, m_pad 3, n_pad 4, k_pad 5, planes_a 6, planes_b 7, residues 8. */
int ozaki2_residue_gemm(ozaki2_handle_t handle, int num_moduli, int m_pad, int n_pad, int k_pad,
                        const void* planes_a, const void* planes_b, int8_t* residues);

/* Steps 3-4 (eqs. os2-C', os2-C'' and the rescaling): from product residues
 * residues[l*plane_stride + i*ldr + j] (any representative in [-128, 127]) computes
 * C'' = rmod(sum_l P_l q_l c_l, P) exactly, rounds it to the nearest double, multiplies by
 * 2^-(shifts_a[i] + shifts_b[j]) and writes C[i + j*ldc] = alpha*y (+ beta*C when beta != 0),
 * for i < m, j < n.  A sentinel shift gives NaN.  Arguments: handle 1, num_moduli 2, m 3, n 4,
 * residues 5, ldr 6, plane_stride 7, shifts_a 8, shifts_b 9, alpha 10, beta 11, C 12, ldc 13. */
int ozaki2_crt(ozaki2_handle_t handle, int num_moduli, int m, int n, const int8_t* residues,
               int ldr, long long plane_stride, const int* shifts_a, const int* shifts_b,
               double alpha, double beta, double* C, int ldc);

/* ---- the whole path without allocation --------------------------------------------------- */
/* Size of the device array that ozaki2_dgemm_noalloc keeps its intermediates in (8 MiB). */
#define OZAKI2_NOALLOC_SCRATCH_BYTES (8u << 20)

/* The emulated DGEMM of ozaki2_dgemm for callers that may not allocate device memory at call
 * time: code whose device memory is budgeted once at start-up (a solver or a serving loop that
 * reserves its memory up front, where a later cudaMalloc can fail, fragment the pool or stall
 * on the implicit device synchronisation that cudaFree brings), or code called back from a host
 * framework that forbids allocation.  The paper has no counterpart; this is a library
 * convenience.
 *
 * It allocates nothing: no cudaMalloc or cudaFree, no handle, no allocating library routine.
 * Its intermediates (shifts, residue planes, product residues, a status word) live in one
 * file-scope device array of OZAKI2_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the
 * library holds until the process exits.  The caller passes the inputs and the output as for
 * ozaki2_dgemm, plus the cudaStream_t (as void*) to queue on.  A, B and C must be memory the
 * device can address (device memory, page-locked host memory, or any host memory on a device
 * with pageable-memory access; otherwise -7, -9 or -12).  Host-resident operands are read, and
 * a host-resident C written, in place over the CPU-GPU link: nothing is staged.
 *
 * Limit: the problem must fit the array, i.e. the workspace of ozaki2_dgemm plus 256 bytes
 * (ozaki2_workspace_size(m, n, k, N) + 256) must not exceed OZAKI2_NOALLOC_SCRATCH_BYTES;
 * m = n = k = 256 fits for every N <= 20.  Larger problems return OZAKI2_ERROR_TOO_LARGE and
 * touch nothing.
 *
 * Set-up: the first call made with a given device current looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it; make that first call before any stream capture.
 * Sharing: every call uses the same array and it keeps the last call's contents, so calls that
 * overlap on the GPU (other streams, other threads) race and must be serialised by the caller.
 * The status word is cleared at the start of each call; device-side status flags are not
 * reported by this entry point.  Failures show in C instead: non-finite lines produce NaN
 * outputs, and if a bounded wait inside the residue GEMM expires (OZAKI2_STATUS_TIMEOUT) every
 * entry of C is set to NaN.  k = 0 or alpha = 0 computes C = beta C for any size (no scratch is
 * used).
 * Argument numbers for errors: as ozaki2_dgemm, stream 15. */
int ozaki2_dgemm_noalloc(char transA, char transB, int m, int n, int k, double alpha,
                         const double* A, int lda, const double* B, int ldb, double beta,
                         double* C, int ldc, int num_moduli, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OZAKI2_H */
