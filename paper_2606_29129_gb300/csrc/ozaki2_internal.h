// ozaki2_internal.h -- internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ozaki2.h"

namespace ozaki2 {

constexpr int kMaxModuli = OZAKI2_MAX_MODULI;
constexpr int kMaxWords = 6;  // 32-bit words of sum_l P_l w_l < N P for N <= 20 (161 bits)
// Default bound of every wait inside the residue-GEMM kernels (OZAKI2_OPT_WAIT_LIMIT_NS).
constexpr unsigned long long kDefaultWaitLimitNs = 2000000000ull;

// Per-N tables derived from Step 1 (Section 2.2) on the host, passed to kernels by value.
struct ConvertTables {
    int N;
    uint32_t p[kMaxModuli];
    uint32_t pow21[kMaxModuli][4];  // 2^(21 j) mod p
    uint32_t bias[kMaxModuli];      // float bits of 1.5 2^23, minus h = (p - 1) / 2
    uint32_t magic39[kMaxModuli];   // ceil(2^39 / p): floor(x / p) = (x magic) >> 39 for every
                                    // x below 2^39 / p, beyond any x formed here
    unsigned long long neg_bias_magic[kMaxModuli];  // -(bias magic39) modulo 2^64
};

struct CrtTables {
    int N;
    uint32_t P[kMaxWords];
    uint32_t negP[kMaxWords];       // 2^(32 kMaxWords) - P: -P modulo any 2^(32 W), W <= kMaxWords
    uint32_t halfP[kMaxWords];      // P/2 (P is even: 256 is always a modulus)
    // Moduli grouped in pairs, g = 0.. : group g holds moduli 2g and 2g+1 (one at the end for
    // odd N), prod_g their product and PG_g = P / prod_g.  P_l = PG_g cf_l with cf_l = prod_g /
    // p_l, and cf_l w_l == cf_l q_l c_l (mod prod_g) for any w_l == q_l c_l (mod p_l), so with
    // K_l = cf_l q_l mod prod_g the group sum v_g = bias_g + sum_{l in g} c_l K_l (bias_g =
    // 256 prod_g keeps it in [0, 2^25)) gives X = sum_g PG_g v_g == sum_l P_l q_l c_l (mod P),
    // and X / P = sum_g v_g / prod_g.
    uint32_t K[kMaxModuli];
    uint32_t Kpair[(kMaxModuli + 1) / 2];  // K_2g | K_2g+1 << 16 (every K_l < prod_g < 2^16)
    uint32_t grp_bias[(kMaxModuli + 1) / 2];
    uint32_t PG[(kMaxModuli + 1) / 2][kMaxWords];
    unsigned long long R46[(kMaxModuli + 1) / 2];  // round(2^46 / prod_g); < 2^32 for a pair
};

struct EpilogueTables {
    int N;
    float p[kMaxModuli];
    float inv_p[kMaxModuli];
    float hi[kMaxModuli];  // largest symmetric representative: (p-1)/2, or 127 for 256
    float lo[kMaxModuli];  // smallest: -(p-1)/2, or -128 for 256
};

struct ModTables {
    int N;
    int moduli[kMaxModuli];
    int inverses[kMaxModuli];
    float pprime;           // P'_prop
    float pprime_fast;      // P'_fast (original fast mode)
    float delta;            // single-up(0.5 / (1 - 4u_32)), eq. (delta)
    ConvertTables conv;
    CrtTables crt;
    EpilogueTables epi;
};

// Stored extent of the bf16 residue planes [N][rows][ld] (K contiguous, row pitch ld elements, a
// multiple of 8 so rows start on 16-byte boundaries).  The residue GEMM runs over m_pad x n_pad x
// k_pad tiles; rows at or beyond `rows` and K at or beyond `ld` are not stored: the TMA reads them
// as zeros.  The library's own layout stores the rows of op(A) and op(B) only (at least one TMA
// box: 128 rows of A, 256 of B, so that no box is larger than the tensor) with ld = k_pad, which
// keeps every row on a 128-byte boundary (a shorter pitch measured slower: rows straddling cache
// lines); the stage entry points keep the padded extents.
// out_rows x out_cols: the part of each m_pad x n_pad plane of product residues that the residue
// GEMM stores (multiples of 32; the reconstruction reads 32 x 32 tiles over m x n only).
struct PlaneGeom {
    int rows_a, rows_b, ld;
    int out_rows, out_cols;
    // rows between consecutive planes of A when the GEMM reads a band of rows out of taller
    // planes (0: rows_a, the planes are stored back to back)
    int plane_rows_a = 0;
};
// bn: width of the residue-GEMM tiles (rows of op(B) in one TMA box: 256, or 128 or 64 for the
// narrower tiles of grouped calls).
inline PlaneGeom compact_planes(int m, int n, int k, int bn = 256) {
    const int ld = (k + 63) / 64 * 64;
    return PlaneGeom{m > 128 ? m : 128, n > bn ? n : bn, ld > 64 ? ld : 64, (m + 31) / 32 * 32,
                     (n + 31) / 32 * 32};
}

// Layout of an encoded operand (ozaki2_encode_operands): int32 shifts of lines_pad lines, then
// bf16 residue planes [N][rows][ld] from off_planes (rows of op(A) or columns of op(B), K
// contiguous).  Side A pads to 128 lines, side B to 256 (one TMA box of the widest tile).
struct OperandLayout {
    int lines_pad, rows, ld;
    int64_t off_planes, bytes;
};
inline OperandLayout operand_layout(bool side_b, int lines, int k, int N) {
    const int align = side_b ? 256 : 128;
    OperandLayout L;
    L.lines_pad = ((lines > 0 ? lines : 1) + align - 1) / align * align;
    L.rows = lines > align ? lines : align;
    const int ld = (k + 63) / 64 * 64;
    L.ld = ld > 64 ? ld : 64;
    L.off_planes = ((int64_t)4 * L.lines_pad + 255) / 256 * 256;
    L.bytes = L.off_planes + ((int64_t)2 * N * L.rows * L.ld + 255) / 256 * 256;
    return L;
}

// One problem of a grouped call, as the grouped kernels see it (device memory).
struct GroupProblem {
    const double* A;
    const double* B;
    double* C;
    int64_t a_ls, a_es;  // element h of row i of op(A): A[i * a_ls + h * a_es]
    int64_t b_ls, b_es;  // element h of column j of op(B): B[j * b_ls + h * b_es]
    int64_t ldc;
    int m, n, k, N;
    int m_pad, n_pad, k_pad;
    PlaneGeom geo;       // stored extent of pa / pb
    double alpha, beta;
    int ab;              // bit 0: alpha != 1, bit 1: beta != 0 (set on the host)
    float pprime;        // P'_prop, or P'_fast in the original fast mode
    float delta;
    int scaling;         // OZAKI2_SCALING_*
    int* e;              // shifts of the rows of op(A)   [m_pad]
    int* f;              // shifts of the columns of op(B) [n_pad]
    void* pa;            // bf16 planes [N][geo.rows_a][geo.ld]
    void* pb;            // bf16 planes [N][geo.rows_b][geo.ld]
    int8_t* res;         // product residues [N][m_pad][n_pad]
};

// Work tables of the grouped kernels: one entry per thread block.
struct ScaleWork {       // 128 lines of one side of one problem
    int problem, side, line0;
};
struct ConvertWork {     // block `block` of one side of one problem (adjacent: a 64 x 64 tile,
    int problem, side, block;  // contiguous: 256 groups of 8 elements)
};
struct CrtWork {         // one 32 x 64 tile of C
    int problem, i0, j0;
};

// One problem of a grouped residue GEMM (device memory, 64-byte aligned for the tensor maps).
struct alignas(64) GroupGemmProblem {
    CUtensorMap ta;      // A planes [N][rows_a][ld], box 64 x 128
    CUtensorMap tb;      // B planes [N][rows_b][ld], box 64 x bn
    int8_t* out;         // product residues [N][m_pad][n_pad]
    int64_t out_ld, out_plane;
    int tiles_m, tiles_n, k_blocks, nchunks;
    int m_live, n_live;  // stored part of each plane of `out` (PlaneGeom::out_rows, out_cols)
    int tile_begin;      // index of this problem's first tile in the grouped launch
    int bn;              // tile width (256, 128 or 64 columns); the B box has bn rows
    int chunk_blocks;    // K blocks of 64 between modular reductions
};

// Fills the tensor maps and tile counts of one grouped-GEMM problem (host); false on failure.
// bn: tile width, 256, 128 or 64 (n_pad a multiple of bn, geo.rows_b >= bn).
bool make_group_gemm_problem(GroupGemmProblem* g, int N, int m_pad, int n_pad, int k_pad,
                             const PlaneGeom& geo, const void* planes_a, const void* planes_b,
                             int8_t* out, int chunk_k, int bn = 256);
int launch_residue_gemm_grouped(const GroupGemmProblem* probs, int count, int total_tiles,
                                const EpilogueTables& t, unsigned* status, int num_sms,
                                int chunk_k, cudaStream_t stream,
                                unsigned long long limit_ns = kDefaultWaitLimitNs);

// The memory layout of a line of a grouped problem: element h of line i at X[i ls + h es];
// lines adjacent (one thread per line) unless es == 1 with ls != 1 (lines contiguous, a warp
// per 32 lines).
constexpr int kLayoutAny = 0, kLayoutAdjacent = 1, kLayoutContiguous = 2;
__host__ __device__ inline bool scale_lines_adjacent(int64_t ls, int64_t es) {
    return es != 1 || ls == 1;
}
// scaling: the mode every problem of the call shares (OZAKI2_SCALING_*).  adjacent_blocks >= 0:
// the work list holds the items of adjacent lines first (that many), then those of contiguous
// lines, and each group runs in a kernel of its own; < 0: one kernel decides per item.
cudaError_t launch_scale_grouped(const GroupProblem* probs, const ScaleWork* work, int blocks,
                                 unsigned* status, cudaStream_t stream,
                                 int scaling = OZAKI2_SCALING_PROPOSED, int adjacent_blocks = -1);
cudaError_t launch_convert_grouped(int N, const GroupProblem* probs, const ConvertWork* work,
                                   int blocks, const ConvertTables& t, unsigned* status,
                                   cudaStream_t stream, bool accurate = false);
cudaError_t launch_crt_grouped(int N, const GroupProblem* probs, const CrtWork* work, int blocks,
                               const CrtTables& t, cudaStream_t stream);
// Blocks of the grouped convert for one side of one problem (rows x ld stored).
int convert_blocks(int lines, int64_t elem_stride, int rows, int ld);

// Residue-GEMM configuration of the problems of a grouped call: the first rule whose bounds
// hold (n <= n_max and k <= k_max) gives the problem's tile width (256, 128 or 64 columns) and K
// chunk (0: the handle's OZAKI2_OPT_CHUNK_K); a problem that no rule matches gets the automatic
// width (auto_tile_n) and the handle's chunk.
struct TileRule {
    int n_max, k_max, tile_n, chunk_k;
};
struct TileRules {
    int count = 0;
    TileRule r[OZAKI2_MAX_TILE_RULES];
};
// Automatic tile width for a problem with n columns of op(B): the fewest estimated cycles per
// 128-row m-tile and K block of 64, a tile taking max(2 bn, (16 KiB + 128 bn) / 96) cycles (its
// MMAs, or loading its A and B blocks at ~96 bytes per cycle and SM); ties go to the wider tile.
int auto_tile_n(int n);
// Tile width and K chunk of a problem under `rules` (chunk_k: the handle's default chunk).
void grouped_tile(const TileRules& rules, int n, int k, int chunk_k, int* bn, int* chunk);

// Grouped calls (grouped.cu).  `rules` and `chunk_k` select each problem's tile width and K chunk.
// enc_a / enc_b: NULL, or per problem NULL or an encoded operand replacing op(A) / op(B) (already
// checked against the problem).
struct Encoded {
    const ozaki2_operand* const* a = nullptr;
    const ozaki2_operand* const* b = nullptr;
};
size_t grouped_workspace_bytes(int count, const ozaki2_problem* probs,
                               const Encoded& enc = Encoded());
int grouped_table_bytes(int count, const ozaki2_problem* probs, const TileRules& rules,
                        int chunk_k, int scaling = OZAKI2_SCALING_PROPOSED,
                        const Encoded& enc = Encoded());
int grouped_check(int count, const ozaki2_problem* probs);
int build_grouped_tables(int count, const ozaki2_problem* probs, char* ws, char* host,
                         const TileRules& rules, int chunk_k,
                         int scaling = OZAKI2_SCALING_PROPOSED, const Encoded& enc = Encoded());
int launch_grouped(int count, const ozaki2_problem* probs, const char* tables_dev,
                   unsigned* status, int num_sms, const TileRules& rules, int chunk_k,
                   cudaStream_t stream, int scaling = OZAKI2_SCALING_PROPOSED,
                   unsigned long long limit_ns = kDefaultWaitLimitNs,
                   const Encoded& enc = Encoded());
char* grouped_tables_in_workspace(int count, const ozaki2_problem* probs, char* ws,
                                  const Encoded& enc = Encoded());
// Encoding of operands (ozaki2_encode_operands): table bytes, the tables (host), the launches.
int encode_table_bytes(int count, const ozaki2_operand* ops);
void build_encode_tables(int count, const ozaki2_operand* ops, int scaling, char* host);
int launch_encode(int count, const ozaki2_operand* ops, const char* tables_dev, unsigned* status,
                  cudaStream_t stream, int scaling = OZAKI2_SCALING_PROPOSED);

// Accurate mode (scale.cu, convert.cu, residue_gemm.cu).
// A-bar plane [rows][ld] (bf16, K contiguous) from the exponent codes of the first pass.
cudaError_t launch_convert_bar(const void* X, int64_t line_stride, int64_t elem_stride,
                               int lines, int len, const int* codes, void* plane, int rows,
                               int ld, unsigned* status, cudaStream_t stream,
                               bool f32 = false);
// Row and column maxima of C-bar = A-bar B-bar into cmax[0, m_pad) and cmax[m_pad, m_pad+n_pad).
int launch_aux_gemm(int m_pad, int n_pad, int k_pad, const PlaneGeom& geo, const void* bar_a,
                    const void* bar_b, uint32_t* cmax, unsigned* status, int num_sms,
                    cudaStream_t stream, unsigned long long limit_ns = kDefaultWaitLimitNs);
// Grouped form: one descriptor per problem (tensor maps over its A-bar / B-bar planes, the
// maxima at `cmax`), and the persistent launch over all their tiles.
bool make_group_aux_problem(GroupGemmProblem* g, int m_pad, int n_pad, int k_pad,
                            const PlaneGeom& geo, const void* bar_a, const void* bar_b,
                            uint32_t* cmax);
int launch_aux_gemm_grouped(const GroupGemmProblem* probs, int count, int total_tiles,
                            unsigned* status, int num_sms, cudaStream_t stream,
                            unsigned long long limit_ns = kDefaultWaitLimitNs);
cudaError_t launch_accu_shift_grouped(const GroupProblem* probs, const ScaleWork* work,
                                      int blocks, cudaStream_t stream);
// Final shifts, in place over the exponent codes.
cudaError_t launch_accu_shift(int* e, int m, int* f, int n, const uint32_t* cmax, int m_pad,
                              float pprime, float delta, cudaStream_t stream);

// Tables for 2 <= N <= 20 (cached, thread safe).  Returns nullptr for other N.
const ModTables* mod_tables(int N);

// ---- launchers (asynchronous on `stream`) ----------------------------------------------------
// Shifts for `lines` lines of length `len`.  Element h of line i is at
//   X[i * line_stride + h * elem_stride]  with either line_stride == 1 (lines adjacent) or
//   elem_stride == 1 (each line contiguous).
// Shifts of the rows of op(A) (m lines) and the columns of op(B) (n lines), both of length len,
// in one launch; strides as for launch_scale.
// f32: the matrices hold floats (SGEMM), else doubles.
// partials: NULL, or device scratch of scale_partials_bytes(m + n, len) bytes, which lets lines
// longer than one norm block split across warps (NULL: one thread per line).
// norms_a / norms_b: NULL, or device doubles that receive the squared norms the shifts come from.
cudaError_t launch_scale_pair(const void* A, int64_t a_ls, int64_t a_es, int m, const void* B,
                              int64_t b_ls, int64_t b_es, int n, int len, float pprime,
                              float delta, int* e, int* f, unsigned* status, cudaStream_t stream,
                              int scaling, bool f32 = false, double* partials = nullptr,
                              double* norms_a = nullptr, double* norms_b = nullptr);
// Scratch bytes of the norm-block sums (and maxima) of `lines` lines of length len: 0 when a
// line fits one block of 256 terms.
inline size_t scale_partials_bytes(int lines, int len) {
    const int64_t nblocks = ((int64_t)len + 255) / 256;
    return nblocks > 1 ? (size_t)(2 * nblocks * (int64_t)lines * 8) : 0;
}

#ifdef __CUDACC__
// The double of the same value as a float, built from the bits with integer operations (the
// conversion instruction runs on the FP64 pipe, which GB300 keeps narrow).  Exact: normal floats
// rebias the exponent; subnormals are normalised; Inf and NaN keep their class.
__device__ __forceinline__ double widen_exact(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint64_t sign = (uint64_t)(b >> 31) << 63;
    const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    uint64_t bits;
    if (e == 0xFFu) {
        bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
    } else if (e != 0u) {
        bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
    } else if (m == 0u) {
        bits = sign;
    } else {
        const int msb = 31 - __clz(m);  // value m 2^-149 = 2^(msb-149) (1.f)
        bits = sign | ((uint64_t)(msb - 149 + 1023) << 52) |
               (((uint64_t)m << (52 - msb)) & ((1ull << 52) - 1));
    }
    return __longlong_as_double((long long)bits);
}
#endif

// Accurate mode: the first scaling pass writes this code for a zero line (a real E is in
// [-1074, 1023], OZAKI2_SHIFT_NONFINITE marks a non-finite line).
constexpr int kAccuZeroLine = INT32_MAX;

// scaling: OZAKI2_SCALING_PROPOSED (pprime = P'_prop) or OZAKI2_SCALING_FAST (pprime = P'_fast).
cudaError_t launch_scale(const double* X, int64_t line_stride, int64_t elem_stride, int lines,
                         int len, float pprime, int* shifts, unsigned* status,
                         cudaStream_t stream, int scaling = OZAKI2_SCALING_PROPOSED,
                         float delta = 0.0f, double* partials = nullptr);

// f32: X holds floats (SGEMM), else doubles.  accurate: the shifts come from accurate mode,
// whose a' may need six more bits than the proposed and fast scalings allow.
// Writes planes [N][rows][ld]: rows at or beyond `lines` and K at or beyond `len` as zeros.
// plane_rows: rows from one plane to the next (0: rows), to convert a band of lines into
// taller planes (planes pointing at the band's first row).
cudaError_t launch_convert(const void* X, int64_t line_stride, int64_t elem_stride, int lines,
                           int len, const int* shifts, const ConvertTables& t, void* planes,
                           int rows, int ld, unsigned* status, cudaStream_t stream,
                           bool f32 = false, bool accurate = false, int plane_rows = 0);

int launch_residue_gemm(int num_moduli, int m_pad, int n_pad, int k_pad, const PlaneGeom& geo,
                        const void* planes_a, const void* planes_b, int8_t* out,
                        const EpilogueTables& t, unsigned* status, int num_sms, int chunk_k,
                        int variant, cudaStream_t stream,
                        unsigned long long limit_ns = kDefaultWaitLimitNs, int64_t out_ld = 0,
                        int64_t out_plane = 0, int group_m = 0, int l2_hints = 0);

// f32: C holds floats (SGEMM: C'' rounded to 24 bits, alpha and beta applied in single
// precision), else doubles.  padded: the residue buffer extends to whole 32 x 32 tiles in every
// plane (true for the library's own layout), which allows 32-bit residue loads.
// max_blocks > 0: at most that many thread blocks, each striding over the 32 x 32 tiles of C.
cudaError_t launch_crt(const int8_t* res, int64_t ldr, int64_t plane, int m, int n,
                       const int* sa, const int* sb, double alpha, double beta, void* C,
                       int64_t ldc, const ModTables& t, unsigned* status, cudaStream_t stream,
                       bool f32 = false, bool padded = false, int max_blocks = 0);

// Device copy of `bytes` from host memory the device can address (page-locked, or any host
// memory on a coherent link): a kernel reads the host memory at the link's rate, where a copy-
// engine upload measured erratic on GB300 after kernels had touched host memory.
// blocks_per_sm: thread blocks per SM of the copy (default 8; 1 leaves room on every SM for a
// kernel running beside it).
cudaError_t launch_stage_in(void* dst, const void* src, size_t bytes, int num_sms,
                            cudaStream_t stream, int blocks_per_sm = 8);

// A 2-D copy between memories the device can address (device, page-locked or coherent host
// memory): `height` rows of `width` bytes, from src (rows spitch bytes apart) to dst (dpitch
// bytes apart).
struct Copy2D {
    void* dst;
    const void* src;
    size_t dpitch, spitch, width, height;
};
// Up to two copies in one launch, each by up to `blocks` thread blocks of 256 threads.
// overlap_previous: launched with programmatic serialization, so that the copies run beside the
// kernel before them in the stream once that kernel's blocks have all started (the residue
// GEMM signals this as it starts); the copy then completes only after that kernel.  The copies
// must not read what that kernel writes.
cudaError_t launch_copies_2d(const Copy2D* copies, int count, int blocks, bool overlap_previous,
                             cudaStream_t stream);

cudaError_t launch_scale_c(int m, int n, double beta, void* C, int64_t ldc,
                           cudaStream_t stream, bool f32 = false);

}  // namespace ozaki2
