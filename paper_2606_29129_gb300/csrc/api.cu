// api.cu -- the C ABI of include/ozaki2.h: handles, workspace, argument checks, the stage entry
// points and the composed emulated DGEMM (Steps 1-4 of Ozaki scheme II, Section 2.2, with the
// scaling of Section 4).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ozaki2_internal.h"

struct ozaki2_context {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = 0;
    unsigned* d_status = nullptr;  // device word of OZAKI2_STATUS_* flags
    void* ws = nullptr;            // workspace (owned unless user_ws)
    size_t ws_bytes = 0;
    bool user_ws = false;
    int chunk_k = 960;             // products accumulated between modular reductions
    int gemm_variant = OZAKI2_GEMM_AUTO;
    int group_m = 0;               // m-tiles per group of the residue-GEMM tile order (0: 16)
    int l2_hints = 1;              // OZAKI2_OPT_L2_HINTS (A tiles evict last: measured faster)
    int host_copies = 0;           // OZAKI2_OPT_HOST_COPIES (kernels: measured steadier)
    int scaling = OZAKI2_SCALING_PROPOSED;  // Algorithm 2, or Algorithm 1 (original fast mode)
    unsigned long long wait_limit_ns = ozaki2::kDefaultWaitLimitNs;  // residue-GEMM wait bound
    ozaki2::TileRules tiles;       // grouped calls: tile width and K chunk by size class
    bool timing = false;           // record stage events in ozaki2_dgemm
    bool timed_call = false;       // a timed call has been queued
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    char* stage = nullptr;         // pinned staging buffer of grouped-call tables
    size_t stage_bytes = 0;
    cudaEvent_t staged = nullptr;  // recorded after the last copy out of `stage`
    bool use_graphs = false;       // replay grouped calls from captured CUDA graphs
    struct GraphEntry {
        std::vector<ozaki2_problem> probs;
        int chunk_k;
        int scaling;
        unsigned long long wait_limit_ns;
        void* tables = nullptr;    // device copy of the call's tables
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t capture_stream = nullptr;
    bool pageable_access = false;  // the device can address ordinary (pageable) host memory
    void* in_ws = nullptr;         // device copies of host-resident A and B (ozaki2_dgemm)
    size_t in_ws_bytes = 0;
    void* out_ws = nullptr;        // device copies of host C's blocks (pipelined ozaki2_dgemm)
    size_t out_ws_bytes = 0;
    // copy-engine transfers of a pipelined ozaki2_dgemm: uploads on up_stream, downloads on
    // down_stream, ordered against the handle's stream by events
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    static constexpr int kCopyEvents = 40;
    cudaEvent_t copy_ev[kCopyEvents] = {};
    // pinned staging of the tables of ozaki2_encode_operands: a ring, so that a call waits only
    // for the copy made kEncodeRing calls earlier
    static constexpr int kEncodeRing = 4;
    char* enc_stage[kEncodeRing] = {};
    size_t enc_stage_bytes[kEncodeRing] = {};
    cudaEvent_t enc_staged[kEncodeRing] = {};
    int enc_next = 0;
};

namespace {
void clear_graphs(ozaki2_context* ctx) {
    for (auto& g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.tables) cudaFree(g.tables);
    }
    ctx->graphs.clear();
}
bool same_problems(const std::vector<ozaki2_problem>& a, int count, const ozaki2_problem* b) {
    return (int)a.size() == count &&
           (count == 0 || memcmp(a.data(), b, sizeof(ozaki2_problem) * (size_t)count) == 0);
}
}  // namespace

namespace {

using namespace ozaki2;

bool is_trans_char(char c) {
    return c == 'N' || c == 'n' || c == 'T' || c == 't' || c == 'C' || c == 'c';
}
bool is_notrans(char c) { return c == 'N' || c == 'n'; }
int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

int check_device(int* dev_out, int* sms_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OZAKI2_ERROR_NO_DEVICE;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return OZAKI2_ERROR_NO_DEVICE;
    if (major != 10 || minor != 3) return OZAKI2_ERROR_NO_DEVICE;  // built for sm_103a only
    if (sms_out) cudaDeviceGetAttribute(sms_out, cudaDevAttrMultiProcessorCount, dev);
    if (dev_out) *dev_out = dev;
    return OZAKI2_SUCCESS;
}

int init_context(ozaki2_context* ctx) {
    int rc = check_device(&ctx->device, &ctx->num_sms);
    if (rc) return rc;
    if (cudaMalloc(&ctx->d_status, 256) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    if (cudaMemset(ctx->d_status, 0, 256) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, ctx->device) !=
        cudaSuccess)
        pageable = 0;
    ctx->pageable_access = pageable != 0;
    return OZAKI2_SUCCESS;
}

// True if the device can address p: device or managed memory, page-locked host memory (mapped
// under unified addressing), or any host memory when the device has pageable-memory access
// (a coherent CPU-GPU link).  Kernels never touch a pointer that fails this check.
bool addressable(const ozaki2_context* ctx, const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return ctx->pageable_access;
    }
    return a.type != cudaMemoryTypeUnregistered || ctx->pageable_access;
}

// True if p is page-locked host memory (allocated so, or registered).
bool page_locked(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// True if p is host memory (page-locked, or pageable on a coherent link) rather than device or
// managed memory.
bool host_resident(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

ozaki2_context* g_default = nullptr;
int g_default_rc = OZAKI2_SUCCESS;
std::once_flag g_default_once;

// handle == NULL -> the process-wide default handle.
int resolve(ozaki2_handle_t h, ozaki2_context** out) {
    if (h) {
        *out = h;
        return OZAKI2_SUCCESS;
    }
    std::call_once(g_default_once, [] {
        g_default = new ozaki2_context();
        g_default_rc = init_context(g_default);
    });
    *out = g_default;
    return g_default_rc;
}

// Make sure the handle has at least `bytes` of workspace.
int ensure_workspace(ozaki2_context* ctx, size_t bytes) {
    if (ctx->ws_bytes >= bytes) return OZAKI2_SUCCESS;
    if (ctx->user_ws) return OZAKI2_ERROR_WORKSPACE;
    if (ctx->ws) {
        // work queued on other streams may still use the old buffer
        if (cudaDeviceSynchronize() != cudaSuccess) return OZAKI2_ERROR_CUDA;
        clear_graphs(ctx);  // captured kernels refer to the old workspace
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return OZAKI2_ERROR_ALLOC;
    }
    ctx->ws_bytes = bytes;
    return OZAKI2_SUCCESS;
}

struct Layout {
    int64_t m_pad, n_pad, k_pad;
    PlaneGeom geo;  // stored extent of the residue planes (no padding rows beyond one TMA box)
    size_t off_e, off_f, off_pa, off_pb, off_res, off_part, total;
};

Layout make_layout(int m, int n, int k, int N) {
    Layout L;
    L.m_pad = round_up(m > 0 ? m : 1, OZAKI2_ROWS_ALIGN_A);
    L.n_pad = round_up(n > 0 ? n : 1, OZAKI2_ROWS_ALIGN_B);
    L.k_pad = round_up(k > 0 ? k : 1, OZAKI2_K_ALIGN);
    L.geo = compact_planes(m, n, k);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (size_t)round_up((int64_t)bytes, 256);
        return o;
    };
    L.off_e = take(sizeof(int) * (size_t)L.m_pad);
    L.off_f = take(sizeof(int) * (size_t)L.n_pad);
    L.off_pa = take((size_t)2 * N * L.geo.rows_a * L.geo.ld);
    L.off_pb = take((size_t)2 * N * L.geo.rows_b * L.geo.ld);
    L.off_res = take((size_t)N * L.m_pad * L.n_pad);
    L.off_part = take(scale_partials_bytes(m + n, k));  // norm-block sums of long lines
    L.total = off;
    return L;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA; }

// Strides of the lines of op(A) (rows) and op(B) (columns) of a column-major matrix.
void rows_of_op(char trans, int64_t ld, int64_t* line_stride, int64_t* elem_stride) {
    if (is_notrans(trans)) { *line_stride = 1; *elem_stride = ld; }
    else { *line_stride = ld; *elem_stride = 1; }
}
void cols_of_op(char trans, int64_t ld, int64_t* line_stride, int64_t* elem_stride) {
    if (is_notrans(trans)) { *line_stride = ld; *elem_stride = 1; }
    else { *line_stride = 1; *elem_stride = ld; }
}

// Accurate mode (Section 2.3): line exponents, A-bar and B-bar in the first residue plane of
// each operand's planes, the maxima of C-bar = A-bar B-bar in the product-residue region (at
// least 4 (m_pad + n_pad) bytes), and the shifts written over the exponents.
int accurate_shifts(ozaki2_context* ctx, const void* A, int64_t als, int64_t aes,
                    const void* B, int64_t bls, int64_t bes, int m, int n, int k,
                    const Layout& L, const ModTables& T, int* e, int* f, void* pa, void* pb,
                    void* cmax_region, bool f32 = false) {
    cudaStream_t st = ctx->stream;
    auto* cmax = static_cast<uint32_t*>(cmax_region);
    int rc;
    if ((rc = cuda_rc(launch_scale_pair(A, als, aes, m, B, bls, bes, n, k, T.pprime, T.delta, e,
                                        f, ctx->d_status, st, OZAKI2_SCALING_ACCURATE, f32))) ||
        (rc = cuda_rc(launch_convert_bar(A, als, aes, m, k, e, pa, L.geo.rows_a, L.geo.ld,
                                         ctx->d_status, st, f32))) ||
        (rc = cuda_rc(launch_convert_bar(B, bls, bes, n, k, f, pb, L.geo.rows_b, L.geo.ld,
                                         ctx->d_status, st, f32))))
        return rc;
    if ((rc = launch_aux_gemm((int)L.m_pad, (int)L.n_pad, (int)L.k_pad, L.geo, pa, pb, cmax,
                              ctx->d_status, ctx->num_sms, st, ctx->wait_limit_ns)))
        return rc;
    return cuda_rc(launch_accu_shift(e, m, f, n, cmax, (int)L.m_pad, T.pprime, T.delta, st));
}

// The emulated GEMM for FP64 (f32 = false) or FP32 (f32 = true) operands and result; alpha and
// beta are passed as doubles (exact for single values).
// Device buffer for the copies of host-resident inputs (grown on demand, like the workspace).
int ensure_input_stage(ozaki2_context* ctx, size_t bytes) {
    if (ctx->in_ws_bytes >= bytes) return OZAKI2_SUCCESS;
    if (ctx->in_ws) {
        if (cudaDeviceSynchronize() != cudaSuccess) return OZAKI2_ERROR_CUDA;
        cudaFree(ctx->in_ws);
        ctx->in_ws = nullptr;
        ctx->in_ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->in_ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return OZAKI2_ERROR_ALLOC;
    }
    ctx->in_ws_bytes = bytes;
    return OZAKI2_SUCCESS;
}

// The streams and events of copy-engine transfers.
int ensure_copy_streams(ozaki2_context* ctx) {
    if (ctx->up_stream) return OZAKI2_SUCCESS;
    bool ok = true;
    for (cudaStream_t* st : {&ctx->down_stream, &ctx->up_stream})
        if (ok && cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) != cudaSuccess) {
            *st = nullptr;
            ok = false;
        }
    for (cudaEvent_t& e : ctx->copy_ev)
        if (ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
            ok = false;
        }
    if (ok) return OZAKI2_SUCCESS;
    // all or nothing: the next call starts again from scratch
    cudaGetLastError();
    for (cudaStream_t* st : {&ctx->down_stream, &ctx->up_stream}) {
        if (*st) cudaStreamDestroy(*st);
        *st = nullptr;
    }
    for (cudaEvent_t& e : ctx->copy_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    return OZAKI2_ERROR_CUDA;
}

// The device buffers of C's blocks, `bytes` in all.
int ensure_output_stage(ozaki2_context* ctx, size_t bytes) {
    if (ctx->out_ws_bytes >= bytes) return OZAKI2_SUCCESS;
    if (ctx->out_ws) {
        if (cudaDeviceSynchronize() != cudaSuccess) return OZAKI2_ERROR_CUDA;
        cudaFree(ctx->out_ws);
        ctx->out_ws = nullptr;
        ctx->out_ws_bytes = 0;
    }
    if (cudaMalloc(&ctx->out_ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return OZAKI2_ERROR_ALLOC;
    }
    ctx->out_ws_bytes = bytes;
    return OZAKI2_SUCCESS;
}

// Host-resident operands, pipelined (proposed or fast scaling, no caller workspace, op(B) = B so
// that its columns are contiguous, n of at least two blocks).  Under these scalings a line's
// shift depends on that line alone (eqs. (proposed-mu), (proposed-nu)), so rows of op(A) and
// columns of op(B) can be scaled, converted and multiplied block by block.  The blocks of C, in
// order: the row blocks A_i of a host-resident op(A) against B's first column block B_0 (one row
// block when A is in device memory, or m is small), then all of A against each later column
// block B_j.  For each block the handle's stream runs the scaling and conversion of its new
// operand block, its residue GEMMs, a copy launched to overlap them that uploads the next
// block's operand block (programmatic dependent launch: the GEMM lets it start once all its
// CTAs are resident, and it takes the room they leave on each SM), then the reconstruction,
// which writes C's block.  The first block's operand blocks are uploaded before it at the link's
// full rate.  Every step computes what the unblocked path computes, so the result is the same
// bits.
//
// Copy engines instead (OZAKI2_OPT_HOST_COPIES = 1, every host operand page-locked): all host
// operand blocks are queued for upload on one copy stream at the start, each awaited by the
// handle's stream where it is first needed; with a host C every block of C is reconstructed
// into a device buffer of its own (uploaded first when beta != 0) and downloaded on a second
// copy stream while the next blocks compute, the last block made small.  No kernel then touches
// host memory.  On GB300 this hides nearly all of the link's traffic when the copy engines run
// at their usual rate, but their rate is erratic (a call now and then takes several times as
// long), so kernels are the default.
constexpr int kPipeMinBlock = 2048;

bool pipeline_applies(const ozaki2_context* ctx, char transB, int n, const void* A,
                      const void* B, const void* C) {
    if (ctx->user_ws || ctx->scaling == OZAKI2_SCALING_ACCURATE || !is_notrans(transB))
        return false;
    if (n < 2 * kPipeMinBlock) return false;
    return host_resident(A) || host_resident(B) || host_resident(C);
}

// Consecutive blocks of lines: block i is [s[i], s[i + 1]); every boundary but the last is a
// multiple of 256 lines.
constexpr int kMaxPipeBlocks = 8;
struct LineBlocks {
    int count = 0;
    int64_t s[kMaxPipeBlocks + 1] = {};
    int64_t start(int i) const { return s[i]; }
    int64_t lines(int i, int64_t) const { return s[i + 1] - s[i]; }
    void add(int64_t len) { s[count + 1] = s[count] + len; ++count; }
};
// `parts` near-equal blocks of the remaining lines, multiples of 256 lines but the last.
void split_even(LineBlocks& b, int64_t total, int parts) {
    const int64_t left = total - b.s[b.count];
    const int64_t size = (left + parts - 1) / parts;
    const int64_t sz = (size + 255) / 256 * 256;
    const int first = b.count;
    while (b.s[b.count] < total) b.add(std::min<int64_t>(sz, total - b.s[b.count]));
    // no sliver at the end: a last block under 256 lines joins the one before it
    if (b.count - first >= 2 && b.s[b.count] - b.s[b.count - 1] < 256) {
        b.s[b.count - 1] = b.s[b.count];
        --b.count;
    }
}
// Column blocks of B: 2 or 4 (4 from 4 kPipeMinBlock lines).  small_tail: the same over all but
// a last block of about lines / 16 (256 to 1024 lines, and what rounding the others to multiples
// of 256 leaves).
LineBlocks line_blocks(int lines, bool small_tail) {
    LineBlocks b;
    int64_t body = lines;
    if (small_tail) {
        const int64_t want = ((int64_t)lines / 16 + 255) / 256 * 256;
        const int64_t tail = std::min<int64_t>(1024, std::max<int64_t>(256, want));
        body = (lines - tail) / 256 * 256;
    }
    split_even(b, body, body / (2 * kPipeMinBlock) >= 2 ? 4 : 2);
    if (body < lines) b.add(lines - body);
    return b;
}
// Row blocks of a host-resident op(A): 1024 rows, then twice as many while that stays below a
// quarter of the rows, then the rest in near-equal blocks of about a quarter.  The pipeline
// cannot start before the first row block and B's first column block are uploaded, and each
// later row block is uploaded beside the residue GEMMs of the one before, which take about
// twice as long per row as its upload: small first blocks growing by two shorten the fill.
LineBlocks row_blocks(int lines) {
    LineBlocks b;
    const int64_t cap = ((int64_t)lines / 4 + 255) / 256 * 256;
    for (int64_t size = 1024; size < cap && lines - b.s[b.count] > 2 * size; size *= 2)
        b.add(size);
    const int64_t left = lines - b.s[b.count];
    const int parts = (int)std::min<int64_t>(kMaxPipeBlocks - b.count,
                                             std::max<int64_t>(1, (left + cap - 1) / cap));
    split_even(b, lines, parts);
    return b;
}

// The copy of a band of lines of a column-major operand into a compact device buffer at dst:
// rows [r0, r0 + h) of op(A) (lines_adjacent: op(A) = A) or columns [r0, r0 + h) of a k x n B.
// The device pitch is a multiple of 16 bytes.
Copy2D band_copy(void* dst, const void* X, int64_t ld, bool lines_adjacent, int64_t r0,
                 int64_t h, int k, size_t esz) {
    Copy2D c;
    c.dst = dst;
    if (lines_adjacent) {  // a run per column of A, h elements of it
        c.src = static_cast<const char*>(X) + (size_t)r0 * esz;
        c.width = (size_t)h * esz;
        c.height = (size_t)k;
    } else {               // a run per line, k elements
        c.src = static_cast<const char*>(X) + (size_t)r0 * (size_t)ld * esz;
        c.width = (size_t)k * esz;
        c.height = (size_t)h;
    }
    c.spitch = (size_t)ld * esz;
    c.dpitch = (c.width + 15) / 16 * 16;
    return c;
}

int dgemm_pipelined(ozaki2_context* ctx, char transA, int m, int n, int k, double alpha,
                    const void* A, int lda, const void* B, int ldb, double beta, void* C, int ldc,
                    int N, bool f32, const Layout& L, const ModTables* T) {
    int rc;
    cudaStream_t S = ctx->stream;
    const size_t esz = f32 ? 4 : 8;
    const bool host_a = host_resident(A), host_b = host_resident(B);
    const bool a_adj = is_notrans(transA);  // rows of op(A) adjacent in memory
    const bool host_c = host_resident(C);
    // copy engines move the host data when every host operand is page-locked
    const bool ce = ctx->host_copies == 1 && (!host_a || page_locked(A)) &&
                    (!host_b || page_locked(B)) && (!host_c || page_locked(C));
    const bool stage_c = ce && host_c;  // C's blocks reconstructed in device memory
    const LineBlocks cb = line_blocks(n, stage_c);
    LineBlocks rb;
    if (host_a && m >= 2 * kPipeMinBlock) rb = row_blocks(m);
    else rb.add(m);
    if (cb.count > kMaxPipeBlocks || rb.count > kMaxPipeBlocks) return OZAKI2_ERROR_CUDA;
    const int nblk = rb.count + cb.count - 1;  // blocks of C

    // block t of C: rows [r0, r0 + h), columns [c0, c0 + cols) of column block j
    struct Blk {
        int64_t r0, h, c0, cols;
        int j;
    };
    auto blk = [&](int t) {
        if (t < rb.count) return Blk{rb.start(t), rb.lines(t, m), 0, cb.lines(0, n), 0};
        const int j = t - rb.count + 1;
        return Blk{0, (int64_t)m, cb.start(j), cb.lines(j, n), j};
    };

    // device memory: copies of A's row blocks and B's column blocks; B's planes per column block
    // (max(cols, 256) rows each)
    size_t a_off[kMaxPipeBlocks] = {}, b_off[kMaxPipeBlocks] = {}, room = 0;
    auto take = [&](size_t bytes) {
        const size_t o = room;
        room += (size_t)round_up((int64_t)bytes, 256);
        return o;
    };
    Copy2D ab[kMaxPipeBlocks] = {}, bb[kMaxPipeBlocks] = {};
    for (int i = 0; i < rb.count && host_a; ++i) {
        ab[i] = band_copy(nullptr, A, lda, a_adj, rb.start(i), rb.lines(i, m), k, esz);
        a_off[i] = take(ab[i].dpitch * ab[i].height);
    }
    for (int j = 0; j < cb.count && host_b; ++j) {
        bb[j] = band_copy(nullptr, B, ldb, false, cb.start(j), cb.lines(j, n), k, esz);
        b_off[j] = take(bb[j].dpitch * bb[j].height);
    }
    if (room && (rc = ensure_input_stage(ctx, room))) return rc;
    char* stage = static_cast<char*>(ctx->in_ws);
    // a device buffer for each block of C, so that no reconstruction waits for a download
    size_t c_off[2 * kMaxPipeBlocks] = {}, c_room = 0;
    for (int t = 0; stage_c && t < nblk; ++t) {
        const Blk b = blk(t);
        c_off[t] = c_room;
        c_room += (size_t)round_up(b.h * b.cols * (int64_t)esz, 256);
    }
    if (stage_c && (rc = ensure_output_stage(ctx, c_room))) return rc;
    if (ce && (rc = ensure_copy_streams(ctx))) return rc;
    for (int i = 0; i < rb.count && host_a; ++i) ab[i].dst = stage + a_off[i];
    for (int j = 0; j < cb.count && host_b; ++j) bb[j].dst = stage + b_off[j];

    char* ws = static_cast<char*>(ctx->ws);
    int* e = reinterpret_cast<int*>(ws + L.off_e);
    int* f = reinterpret_cast<int*>(ws + L.off_f);
    char* pa = ws + L.off_pa;
    int8_t* res = reinterpret_cast<int8_t*>(ws + L.off_res);
    double* part = reinterpret_cast<double*>(ws + L.off_part);
    const float pp = ctx->scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
    const int64_t pa_row = (int64_t)2 * L.geo.ld;  // bytes per row of a plane
    char* pbj[kMaxPipeBlocks];
    int rows_b[kMaxPipeBlocks];
    {
        char* p = ws + L.off_pb;
        for (int j = 0; j < cb.count; ++j) {
            rows_b[j] = (int)std::max<int64_t>(cb.lines(j, n), 256);
            pbj[j] = p;
            p += (int64_t)2 * N * rows_b[j] * L.geo.ld;
        }
    }
    // scaling and conversion of A's row block i (into the same rows of the planes) and of B's
    // column block j (into its own planes)
    auto prep_a = [&](int i) -> int {
        const int64_t r0 = rb.start(i), h = rb.lines(i, m);
        const void* X = A;
        int64_t ls, es;
        rows_of_op(transA, lda, &ls, &es);
        if (host_a) {
            X = ab[i].dst;
            const int64_t w = (int64_t)(ab[i].dpitch / esz);
            ls = a_adj ? 1 : w;
            es = a_adj ? w : 1;
        }
        const int rows_pad = i + 1 == rb.count ? (int)(L.geo.rows_a - r0) : (int)h;
        int r;
        if ((r = cuda_rc(launch_scale_pair(X, ls, es, (int)h, B, 0, 1, 0, k, pp, T->delta,
                                           e + r0, f, ctx->d_status, S, ctx->scaling, f32,
                                           part))) ||
            (r = cuda_rc(launch_convert(X, ls, es, (int)h, k, e + r0, T->conv, pa + r0 * pa_row,
                                        rows_pad, L.geo.ld, ctx->d_status, S, f32, false,
                                        L.geo.rows_a))))
            return r;
        return OZAKI2_SUCCESS;
    };
    auto prep_b = [&](int j) -> int {
        const int64_t c0 = cb.start(j), cols = cb.lines(j, n);
        const void* X = static_cast<const char*>(B) + (size_t)c0 * ldb * esz;
        int64_t ls = ldb;
        if (host_b) {
            X = bb[j].dst;
            ls = (int64_t)(bb[j].dpitch / esz);
        }
        int r;
        if ((r = cuda_rc(launch_scale_pair(A, 0, 1, 0, X, ls, 1, (int)cols, k, pp, T->delta, e,
                                           f + c0, ctx->d_status, S, ctx->scaling, f32,
                                           part))) ||
            (r = cuda_rc(launch_convert(X, ls, 1, (int)cols, k, f + c0, T->conv, pbj[j],
                                        rows_b[j], L.geo.ld, ctx->d_status, S, f32, false))))
            return r;
        return OZAKI2_SUCCESS;
    };

    // block t of C in host memory, and its device buffer (stage_c)
    auto c_host = [&](const Blk& b) {
        return static_cast<char*>(C) + ((size_t)b.c0 * ldc + (size_t)b.r0) * esz;
    };
    auto c_copy = [&](int t, bool down) {
        const Blk b = blk(t);
        char* h = c_host(b);
        char* d = static_cast<char*>(ctx->out_ws) + c_off[t];
        const size_t hp = (size_t)ldc * esz, dp = (size_t)b.h * esz;
        return down ? Copy2D{h, d, hp, dp, dp, (size_t)b.cols}
                    : Copy2D{d, h, dp, hp, dp, (size_t)b.cols};
    };

    // copy engines: every upload queued now, after the work already on the handle's stream
    // (which may still read the staging buffers); events 0-3 order the streams, 4.. the uploads
    cudaEvent_t* ev = ctx->copy_ev;
    int up_ev[2 * kMaxPipeBlocks][3];  // per block: operand uploads and C's, -1 for none
    for (auto& u : up_ev) u[0] = u[1] = u[2] = -1;
    // on every return, the handle's stream waits for both copy streams
    struct JoinCopies {
        ozaki2_context* ctx;
        bool armed = false;
        ~JoinCopies() {
            if (!armed) return;
            if (cudaEventRecord(ctx->copy_ev[1], ctx->down_stream) == cudaSuccess)
                cudaStreamWaitEvent(ctx->stream, ctx->copy_ev[1], 0);
            if (cudaEventRecord(ctx->copy_ev[2], ctx->up_stream) == cudaSuccess)
                cudaStreamWaitEvent(ctx->stream, ctx->copy_ev[2], 0);
        }
    } join{ctx};
    if (ce) {
        if (cudaEventRecord(ev[0], S) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->up_stream, ev[0], 0) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->down_stream, ev[0], 0) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        join.armed = true;
        int u = 4;
        auto up = [&](const Copy2D& c) -> int {
            if (u >= ozaki2_context::kCopyEvents ||
                cudaMemcpy2DAsync(c.dst, c.dpitch, c.src, c.spitch, c.width, c.height,
                                  cudaMemcpyHostToDevice, ctx->up_stream) != cudaSuccess ||
                cudaEventRecord(ev[u], ctx->up_stream) != cudaSuccess)
                return -1;
            return u++;
        };
        for (int t = 0; t < nblk; ++t) {
            if (t < rb.count && host_a && (up_ev[t][0] = up(ab[t])) < 0) return OZAKI2_ERROR_CUDA;
            if ((t == 0 || t >= rb.count) && host_b && (up_ev[t][1] = up(bb[blk(t).j])) < 0)
                return OZAKI2_ERROR_CUDA;
            if (stage_c && beta != 0.0 && (up_ev[t][2] = up(c_copy(t, false))) < 0)
                return OZAKI2_ERROR_CUDA;
        }
    } else {
        // the first block's operand blocks at the link's full rate
        Copy2D first[2];
        int nf = 0;
        if (host_a) first[nf++] = ab[0];
        if (host_b) first[nf++] = bb[0];
        if ((rc = cuda_rc(launch_copies_2d(first, nf, 4 * ctx->num_sms, false, S)))) return rc;
    }
    auto await = [&](int u) {
        return u < 0 || cudaStreamWaitEvent(S, ev[u], 0) == cudaSuccess;
    };
    for (int t = 0; t < nblk; ++t) {
        const Blk b = blk(t);
        if (!await(up_ev[t][0]) || !await(up_ev[t][1])) return OZAKI2_ERROR_CUDA;
        if (t == 0 && ((rc = prep_a(0)) || (rc = prep_b(0)))) return rc;
        if (t > 0 && (rc = t < rb.count ? prep_a(t) : prep_b(b.j))) return rc;
        const bool last_row = b.r0 + b.h >= m;
        const PlaneGeom geo{last_row ? (int)(L.geo.rows_a - b.r0) : (int)b.h, rows_b[b.j],
                            L.geo.ld, (int)round_up(b.h, 32), (int)round_up(b.cols, 32),
                            L.geo.rows_a};
        int8_t* out = res + b.r0 * L.n_pad + b.c0;
        if ((rc = launch_residue_gemm(N, (int)(last_row ? L.m_pad - b.r0 : b.h),
                                      (int)round_up(b.cols, OZAKI2_ROWS_ALIGN_B), (int)L.k_pad,
                                      geo, pa + b.r0 * pa_row, pbj[b.j], out, T->epi,
                                      ctx->d_status, ctx->num_sms, ctx->chunk_k,
                                      ctx->gemm_variant, S, ctx->wait_limit_ns, L.n_pad,
                                      L.m_pad * L.n_pad, ctx->group_m, ctx->l2_hints)))
            return rc;
        if (!ce) {
            // beside the GEMMs: the next block's operand block in
            const Copy2D* next = nullptr;
            if (t + 1 < rb.count && host_a) next = &ab[t + 1];
            if (t + 1 >= rb.count && t + 1 < nblk && host_b) next = &bb[blk(t + 1).j];
            if (next && (rc = cuda_rc(launch_copies_2d(next, 1, ctx->num_sms, true, S))))
                return rc;
        }
        char* Cd = stage_c ? static_cast<char*>(ctx->out_ws) + c_off[t] : c_host(b);
        const int64_t ldd = stage_c ? b.h : ldc;
        if (!await(up_ev[t][2])) return OZAKI2_ERROR_CUDA;
        if ((rc = cuda_rc(launch_crt(out, L.n_pad, L.m_pad * L.n_pad, (int)b.h, (int)b.cols,
                                     e + b.r0, f + b.c0, alpha, beta, Cd, ldd, *T,
                                     ctx->d_status, S, f32, true))))
            return rc;
        if (stage_c) {
            const Copy2D c = c_copy(t, true);
            if (cudaEventRecord(ev[3], S) != cudaSuccess ||
                cudaStreamWaitEvent(ctx->down_stream, ev[3], 0) != cudaSuccess ||
                cudaMemcpy2DAsync(c.dst, c.dpitch, c.src, c.spitch, c.width, c.height,
                                  cudaMemcpyDeviceToHost, ctx->down_stream) != cudaSuccess)
                return OZAKI2_ERROR_CUDA;
        }
    }
    return OZAKI2_SUCCESS;
}

int dgemm_impl(ozaki2_context* ctx, int argbase, char transA, char transB, int m, int n, int k,
               double alpha, const void* A, int lda, const void* B, int ldb, double beta,
               void* C, int ldc, int N, bool f32 = false) {
    if (!is_trans_char(transA)) return -(argbase + 1);
    if (!is_trans_char(transB)) return -(argbase + 2);
    if (m < 0) return -(argbase + 3);
    if (n < 0) return -(argbase + 4);
    if (k < 0) return -(argbase + 5);
    const int arows = is_notrans(transA) ? m : k;
    const int brows = is_notrans(transB) ? k : n;
    if (lda < (arows > 1 ? arows : 1)) return -(argbase + 8);
    if (ldb < (brows > 1 ? brows : 1)) return -(argbase + 10);
    if (ldc < (m > 1 ? m : 1)) return -(argbase + 13);
    if (N < OZAKI2_MIN_MODULI || N > OZAKI2_MAX_MODULI) return -(argbase + 14);
    if (m > 0 && k > 0 && !A) return -(argbase + 7);
    if (k > 0 && n > 0 && !B) return -(argbase + 9);
    if (m > 0 && n > 0 && !C) return -(argbase + 12);
    if (m == 0 || n == 0) return OZAKI2_SUCCESS;
    if (k > 0 && !addressable(ctx, A)) return -(argbase + 7);
    if (k > 0 && !addressable(ctx, B)) return -(argbase + 9);
    if (!addressable(ctx, C)) return -(argbase + 12);
    if (k == 0 || alpha == 0.0)
        return cuda_rc(launch_scale_c(m, n, beta, C, ldc, ctx->stream, f32));
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE && k > OZAKI2_ACCURATE_MAX_K)
        return OZAKI2_ERROR_TOO_LARGE;

    const ModTables* T = mod_tables(N);
    const Layout L = make_layout(m, n, k, N);
    int rc = ensure_workspace(ctx, L.total);
    if (rc) return rc;
    char* ws = static_cast<char*>(ctx->ws);
    int* e = reinterpret_cast<int*>(ws + L.off_e);
    int* f = reinterpret_cast<int*>(ws + L.off_f);
    void* pa = ws + L.off_pa;
    void* pb = ws + L.off_pb;
    int8_t* res = reinterpret_cast<int8_t*>(ws + L.off_res);
    cudaStream_t st = ctx->stream;

    if (!ctx->timing && pipeline_applies(ctx, transB, n, A, B, C))
        return dgemm_pipelined(ctx, transA, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, N, f32,
                               L, T);

    // Host-resident A or B (page-locked, or pageable on a coherent link) are first copied into
    // device memory by a kernel, so the scaling and the conversion, which each read the inputs,
    // read them from HBM.  A handle with a caller-provided workspace allocates nothing and reads
    // them in place.
    if (!ctx->user_ws) {
        const size_t esz = f32 ? 4 : 8;
        const int acols = is_notrans(transA) ? k : m, bcols = is_notrans(transB) ? n : k;
        const size_t a_span = ((size_t)lda * (size_t)(acols - 1) + (size_t)arows) * esz;
        const size_t b_span = ((size_t)ldb * (size_t)(bcols - 1) + (size_t)brows) * esz;
        const bool stage_a = host_resident(A), stage_b = host_resident(B);
        if (stage_a || stage_b) {
            const size_t a_room = stage_a ? (size_t)round_up((int64_t)a_span, 256) : 0;
            if ((rc = ensure_input_stage(ctx, a_room + (stage_b ? b_span : 0)))) return rc;
            char* p = static_cast<char*>(ctx->in_ws);
            if (stage_a) {
                if ((rc = cuda_rc(launch_stage_in(p, A, a_span, ctx->num_sms, st)))) return rc;
                A = p;
            }
            if (stage_b) {
                if ((rc = cuda_rc(launch_stage_in(p + a_room, B, b_span, ctx->num_sms, st))))
                    return rc;
                B = p + a_room;
            }
        }
    }

    auto mark = [&](int i) {
        if (ctx->timing) cudaEventRecord(ctx->ev[i], st);
    };
    int64_t als, aes, bls, bes;
    rows_of_op(transA, lda, &als, &aes);
    cols_of_op(transB, ldb, &bls, &bes);
    mark(0);
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE) {
        if ((rc = accurate_shifts(ctx, A, als, aes, B, bls, bes, m, n, k, L, *T, e, f, pa, pb,
                                  res, f32)))
            return rc;
    } else {
        const float pp = ctx->scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
        double* part = reinterpret_cast<double*>(ws + L.off_part);
        if ((rc = cuda_rc(launch_scale_pair(A, als, aes, m, B, bls, bes, n, k, pp, T->delta, e,
                                            f, ctx->d_status, st, ctx->scaling, f32, part))))
            return rc;
    }
    mark(1);
    const bool accurate = ctx->scaling == OZAKI2_SCALING_ACCURATE;
    if ((rc = cuda_rc(launch_convert(A, als, aes, m, k, e, T->conv, pa, L.geo.rows_a, L.geo.ld,
                                     ctx->d_status, st, f32, accurate))))
        return rc;
    if ((rc = cuda_rc(launch_convert(B, bls, bes, n, k, f, T->conv, pb, L.geo.rows_b, L.geo.ld,
                                     ctx->d_status, st, f32, accurate))))
        return rc;
    mark(2);
    if ((rc = launch_residue_gemm(N, (int)L.m_pad, (int)L.n_pad, (int)L.k_pad, L.geo, pa, pb, res,
                                  T->epi, ctx->d_status, ctx->num_sms, ctx->chunk_k,
                                  ctx->gemm_variant, st, ctx->wait_limit_ns, 0, 0,
                                  ctx->group_m, ctx->l2_hints)))
        return rc;
    mark(3);
    rc = cuda_rc(launch_crt(res, L.n_pad, L.m_pad * L.n_pad, m, n, e, f, alpha, beta, C, ldc, *T,
                            ctx->d_status, st, f32, true));
    mark(4);
    if (ctx->timing) ctx->timed_call = true;
    return rc;
}

}  // namespace

extern "C" {

int ozaki2_create(ozaki2_handle_t* handle) {
    if (!handle) return -1;
    *handle = nullptr;
    auto* ctx = new ozaki2_context();
    int rc = init_context(ctx);
    if (rc) {
        if (ctx->d_status) cudaFree(ctx->d_status);
        delete ctx;
        return rc;
    }
    *handle = ctx;
    return OZAKI2_SUCCESS;
}

int ozaki2_destroy(ozaki2_handle_t handle) {
    if (!handle) return -1;
    cudaStreamSynchronize(handle->stream);
    if (handle->ws && !handle->user_ws) cudaFree(handle->ws);
    if (handle->in_ws) cudaFree(handle->in_ws);
    if (handle->out_ws) cudaFree(handle->out_ws);
    for (cudaStream_t st : {handle->up_stream, handle->down_stream})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (cudaEvent_t e : handle->copy_ev)
        if (e) cudaEventDestroy(e);
    if (handle->d_status) cudaFree(handle->d_status);
    for (auto& e : handle->ev)
        if (e) cudaEventDestroy(e);
    if (handle->staged) cudaEventDestroy(handle->staged);
    for (int i = 0; i < ozaki2_context::kEncodeRing; ++i) {
        if (handle->enc_staged[i]) cudaEventDestroy(handle->enc_staged[i]);
        if (handle->enc_stage[i]) cudaFreeHost(handle->enc_stage[i]);
    }
    clear_graphs(handle);
    if (handle->capture_stream) cudaStreamDestroy(handle->capture_stream);
    if (handle->stage) cudaFreeHost(handle->stage);
    delete handle;
    return OZAKI2_SUCCESS;
}

int ozaki2_set_stream(ozaki2_handle_t handle, void* stream) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return OZAKI2_SUCCESS;
}

int ozaki2_set_option(ozaki2_handle_t handle, int option, int value) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    switch (option) {
        case OZAKI2_OPT_GEMM_VARIANT:
            if (value < OZAKI2_GEMM_AUTO || value > OZAKI2_GEMM_PAIR) return -3;
            ctx->gemm_variant = value;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_CHUNK_K:
            if (value < 64 || value > 960 || value % 64) return -3;
            if (value != ctx->chunk_k) clear_graphs(ctx);
            ctx->chunk_k = value;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_GRAPH:
            if (value != 0 && value != 1) return -3;
            if (!value) clear_graphs(ctx);
            ctx->use_graphs = value != 0;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_SCALING:
            if (value != OZAKI2_SCALING_PROPOSED && value != OZAKI2_SCALING_FAST &&
                value != OZAKI2_SCALING_ACCURATE)
                return -3;
            ctx->scaling = value;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_WAIT_LIMIT_NS:
            if (value < 0) return -3;
            ctx->wait_limit_ns = (unsigned long long)value;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_L2_HINTS:
            if (value < 0 || value > 15 || (value & 3) == 3 || (value >> 2) == 3) return -3;
            ctx->l2_hints = value;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_HOST_COPIES:
            if (value != 0 && value != 1) return -3;
            ctx->host_copies = value;
            return OZAKI2_SUCCESS;
        case OZAKI2_OPT_GROUP_M:
            if (value < 0 || value > 1024) return -3;
            ctx->group_m = value;
            return OZAKI2_SUCCESS;
        default:
            return -2;
    }
}

int ozaki2_set_workspace(ozaki2_handle_t handle, void* workspace, size_t bytes) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255u)) return -2;
    if (ctx->ws && !ctx->user_ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
    }
    ctx->ws = workspace;
    ctx->ws_bytes = workspace ? bytes : 0;
    ctx->user_ws = workspace != nullptr;
    return OZAKI2_SUCCESS;
}

size_t ozaki2_workspace_size(int m, int n, int k, int num_moduli) {
    if (m < 0 || n < 0 || k < 0 || num_moduli < OZAKI2_MIN_MODULI ||
        num_moduli > OZAKI2_MAX_MODULI)
        return 0;
    return make_layout(m, n, k, num_moduli).total;
}

int ozaki2_get_status(ozaki2_handle_t handle, unsigned* flags) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (!flags) return -2;
    unsigned v = 0;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    if (cudaMemcpy(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    if (cudaMemset(ctx->d_status, 0, sizeof(v)) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    *flags = v;
    return OZAKI2_SUCCESS;
}

int ozaki2_set_timing(ozaki2_handle_t handle, int on) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (on && !ctx->ev[0]) {
        for (auto& e : ctx->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    }
    ctx->timing = on != 0;
    return OZAKI2_SUCCESS;
}

int ozaki2_get_timing(ozaki2_handle_t handle, float* ms) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (!ms) return -2;
    if (!ctx->timed_call) return OZAKI2_ERROR_CUDA;
    if (cudaEventSynchronize(ctx->ev[4]) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    for (int i = 0; i < 4; ++i)
        if (cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
    return OZAKI2_SUCCESS;
}

const char* ozaki2_error_string(int code) {
    if (code < 0) return "invalid argument";
    switch (code) {
        case OZAKI2_SUCCESS: return "success";
        case OZAKI2_ERROR_CUDA: return "CUDA runtime error";
        case OZAKI2_ERROR_ALLOC: return "workspace allocation failed";
        case OZAKI2_ERROR_WORKSPACE: return "user workspace too small";
        case OZAKI2_ERROR_NO_DEVICE: return "no sm_103 GPU available";
        case OZAKI2_ERROR_DRIVER: return "tensor map encoder unavailable or failed";
        case OZAKI2_ERROR_TOO_LARGE:
            return "problem exceeds the static scratch of ozaki2_dgemm_noalloc, or k exceeds "
                   "OZAKI2_ACCURATE_MAX_K in accurate mode";
        case OZAKI2_ERROR_MODE: return "entry point not available in the handle's scaling mode";
        default: return "unknown error";
    }
}

int ozaki2_constants(int num_moduli, int* moduli, int* inverses, float* pprime) {
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -1;
    if (!moduli) return -2;
    if (!inverses) return -3;
    if (!pprime) return -4;
    for (int l = 0; l < num_moduli; ++l) {
        moduli[l] = T->moduli[l];
        inverses[l] = T->inverses[l];
    }
    *pprime = T->pprime;
    return OZAKI2_SUCCESS;
}

int ozaki2_dgemm(char transA, char transB, int m, int n, int k, double alpha, const double* A,
                 int lda, const double* B, int ldb, double beta, double* C, int ldc,
                 int num_moduli) {
    ozaki2_context* ctx;
    int rc = resolve(nullptr, &ctx);
    if (rc) return rc;
    return dgemm_impl(ctx, 0, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                      num_moduli);
}

int ozaki2_dgemm_h(ozaki2_handle_t handle, char transA, char transB, int m, int n, int k,
                   double alpha, const double* A, int lda, const double* B, int ldb,
                   double beta, double* C, int ldc, int num_moduli) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    return dgemm_impl(ctx, 1, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                      num_moduli);
}

int ozaki2_sgemm(char transA, char transB, int m, int n, int k, float alpha, const float* A,
                 int lda, const float* B, int ldb, float beta, float* C, int ldc,
                 int num_moduli) {
    ozaki2_context* ctx;
    int rc = resolve(nullptr, &ctx);
    if (rc) return rc;
    return dgemm_impl(ctx, 0, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                      num_moduli, true);
}

int ozaki2_sgemm_h(ozaki2_handle_t handle, char transA, char transB, int m, int n, int k,
                   float alpha, const float* A, int lda, const float* B, int ldb, float beta,
                   float* C, int ldc, int num_moduli) {
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    return dgemm_impl(ctx, 1, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                      num_moduli, true);
}

size_t ozaki2_grouped_workspace_size(int count, const ozaki2_problem* problems) {
    if (count < 0 || (count > 0 && !problems)) return 0;
    if (grouped_check(count, problems)) return 0;
    return grouped_workspace_bytes(count, problems);
}

static int grouped_impl(ozaki2_handle_t handle, int count, const ozaki2_problem* problems,
                        const Encoded& enc) {
    if (count < 0) return -2;
    if (count > 0 && !problems) return -3;
    int rc = grouped_check(count, problems);
    if (rc) return rc;
    if (count == 0) return OZAKI2_SUCCESS;
    const bool encoded = enc.a || enc.b;
    ozaki2_context* ctx;
    if ((rc = resolve(handle, &ctx))) return rc;
    if (encoded && ctx->scaling == OZAKI2_SCALING_ACCURATE) return OZAKI2_ERROR_MODE;
    if ((rc = ensure_workspace(ctx, grouped_workspace_bytes(count, problems, enc)))) return rc;
    if (!ctx->staged &&
        cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    for (int i = 0; ctx->scaling == OZAKI2_SCALING_ACCURATE && i < count; ++i)
        if (problems[i].k > OZAKI2_ACCURATE_MAX_K) return OZAKI2_ERROR_TOO_LARGE;
    const size_t tb =
        (size_t)grouped_table_bytes(count, problems, ctx->tiles, ctx->chunk_k, ctx->scaling, enc);
    char* ws = static_cast<char*>(ctx->ws);
    auto operands_ok = [&]() {
        for (int i = 0; i < count; ++i) {
            const ozaki2_problem& p = problems[i];
            if (p.m <= 0 || p.n <= 0 || p.k <= 0 || p.alpha == 0.0) continue;
            const bool has_a = enc.a && enc.a[i], has_b = enc.b && enc.b[i];
            if (!has_a && !addressable(ctx, p.A)) return -(100 * (i + 1) + 7);
            if (!has_b && !addressable(ctx, p.B)) return -(100 * (i + 1) + 9);
            if (!addressable(ctx, p.C)) return -(100 * (i + 1) + 12);
        }
        return 0;
    };
    if (ctx->use_graphs && !encoded) {
        for (auto& g : ctx->graphs)
            if (g.chunk_k == ctx->chunk_k && g.scaling == ctx->scaling &&
                g.wait_limit_ns == ctx->wait_limit_ns && same_problems(g.probs, count, problems))
                return cudaGraphLaunch(g.exec, ctx->stream) == cudaSuccess ? OZAKI2_SUCCESS
                                                                            : OZAKI2_ERROR_CUDA;
        // First call with these problems: check the operands, upload the tables to a buffer of
        // their own, capture the launches once, keep the instantiated graph.
        if ((rc = operands_ok())) return rc;
        ozaki2_context::GraphEntry g;
        g.probs.assign(problems, problems + count);
        g.chunk_k = ctx->chunk_k;
        g.scaling = ctx->scaling;
        g.wait_limit_ns = ctx->wait_limit_ns;
        std::vector<char> host(tb ? tb : 1);
        if ((rc = build_grouped_tables(count, problems, ws, host.data(), ctx->tiles,
                                       ctx->chunk_k, ctx->scaling)))
            return rc;
        if (cudaMalloc(&g.tables, tb ? tb : 1) != cudaSuccess) {
            cudaGetLastError();
            return OZAKI2_ERROR_ALLOC;
        }
        if (cudaMemcpy(g.tables, host.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(g.tables);
            return OZAKI2_ERROR_CUDA;
        }
        if (!ctx->capture_stream &&
            cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaFree(g.tables);
            return OZAKI2_ERROR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess) {
            cudaFree(g.tables);
            return OZAKI2_ERROR_CUDA;
        }
        rc = launch_grouped(count, problems, static_cast<const char*>(g.tables), ctx->d_status,
                            ctx->num_sms, ctx->tiles, ctx->chunk_k, ctx->capture_stream,
                            ctx->scaling, ctx->wait_limit_ns);
        const cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (rc || ce != cudaSuccess ||
            cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaFree(g.tables);
            cudaGetLastError();
            return rc ? rc : OZAKI2_ERROR_CUDA;
        }
        cudaGraphDestroy(graph);
        ctx->graphs.push_back(std::move(g));
        return cudaGraphLaunch(ctx->graphs.back().exec, ctx->stream) == cudaSuccess
                   ? OZAKI2_SUCCESS
                   : OZAKI2_ERROR_CUDA;
    }
    if ((rc = operands_ok())) return rc;
    if (ctx->stage_bytes < tb) {
        if (cudaEventSynchronize(ctx->staged) != cudaSuccess) return OZAKI2_ERROR_CUDA;
        if (ctx->stage) cudaFreeHost(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (cudaMallocHost(&ctx->stage, tb) != cudaSuccess) {
            cudaGetLastError();
            return OZAKI2_ERROR_ALLOC;
        }
        ctx->stage_bytes = tb;
    }
    // the staging buffer may still be read by the previous call's copy
    if (cudaEventSynchronize(ctx->staged) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    if ((rc = build_grouped_tables(count, problems, ws, ctx->stage, ctx->tiles, ctx->chunk_k,
                                   ctx->scaling, enc)))
        return rc;
    char* tables_dev = grouped_tables_in_workspace(count, problems, ws, enc);
    if (tb && (cudaMemcpyAsync(tables_dev, ctx->stage, tb, cudaMemcpyHostToDevice,
                               ctx->stream) != cudaSuccess ||
               cudaEventRecord(ctx->staged, ctx->stream) != cudaSuccess))
        return OZAKI2_ERROR_CUDA;
    return launch_grouped(count, problems, tables_dev, ctx->d_status, ctx->num_sms, ctx->tiles,
                          ctx->chunk_k, ctx->stream, ctx->scaling, ctx->wait_limit_ns, enc);
}

int ozaki2_dgemm_grouped(ozaki2_handle_t handle, int count, const ozaki2_problem* problems) {
    return grouped_impl(handle, count, problems, Encoded());
}

// 0 if every encoded operand matches its problem, else the negative error of the first that
// does not (argument 7 for op(A), 9 for op(B) of problem i).
static int check_encoded(int count, const ozaki2_problem* problems,
                         const ozaki2_operand* const* enc_a, const ozaki2_operand* const* enc_b,
                         int scaling) {
    auto bad = [&](const ozaki2_operand* o, bool side_b, const ozaki2_problem& p) {
        const bool sb = o->side == 'B' || o->side == 'b';
        const bool sa = o->side == 'A' || o->side == 'a';
        return (side_b ? !sb : !sa) || o->lines != (side_b ? p.n : p.m) || o->k != p.k ||
               o->num_moduli != p.num_moduli || o->scaling != scaling || !o->data ||
               (reinterpret_cast<uintptr_t>(o->data) & 255u);
    };
    for (int i = 0; i < count; ++i) {
        if (enc_a && enc_a[i] && bad(enc_a[i], false, problems[i])) return -(100 * (i + 1) + 7);
        if (enc_b && enc_b[i] && bad(enc_b[i], true, problems[i])) return -(100 * (i + 1) + 9);
    }
    return OZAKI2_SUCCESS;
}

int ozaki2_dgemm_grouped_encoded(ozaki2_handle_t handle, int count,
                                 const ozaki2_problem* problems,
                                 const ozaki2_operand* const* enc_a,
                                 const ozaki2_operand* const* enc_b) {
    if (count < 0) return -2;
    if (count > 0 && !problems) return -3;
    int rc = grouped_check(count, problems);
    if (rc) return rc;
    ozaki2_context* ctx;
    if ((rc = resolve(handle, &ctx))) return rc;
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE && (enc_a || enc_b)) return OZAKI2_ERROR_MODE;
    if ((rc = check_encoded(count, problems, enc_a, enc_b, ctx->scaling))) return rc;
    Encoded enc;
    enc.a = enc_a;
    enc.b = enc_b;
    return grouped_impl(handle, count, problems, enc);
}

size_t ozaki2_grouped_encoded_workspace_size(int count, const ozaki2_problem* problems,
                                             const ozaki2_operand* const* enc_a,
                                             const ozaki2_operand* const* enc_b) {
    if (count < 0 || (count > 0 && !problems)) return 0;
    if (grouped_check(count, problems)) return 0;
    Encoded enc;
    enc.a = enc_a;
    enc.b = enc_b;
    return grouped_workspace_bytes(count, problems, enc);
}

size_t ozaki2_operand_bytes(char side, int lines, int k, int num_moduli) {
    const bool a = side == 'A' || side == 'a', b = side == 'B' || side == 'b';
    if ((!a && !b) || lines < 0 || k < 0 || !mod_tables(num_moduli)) return 0;
    return (size_t)operand_layout(b, lines, k, num_moduli).bytes;
}

int ozaki2_encode_operands(ozaki2_handle_t handle, int count, ozaki2_operand* ops) {
    if (count < 0) return -2;
    if (count > 0 && !ops) return -3;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE) return OZAKI2_ERROR_MODE;
    for (int i = 0; i < count; ++i) {
        ozaki2_operand& o = ops[i];
        const int e = -(100 * (i + 1));
        const bool sa = o.side == 'A' || o.side == 'a', sb = o.side == 'B' || o.side == 'b';
        if (!sa && !sb) return e - 1;
        if (!is_trans_char(o.trans)) return e - 2;
        if (o.lines < 0) return e - 3;
        if (o.k < 0) return e - 4;
        // rows of the stored matrix: op(A) m x k is A (m x k) or A^T; op(B) k x n likewise
        const bool nt = is_notrans(o.trans);
        const int stored_rows = sa ? (nt ? o.lines : o.k) : (nt ? o.k : o.lines);
        if (o.lines > 0 && o.k > 0 && !o.X) return e - 5;
        if (o.ld < (stored_rows > 1 ? stored_rows : 1)) return e - 6;
        if (!mod_tables(o.num_moduli)) return e - 7;
        if (!o.data || (reinterpret_cast<uintptr_t>(o.data) & 255u)) return e - 8;
        if (o.lines > 0 && o.k > 0 && !addressable(ctx, o.X)) return e - 5;
        if (host_resident(o.data)) return e - 8;
        o.scaling = ctx->scaling;
    }
    if (count == 0) return OZAKI2_SUCCESS;
    // lines of length 0: zero shifts, zero planes (no kernel touches them otherwise)
    for (int i = 0; i < count; ++i) {
        const ozaki2_operand& o = ops[i];
        if (o.lines > 0 && o.k == 0) {
            const OperandLayout L = operand_layout(o.side == 'B' || o.side == 'b', o.lines, 0,
                                                   o.num_moduli);
            if (cudaMemsetAsync(o.data, 0, (size_t)L.bytes, ctx->stream) != cudaSuccess)
                return OZAKI2_ERROR_CUDA;
        }
    }
    // Host-resident matrices (page-locked, or pageable on a coherent link) are first copied into
    // device memory by a kernel, as ozaki2_dgemm does, so the scaling and the conversion read
    // them from HBM (the link is crossed once); with a caller workspace they are read in place.
    std::vector<ozaki2_operand> staged(ops, ops + count);
    if (!ctx->user_ws) {
        size_t total = 0;
        std::vector<size_t> span(count, 0);
        for (int i = 0; i < count; ++i) {
            const ozaki2_operand& o = ops[i];
            if (o.lines <= 0 || o.k <= 0 || !host_resident(o.X)) continue;
            const bool sa = o.side == 'A' || o.side == 'a', nt = is_notrans(o.trans);
            const int64_t rows = sa ? (nt ? o.lines : o.k) : (nt ? o.k : o.lines);
            const int64_t cols = sa ? (nt ? o.k : o.lines) : (nt ? o.lines : o.k);
            span[i] = (size_t)((int64_t)o.ld * (cols - 1) + rows) * sizeof(double);
            total += (size_t)round_up((int64_t)span[i], 256);
        }
        if (total) {
            if ((rc = ensure_input_stage(ctx, total))) return rc;
            char* p = static_cast<char*>(ctx->in_ws);
            for (int i = 0; i < count; ++i) {
                if (!span[i]) continue;
                if ((rc = cuda_rc(launch_stage_in(p, ops[i].X, span[i], ctx->num_sms,
                                                  ctx->stream))))
                    return rc;
                staged[i].X = reinterpret_cast<const double*>(p);
                p += round_up((int64_t)span[i], 256);
            }
        }
    }
    ops = staged.data();
    const size_t tb = (size_t)encode_table_bytes(count, ops);
    // the device copy of the tables lives in the workspace; earlier calls on this stream have
    // read theirs before this call's copy lands (stream order)
    if ((rc = ensure_workspace(ctx, tb))) return rc;
    const int slot = ctx->enc_next;
    ctx->enc_next = (slot + 1) % ozaki2_context::kEncodeRing;
    cudaEvent_t& ev = ctx->enc_staged[slot];
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    if (cudaEventSynchronize(ev) != cudaSuccess) return OZAKI2_ERROR_CUDA;
    if (ctx->enc_stage_bytes[slot] < tb) {
        if (ctx->enc_stage[slot]) cudaFreeHost(ctx->enc_stage[slot]);
        ctx->enc_stage[slot] = nullptr;
        ctx->enc_stage_bytes[slot] = 0;
        if (cudaMallocHost(&ctx->enc_stage[slot], tb) != cudaSuccess) {
            cudaGetLastError();
            return OZAKI2_ERROR_ALLOC;
        }
        ctx->enc_stage_bytes[slot] = tb;
    }
    char* host = ctx->enc_stage[slot];
    build_encode_tables(count, ops, ctx->scaling, host);
    char* tables_dev = static_cast<char*>(ctx->ws);
    if (cudaMemcpyAsync(tables_dev, host, tb, cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess ||
        cudaEventRecord(ev, ctx->stream) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    return launch_encode(count, ops, tables_dev, ctx->d_status, ctx->stream, ctx->scaling);
}


int ozaki2_set_grouped_tiles(ozaki2_handle_t handle, int count, const int* n_max,
                             const int* k_max, const int* tile_n, const int* chunk_k) {
    if (count < 0 || count > OZAKI2_MAX_TILE_RULES) return -2;
    if (count > 0 && !n_max) return -3;
    if (count > 0 && !k_max) return -4;
    if (count > 0 && !tile_n) return -5;
    if (count > 0 && !chunk_k) return -6;
    TileRules r;
    r.count = count;
    for (int i = 0; i < count; ++i) {
        const int tn = tile_n[i], ck = chunk_k[i];
        if (tn != 64 && tn != 128 && tn != 256) return -5;
        if (ck != 0 && (ck < 64 || ck > 960 || ck % 64)) return -6;
        r.r[i] = TileRule{n_max[i], k_max[i], tn, ck};
    }
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    clear_graphs(ctx);
    ctx->tiles = r;
    return OZAKI2_SUCCESS;
}

// Scratch for the norm-block sums of lines longer than one block (the handle's workspace), or
// NULL when none is needed or a caller workspace is too small (then one thread per line).
static double* partials_scratch(ozaki2_context* ctx, int lines, int len) {
    const size_t bytes = scale_partials_bytes(lines, len);
    if (!bytes || ensure_workspace(ctx, bytes) != OZAKI2_SUCCESS) return nullptr;
    return static_cast<double*>(ctx->ws);
}

int ozaki2_scale_a(ozaki2_handle_t handle, char transA, int m, int k, const double* A, int lda,
                   int num_moduli, int* shifts) {
    if (!is_trans_char(transA)) return -2;
    if (m < 0) return -3;
    if (k < 0) return -4;
    const int rows = is_notrans(transA) ? m : k;
    if (lda < (rows > 1 ? rows : 1)) return -6;
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -7;
    if (m > 0 && k > 0 && !A) return -5;
    if (m > 0 && !shifts) return -8;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    int64_t ls, es;
    rows_of_op(transA, lda, &ls, &es);
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE) return OZAKI2_ERROR_MODE;
    const float pp = ctx->scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
    return cuda_rc(launch_scale(A, ls, es, m, k, pp, shifts, ctx->d_status, ctx->stream,
                                ctx->scaling, T->delta, partials_scratch(ctx, m, k)));
}

int ozaki2_scale_b(ozaki2_handle_t handle, char transB, int k, int n, const double* B, int ldb,
                   int num_moduli, int* shifts) {
    if (!is_trans_char(transB)) return -2;
    if (k < 0) return -3;
    if (n < 0) return -4;
    const int rows = is_notrans(transB) ? k : n;
    if (ldb < (rows > 1 ? rows : 1)) return -6;
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -7;
    if (n > 0 && k > 0 && !B) return -5;
    if (n > 0 && !shifts) return -8;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    int64_t ls, es;
    cols_of_op(transB, ldb, &ls, &es);
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE) return OZAKI2_ERROR_MODE;
    const float pp = ctx->scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
    return cuda_rc(launch_scale(B, ls, es, n, k, pp, shifts, ctx->d_status, ctx->stream,
                                ctx->scaling, T->delta, partials_scratch(ctx, n, k)));
}

int ozaki2_scale_norms(ozaki2_handle_t handle, char side, char trans, int lines, int k,
                       const double* X, int ld, int num_moduli, int* shifts, double* norms) {
    const bool is_a = side == 'A' || side == 'a';
    if (!is_a && side != 'B' && side != 'b') return -2;
    if (!is_trans_char(trans)) return -3;
    if (lines < 0) return -4;
    if (k < 0) return -5;
    if (lines > 0 && k > 0 && !X) return -6;
    // rows of the stored matrix: op(A) = A is lines x k, op(B) = B is k x lines
    const int rows = is_a == is_notrans(trans) ? lines : k;
    if (ld < (rows > 1 ? rows : 1)) return -7;
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -8;
    if (lines > 0 && !shifts) return -9;
    if (lines > 0 && !norms) return -10;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (ctx->scaling == OZAKI2_SCALING_ACCURATE) return OZAKI2_ERROR_MODE;
    if (lines == 0) return OZAKI2_SUCCESS;
    int64_t ls, es;
    if (is_a) rows_of_op(trans, ld, &ls, &es);
    else cols_of_op(trans, ld, &ls, &es);
    const float pp = ctx->scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
    double* part = partials_scratch(ctx, lines, k);
    if (is_a)
        return cuda_rc(launch_scale_pair(X, ls, es, lines, nullptr, 0, 1, 0, k, pp, T->delta,
                                         shifts, nullptr, ctx->d_status, ctx->stream,
                                         ctx->scaling, false, part, norms, nullptr));
    return cuda_rc(launch_scale_pair(nullptr, 0, 1, 0, X, ls, es, lines, k, pp, T->delta, nullptr,
                                     shifts, ctx->d_status, ctx->stream, ctx->scaling, false,
                                     part, nullptr, norms));
}

int ozaki2_scale_accurate(ozaki2_handle_t handle, char transA, char transB, int m, int n, int k,
                          const double* A, int lda, const double* B, int ldb, int num_moduli,
                          int* e, int* f, unsigned* cmax) {
    if (!is_trans_char(transA)) return -2;
    if (!is_trans_char(transB)) return -3;
    if (m < 0) return -4;
    if (n < 0) return -5;
    if (k < 0) return -6;
    const int arows = is_notrans(transA) ? m : k;
    const int brows = is_notrans(transB) ? k : n;
    if (m > 0 && k > 0 && !A) return -7;
    if (lda < (arows > 1 ? arows : 1)) return -8;
    if (k > 0 && n > 0 && !B) return -9;
    if (ldb < (brows > 1 ? brows : 1)) return -10;
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -11;
    if (m > 0 && !e) return -12;
    if (n > 0 && !f) return -13;
    if (k > OZAKI2_ACCURATE_MAX_K) return OZAKI2_ERROR_TOO_LARGE;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    if (m == 0 && n == 0) return OZAKI2_SUCCESS;
    // A-bar, B-bar and the maxima use the layout of a one-modulus product
    const Layout L = make_layout(m, n, k, 1);
    if ((rc = ensure_workspace(ctx, L.total))) return rc;
    char* ws = static_cast<char*>(ctx->ws);
    int64_t als, aes, bls, bes;
    rows_of_op(transA, lda, &als, &aes);
    cols_of_op(transB, ldb, &bls, &bes);
    if (k == 0) {  // no products: every line is a zero line
        if (m > 0 && cudaMemsetAsync(e, 0, sizeof(int) * (size_t)m, ctx->stream) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        if (n > 0 && cudaMemsetAsync(f, 0, sizeof(int) * (size_t)n, ctx->stream) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        if (cmax &&
            cudaMemsetAsync(cmax, 0, sizeof(unsigned) * ((size_t)m + n), ctx->stream) !=
                cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        return OZAKI2_SUCCESS;
    }
    void* region = ws + L.off_res;
    if ((rc = accurate_shifts(ctx, A, als, aes, B, bls, bes, m, n, k, L, *T, e, f, ws + L.off_pa,
                              ws + L.off_pb, region)))
        return rc;
    if (cmax) {
        const auto* src = static_cast<const uint32_t*>(region);
        if ((m > 0 && cudaMemcpyAsync(cmax, src, sizeof(uint32_t) * (size_t)m,
                                      cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) ||
            (n > 0 && cudaMemcpyAsync(cmax + m, src + L.m_pad, sizeof(uint32_t) * (size_t)n,
                                      cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess))
            return OZAKI2_ERROR_CUDA;
    }
    return OZAKI2_SUCCESS;
}

static int convert_common(ozaki2_handle_t handle, bool is_a, char trans, int lines, int len,
                          const double* X, int ld, const int* shifts, int num_moduli,
                          void* planes, int rows_pad, int k_pad) {
    const int rows = is_a ? (is_notrans(trans) ? lines : len) : (is_notrans(trans) ? len : lines);
    if (ld < (rows > 1 ? rows : 1)) return -6;
    if (!mod_tables(num_moduli)) return -8;
    if (lines > 0 && len > 0 && !X) return -5;
    if (lines > 0 && !shifts) return -7;
    const int align = is_a ? OZAKI2_ROWS_ALIGN_A : OZAKI2_ROWS_ALIGN_B;
    if (rows_pad < lines || rows_pad % align) return -10;
    if (k_pad < len || k_pad % OZAKI2_K_ALIGN) return -11;
    if (!planes || (reinterpret_cast<uintptr_t>(planes) & 15u)) return -9;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    int64_t ls, es;
    if (is_a) rows_of_op(trans, ld, &ls, &es);
    else cols_of_op(trans, ld, &ls, &es);
    // the shifts may come from any scaling mode: use the limb count that covers them all
    return cuda_rc(launch_convert(X, ls, es, lines, len, shifts, mod_tables(num_moduli)->conv,
                                  planes, rows_pad, k_pad, ctx->d_status, ctx->stream, false,
                                  true));
}

int ozaki2_convert_a(ozaki2_handle_t handle, char transA, int m, int k, const double* A, int lda,
                     const int* shifts, int num_moduli, void* planes, int rows_pad, int k_pad) {
    if (!is_trans_char(transA)) return -2;
    if (m < 0) return -3;
    if (k < 0) return -4;
    return convert_common(handle, true, transA, m, k, A, lda, shifts, num_moduli, planes,
                          rows_pad, k_pad);
}

int ozaki2_convert_b(ozaki2_handle_t handle, char transB, int k, int n, const double* B, int ldb,
                     const int* shifts, int num_moduli, void* planes, int rows_pad, int k_pad) {
    if (!is_trans_char(transB)) return -2;
    if (k < 0) return -3;
    if (n < 0) return -4;
    return convert_common(handle, false, transB, n, k, B, ldb, shifts, num_moduli, planes,
                          rows_pad, k_pad);
}

int ozaki2_residue_gemm(ozaki2_handle_t handle, int num_moduli, int m_pad, int n_pad, int k_pad,
                        const void* planes_a, const void* planes_b, int8_t* residues) {
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -2;
    if (m_pad < 0 || m_pad % OZAKI2_ROWS_ALIGN_A) return -3;
    if (n_pad < 0 || n_pad % OZAKI2_ROWS_ALIGN_B) return -4;
    if (k_pad < 0 || k_pad % OZAKI2_K_ALIGN) return -5;
    const bool work = m_pad > 0 && n_pad > 0;
    if (work && k_pad > 0 && (!planes_a || (reinterpret_cast<uintptr_t>(planes_a) & 15u))) return -6;
    if (work && k_pad > 0 && (!planes_b || (reinterpret_cast<uintptr_t>(planes_b) & 15u))) return -7;
    if (work && (!residues || (reinterpret_cast<uintptr_t>(residues) & 15u))) return -8;
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    // the caller's padded layout, every product residue stored
    const PlaneGeom geo{m_pad, n_pad, k_pad, m_pad, n_pad};
    return launch_residue_gemm(num_moduli, m_pad, n_pad, k_pad, geo, planes_a, planes_b, residues,
                               T->epi, ctx->d_status, ctx->num_sms, ctx->chunk_k,
                               ctx->gemm_variant, ctx->stream, ctx->wait_limit_ns, 0, 0,
                               ctx->group_m);
}

int ozaki2_crt(ozaki2_handle_t handle, int num_moduli, int m, int n, const int8_t* residues,
               int ldr, long long plane_stride, const int* shifts_a, const int* shifts_b,
               double alpha, double beta, double* C, int ldc) {
    const ModTables* T = mod_tables(num_moduli);
    if (!T) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (ldr < (n > 1 ? n : 1)) return -6;
    if (plane_stride < (long long)m * ldr) return -7;
    if (ldc < (m > 1 ? m : 1)) return -13;
    if (m > 0 && n > 0) {
        if (!residues) return -5;
        if (!shifts_a) return -8;
        if (!shifts_b) return -9;
        if (!C) return -12;
    }
    ozaki2_context* ctx;
    int rc = resolve(handle, &ctx);
    if (rc) return rc;
    return cuda_rc(launch_crt(residues, ldr, plane_stride, m, n, shifts_a, shifts_b, alpha, beta,
                              C, ldc, *T, ctx->d_status, ctx->stream));
}

}  // extern "C"
