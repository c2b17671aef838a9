// grouped.cu -- many independent emulated DGEMMs in one set of launches: one grouped scaling
// launch, one grouped conversion launch per moduli count, one persistent residue-GEMM launch over
// the tiles of every problem, and one grouped CRT launch per moduli count.  The per-problem
// descriptors and per-block work tables are built on the host, staged in pinned memory and
// copied to the workspace with one asynchronous copy.  Each problem goes through exactly the
// arithmetic of ozaki2_dgemm (Steps 1-4 of Section 2.2 with the scaling of Section 4), so its
// result is bit-identical to a separate call.
#include <string.h>

#include <algorithm>
#include <vector>

#include "ozaki2_internal.h"

namespace ozaki2 {
namespace {

int64_t round_up64(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
bool trans_ok(char c) {
    return c == 'N' || c == 'n' || c == 'T' || c == 't' || c == 'C' || c == 'c';
}
bool notrans(char c) { return c == 'N' || c == 'n'; }

// 0 if the problem is valid, else the number of the offending argument of ozaki2_dgemm.
int check_problem(const ozaki2_problem& p) {
    if (!trans_ok(p.transA)) return 1;
    if (!trans_ok(p.transB)) return 2;
    if (p.m < 0) return 3;
    if (p.n < 0) return 4;
    if (p.k < 0) return 5;
    const int arows = notrans(p.transA) ? p.m : p.k;
    const int brows = notrans(p.transB) ? p.k : p.n;
    if (p.lda < (arows > 1 ? arows : 1)) return 8;
    if (p.ldb < (brows > 1 ? brows : 1)) return 10;
    if (p.ldc < (p.m > 1 ? p.m : 1)) return 13;
    if (!mod_tables(p.num_moduli)) return 14;
    if (p.m > 0 && p.k > 0 && !p.A) return 7;
    if (p.k > 0 && p.n > 0 && !p.B) return 9;
    if (p.m > 0 && p.n > 0 && !p.C) return 12;
    return 0;
}

bool active(const ozaki2_problem& p) {
    return p.m > 0 && p.n > 0 && p.k > 0 && p.alpha != 0.0;
}

struct Plan {
    std::vector<int> idx;           // active problems (indices into the caller's array)
    std::vector<int> bn, chunk;     // tile width and K chunk of each active problem
    std::vector<const ozaki2_operand*> ea, eb;  // encoded op(A) / op(B) of each, or NULL
    std::vector<int64_t> ws_off;    // offset of each active problem's intermediates
    int64_t ws_problems = 0;        // bytes of all intermediates
    // table sections (offsets within the table block)
    int64_t off_gp = 0, off_gg = 0, off_sw = 0, off_cw = 0, off_rw = 0, table_bytes = 0;
    int n_scale = 0, n_conv = 0, n_crt = 0;
    int n_scale_adj = 0;  // scale work items of adjacent lines (first in the list)
    std::vector<int> conv_n, conv_begin, conv_count;  // per distinct N: blocks in the table
    std::vector<int> crt_begin, crt_count;
    int total_tiles = 0;
    // accurate mode: one auxiliary-product descriptor per problem (C-bar = A-bar B-bar)
    bool accurate = false;
    int64_t off_ga = 0;
    int aux_tiles = 0;
};

// Bytes of one problem's intermediates, laid out for 256-wide tiles (the largest layout: with a
// narrower tile the B planes and product residues use a prefix of their regions).  An encoded
// side brings its own shifts and planes.
int64_t problem_bytes(const ozaki2_problem& p, bool enc_a, bool enc_b) {
    const int64_t m_pad = round_up64(p.m, OZAKI2_ROWS_ALIGN_A);
    const int64_t n_pad = round_up64(p.n, OZAKI2_ROWS_ALIGN_B);
    const PlaneGeom geo = compact_planes(p.m, p.n, p.k);
    const int64_t N = p.num_moduli;
    int64_t b = round_up64(N * m_pad * n_pad, 256);
    if (!enc_a) b += round_up64(4 * m_pad, 256) + round_up64(2 * N * geo.rows_a * geo.ld, 256);
    if (!enc_b) b += round_up64(4 * n_pad, 256) + round_up64(2 * N * geo.rows_b * geo.ld, 256);
    return b;
}

// Stored extent of a problem's planes: an encoded B keeps the 256-row layout of its encoding.
PlaneGeom problem_geo(const ozaki2_problem& p, int bn, bool enc_b) {
    PlaneGeom g = compact_planes(p.m, p.n, p.k, bn);
    if (enc_b) g.rows_b = p.n > 256 ? p.n : 256;
    return g;
}

// rules == nullptr: 256-wide tiles for every problem (the largest tables, for sizing).
void make_plan(int count, const ozaki2_problem* probs, Plan& P, const TileRules* rules,
               int chunk_k, int scaling = OZAKI2_SCALING_PROPOSED,
               const Encoded& enc = Encoded()) {
    P.accurate = scaling == OZAKI2_SCALING_ACCURATE;
    for (int i = 0; i < count; ++i)
        if (active(probs[i])) P.idx.push_back(i);
    // order by moduli count so that each conversion / CRT launch covers one contiguous range
    std::stable_sort(P.idx.begin(), P.idx.end(), [&](int a, int b) {
        return probs[a].num_moduli < probs[b].num_moduli;
    });
    int64_t off = 0;
    for (int i : P.idx) {
        P.ea.push_back(enc.a ? enc.a[i] : nullptr);
        P.eb.push_back(enc.b ? enc.b[i] : nullptr);
        P.ws_off.push_back(off);
        off += problem_bytes(probs[i], P.ea.back() != nullptr, P.eb.back() != nullptr);
    }
    P.ws_problems = off;
    int scale = 0, conv = 0, crt = 0, tiles = 0;
    int curN = -1;
    for (size_t a = 0; a < P.idx.size(); ++a) {
        const ozaki2_problem& p = probs[P.idx[a]];
        const bool has_a = P.ea[a] != nullptr, has_b = P.eb[a] != nullptr;
        int bn = 256, chunk = chunk_k;
        // accurate mode's auxiliary product runs on 256-wide tiles over the same planes
        if (rules && !P.accurate) grouped_tile(*rules, p.n, p.k, chunk_k, &bn, &chunk);
        P.bn.push_back(bn);
        P.chunk.push_back(chunk);
        const int64_t m_pad = round_up64(p.m, OZAKI2_ROWS_ALIGN_A);
        const int64_t n_pad = round_up64(p.n, bn);
        const PlaneGeom geo = problem_geo(p, bn, has_b);
        scale += (has_a ? 0 : (p.m + 127) / 128) + (has_b ? 0 : (p.n + 127) / 128);
        const int64_t aes = notrans(p.transA) ? p.lda : 1;
        const int64_t bes = notrans(p.transB) ? 1 : p.ldb;
        const int64_t als = notrans(p.transA) ? 1 : p.lda;
        const int64_t bls = notrans(p.transB) ? p.ldb : 1;
        if (!has_a && scale_lines_adjacent(als, aes)) P.n_scale_adj += (p.m + 127) / 128;
        if (!has_b && scale_lines_adjacent(bls, bes)) P.n_scale_adj += (p.n + 127) / 128;
        const int cb = (has_a ? 0 : convert_blocks(p.m, aes, geo.rows_a, geo.ld)) +
                       (has_b ? 0 : convert_blocks(p.n, bes, geo.rows_b, geo.ld));
        const int rb = ((p.m + 31) / 32) * ((p.n + 63) / 64);  // 32 x 64 CRT tiles
        if (p.num_moduli != curN) {
            curN = p.num_moduli;
            P.conv_n.push_back(curN);
            P.conv_begin.push_back(conv);
            P.conv_count.push_back(0);
            P.crt_begin.push_back(crt);
            P.crt_count.push_back(0);
        }
        P.conv_count.back() += cb;
        P.crt_count.back() += rb;
        conv += cb;
        crt += rb;
        tiles += p.num_moduli * (int)(m_pad / 128) * (int)(n_pad / bn);
        P.aux_tiles += (int)(m_pad / 128) * (int)(n_pad / 256);
    }
    P.n_scale = scale;
    P.n_conv = conv;
    P.n_crt = crt;
    P.total_tiles = tiles;
    const int64_t np = (int64_t)P.idx.size();
    int64_t t = 0;
    P.off_gg = t;  t += round_up64(np * (int64_t)sizeof(GroupGemmProblem), 256);
    P.off_gp = t;  t += round_up64(np * (int64_t)sizeof(GroupProblem), 256);
    P.off_sw = t;  t += round_up64((int64_t)scale * sizeof(ScaleWork), 256);
    P.off_cw = t;  t += round_up64((int64_t)conv * sizeof(ConvertWork), 256);
    P.off_rw = t;  t += round_up64((int64_t)crt * sizeof(CrtWork), 256);
    if (P.accurate) {
        P.off_ga = t;
        t += round_up64(np * (int64_t)sizeof(GroupGemmProblem), 256);
    }
    P.table_bytes = t;
}

}  // namespace

// Bytes of workspace a grouped call needs (intermediates of every problem plus its tables, sized
// for the largest tables, those of accurate mode).
size_t grouped_workspace_bytes(int count, const ozaki2_problem* probs, const Encoded& enc) {
    Plan P;
    make_plan(count, probs, P, nullptr, 960, OZAKI2_SCALING_ACCURATE, enc);
    return (size_t)(P.ws_problems + P.table_bytes + 256);
}

// Builds the tables of a grouped call into `host` (grouped_table_bytes bytes).  `ws` is the device
// workspace holding the problems' intermediates.
int build_grouped_tables(int count, const ozaki2_problem* probs, char* ws, char* host,
                         const TileRules& rules, int chunk_k, int scaling, const Encoded& enc) {
    Plan P;
    make_plan(count, probs, P, &rules, chunk_k, scaling, enc);
    if (P.idx.empty()) return OZAKI2_SUCCESS;
    memset(host, 0, (size_t)P.table_bytes);
    auto* gg = reinterpret_cast<GroupGemmProblem*>(host + P.off_gg);
    auto* ga = reinterpret_cast<GroupGemmProblem*>(host + P.off_ga);
    int aux_begin = 0;
    auto* gp = reinterpret_cast<GroupProblem*>(host + P.off_gp);
    auto* sw = reinterpret_cast<ScaleWork*>(host + P.off_sw);
    auto* cw = reinterpret_cast<ConvertWork*>(host + P.off_cw);
    auto* rw = reinterpret_cast<CrtWork*>(host + P.off_rw);
    int ns_adj = 0, ns_con = P.n_scale_adj, nc = 0, nr = 0, tile_begin = 0;
    for (size_t a = 0; a < P.idx.size(); ++a) {
        const ozaki2_problem& p = probs[P.idx[a]];
        const ModTables* T = mod_tables(p.num_moduli);
        const int bn = P.bn[a];
        const int64_t m_pad = round_up64(p.m, OZAKI2_ROWS_ALIGN_A);
        const int64_t n_pad = round_up64(p.n, bn);
        const int64_t k_pad = round_up64(p.k, OZAKI2_K_ALIGN);
        const int64_t N = p.num_moduli;
        char* base = ws + P.ws_off[a];
        GroupProblem& g = gp[a];
        g.A = p.A;
        g.B = p.B;
        g.C = p.C;
        g.a_ls = notrans(p.transA) ? 1 : p.lda;
        g.a_es = notrans(p.transA) ? p.lda : 1;
        g.b_ls = notrans(p.transB) ? p.ldb : 1;
        g.b_es = notrans(p.transB) ? 1 : p.ldb;
        g.ldc = p.ldc;
        g.m = p.m;
        g.n = p.n;
        g.k = p.k;
        g.N = p.num_moduli;
        g.m_pad = (int)m_pad;
        g.n_pad = (int)n_pad;
        g.k_pad = (int)k_pad;
        const ozaki2_operand* ea = P.ea[a];
        const ozaki2_operand* eb = P.eb[a];
        g.geo = problem_geo(p, bn, eb != nullptr);
        g.alpha = p.alpha;
        g.beta = p.beta;
        g.ab = (p.alpha != 1.0 ? 1 : 0) | (p.beta != 0.0 ? 2 : 0);
        g.scaling = scaling;
        g.pprime = scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
        g.delta = T->delta;
        int64_t o = 0;
        g.res = reinterpret_cast<int8_t*>(base + o);  o += round_up64(N * m_pad * n_pad, 256);
        if (ea) {  // the encoding's shifts and planes (operand_layout)
            char* d = static_cast<char*>(ea->data);
            g.e = reinterpret_cast<int*>(d);
            g.pa = d + operand_layout(false, p.m, p.k, p.num_moduli).off_planes;
        } else {
            g.e = reinterpret_cast<int*>(base + o);  o += round_up64(4 * m_pad, 256);
            g.pa = base + o;  o += round_up64(2 * N * g.geo.rows_a * g.geo.ld, 256);
        }
        if (eb) {
            char* d = static_cast<char*>(eb->data);
            g.f = reinterpret_cast<int*>(d);
            g.pb = d + operand_layout(true, p.n, p.k, p.num_moduli).off_planes;
        } else {
            g.f = reinterpret_cast<int*>(base + o);  o += round_up64(4 * n_pad, 256);
            g.pb = base + o;  o += round_up64(2 * N * g.geo.rows_b * g.geo.ld, 256);
        }
        if (!make_group_gemm_problem(&gg[a], p.num_moduli, (int)m_pad, (int)n_pad, (int)k_pad,
                                     g.geo, g.pa, g.pb, g.res, P.chunk[a], bn))
            return OZAKI2_ERROR_DRIVER;
        gg[a].tile_begin = tile_begin;
        tile_begin += p.num_moduli * gg[a].tiles_m * gg[a].tiles_n;
        if (P.accurate) {
            // A-bar / B-bar live in the first residue plane, the C-bar maxima in the product
            // residues; both are overwritten later by the main stages
            if (!make_group_aux_problem(&ga[a], (int)m_pad, (int)n_pad, (int)k_pad, g.geo, g.pa,
                                        g.pb, reinterpret_cast<uint32_t*>(g.res)))
                return OZAKI2_ERROR_DRIVER;
            ga[a].tile_begin = aux_begin;
            aux_begin += ga[a].tiles_m * ga[a].tiles_n;
        }
        for (int side = 0; side < 2; ++side) {
            if (side ? eb != nullptr : ea != nullptr) continue;  // encoded: nothing to do
            const int lines = side ? p.n : p.m;
            // adjacent lines' items first, then contiguous lines' (one kernel each)
            const bool adj = side ? scale_lines_adjacent(g.b_ls, g.b_es)
                                  : scale_lines_adjacent(g.a_ls, g.a_es);
            int& ns = adj ? ns_adj : ns_con;
            for (int l0 = 0; l0 < lines; l0 += 128) sw[ns++] = ScaleWork{(int)a, side, l0};
            const int64_t es = side ? g.b_es : g.a_es;
            const int cb = convert_blocks(lines, es, side ? g.geo.rows_b : g.geo.rows_a, g.geo.ld);
            for (int b = 0; b < cb; ++b) cw[nc++] = ConvertWork{(int)a, side, b};
        }
        for (int i0 = 0; i0 < p.m; i0 += 32)
            for (int j0 = 0; j0 < p.n; j0 += 64) rw[nr++] = CrtWork{(int)a, i0, j0};
    }
    return OZAKI2_SUCCESS;
}

// Launches every stage of a grouped call whose tables are already at `tables_dev`.
int launch_grouped(int count, const ozaki2_problem* probs, const char* tables_dev,
                   unsigned* status, int num_sms, const TileRules& rules, int chunk_k,
                   cudaStream_t stream, int scaling, unsigned long long limit_ns,
                   const Encoded& enc) {
    Plan P;
    make_plan(count, probs, P, &rules, chunk_k, scaling, enc);
    // quick returns of inactive problems: C = beta C (m, n > 0)
    for (int i = 0; i < count; ++i) {
        const ozaki2_problem& p = probs[i];
        if (p.m > 0 && p.n > 0 && !active(p))
            if (launch_scale_c(p.m, p.n, p.beta, p.C, p.ldc, stream) != cudaSuccess)
                return OZAKI2_ERROR_CUDA;
    }
    if (P.idx.empty()) return OZAKI2_SUCCESS;
    const auto* dgg = reinterpret_cast<const GroupGemmProblem*>(tables_dev + P.off_gg);
    const auto* dgp = reinterpret_cast<const GroupProblem*>(tables_dev + P.off_gp);
    const auto* dsw = reinterpret_cast<const ScaleWork*>(tables_dev + P.off_sw);
    const auto* dcw = reinterpret_cast<const ConvertWork*>(tables_dev + P.off_cw);
    const auto* drw = reinterpret_cast<const CrtWork*>(tables_dev + P.off_rw);
    if (launch_scale_grouped(dgp, dsw, P.n_scale, status, stream, scaling, P.n_scale_adj) !=
        cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    if (P.accurate) {
        // the first pass wrote the line exponents; A-bar and B-bar, the auxiliary product's
        // maxima, then the shifts in place
        if (launch_convert_grouped(1, dgp, dcw, P.n_conv, ConvertTables{}, status, stream) !=
            cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        const auto* dga = reinterpret_cast<const GroupGemmProblem*>(tables_dev + P.off_ga);
        int rc = launch_aux_gemm_grouped(dga, (int)P.idx.size(), P.aux_tiles, status, num_sms,
                                         stream, limit_ns);
        if (rc) return rc;
        if (launch_accu_shift_grouped(dgp, dsw, P.n_scale, stream) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
    }
    for (size_t g = 0; g < P.conv_n.size(); ++g)
        if (launch_convert_grouped(P.conv_n[g], dgp, dcw + P.conv_begin[g], P.conv_count[g],
                                   mod_tables(P.conv_n[g])->conv, status, stream,
                                   P.accurate) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
    int rc = launch_residue_gemm_grouped(dgg, (int)P.idx.size(), P.total_tiles,
                                         mod_tables(OZAKI2_MAX_MODULI)->epi, status, num_sms,
                                         chunk_k, stream, limit_ns);
    if (rc) return rc;
    for (size_t g = 0; g < P.conv_n.size(); ++g)
        if (launch_crt_grouped(P.conv_n[g], dgp, drw + P.crt_begin[g], P.crt_count[g],
                               mod_tables(P.conv_n[g])->crt, stream) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
    return OZAKI2_SUCCESS;
}

// Device address of the tables inside the workspace (after the problems' intermediates).
char* grouped_tables_in_workspace(int count, const ozaki2_problem* probs, char* ws,
                                  const Encoded& enc) {
    Plan P;
    make_plan(count, probs, P, nullptr, 960, OZAKI2_SCALING_PROPOSED, enc);
    return ws + round_up64(P.ws_problems, 256);
}

int grouped_table_bytes(int count, const ozaki2_problem* probs, const TileRules& rules,
                        int chunk_k, int scaling, const Encoded& enc) {
    Plan P;
    make_plan(count, probs, P, &rules, chunk_k, scaling, enc);
    return (int)P.table_bytes;
}

// ---------------------------------------------------------------- encoded operands
// Each operand becomes a one-sided problem of the grouped scaling and conversion kernels (side
// 0 for op(A), side 1 for op(B)) whose shifts and planes are the operand's buffer.  Tables:
// GroupProblem[count], then the scale work, then the conversion work ordered by moduli count.
namespace {
struct EncodePlan {
    std::vector<int> order;  // operands by moduli count
    int n_scale = 0, n_conv = 0;
    std::vector<int> conv_n, conv_begin, conv_count;
    int64_t off_gp = 0, off_sw = 0, off_cw = 0, bytes = 0;
};

bool side_b(const ozaki2_operand& o) { return o.side == 'B' || o.side == 'b'; }

GroupProblem encode_problem(const ozaki2_operand& o, int scaling) {
    GroupProblem g = {};
    const bool b = side_b(o);
    const OperandLayout L = operand_layout(b, o.lines, o.k, o.num_moduli);
    const ModTables* T = mod_tables(o.num_moduli);
    char* d = static_cast<char*>(o.data);
    g.k = o.k;
    g.N = o.num_moduli;
    g.k_pad = (int)round_up64(o.k, OZAKI2_K_ALIGN);
    g.geo = PlaneGeom{L.rows, L.rows, L.ld, 0, 0};
    g.scaling = scaling;
    g.pprime = scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
    g.delta = T->delta;
    g.alpha = 1.0;
    if (!b) {  // rows of op(A): line i, element h at X[i * ls + h * es]
        g.A = o.X;
        g.a_ls = notrans(o.trans) ? 1 : o.ld;
        g.a_es = notrans(o.trans) ? o.ld : 1;
        g.m = o.lines;
        g.m_pad = L.lines_pad;
        g.e = reinterpret_cast<int*>(d);
        g.pa = d + L.off_planes;
    } else {   // columns of op(B)
        g.B = o.X;
        g.b_ls = notrans(o.trans) ? o.ld : 1;
        g.b_es = notrans(o.trans) ? 1 : o.ld;
        g.n = o.lines;
        g.n_pad = L.lines_pad;
        g.f = reinterpret_cast<int*>(d);
        g.pb = d + L.off_planes;
    }
    return g;
}

void make_encode_plan(int count, const ozaki2_operand* ops, EncodePlan& E) {
    for (int i = 0; i < count; ++i)  // (k = 0: the caller clears the encoding)
        if (ops[i].lines > 0 && ops[i].k > 0) E.order.push_back(i);
    std::stable_sort(E.order.begin(), E.order.end(), [&](int a, int b) {
        return ops[a].num_moduli < ops[b].num_moduli;
    });
    int curN = -1;
    for (int i : E.order) {
        const ozaki2_operand& o = ops[i];
        const OperandLayout L = operand_layout(side_b(o), o.lines, o.k, o.num_moduli);
        const int64_t es = side_b(o) ? (notrans(o.trans) ? 1 : o.ld) : (notrans(o.trans) ? o.ld : 1);
        E.n_scale += (o.lines + 127) / 128;
        const int cb = convert_blocks(o.lines, es, L.rows, L.ld);
        if (o.num_moduli != curN) {
            curN = o.num_moduli;
            E.conv_n.push_back(curN);
            E.conv_begin.push_back(E.n_conv);
            E.conv_count.push_back(0);
        }
        E.conv_count.back() += cb;
        E.n_conv += cb;
    }
    int64_t t = 0;
    E.off_gp = t;  t += round_up64((int64_t)count * sizeof(GroupProblem), 256);
    E.off_sw = t;  t += round_up64((int64_t)E.n_scale * sizeof(ScaleWork), 256);
    E.off_cw = t;  t += round_up64((int64_t)E.n_conv * sizeof(ConvertWork), 256);
    E.bytes = t;
}
}  // namespace

int encode_table_bytes(int count, const ozaki2_operand* ops) {
    EncodePlan E;
    make_encode_plan(count, ops, E);
    return (int)E.bytes;
}

void build_encode_tables(int count, const ozaki2_operand* ops, int scaling, char* host) {
    EncodePlan E;
    make_encode_plan(count, ops, E);
    memset(host, 0, (size_t)E.bytes);
    auto* gp = reinterpret_cast<GroupProblem*>(host + E.off_gp);
    auto* sw = reinterpret_cast<ScaleWork*>(host + E.off_sw);
    auto* cw = reinterpret_cast<ConvertWork*>(host + E.off_cw);
    int ns = 0, nc = 0;
    for (int i : E.order) {
        const ozaki2_operand& o = ops[i];
        gp[i] = encode_problem(o, scaling);
        const int side = side_b(o) ? 1 : 0;
        for (int l0 = 0; l0 < o.lines; l0 += 128) sw[ns++] = ScaleWork{i, side, l0};
        const int64_t es = side ? gp[i].b_es : gp[i].a_es;
        const int cb = convert_blocks(o.lines, es, gp[i].geo.rows_a, gp[i].geo.ld);
        for (int b = 0; b < cb; ++b) cw[nc++] = ConvertWork{i, side, b};
    }
}

int launch_encode(int count, const ozaki2_operand* ops, const char* tables_dev, unsigned* status,
                  cudaStream_t stream, int scaling) {
    EncodePlan E;
    make_encode_plan(count, ops, E);
    if (E.order.empty()) return OZAKI2_SUCCESS;
    const auto* dgp = reinterpret_cast<const GroupProblem*>(tables_dev + E.off_gp);
    const auto* dsw = reinterpret_cast<const ScaleWork*>(tables_dev + E.off_sw);
    const auto* dcw = reinterpret_cast<const ConvertWork*>(tables_dev + E.off_cw);
    if (launch_scale_grouped(dgp, dsw, E.n_scale, status, stream, scaling) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    for (size_t g = 0; g < E.conv_n.size(); ++g)
        if (launch_convert_grouped(E.conv_n[g], dgp, dcw + E.conv_begin[g], E.conv_count[g],
                                   mod_tables(E.conv_n[g])->conv, status, stream) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
    return OZAKI2_SUCCESS;
}

int auto_tile_n(int n) {
    int best = 256;
    int64_t best_cost = INT64_MAX;
    for (int bn : {256, 128, 64}) {
        const int64_t tiles = (n + bn - 1) / bn;
        const int64_t mma = 2 * 96 * (int64_t)bn, load = 16384 + 128 * (int64_t)bn;  // x 96
        const int64_t cost = tiles * (mma > load ? mma : load);
        if (cost < best_cost) {  // strictly fewer cycles: ties keep the wider tile
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

void grouped_tile(const TileRules& rules, int n, int k, int chunk_k, int* bn, int* chunk) {
    for (int i = 0; i < rules.count; ++i) {
        const TileRule& r = rules.r[i];
        if (n <= r.n_max && k <= r.k_max) {
            *bn = r.tile_n;
            *chunk = r.chunk_k ? r.chunk_k : chunk_k;
            return;
        }
    }
    *bn = auto_tile_n(n);
    *chunk = chunk_k;
}

int grouped_check(int count, const ozaki2_problem* probs) {
    for (int i = 0; i < count; ++i) {
        const int a = check_problem(probs[i]);
        if (a) return -(100 * (i + 1) + a);
    }
    return OZAKI2_SUCCESS;
}

}  // namespace ozaki2
