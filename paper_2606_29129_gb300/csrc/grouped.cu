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
    std::vector<int64_t> ws_off;    // offset of each active problem's intermediates
    int64_t ws_problems = 0;        // bytes of all intermediates
    // table sections (offsets within the table block)
    int64_t off_gp = 0, off_gg = 0, off_sw = 0, off_cw = 0, off_rw = 0, table_bytes = 0;
    int n_scale = 0, n_conv = 0, n_crt = 0;
    std::vector<int> conv_n, conv_begin, conv_count;  // per distinct N: blocks in the table
    std::vector<int> crt_begin, crt_count;
    int total_tiles = 0;
    // accurate mode: one auxiliary-product descriptor per problem (C-bar = A-bar B-bar)
    bool accurate = false;
    int64_t off_ga = 0;
    int aux_tiles = 0;
};

int64_t problem_bytes(const ozaki2_problem& p) {
    const int64_t m_pad = round_up64(p.m, OZAKI2_ROWS_ALIGN_A);
    const int64_t n_pad = round_up64(p.n, OZAKI2_ROWS_ALIGN_B);
    const PlaneGeom geo = compact_planes(p.m, p.n, p.k);
    const int64_t N = p.num_moduli;
    return round_up64(4 * m_pad, 256) + round_up64(4 * n_pad, 256) +
           round_up64(2 * N * geo.rows_a * geo.ld, 256) +
           round_up64(2 * N * geo.rows_b * geo.ld, 256) + round_up64(N * m_pad * n_pad, 256);
}

void make_plan(int count, const ozaki2_problem* probs, Plan& P,
               int scaling = OZAKI2_SCALING_PROPOSED) {
    P.accurate = scaling == OZAKI2_SCALING_ACCURATE;
    for (int i = 0; i < count; ++i)
        if (active(probs[i])) P.idx.push_back(i);
    // order by moduli count so that each conversion / CRT launch covers one contiguous range
    std::stable_sort(P.idx.begin(), P.idx.end(), [&](int a, int b) {
        return probs[a].num_moduli < probs[b].num_moduli;
    });
    int64_t off = 0;
    for (int i : P.idx) {
        P.ws_off.push_back(off);
        off += problem_bytes(probs[i]);
    }
    P.ws_problems = off;
    int scale = 0, conv = 0, crt = 0, tiles = 0;
    int curN = -1;
    for (int i : P.idx) {
        const ozaki2_problem& p = probs[i];
        const int64_t m_pad = round_up64(p.m, OZAKI2_ROWS_ALIGN_A);
        const int64_t n_pad = round_up64(p.n, OZAKI2_ROWS_ALIGN_B);
        const PlaneGeom geo = compact_planes(p.m, p.n, p.k);
        scale += (p.m + 127) / 128 + (p.n + 127) / 128;
        const int64_t aes = notrans(p.transA) ? p.lda : 1;
        const int64_t bes = notrans(p.transB) ? 1 : p.ldb;
        const int cb = convert_blocks(p.m, aes, geo.rows_a, geo.ld) +
                       convert_blocks(p.n, bes, geo.rows_b, geo.ld);
        const int rb = ((p.m + 31) / 32) * ((p.n + 31) / 32);
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
        tiles += p.num_moduli * (int)(m_pad / 128) * (int)(n_pad / 256);
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
size_t grouped_workspace_bytes(int count, const ozaki2_problem* probs) {
    Plan P;
    make_plan(count, probs, P, OZAKI2_SCALING_ACCURATE);
    return (size_t)(P.ws_problems + P.table_bytes + 256);
}

// Builds the tables of a grouped call into `host` (grouped_table_bytes bytes).  `ws` is the device
// workspace holding the problems' intermediates.
int build_grouped_tables(int count, const ozaki2_problem* probs, char* ws, char* host,
                         int chunk_k, int scaling) {
    Plan P;
    make_plan(count, probs, P, scaling);
    if (P.idx.empty()) return OZAKI2_SUCCESS;
    memset(host, 0, (size_t)P.table_bytes);
    auto* gg = reinterpret_cast<GroupGemmProblem*>(host + P.off_gg);
    auto* ga = reinterpret_cast<GroupGemmProblem*>(host + P.off_ga);
    int aux_begin = 0;
    auto* gp = reinterpret_cast<GroupProblem*>(host + P.off_gp);
    auto* sw = reinterpret_cast<ScaleWork*>(host + P.off_sw);
    auto* cw = reinterpret_cast<ConvertWork*>(host + P.off_cw);
    auto* rw = reinterpret_cast<CrtWork*>(host + P.off_rw);
    int ns = 0, nc = 0, nr = 0, tile_begin = 0;
    for (size_t a = 0; a < P.idx.size(); ++a) {
        const ozaki2_problem& p = probs[P.idx[a]];
        const ModTables* T = mod_tables(p.num_moduli);
        const int64_t m_pad = round_up64(p.m, OZAKI2_ROWS_ALIGN_A);
        const int64_t n_pad = round_up64(p.n, OZAKI2_ROWS_ALIGN_B);
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
        g.geo = compact_planes(p.m, p.n, p.k);
        g.alpha = p.alpha;
        g.beta = p.beta;
        g.ab = (p.alpha != 1.0 ? 1 : 0) | (p.beta != 0.0 ? 2 : 0);
        g.scaling = scaling;
        g.pprime = scaling == OZAKI2_SCALING_FAST ? T->pprime_fast : T->pprime;
        g.delta = T->delta;
        int64_t o = 0;
        g.e = reinterpret_cast<int*>(base + o);  o += round_up64(4 * m_pad, 256);
        g.f = reinterpret_cast<int*>(base + o);  o += round_up64(4 * n_pad, 256);
        g.pa = base + o;  o += round_up64(2 * N * g.geo.rows_a * g.geo.ld, 256);
        g.pb = base + o;  o += round_up64(2 * N * g.geo.rows_b * g.geo.ld, 256);
        g.res = reinterpret_cast<int8_t*>(base + o);
        if (!make_group_gemm_problem(&gg[a], p.num_moduli, (int)m_pad, (int)n_pad, (int)k_pad,
                                     g.geo, g.pa, g.pb, g.res, chunk_k))
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
            const int lines = side ? p.n : p.m;
            for (int l0 = 0; l0 < lines; l0 += 128) sw[ns++] = ScaleWork{(int)a, side, l0};
            const int64_t es = side ? g.b_es : g.a_es;
            const int cb = convert_blocks(lines, es, side ? g.geo.rows_b : g.geo.rows_a, g.geo.ld);
            for (int b = 0; b < cb; ++b) cw[nc++] = ConvertWork{(int)a, side, b};
        }
        for (int i0 = 0; i0 < p.m; i0 += 32)
            for (int j0 = 0; j0 < p.n; j0 += 32) rw[nr++] = CrtWork{(int)a, i0, j0};
    }
    return OZAKI2_SUCCESS;
}

// Launches every stage of a grouped call whose tables are already at `tables_dev`.
int launch_grouped(int count, const ozaki2_problem* probs, const char* tables_dev,
                   unsigned* status, int num_sms, int chunk_k, cudaStream_t stream, int scaling) {
    Plan P;
    make_plan(count, probs, P, scaling);
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
    if (launch_scale_grouped(dgp, dsw, P.n_scale, status, stream) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    if (P.accurate) {
        // the first pass wrote the line exponents; A-bar and B-bar, the auxiliary product's
        // maxima, then the shifts in place
        if (launch_convert_grouped(1, dgp, dcw, P.n_conv, ConvertTables{}, status, stream) !=
            cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        const auto* dga = reinterpret_cast<const GroupGemmProblem*>(tables_dev + P.off_ga);
        int rc = launch_aux_gemm_grouped(dga, (int)P.idx.size(), P.aux_tiles, status, num_sms,
                                         stream);
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
                                         chunk_k, stream);
    if (rc) return rc;
    for (size_t g = 0; g < P.conv_n.size(); ++g)
        if (launch_crt_grouped(P.conv_n[g], dgp, drw + P.crt_begin[g], P.crt_count[g],
                               mod_tables(P.conv_n[g])->crt, stream) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
    return OZAKI2_SUCCESS;
}

// Device address of the tables inside the workspace (after the problems' intermediates).
char* grouped_tables_in_workspace(int count, const ozaki2_problem* probs, char* ws) {
    Plan P;
    make_plan(count, probs, P);
    return ws + round_up64(P.ws_problems, 256);
}

int grouped_table_bytes(int count, const ozaki2_problem* probs, int scaling) {
    Plan P;
    make_plan(count, probs, P, scaling);
    return (int)P.table_bytes;
}

int grouped_check(int count, const ozaki2_problem* probs) {
    for (int i = 0; i < count; ++i) {
        const int a = check_problem(probs[i]);
        if (a) return -(100 * (i + 1) + a);
    }
    return OZAKI2_SUCCESS;
}

}  // namespace ozaki2
