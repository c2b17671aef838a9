// residue_gemm.cu -- Step 3 of Ozaki scheme II: the N residue GEMMs of eq. (os2-C'),
// G_l = rmod(A', p_l) rmod(B', p_l), reduced modulo p_l in the epilogue.
//
// GB300 design.  sm_103a has no integer tcgen05 MMA, so the residues (integers in [-128, 127])
// are stored as bf16, where they are exact, and multiplied on the 5th-generation tensor cores
// with tcgen05.mma kind::f16 into FP32 accumulators in tensor memory (TMEM).  Every product has
// magnitude <= 2^14, so an FP32 accumulator holding a value below 2^24 in magnitude is exact.
// The K loop is cut into chunks of at most 960 (15 x 64); after each chunk the epilogue warps
// reduce the accumulator modulo p_l in place (tcgen05.ld -> r = x - p*rint(x/p) -> tcgen05.st),
// keeping |acc| <= ~0.52 p + 960 * 2^14 < 2^24.  The last chunk's drain produces the symmetric
// residue c_l = rmod(G_l, p_l) as int8.
//
// Pipeline (one CTA per SM, persistent over (modulus, m-tile, n-tile) work):
//   warp 0   TMA producer: 128x64 A and 256x64 B bf16 tiles, 128-byte swizzle, 4 stages.
//   warp 1   TMEM allocator and MMA issuer (one thread): 4 x (M=128, N=256, K=16) per stage.
//   warps 4-11 epilogue: TMEM lanes 32*(warp%4).., one half of the columns each; in-place
//            reductions and the final drain.
// Two TMEM accumulators (2 x 256 columns) hold two tiles whose K chunks are interleaved, so the
// in-place reduction of one tile overlaps the MMAs of the other.
//
// Every mbarrier wait is bounded (globaltimer); on expiry the kernel raises
// OZAKI2_STATUS_TIMEOUT, stops all roles, waits (bounded) for its TMA copies and MMAs, frees
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "ozaki2_internal.h"
#include "sm103_ptx.cuh"

namespace ozaki2 {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4, UMMA_K = 16;
constexpr int A_BYTES = BM * BK * 2;           // 16 KiB
constexpr int B_BYTES = BN * BK * 2;           // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * BN;              // two fp32 accumulators of 128 x 256
constexpr int NUM_THREADS = 384;
constexpr int EPI_WARP0 = 4;       // warps 4..11: two epilogue warps per TMEM lane quarter
constexpr int EPI_WARPS = 8;
constexpr int EPI_COLS = 128;      // accumulator columns drained by one epilogue warp
constexpr int NUM_BARRIERS = 2 * STAGES + 5;   // full, empty, acc_full[2], acc_empty[2], drain
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + NUM_BARRIERS * 8 + 16;
constexpr int GROUP_M = 16;  // m-tiles per group in the tile order of grouped calls (L2 reuse)
// Defaults of single-problem calls, fastest in a sweep on GB300 (8192^3 and 16384^3, N = 16):
// 32 m-tiles of 128 rows for the one-SM kernel, 4 m-tiles of 256 rows for the SM-pair kernel.
constexpr int GROUP_M_SINGLE = 32, GROUP_M_PAIR = 4;

// Instruction descriptor of tcgen05.mma kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
// The same for a tile of bn columns (bn = 64, 128 or 256: N >> 3 at bits 17-22).
__host__ __device__ constexpr uint32_t idesc_for(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}
static_assert(idesc_for(BN) == IDESC, "instruction descriptor");

struct GemmArgs {
    int tiles_m, tiles_n, total_tiles, k_blocks, chunk_blocks, nchunks;
    int group_m;  // m-tiles per group of the tile order
    int l2_hints;  // OZAKI2_L2_*: eviction priorities of the A and B tile loads in L2
    int m_rows;  // rows of the A planes / product residues (m_pad)
    int m_live, n_live;  // product residues stored: rows below m_live, columns below n_live
    int8_t* out;
    int64_t out_ld, out_plane;
    unsigned* status;
    unsigned long long limit_ns;  // bound of every mbarrier wait of the main loops
    EpilogueTables ep;
};

// ---------------------------------------------------------------- PTX wrappers (GEMM only)
// L2 eviction policies for the tile loads (createpolicy): 0 keeps the default.
__device__ __forceinline__ uint64_t l2_policy(int kind) {
    uint64_t p = 0;
    if (kind == 1)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else if (kind == 2)
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// A tile load with an L2 eviction policy (policy 0: none).
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, uint64_t* bar,
                                                 int x, int y, int z, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)),
        "l"(policy)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Nearest integer, ties to even.  (On this power-capped part the single rounding instruction
// measured faster than the two-add magic-number form.)
__device__ __forceinline__ float round_small(float y) { return rintf(y); }

// ---- cluster (2-SM) helpers
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}
// TMA load whose completion is signalled on an mbarrier in either CTA of the pair.
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster_addr, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::"
        "bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar_cluster_addr)
        : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive (once MMAs issued so far complete) on the mbarrier at this offset in both CTAs.
__device__ __forceinline__ void umma_commit_pair_both(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)), "h"((uint16_t)3)
        : "memory");
}
__device__ __forceinline__ void umma_commit_pair_local(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void spin_ns(unsigned long long ns) {
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < ns) {
    }
}

// Tile t -> (modulus l, m-tile, n-tile).  Within a modulus, groups of GROUP_M m-tiles sweep the
// n-tiles so that CTAs running at the same time share A and B panels in L2.
__device__ __forceinline__ void decode_tile(int tile, const GemmArgs& a, int& l, int& mt,
                                            int& nt) {
    const int per_plane = a.tiles_m * a.tiles_n;
    l = tile / per_plane;
    const int idx = tile - l * per_plane;
    const int per_group = a.group_m * a.tiles_n;
    const int g = idx / per_group;
    const int first_m = g * a.group_m;
    const int gsize = min(a.tiles_m - first_m, a.group_m);
    const int r = idx - g * per_group;
    mt = first_m + r % gsize;
    nt = r / gsize;
}

// ---------------------------------------------------------------- tile sources
// Everything the three roles need about one output tile.
struct TileInfo {
    const CUtensorMap* ta;
    const CUtensorMap* tb;
    int l, mt, nt, k_blocks, nchunks;
    int bn;            // tile width: 256, 128 or 64 columns (rows of the B box)
    int chunk_blocks;  // K blocks of 64 between modular reductions
    int8_t* out;
    int64_t out_ld, out_plane;
    int m_live, n_live;  // rows and columns of the product residues that are stored
};

__device__ __forceinline__ void decode_local(int idx, int tiles_m, int tiles_n, int& l, int& mt,
                                             int& nt, int group_m = GROUP_M) {
    const int per_plane = tiles_m * tiles_n;
    l = idx / per_plane;
    const int r0 = idx - l * per_plane;
    const int per_group = group_m * tiles_n;
    const int g = r0 / per_group;
    const int first_m = g * group_m;
    const int gsize = min(tiles_m - first_m, group_m);
    const int r = r0 - g * per_group;
    mt = first_m + r % gsize;
    nt = r / gsize;
}

// One problem; tensor maps in kernel parameters.
struct SingleSource {
    static constexpr bool kPrefetchMaps = false;
    const CUtensorMap* ta;
    const CUtensorMap* tb;
    const GemmArgs* a;
    __device__ __forceinline__ TileInfo get(int t) const {
        TileInfo ti;
        decode_local(t, a->tiles_m, a->tiles_n, ti.l, ti.mt, ti.nt, a->group_m);
        ti.ta = ta;
        ti.tb = tb;
        ti.k_blocks = a->k_blocks;
        ti.nchunks = a->nchunks;
        ti.bn = BN;
        ti.chunk_blocks = a->chunk_blocks;
        ti.out = a->out;
        ti.out_ld = a->out_ld;
        ti.out_plane = a->out_plane;
        ti.m_live = a->m_live;
        ti.n_live = a->n_live;
        return ti;
    }
};

// Many problems; each with its own tensor maps in device memory.  A CTA visits its tiles in
// increasing order, so each role keeps the problem of its last tile and steps forward from it (a
// step or two per tile), with a binary search over the rest when the jump is longer.
struct GroupSource {
    static constexpr bool kPrefetchMaps = true;
    const GroupGemmProblem* probs;
    int count;
    int at = 0;  // problem of the last tile looked up
    __device__ __forceinline__ int find(int t) {
        int lo = at;
#pragma unroll 1
        for (int step = 0; step < 4; ++step) {
            if (lo + 1 >= count || __ldg(&probs[lo + 1].tile_begin) > t) return at = lo;
            ++lo;
        }
        int hi = count - 1;  // last problem whose first tile is <= t
#pragma unroll 1
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&probs[mid].tile_begin) <= t) lo = mid;
            else hi = mid - 1;
        }
        return at = lo;
    }
    __device__ __forceinline__ TileInfo get(int t) {
        const GroupGemmProblem& P = probs[find(t)];
        TileInfo ti;
        decode_local(t - P.tile_begin, P.tiles_m, P.tiles_n, ti.l, ti.mt, ti.nt);
        ti.ta = &P.ta;
        ti.tb = &P.tb;
        ti.k_blocks = P.k_blocks;
        ti.nchunks = P.nchunks;
        ti.bn = P.bn;
        ti.chunk_blocks = P.chunk_blocks;
        ti.out = P.out;
        ti.out_ld = P.out_ld;
        ti.out_plane = P.out_plane;
        ti.m_live = P.m_live;
        ti.n_live = P.n_live;
        return ti;
    }
};

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------- accurate-mode epilogue
// One chunk of the auxiliary product for the 32 rows of this warp (TMEM lane quarter q) and its
// EPI_COLS columns from col0.  Intermediate chunks move x div 4096 into the carry columns;
// the last one forms C-bar and merges the maxima.
__device__ __forceinline__ void aux_epilogue(uint32_t taddr, const TileInfo& ti, int c, int q,
                                             int lane, int col0) {
    const uint32_t carry_addr = taddr + BN;
    const bool last = c + 1 == ti.nchunks;
    uint32_t row_max = 0;
    uint32_t* mx = reinterpret_cast<uint32_t*>(ti.out);
    const int64_t col_base = (int64_t)ti.nt * BN + col0;
#pragma unroll 1
    for (int col = 0; col < EPI_COLS; col += 32) {
        uint32_t v[32], h[32];
        tmem_ld32(taddr + col, v);
        if (c > 0) {
            tmem_ld32(carry_addr + col, h);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) h[j] = 0u;  // 0.0f
        }
        if (!last) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float x = __uint_as_float(v[j]);       // exact integer < 2^24
                const float qq = truncf(x * (1.0f / 4096.0f));
                v[j] = __float_as_uint(fmaf(-qq, 4096.0f, x));
                h[j] = __float_as_uint(__uint_as_float(h[j]) + qq);
            }
            tmem_st32(taddr + col, v);
            tmem_st32(carry_addr + col, h);
        } else {
            uint32_t mine = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const uint32_t cbar = (uint32_t)__uint_as_float(h[j]) * 4096u +
                                      (uint32_t)__uint_as_float(v[j]);
                row_max = cbar > row_max ? cbar : row_max;
                const uint32_t cm = __reduce_max_sync(0xffffffffu, cbar);
                if (lane == j) mine = cm;
            }
            atomicMax(mx + ti.out_ld + col_base + col + lane, mine);
        }
    }
    if (!last) {
        tmem_wait_st();
    } else {
        const int64_t row = (int64_t)ti.mt * BM + q * 32 + lane;
        atomicMax(mx + row, row_max);
    }
}

// ---------------------------------------------------------------- the kernel body
// Tiles t = blockIdx.x + i * gridDim.x of the source, taken two at a time: the two tiles of a
// pair accumulate in the two TMEM buffers and their K chunks alternate (a tile with fewer chunks
// simply drops out), so the reduction of one overlaps the MMAs of the other.
//
// AUX = true computes the auxiliary product C-bar = A-bar B-bar of accurate mode instead (one
// plane of nonnegative integers <= 64, Section 2.3) and keeps only its row and column maxima:
// tiles are taken one at a time, TMEM columns [BN, 2 BN) hold the carries of the exact sum
// (after each chunk the accumulator x < 2^24 is split into x mod 4096, kept, and x div 4096,
// added to the carry column), and the drain forms C-bar = 4096 carry + x as uint32 and merges
// its row and column maxima into `out` (uint32 [rows_pad] then [cols_pad] from offset out_ld).
template <class Src, bool AUX = false>
__device__ __forceinline__ void residue_gemm_body(Src src, int total_tiles,
                                                  const GemmArgs& args) {
    constexpr int PER = AUX ? 1 : 2;  // tiles in flight per CTA (TMEM accumulators in use)
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* smem = smem_raw + pad;
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* acc_full = bars + 2 * STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long lim = args.limit_ns;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tmem_slot)),
            "r"(TMEM_COLS)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int my_tiles = (int)blockIdx.x < total_tiles
                             ? (total_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                             : 0;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0;
        // eviction priorities: A policy in bits 0-1, B policy in bits 2-3 of l2_hints
        const uint64_t pol_a = l2_policy(args.l2_hints & 3), pol_b = l2_policy(args.l2_hints >> 2);
        uint32_t armed_parity[STAGES];
        bool armed[STAGES];
        for (int s = 0; s < STAGES; ++s) armed[s] = false, armed_parity[s] = 0;
        bool ok = true;
        for (int pr = 0; ok && PER * pr < my_tiles; ++pr) {
            const int npair = min(PER, my_tiles - PER * pr);
            TileInfo ti[2];
            for (int s = 0; s < npair; ++s) {
                ti[s] = src.get(blockIdx.x + (PER * pr + s) * gridDim.x);
                if constexpr (Src::kPrefetchMaps) {
                    prefetch_tensormap(ti[s].ta);
                    prefetch_tensormap(ti[s].tb);
                }
            }
            const int maxc = max(ti[0].nchunks, npair > 1 ? ti[1].nchunks : 0);
            for (int c = 0; ok && c < maxc; ++c) {
                for (int s = 0; ok && s < npair; ++s) {
                    if (c >= ti[s].nchunks) continue;
                    const int kb0 = c * ti[s].chunk_blocks;
                    const int kb1 = min(kb0 + ti[s].chunk_blocks, ti[s].k_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, args.status, lim)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[stage], A_BYTES + ti[s].bn * (BK * 2));
                        if (pol_a | pol_b) {
                            tma_load_3d_hint(sA + stage * A_BYTES, ti[s].ta, &full[stage],
                                             kb * BK, ti[s].mt * BM, ti[s].l, pol_a);
                            tma_load_3d_hint(sB + stage * B_BYTES, ti[s].tb, &full[stage],
                                             kb * BK, ti[s].nt * ti[s].bn, ti[s].l, pol_b);
                        } else {
                            tma_load_3d(sA + stage * A_BYTES, ti[s].ta, &full[stage], kb * BK,
                                        ti[s].mt * BM, ti[s].l);
                            tma_load_3d(sB + stage * B_BYTES, ti[s].tb, &full[stage], kb * BK,
                                        ti[s].nt * ti[s].bn, ti[s].l);
                        }
                        armed[stage] = true;
                        armed_parity[stage] = phase;
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
        }
        if (!ok) {  // let every copy this thread started land before the CTA exits
            volatile int no_abort = 0;
            for (int s = 0; s < STAGES; ++s)
                if (armed[s])
                    mbar_wait(&full[s], armed_parity[s], &no_abort, args.status, 100000000ull);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acc_cnt[2] = {0, 0};
        bool ok = true, issued = false;
        for (int pr = 0; ok && PER * pr < my_tiles; ++pr) {
            const int npair = min(PER, my_tiles - PER * pr);
            TileInfo ti[2];
            for (int s = 0; s < npair; ++s)
                ti[s] = src.get(blockIdx.x + (PER * pr + s) * gridDim.x);
            const int maxc = max(ti[0].nchunks, npair > 1 ? ti[1].nchunks : 0);
            for (int c = 0; ok && c < maxc; ++c) {
                for (int s = 0; ok && s < npair; ++s) {
                    if (c >= ti[s].nchunks) continue;
                    if (!mbar_wait(&acc_empty[s], (acc_cnt[s] & 1) ^ 1, abort_flag, args.status,
                                   lim)) {
                        ok = false;
                        break;
                    }
                    ++acc_cnt[s];
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(s * BN);
                    const uint32_t idesc = idesc_for(ti[s].bn);
                    const int kb0 = c * ti[s].chunk_blocks;
                    const int kb1 = min(kb0 + ti[s].chunk_blocks, ti[s].k_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, args.status, lim)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sA + stage * A_BYTES);
                        const uint32_t b0 = smem_u32(sB + stage * B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                            const uint32_t acc = (c > 0 || kb > kb0 || kk > 0) ? 1u : 0u;
                            umma_bf16(d_tmem, sw128_desc(a0 + kk * UMMA_K * 2),
                                      sw128_desc(b0 + kk * UMMA_K * 2), idesc, acc);
                        }
                        issued = true;
                        umma_commit(&empty[stage]);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (ok) umma_commit(&acc_full[s]);
                }
            }
        }
        if (!ok && issued) {  // make sure the MMAs already issued have finished
            volatile int no_abort = 0;
            umma_commit(drain);
            mbar_wait(drain, 0, &no_abort, args.status, 100000000ull);
        }
    } else if (warp >= EPI_WARP0) {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;
        const int half = (warp - EPI_WARP0) >> 2;  // this warp's half of the tile's columns
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t acc_cnt[2] = {0, 0};
        bool ok = true;
        for (int pr = 0; ok && PER * pr < my_tiles; ++pr) {
            const int npair = min(PER, my_tiles - PER * pr);
            TileInfo ti[2];
            for (int s = 0; s < npair; ++s)
                ti[s] = src.get(blockIdx.x + (PER * pr + s) * gridDim.x);
            const int maxc = max(ti[0].nchunks, npair > 1 ? ti[1].nchunks : 0);
            for (int c = 0; ok && c < maxc; ++c) {
                for (int s = 0; ok && s < npair; ++s) {
                    if (c >= ti[s].nchunks) continue;
                    bool got = true;
                    if (lane == 0)
                        got = mbar_wait(&acc_full[s], acc_cnt[s] & 1, abort_flag, args.status,
                                        lim);
                    got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                    if (!got) {
                        ok = false;
                        break;
                    }
                    ++acc_cnt[s];
                    tc_fence_after();
                    const int ncols = ti[s].bn >> 1;  // columns per warp: 128, 64 or 32
                    const int col0 = half * ncols;
                    const uint32_t taddr =
                        tmem_base + lane_base + (uint32_t)(s * BN) + (uint32_t)col0;
                    const int l = ti[s].l;
                    const float p = args.ep.p[l], inv = args.ep.inv_p[l];
                    if (AUX) {
                        aux_epilogue(taddr, ti[s], c, q, lane, col0);
                    } else if (c + 1 < ti[s].nchunks) {
                        // in-place reduction modulo p: |r| <= ~0.52 p
#pragma unroll 1
                        for (int col = 0; col < ncols; col += 32) {
                            uint32_t v[32];
                            tmem_ld32(taddr + col, v);
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const float x = __uint_as_float(v[j]);
                                v[j] = __float_as_uint(fmaf(-round_small(x * inv), p, x));
                            }
                            tmem_st32(taddr + col, v);
                        }
                        tmem_wait_st();
                    } else {
                        // final drain: symmetric residue as int8
                        const float hi = args.ep.hi[l], lo = args.ep.lo[l];
                        // (only rows below m_live and 32-column groups below n_live are stored:
                        // the reconstruction reads no others)
                        const int64_t row = (int64_t)ti[s].mt * BM + q * 32 + lane;
                        const bool row_live = row < ti[s].m_live;
                        const int col_end =
                            min(ncols, ti[s].n_live - ti[s].nt * ti[s].bn - col0);
                        int8_t* dst = ti[s].out + (int64_t)l * ti[s].out_plane +
                                      row * ti[s].out_ld + (int64_t)ti[s].nt * ti[s].bn + col0;
#pragma unroll 1
                        for (int col = 0; col < col_end; col += 32) {
                            uint32_t v[32];
                            tmem_ld32(taddr + col, v);
                            uint32_t packed[8];
#pragma unroll
                            for (int w = 0; w < 8; ++w) {
                                uint32_t word = 0;
#pragma unroll
                                for (int b = 0; b < 4; ++b) {
                                    const float x = __uint_as_float(v[4 * w + b]);
                                    float r = fmaf(-round_small(x * inv), p, x);
                                    r = r > hi ? r - p : r;
                                    r = r < lo ? r + p : r;
                                    word |= ((uint32_t)__float2int_rn(r) & 0xFFu) << (8 * b);
                                }
                                packed[w] = word;
                            }
                            if (row_live) {
                                uint4* o = reinterpret_cast<uint4*>(dst + col);
                                o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                                o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[s]);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();  // lane 0 ran the MMA loop alone; the dealloc is warp-collective
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    residue_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB, const GemmArgs args) {
    // a copy launched after this GEMM with programmatic serialization may run beside it (the
    // pipelined host-operand path); every CTA is resident when it gets here
    pdl_launch_dependents();
    const SingleSource src{&tmA, &tmB, &args};
    residue_gemm_body(src, args.total_tiles, args);
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    residue_gemm_grouped_kernel(const GroupGemmProblem* __restrict__ probs, int count,
                                int total_tiles, const GemmArgs args) {
    const GroupSource src{probs, count};
    residue_gemm_body(src, total_tiles, args);
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    aux_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB, const GemmArgs args) {
    const SingleSource src{&tmA, &tmB, &args};
    residue_gemm_body<SingleSource, true>(src, args.total_tiles, args);
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    aux_gemm_grouped_kernel(const GroupGemmProblem* __restrict__ probs, int count,
                            int total_tiles, const GemmArgs args) {
    const GroupSource src{probs, count};
    residue_gemm_body<GroupSource, true>(src, total_tiles, args);
}

// ---------------------------------------------------------------- the 2-SM kernel
// A cluster of two CTAs on a pair of SMs computes a 256 x 256 tile with tcgen05.mma
// cta_group::2 (M = 256, N = 256, K = 16).  Each CTA loads its own 128 rows of A and its 128-row
// half of B per stage (32 KiB, 6 stages), so each SM takes in two thirds of the bytes per FLOP of
// the 1-SM kernel.  The even CTA (the leader) issues the MMAs; each CTA's TMEM holds its own 128
// rows x 256 columns of the accumulators, which its own epilogue warps reduce and drain exactly as
// in the 1-SM kernel.  Synchronisation across the pair: TMA completions of both CTAs land on the
// leader's full barriers; MMA commits are multicast to both CTAs' empty and acc_full barriers;
// the peer's epilogue warps arrive remotely on the leader's acc_empty barriers.
namespace pair {
constexpr int BM = 256, BN = 256, HALF = 128, STAGES = 6;
constexpr int A_BYTES = HALF * BK * 2;          // 16 KiB
constexpr int B_BYTES = HALF * BK * 2;          // 16 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * BN;
constexpr int NUM_BARRIERS = 2 * STAGES + 5;
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + NUM_BARRIERS * 8 + 16;
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
}  // namespace pair

__global__ void __launch_bounds__(NUM_THREADS, 1)
    residue_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                             const __grid_constant__ CUtensorMap tmB, const GemmArgs args) {
    pdl_launch_dependents();  // as in residue_gemm_kernel
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t* smem = smem_raw + pad;
    uint8_t* sA = smem;
    uint8_t* sB = smem + pair::STAGES * pair::A_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + pair::STAGES * pair::B_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + pair::STAGES;
    uint64_t* acc_full = bars + 2 * pair::STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long lim = args.limit_ns;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cluster = (int)(blockIdx.x >> 1), nclusters = (int)(gridDim.x >> 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < pair::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 2 * EPI_WARPS);   // epilogue warps of both CTAs of the pair
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {  // collective over the pair: one warp in each CTA
        asm volatile(
            "tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tmem_slot)),
            "r"(pair::TMEM_COLS)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int my_tiles = cluster < args.total_tiles
                             ? (args.total_tiles - 1 - cluster) / nclusters + 1
                             : 0;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ TMA producer (both CTAs)
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true, started = false;
        for (int pr = 0; ok && 2 * pr < my_tiles; ++pr) {
            const int npair = min(2, my_tiles - 2 * pr);
            for (int c = 0; ok && c < args.nchunks; ++c) {
                for (int s = 0; ok && s < npair; ++s) {
                    const int tile = cluster + (2 * pr + s) * nclusters;
                    int l, mt, nt;
                    decode_tile(tile, args, l, mt, nt);
                    const int kb0 = c * args.chunk_blocks;
                    const int kb1 = min(kb0 + args.chunk_blocks, args.k_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, args.status, lim)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = map_to_rank(smem_u32(&full[stage]), 0);
                        if (leader) mbar_arrive_expect_tx(&full[stage], 2 * pair::STAGE_BYTES);
                        tma_load_3d_pair(sA + stage * pair::A_BYTES, &tmA, fb, kb * BK,
                                         mt * pair::BM + (int)rank * pair::HALF, l);
                        tma_load_3d_pair(sB + stage * pair::B_BYTES, &tmB, fb, kb * BK,
                                         nt * pair::BN + (int)rank * pair::HALF, l);
                        started = true;
                        if (++stage == pair::STAGES) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
        }
        if (!ok && started) spin_ns(2000000ull);  // let copies already issued land
    } else if (warp == 1 && lane == 0 && leader) {
        // ------------------------------------------------------------ MMA issuer (leader)
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acc_cnt[2] = {0, 0};
        bool ok = true, issued = false;
        for (int pr = 0; ok && 2 * pr < my_tiles; ++pr) {
            const int npair = min(2, my_tiles - 2 * pr);
            for (int c = 0; ok && c < args.nchunks; ++c) {
                for (int s = 0; ok && s < npair; ++s) {
                    if (!mbar_wait(&acc_empty[s], (acc_cnt[s] & 1) ^ 1, abort_flag, args.status,
                                   lim)) {
                        ok = false;
                        break;
                    }
                    ++acc_cnt[s];
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(s * pair::BN);
                    const int kb0 = c * args.chunk_blocks;
                    const int kb1 = min(kb0 + args.chunk_blocks, args.k_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, args.status, lim)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sA + stage * pair::A_BYTES);
                        const uint32_t b0 = smem_u32(sB + stage * pair::B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                            const uint32_t acc = (c > 0 || kb > kb0 || kk > 0) ? 1u : 0u;
                            umma_bf16_pair(d_tmem, sw128_desc(a0 + kk * UMMA_K * 2),
                                           sw128_desc(b0 + kk * UMMA_K * 2), pair::IDESC, acc);
                        }
                        issued = true;
                        umma_commit_pair_both(&empty[stage]);
                        if (++stage == pair::STAGES) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (ok) umma_commit_pair_both(&acc_full[s]);
                }
            }
        }
        if (!ok && issued) {  // make sure the MMAs already issued have finished
            volatile int no_abort = 0;
            umma_commit_pair_local(drain);
            mbar_wait(drain, 0, &no_abort, args.status, 100000000ull);
        }
    } else if (warp >= EPI_WARP0) {
        // ------------------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;
        const int col0 = ((warp - EPI_WARP0) >> 2) * EPI_COLS;  // this warp's half of the columns
        const uint32_t lane_base = ((uint32_t)(q * 32) << 16) + (uint32_t)col0;
        uint32_t acc_cnt[2] = {0, 0};
        const uint32_t empty_remote[2] = {map_to_rank(smem_u32(&acc_empty[0]), 0),
                                          map_to_rank(smem_u32(&acc_empty[1]), 0)};
        bool ok = true;
        for (int pr = 0; ok && 2 * pr < my_tiles; ++pr) {
            const int npair = min(2, my_tiles - 2 * pr);
            for (int c = 0; ok && c < args.nchunks; ++c) {
                for (int s = 0; ok && s < npair; ++s) {
                    const int tile = cluster + (2 * pr + s) * nclusters;
                    int l, mt, nt;
                    decode_tile(tile, args, l, mt, nt);
                    bool got = true;
                    if (lane == 0)
                        got = mbar_wait(&acc_full[s], acc_cnt[s] & 1, abort_flag, args.status,
                                        lim);
                    got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                    if (!got) {
                        ok = false;
                        break;
                    }
                    ++acc_cnt[s];
                    tc_fence_after();
                    const uint32_t taddr = tmem_base + lane_base + (uint32_t)(s * pair::BN);
                    const float p = args.ep.p[l], inv = args.ep.inv_p[l];
                    if (c + 1 < args.nchunks) {
#pragma unroll 1
                        for (int col = 0; col < EPI_COLS; col += 32) {
                            uint32_t v[32];
                            tmem_ld32(taddr + col, v);
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const float x = __uint_as_float(v[j]);
                                v[j] = __float_as_uint(fmaf(-round_small(x * inv), p, x));
                            }
                            tmem_st32(taddr + col, v);
                        }
                        tmem_wait_st();
                    } else {
                        const float hi = args.ep.hi[l], lo = args.ep.lo[l];
                        const int64_t row = (int64_t)mt * pair::BM + (int64_t)rank * pair::HALF + q * 32 + lane;
                        const bool live = row < args.m_rows;
                        int8_t* dst = args.out + (int64_t)l * args.out_plane +
                                      (live ? row : 0) * args.out_ld + (int64_t)nt * pair::BN +
                                      col0;
#pragma unroll 1
                        for (int col = 0; col < EPI_COLS; col += 32) {
                            uint32_t v[32];
                            tmem_ld32(taddr + col, v);
                            uint32_t packed[8];
#pragma unroll
                            for (int w = 0; w < 8; ++w) {
                                uint32_t word = 0;
#pragma unroll
                                for (int b = 0; b < 4; ++b) {
                                    const float x = __uint_as_float(v[4 * w + b]);
                                    float r = fmaf(-round_small(x * inv), p, x);
                                    r = r > hi ? r - p : r;
                                    r = r < lo ? r + p : r;
                                    word |= ((uint32_t)__float2int_rn(r) & 0xFFu) << (8 * b);
                                }
                                packed[w] = word;
                            }
                            if (live) {
                                uint4* o = reinterpret_cast<uint4*>(dst + col);
                                o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                                o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (leader) mbar_arrive(&acc_empty[s]);
                        else mbar_arrive_cluster(empty_remote[s]);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(pair::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D map over residue planes [N][rows][ld] (bf16, K contiguous), box 64 x box_rows x 1; the
// boxes of the tile grid that reach beyond rows or ld read zeros.
// rows: the rows the GEMM may read from each plane (rows beyond read as zeros); plane_rows: the
// rows from one plane to the next (0: rows).
bool encode_planes(CUtensorMap* map, const void* base, int N, int rows, int ld, int box_rows,
                   int plane_rows = 0) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    if (plane_rows <= 0) plane_rows = rows;
    if (plane_rows < rows) return false;
    cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)N};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)plane_rows * (cuuint64_t)ld * 2};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The dynamic shared-memory limit is a per-device attribute of a kernel: set it once for each
// device a launch is made on (bit d of `done` marks device d).
std::mutex g_attr_mu;
cudaError_t ensure_smem_attr(const void* kernel, int bytes, uint64_t& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    const uint64_t bit = dev < 64 ? 1ull << dev : 0;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (bit && (done & bit)) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}
uint64_t g_attr_grouped = 0, g_attr_aux = 0, g_attr_aux_grouped = 0, g_attr_pair = 0,
         g_attr_single = 0;

}  // namespace

// K blocks (of 64) between modular reductions: at most chunk_k / 64 (and at most 15: <= 960
// products keep the fp32 accumulator exact), spread evenly over the same number of chunks, so
// that no chunk is a short remainder (k = 1024: 8 + 8 blocks rather than 15 + 1).
static int chunk_blocks_of(int chunk_k, int k_blocks) {
    int cb = chunk_k / BK;
    if (cb < 1) cb = 1;
    if (cb > 15) cb = 15;
    if (k_blocks <= 0) return cb;
    const int nchunks = (k_blocks + cb - 1) / cb;
    return (k_blocks + nchunks - 1) / nchunks;
}

bool make_group_gemm_problem(GroupGemmProblem* g, int N, int m_pad, int n_pad, int k_pad,
                             const PlaneGeom& geo, const void* planes_a, const void* planes_b,
                             int8_t* out, int chunk_k, int bn) {
    if (bn != 64 && bn != 128 && bn != BN) return false;
    if (n_pad % bn || geo.rows_b < bn) return false;
    if (!encode_planes(&g->ta, planes_a, N, geo.rows_a, geo.ld, BM) ||
        !encode_planes(&g->tb, planes_b, N, geo.rows_b, geo.ld, bn))
        return false;
    const int cb = chunk_blocks_of(chunk_k, k_pad / BK);
    g->out = out;
    g->out_ld = n_pad;
    g->out_plane = (int64_t)m_pad * n_pad;
    g->bn = bn;
    g->chunk_blocks = cb;
    g->tiles_m = m_pad / BM;
    g->tiles_n = n_pad / bn;
    g->k_blocks = k_pad / BK;
    g->nchunks = (g->k_blocks + cb - 1) / cb;
    g->m_live = geo.out_rows;
    g->n_live = geo.out_cols;
    g->tile_begin = 0;
    return true;
}

int launch_residue_gemm_grouped(const GroupGemmProblem* probs, int count, int total_tiles,
                                const EpilogueTables& t, unsigned* status, int num_sms,
                                int chunk_k, cudaStream_t stream, unsigned long long limit_ns) {
    if (count <= 0 || total_tiles <= 0) return OZAKI2_SUCCESS;
    if (ensure_smem_attr((const void*)residue_gemm_grouped_kernel, (int)SMEM_BYTES,
                         g_attr_grouped) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    GemmArgs a = {};
    a.chunk_blocks = 15;  // unused: each problem carries its own chunk
    a.status = status;
    a.limit_ns = limit_ns;
    a.ep = t;
    const int grid = total_tiles < num_sms ? total_tiles : num_sms;
    residue_gemm_grouped_kernel<<<grid, NUM_THREADS, SMEM_BYTES, stream>>>(probs, count,
                                                                          total_tiles, a);
    return cudaGetLastError() == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
}

// Products accumulated between carry passes of the auxiliary product: 63 x 64 x 64^2 plus a
// kept remainder below 4096 stays under 2^24, where fp32 sums of integers are exact.
constexpr int kAuxChunkBlocks = 63;

int launch_aux_gemm(int m_pad, int n_pad, int k_pad, const PlaneGeom& geo, const void* bar_a,
                    const void* bar_b, uint32_t* cmax, unsigned* status, int num_sms,
                    cudaStream_t stream, unsigned long long limit_ns) {
    if (m_pad == 0 || n_pad == 0) return OZAKI2_SUCCESS;
    if (cudaMemsetAsync(cmax, 0, sizeof(uint32_t) * ((size_t)m_pad + n_pad), stream) !=
        cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    if (k_pad == 0) return OZAKI2_SUCCESS;
    GemmArgs a = {};
    a.k_blocks = k_pad / BK;
    a.chunk_blocks = kAuxChunkBlocks;
    a.nchunks = (a.k_blocks + kAuxChunkBlocks - 1) / kAuxChunkBlocks;
    a.group_m = GROUP_M;
    a.m_rows = m_pad;
    a.out = reinterpret_cast<int8_t*>(cmax);
    a.out_ld = m_pad;
    a.out_plane = 0;
    a.status = status;
    a.limit_ns = limit_ns;
    CUtensorMap ta, tb;
    if (!encode_planes(&ta, bar_a, 1, geo.rows_a, geo.ld, BM) ||
        !encode_planes(&tb, bar_b, 1, geo.rows_b, geo.ld, BN))
        return OZAKI2_ERROR_DRIVER;
    if (ensure_smem_attr((const void*)aux_gemm_kernel, (int)SMEM_BYTES, g_attr_aux) !=
        cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    a.tiles_m = m_pad / BM;
    a.tiles_n = n_pad / BN;
    a.total_tiles = a.tiles_m * a.tiles_n;
    const int grid = a.total_tiles < num_sms ? a.total_tiles : num_sms;
    aux_gemm_kernel<<<grid, NUM_THREADS, SMEM_BYTES, stream>>>(ta, tb, a);
    return cudaGetLastError() == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
}

bool make_group_aux_problem(GroupGemmProblem* g, int m_pad, int n_pad, int k_pad,
                            const PlaneGeom& geo, const void* bar_a, const void* bar_b,
                            uint32_t* cmax) {
    if (!encode_planes(&g->ta, bar_a, 1, geo.rows_a, geo.ld, BM) ||
        !encode_planes(&g->tb, bar_b, 1, geo.rows_b, geo.ld, BN))
        return false;
    g->out = reinterpret_cast<int8_t*>(cmax);
    g->out_ld = m_pad;  // the column maxima follow the m_pad row maxima
    g->out_plane = 0;
    g->bn = BN;
    g->chunk_blocks = kAuxChunkBlocks;
    g->tiles_m = m_pad / BM;
    g->tiles_n = n_pad / BN;
    g->k_blocks = k_pad / BK;
    g->nchunks = (g->k_blocks + kAuxChunkBlocks - 1) / kAuxChunkBlocks;
    g->tile_begin = 0;
    return true;
}

int launch_aux_gemm_grouped(const GroupGemmProblem* probs, int count, int total_tiles,
                            unsigned* status, int num_sms, cudaStream_t stream,
                            unsigned long long limit_ns) {
    if (count <= 0 || total_tiles <= 0) return OZAKI2_SUCCESS;
    if (ensure_smem_attr((const void*)aux_gemm_grouped_kernel, (int)SMEM_BYTES,
                         g_attr_aux_grouped) != cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    GemmArgs a = {};
    a.chunk_blocks = kAuxChunkBlocks;
    a.status = status;
    a.limit_ns = limit_ns;
    const int grid = total_tiles < num_sms ? total_tiles : num_sms;
    aux_gemm_grouped_kernel<<<grid, NUM_THREADS, SMEM_BYTES, stream>>>(probs, count, total_tiles,
                                                                      a);
    return cudaGetLastError() == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
}

int launch_residue_gemm(int num_moduli, int m_pad, int n_pad, int k_pad, const PlaneGeom& geo,
                        const void* planes_a, const void* planes_b, int8_t* out,
                        const EpilogueTables& t, unsigned* status, int num_sms, int chunk_k,
                        int variant, cudaStream_t stream, unsigned long long limit_ns,
                        int64_t out_ld, int64_t out_plane, int group_m, int l2_hints) {
    if (m_pad == 0 || n_pad == 0) return OZAKI2_SUCCESS;
    if (out_ld <= 0) out_ld = n_pad;
    if (out_plane <= 0) out_plane = (int64_t)m_pad * out_ld;
    GemmArgs a = {};
    a.l2_hints = l2_hints;
    a.k_blocks = k_pad / BK;
    const int cb = chunk_blocks_of(chunk_k, a.k_blocks);
    a.chunk_blocks = cb;
    a.nchunks = a.k_blocks > 0 ? (a.k_blocks + cb - 1) / cb : 0;
    a.m_rows = m_pad;
    a.m_live = geo.out_rows;
    a.n_live = geo.out_cols;
    a.out = out;
    a.out_ld = out_ld;
    a.out_plane = out_plane;
    a.group_m = group_m;  // 0: the kernel's default, set below
    a.status = status;
    a.limit_ns = limit_ns;
    a.ep = t;
    if (a.k_blocks == 0) {  // empty inner dimension: every product residue is zero
        if (out_ld != n_pad || out_plane != (int64_t)m_pad * n_pad) return OZAKI2_ERROR_CUDA;
        cudaError_t e = cudaMemsetAsync(out, 0, (size_t)num_moduli * m_pad * n_pad, stream);
        return e == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
    }
    // Automatic choice, from timings on GB300 (square DGEMMs, N = 16): the SM-pair kernel is
    // 2-3% faster when both padded dimensions lie in [2048, 8192]; the one-SM kernel is faster
    // below (equal at 1024) and 11% faster at 16384, where 304 tiles in flight fill the machine.
    const bool auto_pair = m_pad >= 2048 && n_pad >= 2048 && m_pad <= 8192 && n_pad <= 8192;
    const bool use_pair =
        variant == OZAKI2_GEMM_PAIR || (variant == OZAKI2_GEMM_AUTO && auto_pair);
    CUtensorMap ta, tb;
    if (use_pair) {
        if (!encode_planes(&ta, planes_a, num_moduli, geo.rows_a, geo.ld, pair::HALF,
                           geo.plane_rows_a) ||
            !encode_planes(&tb, planes_b, num_moduli, geo.rows_b, geo.ld, pair::HALF))
            return OZAKI2_ERROR_DRIVER;
        if (ensure_smem_attr((const void*)residue_gemm_pair_kernel, (int)pair::SMEM_BYTES,
                             g_attr_pair) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        if (a.group_m <= 0) a.group_m = GROUP_M_PAIR;
        a.tiles_m = (m_pad + pair::BM - 1) / pair::BM;
        a.tiles_n = n_pad / pair::BN;
        a.total_tiles = a.tiles_m * a.tiles_n * num_moduli;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(NUM_THREADS);
        cfg.dynamicSmemBytes = pair::SMEM_BYTES;
        cfg.stream = stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int max_clusters = num_sms / 2;
        cfg.gridDim = dim3(2 * max_clusters);
        int q = 0;
        if (cudaOccupancyMaxActiveClusters(&q, residue_gemm_pair_kernel, &cfg) == cudaSuccess &&
            q > 0 && q < max_clusters)
            max_clusters = q;
        cudaGetLastError();
        const int clusters = a.total_tiles < max_clusters ? a.total_tiles : max_clusters;
        cfg.gridDim = dim3(2 * clusters);
        if (cudaLaunchKernelEx(&cfg, residue_gemm_pair_kernel, ta, tb, a) != cudaSuccess)
            return OZAKI2_ERROR_CUDA;
        return cudaGetLastError() == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
    }
    if (!encode_planes(&ta, planes_a, num_moduli, geo.rows_a, geo.ld, BM, geo.plane_rows_a) ||
        !encode_planes(&tb, planes_b, num_moduli, geo.rows_b, geo.ld, BN))
        return OZAKI2_ERROR_DRIVER;
    if (ensure_smem_attr((const void*)residue_gemm_kernel, (int)SMEM_BYTES, g_attr_single) !=
        cudaSuccess)
        return OZAKI2_ERROR_CUDA;
    if (a.group_m <= 0) a.group_m = GROUP_M_SINGLE;
    a.tiles_m = m_pad / BM;
    a.tiles_n = n_pad / BN;
    a.total_tiles = a.tiles_m * a.tiles_n * num_moduli;
    const int grid = a.total_tiles < num_sms ? a.total_tiles : num_sms;
    residue_gemm_kernel<<<grid, NUM_THREADS, SMEM_BYTES, stream>>>(ta, tb, a);
    return cudaGetLastError() == cudaSuccess ? OZAKI2_SUCCESS : OZAKI2_ERROR_CUDA;
}

}  // namespace ozaki2
