"""Autotuning per size class: the number of moduli N (by accuracy) and the residue-GEMM
configuration, kernel variant (tile shape) and K chunk (by time).

More moduli make P larger, so the scaled integers keep more bits and the emulated product is
more accurate (Section 2.2; the error falls roughly 16-20x per modulus).  The cost grows
linearly in N.  For each size class this module measures, on synthetic inputs drawn like the
paper's (eq. random-matrix-generation), the maximum relative error of the emulation for each
candidate N, and that of cuBLAS DGEMM on the same inputs.  The reference is the emulation with
N = 20, whose error is at the level of one rounding of the result (~1e-16), far below the
errors being compared.  `choose_n` then picks the smallest N that is not worse than cuBLAS
(equal accuracy) or that meets a stated relative-error target.  `tune_tiles` and
`tune_grouped_chunk` / `tune_grouped_tiles` time the residue-GEMM configurations (see below).
"""
from __future__ import annotations

import math

from . import ozaki2 as oz

# Size classes by inner dimension k: the error of both methods grows with k.
CLASS_EDGES = (64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384)


def size_class(k: int) -> int:
    """Index of the smallest class edge >= k (the last class for larger k)."""
    for i, e in enumerate(CLASS_EDGES):
        if k <= e:
            return i
    return len(CLASS_EDGES) - 1


def _max_rel(C, R):
    import torch

    nz = R != 0
    d = (C - R).abs()
    return float(torch.where(nz, d / R.abs().clamp_min(1e-300), torch.zeros_like(d)).max())


def calibrate(ks=None, candidates=range(8, 21), phis=(0.5, 1.0, 2.0), samples=1, seed=0,
              device="cuda", reference=None, max_mn=4096):
    """Errors per size class: {class: {"N": {N: err}, "cublas": err}} (max over phis/samples).

    Each class is measured on a square problem of its edge size (m = n = k, m and n capped at
    max_mn for the calibration cost; the error depends mainly on k).  `reference(A, B, m, n, k)`
    returns (rows, cols, C_ref) with C_ref an exact-enough product on the entries (rows, cols)
    (torch tensors, C_ref indexed [cols][rows] like the column-major result); by default it is
    the emulation with N = 20 on every entry, whose error (about one rounding of the result) is
    far below the errors being compared down to targets of ~1e-14."""
    import torch

    from synthetic import paper_matrix_torch  # the shared input generator

    ks = ks or CLASS_EDGES
    out = {}
    h = oz.Handle()

    def emulated_reference(A, B, m, n, k):
        ref = torch.empty((n, m), dtype=torch.float64, device=device)
        oz._check("ozaki2_dgemm", oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0,
                                                  ref, m, 20, h))
        return None, None, ref

    reference = reference or emulated_reference
    for ci, k in enumerate(ks):
        m = n = min(k, max_mn)
        errs = {N: 0.0 for N in candidates}
        cub = 0.0
        for phi in phis:
            for s in range(samples):
                A = paper_matrix_torch(m, k, phi, seed + 17 * ci + 3 * s + 1, device=device)
                B = paper_matrix_torch(k, n, phi, seed + 17 * ci + 3 * s + 2, device=device)
                rows, cols, ref = reference(A, B, m, n, k)

                def pick(X):
                    return X if rows is None else X[cols][:, rows]

                C = torch.empty((n, m), dtype=torch.float64, device=device)
                for N in candidates:
                    oz._check("ozaki2_dgemm", oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k,
                                                              0.0, C, m, N, h))
                    errs[N] = max(errs[N], _max_rel(pick(C), ref))
                Cd = torch.matmul(B.view(n, k), A.view(k, m))
                cub = max(cub, _max_rel(pick(Cd), ref))
        out[size_class(k)] = {"k": k, "N": errs, "cublas": cub}
    return out


def choose_n(table, k: int, target: float | None = None, default: int = 16,
             margin: float = 1.0) -> int:
    """Smallest calibrated N whose error is <= target / margin (or <= cuBLAS DGEMM's / margin
    when target is None) for the size class of k; `default` if the class was not calibrated.
    A margin above 1 covers problems of the class whose error ratio to cuBLAS exceeds the
    calibration problem's (the ratio of maximum relative errors varies from problem to
    problem)."""
    entry = table.get(size_class(k))
    if entry is None:
        return default
    bound = (entry["cublas"] if target is None else target) / margin
    for N in sorted(entry["N"]):
        if entry["N"][N] <= bound:
            return N
    return max(entry["N"])


def table_to_json(table):
    return {str(c): {"k": v["k"], "cublas": v["cublas"],
                     "N": {str(N): e for N, e in v["N"].items()}} for c, v in table.items()}


def table_from_json(d):
    return {int(c): {"k": v["k"], "cublas": v["cublas"],
                     "N": {int(N): e for N, e in v["N"].items()}} for c, v in d.items()}


CALIBRATION_FILE = "calibration_gb300.json"


def load_calibration(path=None):
    """The committed calibration table (errors against the double-double reference, measured
    on GB300 by `bench.py --calibrate`), or None when the file is absent."""
    import json
    import os

    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), CALIBRATION_FILE)
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return table_from_json(json.load(fh)["table"])


def log2_gap(a: float, b: float) -> float:
    return math.log2(max(a, 1e-300) / max(b, 1e-300))


# ---- residue-GEMM configuration (timing autotuning) ------------------------------------------
# The residue GEMM has two kernels, 128 x 256 tiles with one CTA per SM (OZAKI2_GEMM_SINGLE) and
# 256 x 256 tiles on SM pairs (OZAKI2_GEMM_PAIR), and a K chunk between the in-place modular
# reductions (OZAKI2_OPT_CHUNK_K, at most 960 products to keep the FP32 accumulator exact).  The
# product residues, and so the results, are bit-identical for every configuration; only the time
# differs, so the choice is made by timing.
TILE_VARIANTS = (oz.GEMM_SINGLE, oz.GEMM_PAIR)
CHUNKS = (960, 640, 448, 320)


def best_config(timings):
    """The fastest configuration of a {config: ms} mapping (the first listed on a tie)."""
    order = list(timings)
    return min(order, key=lambda c: (timings[c], order.index(c)))


def _time_ms(fn, reps):
    import torch

    fn()  # warm-up (and, for grouped calls, the graph capture)
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune_tiles(sizes=(1024, 2048, 4096, 8192, 16384), N=16, variants=TILE_VARIANTS,
               chunks=CHUNKS, reps=3, seed=0, device="cuda", groups=(0,)):
    """Times ozaki2_dgemm on m = n = k = size for every (kernel variant, K chunk, tile-order
    group size; 0 = the library's default) and returns {size_class(size): {"size": size,
    "ms": {(variant, chunk, group): ms}, "best": (variant, chunk, group)}}."""
    import torch

    import synthetic

    out = {}
    for size in sizes:
        m = n = k = size
        A = synthetic.paper_matrix_torch(m, k, 1.0, seed + 3 * size + 1, device=device)
        B = synthetic.paper_matrix_torch(k, n, 1.0, seed + 3 * size + 2, device=device)
        C = torch.empty((n, m), dtype=torch.float64, device=device)
        h = oz.Handle()
        ms = {}
        for variant in variants:
            for chunk in chunks:
                for group in groups:
                    h.set_option(oz.OPT_GEMM_VARIANT, variant)
                    h.set_option(oz.OPT_CHUNK_K, chunk)
                    h.set_option(oz.OPT_GROUP_M, group)

                    def call():
                        oz._check("ozaki2_dgemm", oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B,
                                                                  k, 0.0, C, m, N, h))

                    ms[(variant, chunk, group)] = _time_ms(call, reps)
        out[size_class(k)] = {"size": size, "ms": ms, "best": best_config(ms)}
    return out


def apply_tiles(handle, table, k: int) -> bool:
    """Sets the handle's kernel variant and K chunk to the tuned ones of k's size class; False
    (handle unchanged) when the class was not tuned."""
    entry = table.get(size_class(k))
    if entry is None:
        return False
    variant, chunk, *group = entry["best"]
    handle.set_option(oz.OPT_GEMM_VARIANT, variant)
    handle.set_option(oz.OPT_CHUNK_K, chunk)
    handle.set_option(oz.OPT_GROUP_M, group[0] if group else 0)
    return True


# Size classes of grouped calls for the residue-GEMM tile configuration, by the number of columns
# n of op(B) (the tile width is the number of columns of C one tile covers: 256, 128 or 64).
GROUPED_N_EDGES = (64, 128, 256, 512, 1 << 30)
TILE_WIDTHS = oz.TILE_WIDTHS
_ANY_K = 1 << 30


def grouped_rules(config):
    """ozaki2_set_grouped_tiles rules from {n_edge: (tile_n, chunk_k)} (classes by n)."""
    return [(edge, _ANY_K, tn, ck) for edge, (tn, ck) in sorted(config.items())]


def tune_grouped_tiles(call, handle, n_edges=GROUPED_N_EDGES, widths=TILE_WIDTHS,
                       chunks=CHUNKS, reps=3, rounds=1):
    """Tile width and K chunk per size class (classes by n, the edges `n_edges`) for a grouped
    call: `call()` issues the grouped call on `handle`.  Coordinate descent from the automatic
    configuration: for each class in turn, each tile width, then each chunk, is timed with the
    other classes at their current best; a change is kept only when it is faster.  Leaves the
    best rules set on the handle and returns a dict with the rules, the start and best times
    and every timing.  Results are bit-identical for every configuration."""
    handle.set_grouped_tiles([])
    base = _time_ms(call, reps)
    # start: every class at its automatic width (as the library picks it) and the handle's chunk
    config = {e: (_auto_width(e), 0) for e in n_edges}
    handle.set_grouped_tiles(grouped_rules(config))
    best = _time_ms(call, reps)
    trials = {"auto": base, "start": best}
    for _ in range(rounds):
        for e in n_edges:
            for tn in widths:
                if tn == config[e][0]:
                    continue
                trial = dict(config)
                trial[e] = (tn, config[e][1])
                handle.set_grouped_tiles(grouped_rules(trial))
                t = _time_ms(call, reps)
                trials[f"n<={e}:tile={tn},chunk={config[e][1]}"] = t
                if t < best:
                    best, config = t, trial
            for ck in chunks:
                if ck == config[e][1]:
                    continue
                trial = dict(config)
                trial[e] = (config[e][0], ck)
                handle.set_grouped_tiles(grouped_rules(trial))
                t = _time_ms(call, reps)
                trials[f"n<={e}:tile={config[e][0]},chunk={ck}"] = t
                if t < best:
                    best, config = t, trial
    if base <= best:  # the automatic choice was not beaten
        handle.set_grouped_tiles([])
        return {"rules": [], "auto_ms": base, "best_ms": base, "trials": trials}
    handle.set_grouped_tiles(grouped_rules(config))
    return {"rules": grouped_rules(config), "auto_ms": base, "best_ms": best, "trials": trials}


def _auto_width(n_edge: int) -> int:
    """The library's automatic width for the widest problem of a class (64 for n <= 64, 128 for
    n <= 128, else 256)."""
    return 64 if n_edge <= 64 else 128 if n_edge <= 128 else 256


def tune_grouped_chunk(call, handle, chunks=CHUNKS, reps=3):
    """K chunk for a grouped call (one kernel, one tile shape for every problem): times `call()`,
    which issues the grouped call on `handle`, for each chunk; leaves the fastest set on the
    handle and returns ({chunk: ms}, best chunk)."""
    ms = {}
    for chunk in chunks:
        handle.set_option(oz.OPT_CHUNK_K, chunk)
        ms[chunk] = _time_ms(call, reps)
    best = best_config(ms)
    handle.set_option(oz.OPT_CHUNK_K, best)
    return ms, best


def tiles_to_json(table):
    def best(b):
        out = {"variant": b[0], "chunk_k": b[1]}
        if len(b) > 2:
            out["group_m"] = b[2]
        return out

    return {str(c): {"size": v["size"], "best": best(v["best"]),
                     "ms": {"/".join(str(x) for x in key): t for key, t in v["ms"].items()}}
            for c, v in table.items()}
