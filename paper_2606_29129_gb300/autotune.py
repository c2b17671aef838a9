"""Choice of the number of moduli N per size class (accuracy autotuning).

More moduli make P larger, so the scaled integers keep more bits and the emulated product is
more accurate (Section 2.2; the error falls roughly 16-20x per modulus).  The cost grows
linearly in N.  For each size class this module measures, on synthetic inputs drawn like the
paper's (eq. random-matrix-generation), the maximum relative error of the emulation for each
candidate N, and that of cuBLAS DGEMM on the same inputs.  The reference is the emulation with
N = 20, whose error is at the level of one rounding of the result (~1e-16), far below the
errors being compared.  `choose_n` then picks the smallest N that is not worse than cuBLAS
(equal accuracy) or that meets a stated relative-error target.
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
              device="cuda"):
    """Errors per size class: {class: {"N": {N: err}, "cublas": err}} (max over phis/samples).

    Each class is measured on a square problem of its edge size (m = n = k, capped at 4096 for
    the calibration cost; the error depends mainly on k)."""
    import torch

    from synthetic import paper_matrix_torch  # the shared input generator

    ks = ks or CLASS_EDGES
    out = {}
    h = oz.Handle()
    for ci, k in enumerate(ks):
        m = n = min(k, 4096)
        errs = {N: 0.0 for N in candidates}
        cub = 0.0
        for phi in phis:
            for s in range(samples):
                A = paper_matrix_torch(m, k, phi, seed + 17 * ci + 3 * s + 1, device=device)
                B = paper_matrix_torch(k, n, phi, seed + 17 * ci + 3 * s + 2, device=device)
                ref = torch.empty((n, m), dtype=torch.float64, device=device)
                oz._check("ozaki2_dgemm", oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0,
                                                          ref, m, 20, h))
                C = torch.empty_like(ref)
                for N in candidates:
                    oz._check("ozaki2_dgemm", oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k,
                                                              0.0, C, m, N, h))
                    errs[N] = max(errs[N], _max_rel(C, ref))
                Cd = torch.matmul(B.view(n, k), A.view(k, m))
                cub = max(cub, _max_rel(Cd, ref))
        out[size_class(k)] = {"k": k, "N": errs, "cublas": cub}
    return out


def choose_n(table, k: int, target: float | None = None, default: int = 16) -> int:
    """Smallest calibrated N whose error is <= target (or <= cuBLAS DGEMM's when target is None)
    for the size class of k; `default` if the class was not calibrated."""
    entry = table.get(size_class(k))
    if entry is None:
        return default
    bound = entry["cublas"] if target is None else target
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


def log2_gap(a: float, b: float) -> float:
    return math.log2(max(a, 1e-300) / max(b, 1e-300))
