"""The autotuner on the GPU: the timed residue-GEMM configurations all give bit-identical
results, and the tuned handle computes the same product as the default one."""
import numpy as np
import pytest

import synthetic
import _gpu

pytestmark = pytest.mark.gpu


def test_tune_tiles_and_apply(orc):
    import torch

    from paper_2606_29129_gb300 import autotune
    from paper_2606_29129_gb300 import ozaki2 as oz

    table = autotune.tune_tiles(sizes=(512,), N=14, chunks=(960, 320), reps=1, groups=(0, 2))
    entry = table[autotune.size_class(512)]
    assert set(entry["ms"]) == {(v, c, g) for v in autotune.TILE_VARIANTS for c in (960, 320)
                                for g in (0, 2)}
    assert entry["best"] in entry["ms"] and all(t > 0 for t in entry["ms"].values())
    m, n, k, N = 300, 520, 512, 14
    A = synthetic.paper_matrix(m, k, 1.0, 61)
    B = synthetic.paper_matrix(k, n, 1.0, 62)
    ref = _gpu.dgemm(oz, A, B, m, n, k, N)
    for variant in autotune.TILE_VARIANTS:
        for chunk in (960, 320):
            for group in (0, 1, 3):
                h = oz.Handle()
                h.set_option(oz.OPT_GEMM_VARIANT, variant)
                h.set_option(oz.OPT_CHUNK_K, chunk)
                h.set_option(oz.OPT_GROUP_M, group)
                assert _gpu.same_bits(_gpu.dgemm(oz, A, B, m, n, k, N, handle=h), ref)
    h = oz.Handle()
    assert autotune.apply_tiles(h, table, k)
    assert _gpu.same_bits(_gpu.dgemm(oz, A, B, m, n, k, N, handle=h), ref)
    assert _gpu.same_bits(ref, orc.dgemm(A, B, m, n, k, N))
    torch.cuda.synchronize()


def test_tune_grouped_chunk():
    import torch

    from paper_2606_29129_gb300 import autotune
    from paper_2606_29129_gb300 import ozaki2 as oz

    sizes = [(100, 300, 700), (257, 64, 1500), (64, 64, 64)]
    items = []
    for i, (m, n, k) in enumerate(sizes):
        A = torch.from_numpy(synthetic.paper_matrix(m, k, 1.0, 70 + 2 * i)).cuda()
        B = torch.from_numpy(synthetic.paper_matrix(k, n, 1.0, 71 + 2 * i)).cuda()
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        items.append(dict(m=m, n=n, k=k, A=A, lda=m, B=B, ldb=k, C=C, ldc=m, num_moduli=15))
    probs = oz.problems_array(items)
    h = oz.Handle()
    h.set_option(oz.OPT_GRAPH, 1)

    def call():
        _gpu.ok(oz.ozaki2_dgemm_grouped(len(items), probs, h), "grouped")

    call()
    torch.cuda.synchronize()
    first = [it["C"].cpu().numpy().copy() for it in items]
    ms, best = autotune.tune_grouped_chunk(call, h, chunks=(960, 448), reps=1)
    assert set(ms) == {960, 448} and best in ms
    call()
    torch.cuda.synchronize()
    for it, ref in zip(items, first):
        assert _gpu.same_bits(it["C"].cpu().numpy(), ref)
