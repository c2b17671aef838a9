"""GPU parity of ozaki2_dgemm_grouped: every problem of a grouped call is bit-identical to a
separate ozaki2_dgemm on the same inputs, and to the oracle on a sample."""
import numpy as np
import pytest

import synthetic
import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oz():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu-marked tests")
    from paper_2606_29129_gb300 import ozaki2

    return ozaki2


def make_batch(rng, count, lo, hi, moduli, quick=False):
    """Problems with log-uniform sizes in [lo, hi]; device inputs and outputs per problem."""
    import torch

    items = []
    for i in range(count):
        m, n, k = (int(np.exp(rng.uniform(np.log(lo), np.log(hi + 1)))) for _ in range(3))
        tA, tB = rng.choice(["N", "T"]), rng.choice(["N", "T"])
        phi = (0.5, 1.0)[i % 2]
        N = int(rng.choice(moduli))
        alpha, beta = 1.0, 0.0
        if i % 7 == 3:
            alpha, beta = -1.5, 0.5
        if quick and i % 11 == 5:
            k = 0
        if quick and i % 13 == 6:
            alpha = 0.0
        A = synthetic.paper_matrix(m, k, phi, 5000 + i) if tA == "N" else \
            synthetic.paper_matrix(k, m, phi, 5000 + i)
        B = synthetic.paper_matrix(k, n, phi, 6000 + i) if tB == "N" else \
            synthetic.paper_matrix(n, k, phi, 6000 + i)
        Cin = synthetic.paper_matrix(m, n, 1.0, 7000 + i)
        lda = max(1, m if tA == "N" else k)
        ldb = max(1, k if tB == "N" else n)
        items.append(dict(transA=tA, transB=tB, m=m, n=n, k=k, alpha=alpha, beta=beta,
                          num_moduli=N, A_np=A, B_np=B, Cin=Cin, lda=lda, ldb=ldb, ldc=max(1, m),
                          A=_gpu.dev(A) if A.size else torch.zeros(1, dtype=torch.float64,
                                                                 device="cuda"),
                          B=_gpu.dev(B) if B.size else torch.zeros(1, dtype=torch.float64,
                                                                 device="cuda"),
                          C=_gpu.dev(Cin)))
    return items


def run_grouped(oz, items, handle=None):
    import torch

    arr = oz.problems_array(items)
    _gpu.ok(oz.ozaki2_dgemm_grouped(len(items), arr, handle), "dgemm_grouped")
    torch.cuda.synchronize()
    return [it["C"].cpu().numpy() for it in items]


def run_separately(oz, it):
    return _gpu.dgemm(oz, it["A_np"], it["B_np"], it["m"], it["n"], it["k"], it["num_moduli"],
                      it["transA"], it["transB"], it["alpha"], it["beta"], it["Cin"],
                      it["lda"], it["ldb"])


def test_grouped_mixed_batch(oz, orc):
    rng = np.random.default_rng(11)
    items = make_batch(rng, 40, 1, 300, [8, 14, 16, 20], quick=True)
    got = run_grouped(oz, items)
    for i, it in enumerate(items):
        ref = run_separately(oz, it)
        assert _gpu.same_bits(got[i], ref), i
    for i in (0, 1, 2, 9):
        it = items[i]
        ref = orc.dgemm(it["A_np"], it["B_np"], it["m"], it["n"], it["k"], it["num_moduli"],
                        it["transA"], it["transB"], it["alpha"], it["beta"], it["Cin"],
                        lda=it["lda"], ldb=it["ldb"])
        assert _gpu.same_bits(got[i], ref), i


def test_grouped_twice_with_different_batches(oz):
    h = oz.Handle()
    for seed in (3, 4):
        rng = np.random.default_rng(seed)
        items = make_batch(rng, 12, 16, 400, [14, 16])
        got = run_grouped(oz, items, h)
        for i, it in enumerate(items):
            assert _gpu.same_bits(got[i], run_separately(oz, it)), (seed, i)


def test_grouped_batch_of_512(oz, orc):
    """The batched workload: 512 problems, m, n, k log-uniform in [64, 2048], phi alternating."""
    rng = np.random.default_rng(512)
    items = make_batch(rng, 512, 64, 2048, [14, 16])
    got = run_grouped(oz, items)
    for i, it in enumerate(items):
        assert _gpu.same_bits(got[i], run_separately(oz, it)), i
    small = sorted(range(len(items)), key=lambda i: items[i]["m"] * items[i]["n"] * items[i]["k"])
    for i in small[:6]:
        it = items[i]
        ref = orc.dgemm(it["A_np"], it["B_np"], it["m"], it["n"], it["k"], it["num_moduli"],
                        it["transA"], it["transB"], it["alpha"], it["beta"], it["Cin"],
                        lda=it["lda"], ldb=it["ldb"])
        assert _gpu.same_bits(got[i], ref), i


def test_grouped_argument_errors(oz):
    import torch

    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    good = dict(m=4, n=4, k=4, A=buf, lda=4, B=buf, ldb=4, C=buf, ldc=4, num_moduli=14)
    bad_ld = dict(good, lda=2)
    bad_n = dict(good, num_moduli=1)
    arr = oz.problems_array([good, bad_ld])
    assert oz.ozaki2_dgemm_grouped(2, arr) == -(100 * 2 + 8)
    arr = oz.problems_array([bad_n, good])
    assert oz.ozaki2_dgemm_grouped(2, arr) == -(100 * 1 + 14)
    assert oz.ozaki2_dgemm_grouped(-1, arr) == -2
    assert oz.ozaki2_dgemm_grouped(0, arr) == 0


def test_grouped_cuda_graph_replay(oz):
    """With OZAKI2_OPT_GRAPH the first call captures the launches into a CUDA graph; later calls
    with the same problem list replay it, reading the current contents of A, B and C."""
    import torch

    rng = np.random.default_rng(21)
    items = make_batch(rng, 24, 32, 700, [14, 16, 20])
    h = oz.Handle()
    h.set_option(oz.OPT_GRAPH, 1)
    arr = oz.problems_array(items)
    for rep in range(3):
        if rep == 2:  # new data in the same buffers
            for i, it in enumerate(items):
                it["A_np"] = it["A_np"] * 3.0 + 1.0
                it["A"].copy_(torch.from_numpy(it["A_np"]))
        for it in items:
            it["C"].copy_(torch.from_numpy(np.ascontiguousarray(it["Cin"])))
        _gpu.ok(oz.ozaki2_dgemm_grouped(len(items), arr, h), "grouped graph call")
        torch.cuda.synchronize()
        for i, it in enumerate(items):
            assert _gpu.same_bits(it["C"].cpu().numpy(), run_separately(oz, it)), (rep, i)


@pytest.mark.parametrize("rules", [
    [(1 << 30, 1 << 30, 64, 64)],                       # every problem on 64-wide tiles
    [(1 << 30, 1 << 30, 128, 320)],                     # 128-wide tiles, K chunk 320
    [(1 << 30, 1 << 30, 256, 960)],                     # 256-wide tiles
    [(64, 1 << 30, 64, 128), (128, 200, 128, 0), (1 << 30, 1 << 30, 256, 192)],  # by class
    [],                                                 # automatic width per problem
])
def test_grouped_tile_widths_match_oracle(oz, orc, rules):
    """Each tile width of the grouped residue GEMM (256, 128 and 64 columns) and several K chunks,
    chosen per size class: every problem bit-identical to the oracle."""
    rng = np.random.default_rng(77)
    items = make_batch(rng, 14, 1, 420, [8, 14, 20])
    h = oz.Handle()
    h.set_grouped_tiles(rules)
    got = run_grouped(oz, items, h)
    for i, it in enumerate(items):
        ref = orc.dgemm(it["A_np"], it["B_np"], it["m"], it["n"], it["k"], it["num_moduli"],
                        it["transA"], it["transB"], it["alpha"], it["beta"], it["Cin"],
                        lda=it["lda"], ldb=it["ldb"])
        assert _gpu.same_bits(got[i], ref), (rules, i, it["m"], it["n"], it["k"])


def test_grouped_tile_rules_errors(oz):
    h = oz.Handle()
    with pytest.raises(oz.Ozaki2Error):
        h.set_grouped_tiles([(64, 64, 96, 0)])          # not a supported width
    with pytest.raises(oz.Ozaki2Error):
        h.set_grouped_tiles([(64, 64, 64, 1000)])       # chunk above 960
    with pytest.raises(oz.Ozaki2Error):
        h.set_grouped_tiles([(1, 1, 64, 0)] * (oz.MAX_TILE_RULES + 1))
    h.set_grouped_tiles([])
