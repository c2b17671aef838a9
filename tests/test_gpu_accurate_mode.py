"""GPU parity of accurate mode (Section 2.3), selected with OZAKI2_OPT_SCALING =
OZAKI2_SCALING_ACCURATE: the exponents, A-bar/B-bar, the auxiliary product C-bar = A-bar B-bar on
the tensor cores (its row and column maxima), the shifts, and whole products, all bit-identical to
the oracle's accurate mode; grouped calls identical to separate ones."""
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


@pytest.fixture(scope="module")
def accu(oz):
    h = oz.Handle()
    h.set_option(oz.OPT_SCALING, oz.SCALING_ACCURATE)
    return h


def gpu_accurate_shifts(oz, A, B, m, n, k, N, tA="N", tB="N", lda=None, ldb=None, handle=None):
    import torch

    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    e = torch.zeros(max(m, 1), dtype=torch.int32, device="cuda")
    f = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    cm = torch.zeros(max(m + n, 1), dtype=torch.int32, device="cuda")
    dA = _gpu.dev(A) if A.size else torch.zeros(1, dtype=torch.float64, device="cuda")
    dB = _gpu.dev(B) if B.size else torch.zeros(1, dtype=torch.float64, device="cuda")
    _gpu.ok(oz.ozaki2_scale_accurate(tA, tB, m, n, k, dA, lda, dB, ldb, N, e, f, cm, handle),
            "scale_accurate")
    torch.cuda.synchronize()
    cmax = cm.cpu().numpy().view(np.uint32).astype(np.int64)
    return e.cpu().numpy()[:m], f.cpu().numpy()[:n], cmax[:m], cmax[m:m + n]


def test_stage_entries_and_errors(oz, accu):
    import torch

    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    sh = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert oz.ozaki2_scale_a("N", 4, 4, buf, 4, 14, sh, accu) == oz.ERROR_MODE
    assert oz.ozaki2_scale_b("N", 4, 4, buf, 4, 14, sh, accu) == oz.ERROR_MODE
    assert oz.ozaki2_scale_accurate("N", "N", 4, 4, oz.ACCURATE_MAX_K + 1, buf, 4, buf,
                                    oz.ACCURATE_MAX_K + 1, 14, sh, sh) == oz.ERROR_TOO_LARGE
    assert oz.ozaki2_scale_accurate("X", "N", 4, 4, 4, buf, 4, buf, 4, 14, sh, sh) == -2
    assert oz.ozaki2_scale_accurate("N", "N", 4, 4, 4, buf, 3, buf, 4, 14, sh, sh) == -8
    assert oz.ozaki2_scale_accurate("N", "N", 4, 4, 4, buf, 4, buf, 4, 1, sh, sh) == -11
    C = torch.zeros(16, dtype=torch.float64, device="cuda")
    big = oz.ACCURATE_MAX_K + 1
    assert oz.ozaki2_dgemm("N", "N", 1, 1, big, 1.0, buf, 1, buf, big, 0.0, C, 1, 14,
                           accu) == oz.ERROR_TOO_LARGE


@pytest.mark.parametrize("shape", [(5, 4, 7), (203, 301, 150), (130, 257, 4100), (64, 48, 9000)])
@pytest.mark.parametrize("trans", [("N", "N"), ("T", "T"), ("T", "N")])
def test_shifts_and_cbar_maxima_match_oracle(oz, orc, shape, trans):
    """Shapes cover ragged tiles, one and several carry chunks of C-bar (k > 4032), both memory
    orders of each operand; the inputs include zero lines, a non-finite line, a line whose
    products all vanish, and a subnormal-heavy line."""
    m, n, k = shape
    tA, tB = trans
    N = 16
    A = synthetic.paper_matrix(m, k, 1.0, 41) if tA == "N" else synthetic.paper_matrix(k, m, 1.0, 41)
    B = synthetic.paper_matrix(k, n, 2.0, 42) if tB == "N" else synthetic.paper_matrix(n, k, 2.0, 42)
    Av = A if tA == "T" else synthetic.colmajor_view(A)      # Av[i, h] = op(A)[i, h]
    Bv = synthetic.colmajor_view(B) if tB == "N" else B      # Bv[h, j] = op(B)[h, j]
    if m > 4 and n > 3:
        Av[0, :] = 0.0
        Av[1, min(3, k - 1)] = np.inf
        Av[2, :] = 0.0
        Av[2, 0] = 3.0
        Bv[0, :] = 0.0                                       # row 2 of C-bar vanishes
        Av[3, :] *= 1e-310
        Bv[:, 1] = 0.0                                       # a zero column of op(B)
    ref = orc.accurate_shifts(A, B, m, n, k, N, tA, tB)
    got = gpu_accurate_shifts(oz, A, B, m, n, k, N, tA, tB)
    for name, r, g in zip(("e", "f", "rowmax", "colmax"), ref, got):
        assert np.array_equal(r, g), (name, np.nonzero(r != g)[0][:5])


def test_cbar_at_the_largest_k(oz, orc):
    """k = 2^20 - 1 with every a-bar = b-bar = 64: C-bar = 4096 k = 2^32 - 4096, the largest
    value the uint32 maxima hold; many carry chunks."""
    m, n, k, N = 2, 3, 1048575, 20
    A = np.full((k, m), 1.99)
    B = np.full((n, k), -1.99)
    e, f, rm, cm = gpu_accurate_shifts(oz, A, B, m, n, k, N)
    re, rf, rrm, rcm = orc.accurate_shifts(A, B, m, n, k, N)
    assert np.all(rm == 4096 * k) and np.all(cm == 4096 * k)
    assert np.array_equal(rm, rrm) and np.array_equal(cm, rcm)
    assert np.array_equal(e, re) and np.array_equal(f, rf)


@pytest.mark.parametrize("shape", [(96, 80, 200), (257, 130, 1000), (129, 300, 5000)])
@pytest.mark.parametrize("trans", [("N", "N"), ("T", "N"), ("N", "T")])
def test_accurate_dgemm_bits_match_oracle(oz, orc, accu, shape, trans):
    m, n, k = shape
    tA, tB = trans
    N = 14 if k < 1500 else 18
    A = synthetic.paper_matrix(m, k, 1.0, 51) if tA == "N" else synthetic.paper_matrix(k, m, 1.0, 51)
    B = synthetic.paper_matrix(k, n, 1.0, 52) if tB == "N" else synthetic.paper_matrix(n, k, 1.0, 52)
    Cin = synthetic.paper_matrix(m, n, 1.0, 53)
    lda, ldb = A.shape[-1], B.shape[-1]
    got = _gpu.dgemm(oz, A, B, m, n, k, N, tA, tB, 0.75, -2.0, Cin, lda, ldb, handle=accu)
    ref = orc.dgemm_mode(A, B, m, n, k, N, orc.ACCURATE_MODE, tA, tB, 0.75, -2.0, Cin, lda, ldb)
    assert _gpu.same_bits(got, ref)


@pytest.mark.parametrize("N", [4, 10, 15, 20])
def test_accurate_dgemm_edge_moduli_and_extremes(oz, orc, accu, N):
    """Moduli counts whose limb count grew for accurate mode's wider a', with rows of wildly
    different magnitude (the largest a' of accurate mode) and a vanishing row."""
    m, n, k = 70, 33, 300
    A = synthetic.paper_matrix(m, k, 2.0, 60 + N)
    B = synthetic.paper_matrix(k, n, 2.0, 70 + N)
    Av, Bv = synthetic.colmajor_view(A), synthetic.colmajor_view(B)
    Av[5, :] = 0.0
    Av[5, 7] = 1e200
    Av[5, 8] = 1e-200
    Bv[7, :] = 1e-250                                        # tiny b-bar = 1 against a-bar = 64
    Av[6, :] = 0.0
    Av[6, 9] = 2.0
    Bv[9, :] = 0.0                                           # row 6 vanishes
    got = _gpu.dgemm(oz, A, B, m, n, k, N, handle=accu)
    ref = orc.dgemm_mode(A, B, m, n, k, N, orc.ACCURATE_MODE)
    assert _gpu.same_bits(got, ref)


def test_accurate_mode_scale_invariance_on_gpu(oz, orc, accu):
    """Fig. 2: accurate mode keeps its accuracy for every alpha = 2^s; the GPU result scales
    exactly by alpha^2 and equals the oracle."""
    m, n, k, N = 300, 200, 1024, 20
    A0 = synthetic.paper_matrix(m, k, 0.5, 11)
    B0 = synthetic.paper_matrix(k, n, 0.5, 12)
    C0 = _gpu.dgemm(oz, A0, B0, m, n, k, N, handle=accu)
    assert _gpu.same_bits(C0, orc.dgemm_mode(A0, B0, m, n, k, N, orc.ACCURATE_MODE))
    for s in (-5, -3, 4, 10):
        C = _gpu.dgemm(oz, A0 * 2.0**s, B0 * 2.0**s, m, n, k, N, handle=accu)
        assert np.array_equal(C, C0 * 4.0**s), s


def test_accurate_all_ones(oz, accu):
    for s in (-6, -2, 0, 5):
        m, n, k, N = 40, 24, 1024, 20
        A = synthetic.ones_matrix(m, k, 2.0**s)
        B = synthetic.ones_matrix(k, n, 2.0**s)
        C = _gpu.dgemm(oz, A, B, m, n, k, N, handle=accu)
        assert np.all(C == k * 4.0**s)


def test_accurate_grouped_equals_separate(oz, accu):
    import torch

    rng = np.random.default_rng(9)
    items = []
    for i in range(12):
        m, n, k = (int(v) for v in rng.integers(1, 500, size=3))
        if i == 3:
            k = 5000
        N = int(rng.choice([8, 14, 20]))
        A = synthetic.paper_matrix(m, k, 1.0, 300 + i) * 2.0 ** int(rng.integers(-50, 50))
        B = synthetic.paper_matrix(k, n, 2.0, 400 + i)
        items.append(dict(m=m, n=n, k=k, num_moduli=N, A_np=A, B_np=B, lda=m, ldb=k, ldc=m,
                          A=_gpu.dev(A), B=_gpu.dev(B),
                          C=torch.zeros((n, m), dtype=torch.float64, device="cuda")))
    arr = oz.problems_array(items)
    for rep in range(2):   # the second call reuses the handle's workspace and staging
        _gpu.ok(oz.ozaki2_dgemm_grouped(len(items), arr, accu), "grouped accurate")
        torch.cuda.synchronize()
        for i, it in enumerate(items):
            ref = _gpu.dgemm(oz, it["A_np"], it["B_np"], it["m"], it["n"], it["k"],
                             it["num_moduli"], handle=accu)
            assert _gpu.same_bits(it["C"].cpu().numpy(), ref), (rep, i)
