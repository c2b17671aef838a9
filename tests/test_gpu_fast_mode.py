"""GPU parity of the original fast mode (Section 2.3, Algorithm 1), selected per handle with
OZAKI2_OPT_SCALING: shifts and whole products bit-identical to the oracle's fast mode, the
failure region of the all-ones example of Section 3.1 reproduced, grouped calls identical to
separate ones."""
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
def fast(oz):
    h = oz.Handle()
    h.set_option(oz.OPT_SCALING, oz.SCALING_FAST)
    return h


def test_scaling_option_values(oz):
    h = oz.Handle()
    assert oz.lib().ozaki2_set_option(h.h, oz.OPT_SCALING, 3) == -3
    assert oz.lib().ozaki2_set_option(h.h, oz.OPT_SCALING, -1) == -3
    assert oz.lib().ozaki2_set_option(h.h, oz.OPT_SCALING, oz.SCALING_FAST) == 0
    assert oz.lib().ozaki2_set_option(h.h, oz.OPT_SCALING, oz.SCALING_PROPOSED) == 0


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("N", [8, 14, 20])
def test_fast_shifts_match_oracle(oz, orc, fast, trans, N):
    """Both memory orders of both sides (the adjacent-line and contiguous-line kernels), with
    scaled copies spanning the exponent range, zero lines, a single huge entry per line and
    non-finite lines."""
    m, k = 203, 301
    rng = np.random.default_rng(N)
    base = synthetic.paper_matrix(m, k, 1.0, 900 + N)            # storage (k, m)
    for s in (-1000, -300, -40, -3, 0, 2, 40, 300, 960):
        X = base * 2.0**s
        if trans == "T":
            X = np.ascontiguousarray(X.T)                           # storage (m, k): op = ^T
        Xv = X if trans == "N" else X.T                             # Xv[h, i] = op(A)[i, h]
        Xv[:, 5] = 0.0
        Xv[7, 9] = 1e300 if s > 0 else 1e-300
        if s == 0:
            Xv[3, 11] = np.inf
            Xv[4, 12] = np.nan
        ld = X.shape[-1]
        ref = orc.shifts_mode(X, m, k, N, orc.FAST_MODE, side=0, trans=trans, ld=ld)
        got = _gpu.shifts_a(oz, X, m, k, N, trans=trans, lda=ld, handle=fast)
        assert np.array_equal(got, ref), (s, np.nonzero(got != ref)[0][:5])
        # the same storage read as op(B) (k x m) with the other transpose
        tb = "T" if trans == "N" else "N"
        ref_b = orc.shifts_mode(X, m, k, N, orc.FAST_MODE, side=1, trans=tb, ld=ld)
        got_b = _gpu.shifts_b(oz, X, k, m, N, trans=tb, ldb=ld, handle=fast)
        assert np.array_equal(got_b, ref_b), s


def test_fast_shifts_differ_from_proposed(oz, orc, fast):
    """The option really switches the algorithm: for alpha = 1 inputs fast mode keeps about one
    bit less than the proposed scaling (P'_fast = P'_prop - 1)."""
    m, k, N = 64, 256, 16
    A = synthetic.paper_matrix(m, k, 0.5, 77)
    e_fast = _gpu.shifts_a(oz, A, m, k, N, handle=fast)
    e_prop = _gpu.shifts_a(oz, A, m, k, N)
    assert not np.array_equal(e_fast, e_prop)
    assert np.array_equal(e_prop, orc.shifts_mode(A, m, k, N, orc.PROPOSED_MODE))


@pytest.mark.parametrize("shape", [(96, 80, 200), (257, 130, 1000), (129, 300, 2000)])
@pytest.mark.parametrize("trans", [("N", "N"), ("T", "N"), ("N", "T")])
def test_fast_dgemm_bits_match_oracle(oz, orc, fast, shape, trans):
    m, n, k = shape
    tA, tB = trans
    N = 14 if k < 1500 else 18
    A = synthetic.paper_matrix(m, k, 1.0, 31) if tA == "N" else synthetic.paper_matrix(k, m, 1.0, 31)
    B = synthetic.paper_matrix(k, n, 1.0, 32) if tB == "N" else synthetic.paper_matrix(n, k, 1.0, 32)
    Cin = synthetic.paper_matrix(m, n, 1.0, 33)
    lda, ldb = A.shape[-1], B.shape[-1]
    got = _gpu.dgemm(oz, A, B, m, n, k, N, tA, tB, -1.25, 0.5, Cin, lda, ldb, handle=fast)
    ref = orc.dgemm_mode(A, B, m, n, k, N, orc.FAST_MODE, tA, tB, -1.25, 0.5, Cin, lda, ldb)
    assert _gpu.same_bits(got, ref)


@pytest.mark.parametrize("s", [-6, -2, 0, 3])
def test_all_ones_failure_region_on_gpu(oz, orc, fast, s):
    """Section 3.1 / Fig. 3: N = 20, A = B = 2^s 1 with k = 1024.  Fast mode breaks down for
    2^s <= 2^-2 (relative error ~1); the proposed scaling returns k 4^s exactly everywhere.  The
    GPU bits equal the oracle's in both modes."""
    m, n, k, N = 40, 24, 1024, 20
    alpha = 2.0**s
    A = synthetic.ones_matrix(m, k, alpha)
    B = synthetic.ones_matrix(k, n, alpha)
    exact = k * alpha * alpha
    Cf = _gpu.dgemm(oz, A, B, m, n, k, N, handle=fast)
    Cp = _gpu.dgemm(oz, A, B, m, n, k, N)
    assert _gpu.same_bits(Cf, orc.dgemm_mode(A, B, m, n, k, N, orc.FAST_MODE))
    assert np.all(Cp == exact)
    if s <= -2:
        assert np.all(np.abs(Cf - exact) / exact > 0.5)
    else:
        assert np.all(Cf == exact)


def test_fast_mode_grouped_equals_separate(oz, fast):
    import torch

    rng = np.random.default_rng(5)
    items = []
    for i in range(10):
        m, n, k = (int(v) for v in rng.integers(1, 400, size=3))
        N = int(rng.choice([8, 14, 20]))
        A = synthetic.paper_matrix(m, k, 1.0, 100 + i) * 2.0 ** int(rng.integers(-50, 50))
        B = synthetic.paper_matrix(k, n, 1.0, 200 + i)
        items.append(dict(m=m, n=n, k=k, num_moduli=N, A_np=A, B_np=B, lda=m, ldb=k, ldc=m,
                          A=_gpu.dev(A), B=_gpu.dev(B),
                          C=torch.zeros((n, m), dtype=torch.float64, device="cuda")))
    arr = oz.problems_array(items)
    _gpu.ok(oz.ozaki2_dgemm_grouped(len(items), arr, fast), "grouped fast")
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        ref = _gpu.dgemm(oz, it["A_np"], it["B_np"], it["m"], it["n"], it["k"], it["num_moduli"],
                         handle=fast)
        assert _gpu.same_bits(it["C"].cpu().numpy(), ref), i


@pytest.mark.parametrize("s", [-5, 0])
def test_fast_mode_breakdown_on_random_phi_half(oz, orc, fast, s):
    """Section 3.2 / Fig. 2: random inputs with phi = 0.5, m = n = k = 1024, N = 20, scaled by
    2^s.  Below alpha = 2^-3 the fast-mode scaling lets some |(A'B')_ij| pass P/2, so those
    entries come out with relative error ~1; the proposed scaling keeps every entry.  GPU and
    oracle agree bit for bit in both modes."""
    m = n = k = 1024
    N = 20
    A = synthetic.paper_matrix(m, k, 0.5, 11) * 2.0**s
    B = synthetic.paper_matrix(k, n, 0.5, 12) * 2.0**s
    Cf = _gpu.dgemm(oz, A, B, m, n, k, N, handle=fast)
    Cp = _gpu.dgemm(oz, A, B, m, n, k, N)
    assert _gpu.same_bits(Cf, orc.dgemm_mode(A, B, m, n, k, N, orc.FAST_MODE))
    # entries where the two modes differ most, checked against double-double
    d = np.abs(Cf - Cp).max(axis=1)                    # per column j of C (storage row)
    J = np.sort(np.argsort(d)[-4:]).astype(np.int32)
    dr = np.abs(Cf - Cp).max(axis=0)
    I = np.sort(np.argsort(dr)[-4:]).astype(np.int32)
    hi, lo = orc.dd_block(A, B, k, I, J)
    err_f, _ = orc.max_rel_error(Cf[np.ix_(J, I)], hi, lo)
    err_p, _ = orc.max_rel_error(Cp[np.ix_(J, I)], hi, lo)
    assert err_p < 1e-15
    if s <= -3:
        assert err_f > 0.5
    else:
        assert err_f < 1e-14
