"""GPU parity of each stage of the path against the oracle, through the C ABI, bit for bit.

Stages: scaling (Algorithm 2), conversion to residues (Step 2), residue GEMMs (eq. os2-C'),
CRT and rescaling (eqs. os2-C'', Step 4).  Each stage is fed the same inputs as the oracle; the
later stages are fed oracle-made or synthetic inputs so that each is checked on its own.
"""
import math

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


SHAPES = [(1, 1), (17, 7), (129, 1023), (300, 1025), (64, 2000), (257, 64)]


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("phi", [0.5, 4.0])
def test_scale_matches_oracle(oz, orc, trans, shape, phi):
    lines, k = shape
    N = 14
    seed = 31 * lines + k
    if trans == "N":
        A = synthetic.paper_matrix(lines, k, phi, seed)
    else:
        A = synthetic.paper_matrix(k, lines, phi, seed)
    e_ref, _ = orc.shifts_a(A, lines, k, N, trans=trans)
    assert np.array_equal(_gpu.shifts_a(oz, A, lines, k, N, trans), e_ref)
    # the same storage read as op(B) columns (transposed meaning of trans)
    tb = "T" if trans == "N" else "N"
    f_ref, _ = orc.shifts_b(A, k, lines, N, trans=tb)
    assert np.array_equal(_gpu.shifts_b(oz, A, k, lines, N, tb), f_ref)
    assert np.array_equal(f_ref, e_ref)


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("shape", [(40, 4097), (70, 6000), (33, 2304)])
@pytest.mark.parametrize("mode", ["proposed", "fast"])
def test_scale_long_lines_match_oracle(oz, orc, trans, shape, mode):
    """Lines of many norm blocks (k > 2048: more than one round of the warps that split a line's
    blocks), both memory layouts, both scalings that take the squared norm."""
    lines, k = shape
    N = 16
    A = synthetic.paper_matrix(lines, k, 2.0, 7 * k) if trans == "N" else \
        synthetic.paper_matrix(k, lines, 2.0, 7 * k)
    h = oz.Handle()
    omode = orc.PROPOSED_MODE
    if mode == "fast":
        h.set_option(oz.OPT_SCALING, oz.SCALING_FAST)
        omode = orc.FAST_MODE
    ld = A.shape[-1]
    e_ref = orc.shifts_mode(A, lines, k, N, omode, side=0, trans=trans, ld=ld)
    assert np.array_equal(_gpu.shifts_a(oz, A, lines, k, N, trans, ld, handle=h), e_ref)
    tb = "T" if trans == "N" else "N"
    f_ref = orc.shifts_mode(A, lines, k, N, omode, side=1, trans=tb, ld=ld)
    assert np.array_equal(_gpu.shifts_b(oz, A, k, lines, N, tb, ld, handle=h), f_ref)


@pytest.mark.parametrize("N", [2, 8, 20])
@pytest.mark.parametrize("alpha", [2.0**40, 2.0**-40, 3.7e20, 3.7e-20, 1e-160])
def test_scale_extreme_magnitudes(oz, orc, N, alpha):
    m, k = 96, 333
    A = synthetic.paper_matrix(m, k, 2.0, 5) * alpha
    A[:, 3] = 0.0
    e_ref, _ = orc.shifts_a(A, m, k, N)
    assert np.array_equal(_gpu.shifts_a(oz, A, m, k, N), e_ref)


def _log2_sweep_rows():
    """2^23 rows (1, v_j) whose squared norms are exactly 1 + j 2^-23, j = 0 .. 2^23 - 1, under
    the single-precision norm: v_j is the least single with v_j^2 > (j - 1) 2^-23, and
    single-up(1 + v_j^2) = 1 + j 2^-23 because the squares of neighbouring singles below 1 lie
    closer than 2^-23."""
    m = 1 << 23
    j = np.arange(m, dtype=np.float64)
    t = (j - 1) * 2.0**-23
    v = np.sqrt(np.maximum(t, 0)).astype(np.float32)
    for _ in range(4):
        up = (v.astype(np.float64) ** 2 <= t) & (j > 0)
        v = np.where(up, np.nextafter(v, np.float32(np.inf)), v)
        pv = np.nextafter(v, np.float32(0))
        v = np.where((pv.astype(np.float64) ** 2 > t) & (pv > 0), pv, v)
    v[0] = 0.0
    assert (v.astype(np.float64) ** 2 <= j * 2.0**-23).all()
    return np.ascontiguousarray(np.stack([np.ones(m), v.astype(np.float64)])), m


def test_scale_log2_argument_sweep(oz, orc):
    """Rows whose squared norms sweep every single-precision mantissa in [1, 2): the GPU's
    logarithm step and the oracle's agree on all of them."""
    A, m = _log2_sweep_rows()          # column-major m x 2, lda = m
    _, nr = orc.shifts_a(A, m, 2, 14)
    assert np.array_equal(np.asarray(nr), 1.0 + np.arange(m) * 2.0**-23)
    for N in (14, 20):
        e_ref, _ = orc.shifts_a(A, m, 2, N)
        assert np.array_equal(_gpu.shifts_a(oz, A, m, 2, N), e_ref)


def test_scale_nonfinite_flag(oz, orc):
    m, k = 40, 50
    A = synthetic.paper_matrix(m, k, 1.0, 8)
    A[3, 5] = np.nan     # row 5
    A[7, 9] = np.inf     # row 9
    A[:, 11] = 1e200     # row 11: squared norm overflows
    h = oz.Handle()
    import torch

    out = torch.zeros(m, dtype=torch.int32, device="cuda")
    _gpu.ok(oz.ozaki2_scale_a("N", m, k, _gpu.dev(A), m, 14, out, handle=h))
    e = out.cpu().numpy()
    e_ref, _ = orc.shifts_a(A, m, k, 14)
    assert np.array_equal(e, e_ref)
    assert set(np.nonzero(e == oz.SHIFT_NONFINITE)[0]) == {5, 9, 11}
    assert h.status() & oz.STATUS_NONFINITE
    assert h.status() == 0   # reading clears the flags


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("shape", [(1, 1), (31, 65), (129, 1023), (200, 77)])
@pytest.mark.parametrize("N", [2, 14, 17, 20])
def test_convert_a_matches_oracle(oz, orc, trans, shape, N):
    m, k = shape
    phi = 4.0
    A = synthetic.paper_matrix(m, k, phi, 3 * m + k) if trans == "N" else \
        synthetic.paper_matrix(k, m, phi, 3 * m + k)
    e, _ = orc.shifts_a(A, m, k, N, trans=trans)
    R_ref = orc.residues_a(A, m, k, e, N, trans=trans)
    P = _gpu.planes_a(oz, A, m, k, e, N, trans)
    assert np.array_equal(P[:, :m, :k], R_ref)
    assert not P[:, m:, :].any() and not P[:, :, k:].any()   # padding is zero


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("N", [8, 14, 20])
def test_convert_b_matches_oracle(oz, orc, trans, N):
    k, n = 300, 270
    B = synthetic.paper_matrix(k, n, 2.0, 77) if trans == "N" else \
        synthetic.paper_matrix(n, k, 2.0, 77)
    f, _ = orc.shifts_b(B, k, n, N, trans=trans)
    R_ref = orc.residues_b(B, k, n, f, N, trans=trans)
    P = _gpu.planes_b(oz, B, k, n, f, N, trans)
    assert np.array_equal(P[:, :n, :k], R_ref)
    assert not P[:, n:, :].any() and not P[:, :, k:].any()


def test_convert_special_values(oz, orc):
    """Subnormals, signed zeros, a zero row, a sentinel row and wide magnitudes."""
    m, k, N = 8, 64, 20
    A = synthetic.paper_matrix(m, k, 4.0, 9)
    A[:, 0] = 0.0
    A[0, 1] = 5e-324
    A[1, 1] = -0.0
    A[2, 1] = -2.5e-310
    A[:, 2] *= 1e-300
    e, _ = orc.shifts_a(A, m, k, N)
    e[3] = oz.SHIFT_NONFINITE
    R_ref = orc.residues_a(A, m, k, e, N)
    assert not R_ref[:, 3, :].any()
    P = _gpu.planes_a(oz, A, m, k, e, N)
    assert np.array_equal(P[:, :m, :k], R_ref)


def random_residues(rng, N, rows, kk, p, fill_k=None):
    R = np.zeros((N, rows, kk), np.int64)
    for l in range(N):
        lo, hi = (-128, 127) if p[l] == 256 else (-(p[l] - 1) // 2, (p[l] - 1) // 2)
        R[l] = rng.integers(lo, hi + 1, size=(rows, kk))
    if fill_k is not None:
        R[:, :, fill_k:] = 0
    return R


VARIANTS = ["single", "pair"]


def variant_code(oz, name):
    return {"single": oz.GEMM_SINGLE, "pair": oz.GEMM_PAIR}[name]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dims", [(128, 256, 64), (256, 512, 1024), (384, 256, 3008),
                                  (128, 256, 16384), (640, 768, 320)])
@pytest.mark.parametrize("N", [2, 14, 20])
def test_residue_gemm_matches_oracle(oz, orc, dims, N, variant):
    mp, npad, kp = dims
    rng = np.random.default_rng(mp + npad + kp + N)
    p = orc.constants(N)["p"]
    RA = random_residues(rng, N, mp, kp, p)
    RB = random_residues(rng, N, npad, kp, p)
    c = _gpu.residue_gemm(oz, RA, RB, variant_code(oz, variant))
    rows = np.arange(0, mp, 7 if kp > 4096 else 1)
    c_ref = orc.residue_products(RA[:, rows].astype(np.int8), RB.astype(np.int8))
    assert np.array_equal(c[:, rows], c_ref)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("kp", [960, 1024, 1088, 2048, 65536])
def test_residue_gemm_accumulation_extremes(oz, orc, kp, variant):
    """Worst-case magnitudes for the FP32 accumulator: every product (-128)^2 = 2^14 on the
    modulus 256, and +-127 patterns on the others, across reduction-chunk boundaries."""
    N, mp, npad = 3, 128, 256
    RA = np.zeros((N, mp, kp), np.int64)
    RB = np.zeros((N, npad, kp), np.int64)
    RA[0] = -128
    RB[0] = -128
    RB[0, 1::2] = 127            # odd columns: -128 * 127 products
    RA[1] = 127
    RB[1] = 127
    RB[1, ::3] = -127
    sgn = np.where(np.arange(kp) % 2 == 0, 1, -1)
    RA[2] = 126 * sgn
    RB[2] = 126
    c = _gpu.residue_gemm(oz, RA, RB, variant_code(oz, variant))
    c_ref = orc.residue_products(RA[:, :16].astype(np.int8), RB.astype(np.int8))
    assert np.array_equal(c[:, :16], c_ref)
    assert np.array_equal(c[:, 16:], np.broadcast_to(c[:, :1], c[:, 16:].shape))


@pytest.mark.parametrize("variant", VARIANTS)
def test_residue_gemm_many_tiles(oz, orc, variant):
    """More tiles than SMs: the persistent loop, tile pairs and the tile order."""
    N, mp, npad, kp = 14, 2048, 2048, 192
    rng = np.random.default_rng(4)
    p = orc.constants(N)["p"]
    RA = random_residues(rng, N, mp, kp, p)
    RB = random_residues(rng, N, npad, kp, p)
    c = _gpu.residue_gemm(oz, RA, RB, variant_code(oz, variant))
    rows = np.arange(3, mp, 61)
    c_ref = orc.residue_products(RA[:, rows].astype(np.int8), RB.astype(np.int8))
    assert np.array_equal(c[:, rows], c_ref)


@pytest.mark.parametrize("N", [2, 8, 14, 16, 17, 20])
def test_crt_matches_oracle(oz, orc, N):
    m, n = 100, 70
    rng = np.random.default_rng(N)
    mp, npad = 128, 256
    c = rng.integers(-128, 128, size=(N, mp, npad)).astype(np.int8)
    e = rng.integers(-60, 60, size=m).astype(np.int32)
    f = rng.integers(-60, 60, size=n).astype(np.int32)
    C_ref = orc.crt(np.ascontiguousarray(c[:, :m, :n]), e, f)
    assert _gpu.same_bits(_gpu.crt(oz, c, e, f, m, n), C_ref)
    Cin = synthetic.paper_matrix(m, n, 1.0, 5)
    C_ref = orc.crt(np.ascontiguousarray(c[:, :m, :n]), e, f, alpha=-1.5, beta=0.25, Cin=Cin)
    assert _gpu.same_bits(_gpu.crt(oz, c, e, f, m, n, -1.5, 0.25, Cin), C_ref)


@pytest.mark.parametrize("N", [2, 14, 20])
def test_crt_extreme_integers_and_exponents(oz, orc, N):
    """Residues of chosen integers at the ends of the symmetric range (where the quotient
    estimate sits next to a half-integer), ties of the final rounding, and shifts that push
    results into the subnormal range or past overflow; sentinel shifts give NaN."""
    P = orc.constants(N)["P"]
    half = (P - 1) // 2
    xs = [0, 1, -1, half, -half, half - 1, -(half - 1), half // 3, -(half // 7),
          2**53 + 1, (2**53 + 1) * 2**20 + 2**19, -(2**60 + 2**7 + 1)]
    rng = np.random.default_rng(N)
    xs += [int(v) for v in rng.integers(-2**62, 2**62, size=20)]
    xs = [x for x in xs if abs(x) <= half]
    m, n = len(xs), 6
    res = orc.int_residues(xs, N)                          # (m, N)
    c = np.zeros((N, 128, 256), np.int8)
    for j in range(n):
        c[:, :m, j] = res.T
    e = np.zeros(m, np.int32)
    f = np.array([0, 1100, -900, 1074, -1023, 0], np.int32)
    e[-1] = oz.SHIFT_NONFINITE
    C_ref = orc.crt(np.ascontiguousarray(c[:, :m, :n]), e, f)
    C = _gpu.crt(oz, c, e, f, m, n)
    assert _gpu.same_bits(C, C_ref)
    for i, x in enumerate(xs[:-1]):
        assert C[0, i] == float(x)
    assert np.isnan(C[:, m - 1]).all()


def _norm_lines(k):
    """Rows whose squared norms reach every branch of the single-precision reading: the block
    maximum rising late, terms far below it (subnormal singles), subnormal doubles, zeros,
    overflow to +Inf, Inf and NaN entries, and wide random magnitudes; zero-padded to k."""
    g = np.random.Generator(np.random.PCG64(91))
    rows = [
        np.sort(np.abs(g.standard_normal(300))) * 2.0 ** g.integers(-60, 60, 300),
        g.standard_normal(600) * np.exp(16.0 * g.standard_normal(600)),
        np.concatenate([g.random(100) * 2.0**-140, [1.5], g.random(100) * 2.0**-75]),
        g.random(300) * 5e-310,
        np.concatenate([g.random(50) * 5e-310, g.random(50) * 1e-300, [0.0] * 20]),
        np.concatenate([g.random(10), [1e200], g.random(10)]),
        np.concatenate([g.random(10), [np.inf], g.random(10)]),
        np.concatenate([g.random(300), [np.nan], g.random(10)]),
        np.concatenate([[2.0**-1000], g.random(5) * 2.0**1000]),
        g.random(400) * 2.0**-1060,
        np.zeros(5),
    ]
    rows += list(g.standard_normal((40, k)) * np.exp(8.0 * g.standard_normal((40, k))))
    M = np.zeros((len(rows), k))
    for i, r in enumerate(rows):
        M[i, :min(len(r), k)] = r[:k]
    return M


@pytest.mark.parametrize("k", [200, 700, 2048])
@pytest.mark.parametrize("side", ["A", "B"])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_scale_norms_match_oracle(oz, orc, k, side, trans):
    """The squared norms the product's scaling kernels compute (one thread per line for lines of
    one block, the split kernels for longer ones, both memory layouts) equal the oracle's bit
    for bit on lines that reach every branch of the single-precision reading, and so do the
    shifts."""
    import torch

    M = _norm_lines(k)                       # lines x k: the mathematical rows of op(A)
    lines = M.shape[0]
    if side == "A":
        # op(A) = M: A is M (trans N) or M^T (trans T), stored column-major
        store = np.ascontiguousarray(M.T if trans == "N" else M)
        ld = lines if trans == "N" else k
        e_ref, nr_ref = orc.shifts_a(store, lines, k, 16, trans=trans, lda=ld)
    else:
        # op(B) = M^T (k x lines): B is M^T (trans N) or M (trans T)
        store = np.ascontiguousarray(M if trans == "N" else M.T)
        ld = k if trans == "N" else lines
        e_ref, nr_ref = orc.shifts_b(store, k, lines, 16, trans=trans, ldb=ld)
    shifts = torch.zeros(lines, dtype=torch.int32, device="cuda")
    norms = torch.zeros(lines, dtype=torch.float64, device="cuda")
    _gpu.ok(oz.ozaki2_scale_norms(side, trans, lines, k, _gpu.dev(store), ld, 16, shifts, norms),
            "scale_norms")
    torch.cuda.synchronize()
    got = norms.cpu().numpy()
    nr_ref = np.asarray(nr_ref)
    assert np.array_equal(got.view(np.int64)[~np.isnan(got)],
                          nr_ref.view(np.int64)[~np.isnan(got)])
    assert np.array_equal(np.isnan(got), np.isnan(nr_ref))
    assert np.array_equal(shifts.cpu().numpy(), e_ref)
