"""GPU parity of the whole emulated DGEMM (ozaki2_dgemm through the C ABI) against the oracle.

Bit-exact comparison of C for every shape, transpose, moduli count and alpha/beta case; the
all-ones worked example of Section 3.1 (exact result); scale invariance (Section 4); quick
returns and argument errors; and, at the full benchmark size, every shift plus a sampled block
of C covering every output tile.
"""
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


def make(m, n, k, phi, seed, transA="N", transB="N"):
    A = synthetic.paper_matrix(m, k, phi, seed) if transA == "N" else \
        synthetic.paper_matrix(k, m, phi, seed)
    B = synthetic.paper_matrix(k, n, phi, seed + 1) if transB == "N" else \
        synthetic.paper_matrix(n, k, phi, seed + 1)
    return A, B


def test_config1_256_cubed(oz, orc):
    """m = n = k = 256, phi = 1, N = 14 (the small configuration), against the oracle."""
    m = n = k = 256
    A, B = make(m, n, k, 1.0, synthetic.seed_for(1, 0, 1))
    C = _gpu.dgemm(oz, A, B, m, n, k, 14)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 14))
    # rigorous truncation bound per entry (a' = mu a - d, |d| < 1; one rounding of C''):
    # |C - AB| <= 2^-f_j sum|a_i.| + 2^-e_i sum|b_.j| + k 2^-(e_i+f_j) + 2^-53 |C|
    hi, lo = orc.dd_block(A, B, k, list(range(m)), list(range(n)))
    e, _ = orc.shifts_a(A, m, k, 14)
    f, _ = orc.shifts_b(B, k, n, 14)
    ra = np.abs(synthetic.colmajor_view(A)).sum(axis=1)          # (m,)
    cb = np.abs(synthetic.colmajor_view(B)).sum(axis=0)          # (n,)
    ei, fj = 2.0 ** -e.astype(np.float64), 2.0 ** -f.astype(np.float64)
    bound = (ra[None, :] * fj[:, None] + cb[:, None] * ei[None, :] + k * fj[:, None] * ei[None, :]
             + np.abs(C) * 2.0**-53) * 1.001                      # storage (n, m)
    assert np.all(np.abs((C - hi) - lo) <= bound)
    err, _ = orc.max_rel_error(C, hi, lo)
    assert err < 1e-9


SHAPES = [(1, 1, 1), (3, 5, 7), (129, 257, 1025), (300, 200, 64), (128, 256, 960),
          (127, 255, 961), (40, 600, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("trans", ["NN", "TN", "NT", "TT"])
def test_shapes_and_transposes(oz, orc, shape, trans):
    m, n, k = shape
    tA, tB = trans
    A, B = make(m, n, k, 2.0, sum(shape), tA, tB)
    C = _gpu.dgemm(oz, A, B, m, n, k, 14, tA, tB)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 14, tA, tB))


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("chunk", [64, 512, 960])
def test_gemm_variants_and_chunks(oz, orc, variant, chunk):
    """Both residue-GEMM kernels and several reduction chunk lengths give the same bits."""
    m, n, k = 300, 520, 1500
    A, B = make(m, n, k, 1.0, 61)
    h = oz.Handle()
    h.set_option(oz.OPT_CHUNK_K, chunk)
    C = _gpu.dgemm(oz, A, B, m, n, k, 16, handle=h, variant=variant)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 16))


@pytest.mark.parametrize("hints", [0, 1, 2, 4, 8, 1 | (2 << 2)])
def test_l2_hints_change_nothing(oz, orc, hints):
    """The L2 eviction policies of the residue GEMM's tile loads change the timing only."""
    m, n, k = 260, 530, 1100
    A, B = make(m, n, k, 1.0, 67)
    h = oz.Handle()
    h.set_option(oz.OPT_L2_HINTS, hints)
    C = _gpu.dgemm(oz, A, B, m, n, k, 15, handle=h, variant=1)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 15))


def test_l2_hints_option_checks(oz):
    h = oz.Handle()
    for bad in (-1, 3, 12, 16):
        assert oz.lib().ozaki2_set_option(h.h, oz.OPT_L2_HINTS, bad) == -3
    for bad in (-1, 2):
        assert oz.lib().ozaki2_set_option(h.h, oz.OPT_HOST_COPIES, bad) == -3


@pytest.mark.parametrize("N", list(range(2, 21)))
@pytest.mark.parametrize("phi", [0.5, 4.0])
def test_moduli_counts(oz, orc, N, phi):
    """Every moduli count: the reconstruction's word count, the word its rounding window starts
    in (one lower for N = 4, 8, 12, whose top word is always zero, and a second choice for
    N = 5, 9, 13, 17) and its pair grouping (odd N ends on a single modulus) all change with N."""
    m, n, k = 150, 130, 700
    A, B = make(m, n, k, phi, N)
    C = _gpu.dgemm(oz, A, B, m, n, k, N)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, N))


def test_alpha_beta(oz, orc):
    m, n, k = 70, 90, 110
    A, B = make(m, n, k, 1.0, 3)
    Cin = synthetic.paper_matrix(m, n, 1.0, 9)
    for alpha, beta in [(1.0, 0.0), (-2.5, 0.0), (1.0, 1.0), (0.3, -0.7)]:
        C = _gpu.dgemm(oz, A, B, m, n, k, 14, alpha=alpha, beta=beta, Cin=Cin)
        ref = orc.dgemm(A, B, m, n, k, 14, alpha=alpha, beta=beta, Cin=Cin)
        assert _gpu.same_bits(C, ref), (alpha, beta)
    nan_in = np.full_like(Cin, np.nan)    # beta = 0 never reads C
    C = _gpu.dgemm(oz, A, B, m, n, k, 14, beta=0.0, Cin=nan_in)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 14))


def test_quick_returns(oz):
    import torch

    m, n = 5, 4
    Cin = synthetic.paper_matrix(m, n, 1.0, 1)
    C = _gpu.dgemm(oz, np.zeros((0, m)), np.zeros((n, 0)), m, n, 0, 14, alpha=2.0, beta=0.5,
                   Cin=Cin, lda=m, ldb=1)
    assert np.array_equal(C, 0.5 * Cin)
    A, B = make(m, n, 3, 1.0, 2)
    C = _gpu.dgemm(oz, A, B, m, n, 3, 14, alpha=0.0, beta=0.0, Cin=Cin)
    assert np.all(C == 0.0)
    # m = 0: nothing happens, nothing is read
    _gpu.ok(oz.ozaki2_dgemm("N", "N", 0, n, 3, 1.0, None, 1, _gpu.dev(B), 3, 0.0, None, 1, 14))
    torch.cuda.synchronize()


def test_argument_errors(oz):
    import torch

    A = torch.zeros(64, dtype=torch.float64, device="cuda")
    call = lambda *a: oz.ozaki2_dgemm(*a)  # noqa: E731
    assert call("X", "N", 4, 4, 4, 1.0, A, 4, A, 4, 0.0, A, 4, 14) == -2
    assert call("N", "Q", 4, 4, 4, 1.0, A, 4, A, 4, 0.0, A, 4, 14) == -3
    assert call("N", "N", -1, 4, 4, 1.0, A, 4, A, 4, 0.0, A, 4, 14) == -4
    assert call("N", "N", 4, 4, 4, 1.0, A, 3, A, 4, 0.0, A, 4, 14) == -9
    assert call("N", "N", 4, 4, 4, 1.0, A, 4, A, 3, 0.0, A, 4, 14) == -11
    assert call("N", "N", 4, 4, 4, 1.0, A, 4, A, 4, 0.0, A, 3, 14) == -14
    assert call("N", "N", 4, 4, 4, 1.0, A, 4, A, 4, 0.0, A, 4, 1) == -15
    assert call("N", "N", 4, 4, 4, 1.0, A, 4, A, 4, 0.0, A, 4, 21) == -15
    assert call("N", "N", 4, 4, 4, 1.0, None, 4, A, 4, 0.0, A, 4, 14) == -8


def test_user_workspace(oz, orc):
    import torch

    m, n, k = 64, 80, 96
    A, B = make(m, n, k, 1.0, 5)
    h = oz.Handle()
    need = oz.ozaki2_workspace_size(m, n, k, 14)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h.set_workspace(ws, need)
    C = _gpu.dgemm(oz, A, B, m, n, k, 14, handle=h)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 14))
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    h.set_workspace(small, need // 2)
    Cd = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    rc = oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, _gpu.dev(A), m, _gpu.dev(B), k, 0.0, Cd, m, 14,
                         h)
    assert rc == 3   # OZAKI2_ERROR_WORKSPACE


@pytest.mark.parametrize("k", [1024, 16384])
@pytest.mark.parametrize("s", [-10, -2, 0, 10])
def test_all_ones_exact(oz, k, s):
    """All-ones example (Section 3.1), N = 20: the proposed scaling never breaks the CRT and the
    product is exactly k alpha^2, like cuBLAS (Fig. 3 caption)."""
    m, n = 64, 48
    alpha = 2.0**s
    A = synthetic.ones_matrix(m, k, alpha)
    B = synthetic.ones_matrix(k, n, alpha)
    C = _gpu.dgemm(oz, A, B, m, n, k, 20)
    assert np.all(C == k * alpha * alpha)


@pytest.mark.parametrize("s", [40, -40])
def test_scale_invariance(oz, orc, s):
    m, n, k = 100, 90, 500
    A, B = make(m, n, k, 2.0, 17)
    C0 = _gpu.dgemm(oz, A, B, m, n, k, 14)
    C1 = _gpu.dgemm(oz, A * 2.0**s, B * 2.0**s, m, n, k, 14)
    assert np.array_equal(C1, C0 * 2.0 ** (2 * s))


def test_nonfinite_inputs(oz, orc):
    m, n, k = 30, 20, 40
    A, B = make(m, n, k, 1.0, 23)
    A[4, 7] = np.nan      # row 7 of A
    B[2, 3] = np.inf      # column 2 of B
    h = oz.Handle()
    C = _gpu.dgemm(oz, A, B, m, n, k, 14, handle=h)
    assert _gpu.same_bits(C, orc.dgemm(A, B, m, n, k, 14))
    assert np.isnan(C[:, 7]).all() and np.isnan(C[2, :]).all()
    assert h.status() & oz.STATUS_NONFINITE


def test_torch_convenience(oz, orc):
    import torch

    from paper_2606_29129_gb300 import dgemm

    m, n, k = 33, 44, 55
    A = torch.randn(m, k, dtype=torch.float64, device="cuda")
    B = torch.randn(k, n, dtype=torch.float64, device="cuda")
    C = dgemm(A, B, num_moduli=16)
    # row-major (m, k) storage is the column-major k x m matrix A^T, so op = 'T' recovers A
    ref = orc.dgemm(A.cpu().numpy(), B.cpu().numpy(), m, n, k, 16, "T", "T", lda=k, ldb=n)
    assert _gpu.same_bits(C.cpu().numpy().T, ref)


FULL_CASES = [
    # square (the benchmark's problem and the accuracy sweep's sizes, phi, scaled copies)
    (8192, 8192, 8192, 14, 1.0, 1.0),
    (16384, 16384, 16384, 16, 1.0, 1.0),
    (16384, 16384, 16384, 16, 0.5, 2.0**40),
    (8192, 8192, 8192, 20, 2.0, 3.7e-20),
    # rectangular
    (16384, 16384, 1024, 14, 1.0, 1.0),
    (1024, 1024, 65536, 18, 1.0, 1.0),
    (65536, 256, 4096, 14, 1.0, 1.0),
    (65536, 256, 4096, 18, 1.0, 3.7e20),
]


@pytest.mark.parametrize("m,n,k,N,phi,alpha", FULL_CASES)
def test_full_size_sampled(oz, orc, m, n, k, N, phi, alpha):
    """Full sizes in the benchmark's launch configuration (one ozaki2_dgemm call): every row and
    column shift equals the oracle's, and a block of C with one row in every 128-row tile and
    one column in every 256-column tile is bit-identical to the oracle's."""
    import torch

    A = synthetic.paper_matrix_torch(m, k, phi, synthetic.seed_for(2, 1, 1)) * alpha
    B = synthetic.paper_matrix_torch(k, n, phi, synthetic.seed_for(2, 1, 2)) * alpha
    C = torch.empty((n, m), dtype=torch.float64, device="cuda")
    _gpu.ok(oz.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, N))
    e = torch.empty(m, dtype=torch.int32, device="cuda")
    f = torch.empty(n, dtype=torch.int32, device="cuda")
    _gpu.ok(oz.ozaki2_scale_a("N", m, k, A, m, N, e))
    _gpu.ok(oz.ozaki2_scale_b("N", k, n, B, k, N, f))
    torch.cuda.synchronize()
    A_h, B_h = A.cpu().numpy(), B.cpu().numpy()
    e_ref, _ = orc.shifts_a(A_h, m, k, N)
    f_ref, _ = orc.shifts_b(B_h, k, n, N)
    assert np.array_equal(e.cpu().numpy(), e_ref)
    assert np.array_equal(f.cpu().numpy(), f_ref)
    rng = np.random.default_rng(m + n + k)
    I = np.minimum(np.arange(0, m, 128) + rng.integers(0, 128, size=(m + 127) // 128), m - 1)
    J = np.minimum(np.arange(0, n, 256) + rng.integers(0, 256, size=(n + 255) // 256), n - 1)
    if len(I) > 256:
        I = np.sort(rng.choice(I, 256, replace=False))
    blk = orc.dgemm_block(A_h, B_h, m, n, k, N, I, J, e=e_ref, f=f_ref)
    Jd = torch.from_numpy(J.astype(np.int64)).cuda()
    Id = torch.from_numpy(I.astype(np.int64)).cuda()
    got = C[Jd][:, Id].cpu().numpy()
    assert _gpu.same_bits(got, blk)


def test_host_resident_operands(oz, orc):
    """A, B and C in page-locked host memory: the kernels read and write it over the CPU-GPU
    link and the result is bit-identical to the device-memory call."""
    import torch

    m, n, k, N = 300, 200, 500, 14
    A, B = make(m, n, k, 1.0, 77)
    Cin = synthetic.paper_matrix(m, n, 1.0, 78)
    ref = _gpu.dgemm(oz, A, B, m, n, k, N, alpha=0.5, beta=-1.0, Cin=Cin)
    Ah = torch.from_numpy(np.ascontiguousarray(A)).pin_memory()
    Bh = torch.from_numpy(np.ascontiguousarray(B)).pin_memory()
    Ch = torch.from_numpy(np.ascontiguousarray(Cin)).pin_memory()
    _gpu.ok(oz.ozaki2_dgemm("N", "N", m, n, k, 0.5, Ah, m, Bh, k, -1.0, Ch, m, N), "host dgemm")
    torch.cuda.synchronize()
    assert _gpu.same_bits(Ch.numpy(), ref)
    assert _gpu.same_bits(ref, orc.dgemm(A, B, m, n, k, N, alpha=0.5, beta=-1.0, Cin=Cin))


def _pinned_view(a, offset_elems):
    """Page-locked host copy of `a` (flattened) starting `offset_elems` elements into its buffer,
    so that the view is not 16-byte aligned when the offset is odd."""
    import torch

    flat = np.ascontiguousarray(a).reshape(-1)
    buf = torch.empty(flat.size + offset_elems, dtype=torch.from_numpy(flat[:1]).dtype).pin_memory()
    view = buf[offset_elems:]
    view.copy_(torch.from_numpy(flat))
    return buf, view


@pytest.mark.parametrize("trans", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("own_workspace", [False, True])
def test_host_operands_unaligned_transposed(oz, orc, trans, own_workspace):
    """Host-resident A and B one element past a 16-byte boundary, any transpose: the handle stages
    them into device memory (8-byte copies), or with a caller-provided workspace reads them in
    place; either way C is bit-identical to the device-memory call and to the oracle."""
    import torch

    tA, tB = trans
    m, n, k, N = 130, 257, 333, 15
    A, B = make(m, n, k, 1.0, 91, tA, tB)
    lda, ldb = A.shape[-1], B.shape[-1]
    ref = _gpu.dgemm(oz, A, B, m, n, k, N, tA, tB, lda=lda, ldb=ldb)
    keep_a, Ah = _pinned_view(A, 1)
    keep_b, Bh = _pinned_view(B, 1)
    h = oz.Handle()
    if own_workspace:
        ws = torch.empty(oz.ozaki2_workspace_size(m, n, k, N), dtype=torch.uint8, device="cuda")
        h.set_workspace(ws, ws.numel())
    C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    _gpu.ok(oz.ozaki2_dgemm(tA, tB, m, n, k, 1.0, Ah, lda, Bh, ldb, 0.0, C, m, N, h),
            "host dgemm")
    torch.cuda.synchronize()
    assert _gpu.same_bits(C.cpu().numpy(), ref)
    assert _gpu.same_bits(ref, orc.dgemm(A, B, m, n, k, N, tA, tB))
    del keep_a, keep_b


@pytest.mark.parametrize("case", [
    # (m, n, k, transA, host A, host B, host C, scaling, dtype, beta[, lda and ldb padding])
    (200, 4700, 600, "N", True, True, True, "proposed", "f64", -0.5),
    (200, 4700, 600, "N", True, True, True, "proposed", "f64", 0.0),
    (150, 9000, 300, "T", True, True, True, "proposed", "f64", 0.0),
    (96, 8300, 257, "N", False, True, False, "proposed", "f64", -0.5),
    (128, 4100, 1000, "N", False, False, True, "fast", "f64", 0.0),
    (160, 5000, 400, "T", True, True, True, "proposed", "f32", 0.0),
    (160, 5000, 400, "N", True, False, True, "proposed", "f32", 2.0),
    # m >= 4096 with host A: A's row blocks within the first column block (ragged last blocks)
    (4500, 4300, 300, "N", True, True, True, "proposed", "f64", 0.0),
    (8300, 4200, 200, "T", True, True, True, "proposed", "f64", 0.0, 3),
    (4200, 8500, 190, "N", True, True, True, "proposed", "f64", 0.0, 5),
    (4200, 4500, 200, "N", True, False, True, "proposed", "f32", 0.0),
    (4200, 4500, 200, "T", True, True, False, "proposed", "f64", -0.5),
    (4200, 4500, 130, "N", True, True, True, "proposed", "f64", 1.5),
    # row blocks growing from 1024 (1024, 2048, then near-equal quarters, the last ragged)
    (12345, 4500, 190, "N", True, True, True, "proposed", "f64", 0.0),
])
@pytest.mark.parametrize("copies", [0, 1])
def test_host_operands_pipelined_over_column_blocks(oz, orc, case, copies):
    """n >= 4096 with host-resident operands: the call pipelines the column blocks of op(B) and,
    within the first, the row blocks of a host-resident op(A) with m >= 4096 (each later operand
    block uploaded by a copy that overlaps the previous block's residue GEMMs; a host-resident C
    written block by block by the reconstruction), or with copy engines (copies = 1: uploads
    queued on a copy stream, C's blocks reconstructed in device memory and downloaded on
    another).  C is bit-identical to the call on device memory, and to the oracle on a sample
    that takes rows and columns from every block."""
    import torch

    m, n, k, tA, ha, hb, hc, scaling, dtype, beta = case[:10]
    pad = case[10] if len(case) > 10 else 0
    N = 14
    A, B = make(m, n, k, 1.0, 4 * n + m, tA, "N")
    if pad:  # leading dimensions beyond the rows of the stored matrices
        A = np.pad(A, ((0, 0), (0, pad)))
        B = np.pad(B, ((0, 0), (0, pad)))
    Cin = synthetic.paper_matrix(m, n, 1.0, 5)
    f32 = dtype == "f32"
    if f32:
        A, B, Cin = A.astype(np.float32), B.astype(np.float32), Cin.astype(np.float32)
    lda, ldb = A.shape[-1], B.shape[-1]
    gemm = oz.ozaki2_sgemm if f32 else oz.ozaki2_dgemm
    h = oz.Handle()
    h.set_option(oz.OPT_SCALING, oz.SCALING_FAST if scaling == "fast" else oz.SCALING_PROPOSED)
    h.set_option(oz.OPT_HOST_COPIES, copies)

    def dev_or_host(x, host):
        t = torch.from_numpy(np.ascontiguousarray(x))
        return t.pin_memory() if host else t.cuda()

    Cd = _gpu.dev(Cin)
    _gpu.ok(gemm(tA, "N", m, n, k, 0.75, _gpu.dev(A), lda, _gpu.dev(B), ldb, beta, Cd, m, N, h),
            "device call")
    Ah, Bh, Ch = dev_or_host(A, ha), dev_or_host(B, hb), dev_or_host(Cin, hc)
    _gpu.ok(gemm(tA, "N", m, n, k, 0.75, Ah, lda, Bh, ldb, beta, Ch, m, N, h), "pipelined call")
    torch.cuda.synchronize()
    assert h.status() == 0
    got = Ch.cpu().numpy()
    assert _gpu.same_bits(got, Cd.cpu().numpy())
    rng = np.random.default_rng(n)
    I = np.sort(np.concatenate([rng.choice(m, size=24, replace=False), [0, m - 1]]))
    I = np.unique(I).astype(np.int32)
    J = np.sort(np.concatenate([rng.choice(n, size=40, replace=False), [0, n - 1]]))
    J = np.unique(J).astype(np.int32)
    mode = orc.FAST_MODE if scaling == "fast" else orc.PROPOSED_MODE
    if f32:
        want = orc.sgemm_block(A, B, k, N, I, J, tA, "N", 0.75, beta,
                               np.ascontiguousarray(Cin[np.ix_(J, I)]), lda=lda, ldb=ldb)
    elif mode == orc.PROPOSED_MODE:
        want = orc.dgemm_block(A, B, m, n, k, N, I, J, tA, "N", 0.75, beta,
                               np.ascontiguousarray(Cin[np.ix_(J, I)]), lda=lda, ldb=ldb)
    else:
        full = orc.dgemm_mode(A, B, m, n, k, N, mode, tA, "N", 0.75, beta, Cin, lda, ldb)
        want = full[np.ix_(J, I)]
    assert _gpu.same_bits(got[np.ix_(J, I)], want)
