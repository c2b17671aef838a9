"""GPU parity of the emulated SGEMM (ozaki2_sgemm through the C ABI) against the oracle: every
shape, transpose, moduli count (the paper's range 3..12 and beyond), alpha/beta, scaling mode,
subnormal and overflowing outputs bit for bit; at the full size, a sampled block covering every
output tile."""
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


def f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def gpu_sgemm(oz, A, B, m, n, k, N, tA="N", tB="N", alpha=1.0, beta=0.0, Cin=None, lda=None,
              ldb=None, handle=None):
    import torch

    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    C = torch.zeros((max(n, 1), max(m, 1)), dtype=torch.float32, device="cuda") if Cin is None \
        else _gpu.dev(f32(Cin))
    dA = _gpu.dev(A) if A.size else torch.zeros(1, dtype=torch.float32, device="cuda")
    dB = _gpu.dev(B) if B.size else torch.zeros(1, dtype=torch.float32, device="cuda")
    _gpu.ok(oz.ozaki2_sgemm(tA, tB, m, n, k, alpha, dA, lda, dB, ldb, beta, C, max(m, 1), N,
                            handle), "sgemm")
    torch.cuda.synchronize()
    return C.cpu().numpy()


def make(m, n, k, phi, seed, tA="N", tB="N"):
    A = synthetic.paper_matrix(m, k, phi, seed) if tA == "N" else synthetic.paper_matrix(k, m, phi, seed)
    B = synthetic.paper_matrix(k, n, phi, seed + 1) if tB == "N" else \
        synthetic.paper_matrix(n, k, phi, seed + 1)
    return f32(A), f32(B)


SHAPES = [(1, 1, 1), (3, 5, 7), (129, 257, 1025), (300, 200, 64), (127, 255, 961), (40, 600, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("trans", ["NN", "TN", "NT", "TT"])
def test_shapes_and_transposes(oz, orc, shape, trans):
    m, n, k = shape
    A, B = make(m, n, k, 1.0, 11, trans[0], trans[1])
    got = gpu_sgemm(oz, A, B, m, n, k, 7, trans[0], trans[1])
    ref = orc.sgemm(A, B, m, n, k, 7, trans[0], trans[1])
    assert _gpu.same_bits(got, ref)


@pytest.mark.parametrize("N", [2, 3, 5, 8, 10, 12, 15, 20])
@pytest.mark.parametrize("phi", [0.0, 1.5])
def test_moduli_counts(oz, orc, N, phi):
    m, n, k = 70, 90, 500
    A, B = make(m, n, k, phi, 20 + N)
    assert _gpu.same_bits(gpu_sgemm(oz, A, B, m, n, k, N), orc.sgemm(A, B, m, n, k, N))


def test_alpha_beta_and_quick_returns(oz, orc):
    m, n, k, N = 65, 33, 129, 8
    A, B = make(m, n, k, 1.0, 5)
    Cin = f32(np.random.default_rng(1).standard_normal((n, m)))
    for alpha, beta in ((1.0, 0.0), (-0.75, 0.5), (2.0, 1.0), (0.0, 3.0)):
        got = gpu_sgemm(oz, A, B, m, n, k, N, alpha=alpha, beta=beta, Cin=Cin)
        ref = orc.sgemm(A, B, m, n, k, N, alpha=alpha, beta=beta, Cin=Cin)
        assert _gpu.same_bits(got, ref), (alpha, beta)
    got = gpu_sgemm(oz, A[:0], B[:, :0], m, n, 0, N, beta=0.5, Cin=Cin, lda=m, ldb=1)
    assert np.array_equal(got, np.float32(0.5) * Cin)


@pytest.mark.parametrize("scale", [2.0**-70, 2.0**-64, 2.0**62, 2.0**66])
def test_subnormal_and_overflow_outputs(oz, orc, scale):
    m, n, k, N = 40, 30, 64, 10
    A, B = make(m, n, k, 0.5, 7)
    A, B = f32(A * scale), f32(B * scale)
    assert _gpu.same_bits(gpu_sgemm(oz, A, B, m, n, k, N), orc.sgemm(A, B, m, n, k, N))


@pytest.mark.parametrize("mode", ["fast", "accurate"])
def test_scaling_modes(oz, orc, mode):
    h = oz.Handle()
    code = oz.SCALING_FAST if mode == "fast" else oz.SCALING_ACCURATE
    h.set_option(oz.OPT_SCALING, code)
    for (m, n, k), phi in (((129, 70, 700), 1.0), ((64, 200, 5000), 0.5)):
        A, B = make(m, n, k, phi, 40)
        got = gpu_sgemm(oz, A, B, m, n, k, 9, handle=h)
        ref = orc.sgemm(A, B, m, n, k, 9, mode=code)
        assert _gpu.same_bits(got, ref), (m, n, k)


def test_nonfinite_inputs(oz, orc):
    m, n, k, N = 20, 12, 40, 6
    A, B = make(m, n, k, 1.0, 3)
    synthetic.colmajor_view(A)[2, 5] = np.inf
    synthetic.colmajor_view(B)[7, 3] = np.nan
    assert _gpu.same_bits(gpu_sgemm(oz, A, B, m, n, k, N), orc.sgemm(A, B, m, n, k, N))


@pytest.mark.parametrize("size,N", [(8192, 8), (16384, 7)])
def test_full_size_sampled(oz, orc, size, N):
    """One ozaki2_sgemm call at full size: a block with one row in every 128-row tile and one
    column in every 256-column tile, bit-identical to the oracle's (whose shifts for those lines
    come from the same widened lines)."""
    import torch

    m = n = k = size
    A = synthetic.paper_matrix_torch(m, k, 1.0, synthetic.seed_for(2, 1, 1)).float()
    B = synthetic.paper_matrix_torch(k, n, 1.0, synthetic.seed_for(2, 1, 2)).float()
    C = torch.empty((n, m), dtype=torch.float32, device="cuda")
    _gpu.ok(oz.ozaki2_sgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, N))
    torch.cuda.synchronize()
    rng = np.random.default_rng(size)
    I = np.arange(0, m, 128) + rng.integers(0, 128, size=m // 128)
    J = np.arange(0, n, 256) + rng.integers(0, 256, size=n // 256)
    blk = orc.sgemm_block(A.cpu().numpy(), B.cpu().numpy(), k, N, I, J)
    got = C[torch.from_numpy(J).cuda()][:, torch.from_numpy(I).cuda()].cpu().numpy()
    assert _gpu.same_bits(got, blk)


def test_torch_convenience(oz, orc):
    import torch

    from paper_2606_29129_gb300 import sgemm

    m, n, k = 33, 44, 55
    A = torch.randn(m, k, dtype=torch.float32, device="cuda")
    B = torch.randn(k, n, dtype=torch.float32, device="cuda")
    C = sgemm(A, B)
    ref = orc.sgemm(A.cpu().numpy(), B.cpu().numpy(), m, n, k, 8, "T", "T", lda=k, ldb=n)
    assert _gpu.same_bits(C.cpu().numpy().T, ref)


@pytest.mark.parametrize("offset", [1, 2, 4])
def test_host_operands_unaligned(oz, orc, offset):
    """Host-resident float A, B and C (A and B `offset` floats past a 16-byte boundary: 4- and
    8-byte staging copies): bit-identical to the device-memory call and to the oracle."""
    import torch

    m, n, k, N = 200, 130, 517, 8
    A, B = make(m, n, k, 1.0, 93)
    ref = gpu_sgemm(oz, A, B, m, n, k, N)
    bufs = []
    views = []
    for X in (A, B):
        flat = X.reshape(-1)
        buf = torch.empty(flat.size + offset, dtype=torch.float32).pin_memory()
        buf[offset:].copy_(torch.from_numpy(flat))
        bufs.append(buf)
        views.append(buf[offset:])
    Ch = torch.zeros((n, m), dtype=torch.float32).pin_memory()
    _gpu.ok(oz.ozaki2_sgemm("N", "N", m, n, k, 1.0, views[0], m, views[1], k, 0.0, Ch, m, N),
            "host sgemm")
    torch.cuda.synchronize()
    assert _gpu.same_bits(Ch.numpy(), ref)
    assert _gpu.same_bits(ref, orc.sgemm(A, B, m, n, k, N))
