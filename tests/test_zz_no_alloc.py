"""ozaki2_dgemm_noalloc: the emulated DGEMM for callers that may not allocate device memory when
they call it (their device memory is budgeted up front, or they run inside a host framework's
callback that forbids allocation).  It keeps its intermediates in a static device array of the
library instead of a workspace.

Called through the C ABI and compared with ozaki2_dgemm and with the CPU oracle, bit for bit (the
tolerance of the other parity tests), on two calls in a row with different inputs, since the
array keeps the previous call's contents.  The file is named to be collected last."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def _op_storage(rows, cols, trans, ld, phi, seed):
    """Column-major storage of a matrix X with op(X) rows x cols, leading dimension ld."""
    r, c = (rows, cols) if trans == "N" else (cols, rows)
    X = synthetic.paper_matrix(r, c, phi, seed)           # storage (c, r), ld = r
    S = np.zeros((c, ld), np.float64)
    S[:, :r] = X
    return S


@pytest.mark.parametrize("transA,transB", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_noalloc_matches_dgemm_and_oracle_on_two_calls(orc, transA, transB):
    import torch

    from paper_2606_29129_gb300 import ozaki2

    L = ozaki2.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    m, n, k, N = 250, 190, 237, 20
    assert ozaki2.ozaki2_workspace_size(m, n, k, N) + 256 <= ozaki2.NOALLOC_SCRATCH_BYTES
    for call, seed in enumerate((41, 77)):
        lda = (m if transA == "N" else k) + 5
        ldb = (k if transB == "N" else n) + 3
        A_np = _op_storage(m, k, transA, lda, 1.0, seed)
        B_np = _op_storage(k, n, transB, ldb, 2.0, seed + 1)
        A = torch.from_numpy(A_np).to(dev)
        B = torch.from_numpy(B_np).to(dev)
        ref = torch.zeros((n, m), dtype=torch.float64, device=dev)
        assert ozaki2.ozaki2_dgemm(transA, transB, m, n, k, 1.0, A, lda, B, ldb, 0.0, ref, m,
                                   N) == 0
        C = torch.full((n, m), float("nan"), dtype=torch.float64, device=dev)
        rc = L.ozaki2_dgemm_noalloc(transA.encode(), transB.encode(), m, n, k, 1.0,
                                    A.data_ptr(), lda, B.data_ptr(), ldb, 0.0, C.data_ptr(), m,
                                    N, stream)
        assert rc == 0, f"call {call}: {rc}"
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        assert np.array_equal(got.view(np.int64), ref.cpu().numpy().view(np.int64)), \
            f"call {call} differs from ozaki2_dgemm"
        want = orc.dgemm(A_np, B_np, m, n, k, N, transA=transA, transB=transB, lda=lda, ldb=ldb)
        assert np.array_equal(got.view(np.int64), want.view(np.int64)), \
            f"call {call} differs from the oracle"


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch

    from paper_2606_29129_gb300 import ozaki2

    L = ozaki2.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    m = n = k = 1024
    A = synthetic.paper_matrix_torch(m, k, 1.0, 5, device=dev)
    B = synthetic.paper_matrix_torch(k, n, 1.0, 6, device=dev)
    C = torch.full((n, m), 3.0, dtype=torch.float64, device=dev)
    rc = L.ozaki2_dgemm_noalloc(b"N", b"N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0,
                                C.data_ptr(), m, 14, stream)
    assert rc == ozaki2.ERROR_TOO_LARGE
    torch.cuda.synchronize()
    assert bool((C == 3.0).all())
    # C = beta C needs no scratch: accepted at any size
    rc = L.ozaki2_dgemm_noalloc(b"N", b"N", m, n, k, 0.0, A.data_ptr(), m, B.data_ptr(), k, 0.5,
                                C.data_ptr(), m, 14, stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert bool((C == 1.5).all())
