"""ozaki2_dgemm_noalloc: the emulated DGEMM for callers that may not allocate device memory when
they call it (their device memory is budgeted up front, or they run inside a host framework's
callback that forbids allocation).  It keeps its intermediates in a static device array of the
library instead of a workspace.

Called through the C ABI and compared with ozaki2_dgemm, bit for bit (the tolerance of the other
parity tests), on two calls in a row with different inputs, since the array keeps the previous
call's contents.  The file is named to be collected last."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def _inputs(m, n, k, seed, device):
    A = synthetic.paper_matrix_torch(m, k, 1.0, seed, device=device)      # column-major m x k
    B = synthetic.paper_matrix_torch(k, n, 2.0, seed + 1, device=device)  # column-major k x n
    return A, B


def test_noalloc_matches_dgemm_on_two_calls():
    import torch

    from paper_2606_29129_gb300 import ozaki2

    L = ozaki2.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    m, n, k, N = 250, 190, 256, 20
    assert ozaki2.ozaki2_workspace_size(m, n, k, N) + 256 <= ozaki2.NOALLOC_SCRATCH_BYTES
    for call, seed in enumerate((41, 77)):
        A, B = _inputs(m, n, k, seed, dev)
        ref = torch.zeros((n, m), dtype=torch.float64, device=dev)
        assert ozaki2.ozaki2_dgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, ref, m, N) == 0
        C = torch.full((n, m), float("nan"), dtype=torch.float64, device=dev)
        rc = L.ozaki2_dgemm_noalloc(b"N", b"N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k,
                                    0.0, C.data_ptr(), m, N, stream)
        assert rc == 0, f"call {call}: {rc}"
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        want = ref.cpu().numpy()
        assert np.array_equal(got.view(np.int64), want.view(np.int64)), f"call {call} differs"


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch

    from paper_2606_29129_gb300 import ozaki2

    L = ozaki2.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    m = n = k = 1024
    A, B = _inputs(m, n, k, 5, dev)
    C = torch.full((n, m), 3.0, dtype=torch.float64, device=dev)
    rc = L.ozaki2_dgemm_noalloc(b"N", b"N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0,
                                C.data_ptr(), m, 14, stream)
    assert rc == ozaki2.ERROR_TOO_LARGE
    torch.cuda.synchronize()
    assert bool((C == 3.0).all())
