"""The continuous-batching server on the GPU: every request's result is bit-identical to the
same request computed alone by ozaki2_dgemm with the same number of moduli."""
import numpy as np
import pytest

import synthetic
import _gpu

pytestmark = pytest.mark.gpu

CAL = {c: {"k": 0, "cublas": 1e-13, "N": {12: 1e-9, 14: 1e-12, 16: 1e-14, 18: 1e-16}}
       for c in range(9)}


def test_served_results_equal_results_alone():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu-marked tests")
    from paper_2606_29129_gb300 import ozaki2 as oz
    from paper_2606_29129_gb300.serve import GpuExecutor, Request, Server

    rng = np.random.default_rng(9)
    reqs = []
    for i in range(30):
        m, n, k = (int(v) for v in rng.integers(8, 400, size=3))
        target = [1e-10, 1e-13, 1e-15][i % 3]
        A = synthetic.paper_matrix(m, k, 1.0, 900 + i)
        B = synthetic.paper_matrix(k, n, 1.0, 950 + i)
        reqs.append(Request(rid=i, m=m, n=n, k=k, target=target, A=A, B=B))
    ex = GpuExecutor(slots=2, slot_workspace_bytes=256 << 20)
    srv = Server(ex, io_budget_bytes=24 << 20, max_batch=8, calibration=CAL)
    for r in reqs[:10]:
        srv.submit(r)
    srv.step()
    for r in reqs[10:]:        # the rest arrive while the first batches run
        srv.submit(r)
    srv.run_until_idle()
    assert len(srv.finished) == 30 and all(r.error is None for r in srv.finished)
    assert srv.peak_io <= srv.io_budget
    for r in reqs:
        alone = _gpu.dgemm(oz, r.A, r.B, r.m, r.n, r.k, r.num_moduli)
        assert _gpu.same_bits(r.C, alone), r.rid
    assert {r.num_moduli for r in reqs} == {14, 16, 18}
