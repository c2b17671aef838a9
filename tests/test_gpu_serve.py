"""The continuous-batching server on the GPU: every request's result is bit-identical to the
same request computed alone by ozaki2_dgemm with the same number of moduli, and to the CPU oracle
(Steps 1-4 of Section 2.2 with the scaling of Section 4)."""
import numpy as np
import pytest

import synthetic
import _gpu

pytestmark = pytest.mark.gpu

CAL = {c: {"k": 0, "cublas": 1e-13, "N": {12: 1e-9, 14: 1e-12, 16: 1e-14, 18: 1e-16}}
       for c in range(9)}


def test_served_results_equal_results_alone(orc):
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
        want = orc.dgemm(r.A, r.B, r.m, r.n, r.k, r.num_moduli)
        assert _gpu.same_bits(r.C, want), f"request {r.rid} differs from the oracle"
    assert {r.num_moduli for r in reqs} == {14, 16, 18}


def test_served_with_residue_cache_equal_oracle(orc):
    """With the residue cache: operands shared between requests (keys) are encoded once and
    reused, operands without keys are private; every result is bit-identical to the oracle, and
    the cache stays within its capacity while evicting."""
    from paper_2606_29129_gb300 import ozaki2 as oz
    from paper_2606_29129_gb300.serve import GpuExecutor, Request, Server

    rng = np.random.default_rng(19)
    pool = []
    for i in range(6):
        m, n, k = (int(v) for v in rng.integers(16, 300, size=3))
        pool.append((m, n, k, synthetic.paper_matrix(m, k, 1.0, 1200 + i),
                     synthetic.paper_matrix(k, n, 0.5, 1300 + i)))
    ex = GpuExecutor(slots=2, slot_workspace_bytes=128 << 20, cache_bytes=24 << 20)
    srv = Server(ex, io_budget_bytes=64 << 20, max_batch=5, calibration=CAL)
    reqs = []
    for i in range(36):
        m, n, k, A, B = pool[int(rng.integers(0, len(pool)))]
        keyed = i % 5 != 4
        r = Request(rid=i, m=m, n=n, k=k, target=[1e-10, 1e-13, 1e-15][i % 3], A=A, B=B,
                    a_key=(id(A) if keyed else None), b_key=(id(B) if keyed else None))
        reqs.append(r)
        srv.submit(r)
        if i % 6 == 5:
            srv.step()
    srv.run_until_idle()
    assert len(srv.finished) == 36 and all(r.error is None for r in srv.finished)
    assert ex.cache.peak <= ex.cache.capacity
    assert ex.cache.hits > 0
    for r in reqs:
        want = orc.dgemm(r.A, r.B, r.m, r.n, r.k, r.num_moduli)
        assert _gpu.same_bits(r.C, want), f"request {r.rid} differs from the oracle"
        alone = _gpu.dgemm(oz, r.A, r.B, r.m, r.n, r.k, r.num_moduli)
        assert _gpu.same_bits(r.C, alone), r.rid
    bd = ex.breakdown()
    # keyed misses plus private operands; the hits were not encoded again
    assert ex.cache.misses <= bd["encoded_operands"] < 2 * len(reqs)
