"""Failure handling of the residue-GEMM kernels: every wait inside them is bounded.  A test-only
bound of 0 ns (OZAKI2_OPT_WAIT_LIMIT_NS) makes the first wait that does not succeed at once run
out, with nothing else wrong: the kernel must raise OZAKI2_STATUS_TIMEOUT, stop its roles, let
its copies and tensor-core work finish, free its tensor memory and return, so that the context
stays usable.  The same handle's next call, with the default bound, must then be bit-identical to
the CPU oracle.  Covered: the one-SM kernel, the SM-pair kernel, the grouped kernel and the
auxiliary product of accurate mode."""
import numpy as np
import pytest

import synthetic
import _gpu

pytestmark = pytest.mark.gpu

DEFAULT_LIMIT_NS = 2_000_000_000


def _inputs(m, n, k, seed):
    return synthetic.paper_matrix(m, k, 1.0, seed), synthetic.paper_matrix(k, n, 1.0, seed + 1)


@pytest.mark.parametrize("variant,scaling", [("single", "proposed"), ("pair", "proposed"),
                                             ("single", "accurate")])
def test_expired_wait_raises_timeout_then_next_call_is_exact(orc, variant, scaling):
    from paper_2606_29129_gb300 import ozaki2 as oz

    m, n, k, N = 512, 512, 700, 14
    A, B = _inputs(m, n, k, 300)
    h = oz.Handle()
    h.set_option(oz.OPT_GEMM_VARIANT, oz.GEMM_SINGLE if variant == "single" else oz.GEMM_PAIR)
    mode = oz.SCALING_PROPOSED if scaling == "proposed" else oz.SCALING_ACCURATE
    h.set_option(oz.OPT_SCALING, mode)
    h.set_option(oz.OPT_WAIT_LIMIT_NS, 0)
    _gpu.dgemm(oz, A, B, m, n, k, N, handle=h)
    assert h.status() & oz.STATUS_TIMEOUT, "a 0 ns bound must make a wait run out"
    h.set_option(oz.OPT_WAIT_LIMIT_NS, DEFAULT_LIMIT_NS)
    got = _gpu.dgemm(oz, A, B, m, n, k, N, handle=h)
    assert h.status() == 0
    if scaling == "proposed":
        want = orc.dgemm(A, B, m, n, k, N)
    else:
        want = orc.dgemm_mode(A, B, m, n, k, N, orc.ACCURATE_MODE)
    assert _gpu.same_bits(got, want)


def test_expired_wait_in_grouped_call(orc):
    import torch

    from paper_2606_29129_gb300 import ozaki2 as oz

    sizes = [(300, 200, 500), (128, 700, 64), (900, 100, 1000)]
    N = 16
    data = [_inputs(m, n, k, 400 + 10 * i) for i, (m, n, k) in enumerate(sizes)]
    dev = [(_gpu.dev(A), _gpu.dev(B)) for A, B in data]
    outs = [torch.zeros((n, m), dtype=torch.float64, device="cuda") for m, n, _ in sizes]
    probs = oz.problems_array([dict(m=m, n=n, k=k, A=dA, lda=m, B=dB, ldb=k, C=C, ldc=m,
                                    num_moduli=N)
                               for (m, n, k), (dA, dB), C in zip(sizes, dev, outs)])
    h = oz.Handle()
    h.set_option(oz.OPT_WAIT_LIMIT_NS, 0)
    assert oz.ozaki2_dgemm_grouped(len(sizes), probs, h) == 0
    assert h.status() & oz.STATUS_TIMEOUT
    h.set_option(oz.OPT_WAIT_LIMIT_NS, DEFAULT_LIMIT_NS)
    assert oz.ozaki2_dgemm_grouped(len(sizes), probs, h) == 0
    assert h.status() == 0
    for (m, n, k), (A, B), C in zip(sizes, data, outs):
        assert _gpu.same_bits(C.cpu().numpy(), orc.dgemm(A, B, m, n, k, N)), (m, n, k)


def test_wait_limit_option_range():
    from paper_2606_29129_gb300 import ozaki2 as oz

    h = oz.Handle()
    with pytest.raises(oz.Ozaki2Error):
        h.set_option(oz.OPT_WAIT_LIMIT_NS, -1)
    h.set_option(oz.OPT_WAIT_LIMIT_NS, DEFAULT_LIMIT_NS)
