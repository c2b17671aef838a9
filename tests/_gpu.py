"""Helpers for the GPU parity tests: run each stage through the C ABI on torch buffers."""
from __future__ import annotations

import numpy as np


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def ok(rc, what="call"):
    assert rc == 0, f"{what} returned {rc}"


def round_up(v, a):
    return (max(v, 1) + a - 1) // a * a


def shifts_a(oz, A_np, m, k, N, trans="N", lda=None, handle=None):
    import torch

    lda = lda if lda is not None else A_np.shape[-1]
    out = torch.zeros(max(m, 1), dtype=torch.int32, device="cuda")
    ok(oz.ozaki2_scale_a(trans, m, k, dev(A_np), lda, N, out, handle), "scale_a")
    torch.cuda.synchronize()
    return out.cpu().numpy()[:m]


def shifts_b(oz, B_np, k, n, N, trans="N", ldb=None, handle=None):
    import torch

    ldb = ldb if ldb is not None else B_np.shape[-1]
    out = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    ok(oz.ozaki2_scale_b(trans, k, n, dev(B_np), ldb, N, out, handle), "scale_b")
    torch.cuda.synchronize()
    return out.cpu().numpy()[:n]


def planes_a(oz, A_np, m, k, e, N, trans="N", lda=None):
    """bf16 residue planes of op(A) read back as int (N, rows_pad, k_pad)."""
    import torch

    lda = lda if lda is not None else A_np.shape[-1]
    rp, kp = round_up(m, oz.ROWS_ALIGN_A), round_up(k, oz.K_ALIGN)
    planes = torch.full((N, rp, kp), 7.0, dtype=torch.bfloat16, device="cuda")
    ok(oz.ozaki2_convert_a(trans, m, k, dev(A_np), lda, dev(np.asarray(e, np.int32)), N, planes,
                           rp, kp), "convert_a")
    torch.cuda.synchronize()
    return planes.float().cpu().numpy().astype(np.int64)


def planes_b(oz, B_np, k, n, f, N, trans="N", ldb=None):
    import torch

    ldb = ldb if ldb is not None else B_np.shape[-1]
    rp, kp = round_up(n, oz.ROWS_ALIGN_B), round_up(k, oz.K_ALIGN)
    planes = torch.full((N, rp, kp), 7.0, dtype=torch.bfloat16, device="cuda")
    ok(oz.ozaki2_convert_b(trans, k, n, dev(B_np), ldb, dev(np.asarray(f, np.int32)), N, planes,
                           rp, kp), "convert_b")
    torch.cuda.synchronize()
    return planes.float().cpu().numpy().astype(np.int64)


def residue_gemm(oz, RA, RB, variant=None):
    """RA (N, m_pad, k_pad), RB (N, n_pad, k_pad) integer arrays -> int8 (N, m_pad, n_pad).
    variant: None (automatic) or one of oz.GEMM_SINGLE / oz.GEMM_PAIR."""
    import torch

    h = None
    if variant is not None:
        h = oz.Handle()
        h.set_option(oz.OPT_GEMM_VARIANT, variant)
    N, mp, kp = RA.shape
    npad = RB.shape[1]
    pa = torch.from_numpy(np.ascontiguousarray(RA, dtype=np.float32)).to(torch.bfloat16).cuda()
    pb = torch.from_numpy(np.ascontiguousarray(RB, dtype=np.float32)).to(torch.bfloat16).cuda()
    out = torch.full((N, mp, npad), 99, dtype=torch.int8, device="cuda")
    ok(oz.ozaki2_residue_gemm(N, mp, npad, kp, pa, pb, out, handle=h), "residue_gemm")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def crt(oz, c, e, f, m, n, alpha=1.0, beta=0.0, Cin=None):
    """c int8 (N, m_pad, n_pad) -> C column-major storage (n, m)."""
    import torch

    N, mp, npad = c.shape
    C = torch.zeros((n, m), dtype=torch.float64, device="cuda") if Cin is None else dev(Cin)
    ok(oz.ozaki2_crt(N, m, n, dev(c), npad, mp * npad, dev(np.asarray(e, np.int32)),
                     dev(np.asarray(f, np.int32)), alpha, beta, C, max(m, 1)), "crt")
    torch.cuda.synchronize()
    return C.cpu().numpy()


def dgemm(oz, A_np, B_np, m, n, k, N, transA="N", transB="N", alpha=1.0, beta=0.0, Cin=None,
          lda=None, ldb=None, handle=None, variant=None):
    import torch

    lda = lda if lda is not None else A_np.shape[-1]
    ldb = ldb if ldb is not None else B_np.shape[-1]
    if variant is not None:
        handle = handle or oz.Handle()
        handle.set_option(oz.OPT_GEMM_VARIANT, variant)
    C = torch.zeros((max(n, 1), max(m, 1)), dtype=torch.float64, device="cuda") if Cin is None \
        else dev(Cin)
    A = dev(A_np) if A_np.size else torch.zeros(1, dtype=torch.float64, device="cuda")
    B = dev(B_np) if B_np.size else torch.zeros(1, dtype=torch.float64, device="cuda")
    ok(oz.ozaki2_dgemm(transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, max(m, 1), N,
                       handle), "dgemm")
    torch.cuda.synchronize()
    return C.cpu().numpy()


def same_bits(a, b) -> bool:
    """Bit equality of float arrays, treating every NaN as equal."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    if not np.array_equal(na, nb):
        return False
    return np.array_equal(a[~na].view(np.int64), b[~nb].view(np.int64))
