"""Device-resident encoded operands (ozaki2_encode_operands, ozaki2_dgemm_grouped_encoded): under
the proposed scaling (Section 4) the shift of a row of op(A) depends on that row only and the
shift of a column of op(B) on that column only, so an operand's shifts and residue planes
(Step 2) can be computed once and reused.  Checked against the oracle: the encoding itself
(shifts and residues, bit for bit), and every product that reads encoded operands (fully,
partly or not at all encoded; one operand shared by several products), bit for bit."""
import numpy as np
import pytest

import synthetic
import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oz():
    from paper_2606_29129_gb300 import ozaki2

    return ozaki2


def _operand(oz, side, trans, lines, k, N, X_np, ld):
    import torch

    data = torch.empty(oz.ozaki2_operand_bytes(side, lines, k, N), dtype=torch.uint8,
                       device="cuda")
    X = _gpu.dev(X_np)
    return dict(side=side, trans=trans, lines=lines, k=k, X=X, ld=ld, num_moduli=N, data=data)


def _stored(rows, cols, phi, seed):
    return synthetic.paper_matrix(rows, cols, phi, seed)


def test_encoding_matches_oracle_shifts_and_residues(oz, orc):
    import torch

    cases = [("A", "N", 200, 130, 14), ("A", "T", 77, 300, 20), ("B", "N", 300, 97, 8),
             ("B", "T", 129, 64, 16)]
    ops, mats = [], []
    for i, (side, trans, lines, k, N) in enumerate(cases):
        if side == "A":
            rows, cols = (lines, k) if trans == "N" else (k, lines)
        else:
            rows, cols = (k, lines) if trans == "N" else (lines, k)
        X = _stored(rows, cols, 1.0, 800 + i)
        mats.append(X)
        ops.append(_operand(oz, side, trans, lines, k, N, X, rows))
    arr = oz.operands_array(ops)
    _gpu.ok(oz.ozaki2_encode_operands(len(ops), arr), "encode")
    torch.cuda.synchronize()
    for i, ((side, trans, lines, k, N), X, o) in enumerate(zip(cases, mats, ops)):
        assert arr[i].scaling == oz.SCALING_PROPOSED
        raw = o["data"].cpu().numpy()
        align = 128 if side == "A" else 256
        lines_pad = (lines + align - 1) // align * align
        rows = max(lines, align)
        ld = max(64, (k + 63) // 64 * 64)
        off = (4 * lines_pad + 255) // 256 * 256
        shifts = raw[: 4 * lines].view(np.int32)
        planes = raw[off: off + 2 * N * rows * ld].view(np.uint16).reshape(N, rows, ld)
        res = (planes.astype(np.uint32) << 16).view(np.float32).astype(np.int64)
        if side == "A":
            e, _ = orc.shifts_a(X, lines, k, N, trans, X.shape[-1])
            R = orc.residues_a(X, lines, k, e, N, trans, X.shape[-1])
        else:
            e, _ = orc.shifts_b(X, k, lines, N, trans, X.shape[-1])
            R = orc.residues_b(X, k, lines, e, N, trans, X.shape[-1])
        assert np.array_equal(shifts, e), i
        assert np.array_equal(res[:, :lines, :k], R.astype(np.int64)), i
        assert not res[:, lines:, :].any() and not res[:, :, k:].any(), i


@pytest.mark.parametrize("scaling", ["proposed", "fast"])
def test_grouped_encoded_matches_oracle(oz, orc, scaling):
    import torch

    rng = np.random.default_rng(123)
    h = oz.Handle()
    mode = oz.SCALING_PROPOSED if scaling == "proposed" else oz.SCALING_FAST
    h.set_option(oz.OPT_SCALING, mode)
    # four A operands and four B operands; products pair them (some share an operand)
    N = 16
    k = 333
    As, Bs, ops = [], [], []
    for i in range(4):
        m = int(rng.integers(40, 400))
        tA = "N" if i % 2 == 0 else "T"
        A = _stored(m, k, 1.0, 900 + i) if tA == "N" else _stored(k, m, 1.0, 900 + i)
        As.append((m, tA, A))
        ops.append(_operand(oz, "A", tA, m, k, N, A, A.shape[-1]))
    for j in range(4):
        n = int(rng.integers(30, 500))
        tB = "N" if j % 2 == 1 else "T"
        B = _stored(k, n, 0.5, 950 + j) if tB == "N" else _stored(n, k, 0.5, 950 + j)
        Bs.append((n, tB, B))
        ops.append(_operand(oz, "B", tB, n, k, N, B, B.shape[-1]))
    arr = oz.operands_array(ops)
    _gpu.ok(oz.ozaki2_encode_operands(len(ops), arr, h), "encode")
    pairs = [(0, 0, "ab"), (0, 1, "ab"), (1, 2, "a"), (2, 3, "b"), (3, 3, ""), (1, 0, "ab")]
    probs, outs, ea, eb = [], [], [], []
    for a, b, which in pairs:
        m, tA, A = As[a]
        n, tB, B = Bs[b]
        C = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        outs.append(C)
        probs.append(dict(transA=tA, transB=tB, m=m, n=n, k=k, A=_gpu.dev(A), lda=A.shape[-1],
                          B=_gpu.dev(B), ldb=B.shape[-1], C=C, ldc=m, num_moduli=N))
        ea.append(a if "a" in which else None)
        eb.append(4 + b if "b" in which else None)
    parr = oz.problems_array(probs)
    refs_a = oz.encoded_refs(arr, ea)
    refs_b = oz.encoded_refs(arr, eb)
    assert oz.ozaki2_grouped_encoded_workspace_size(len(probs), parr, refs_a, refs_b) > 0
    _gpu.ok(oz.ozaki2_dgemm_grouped_encoded(len(probs), parr, refs_a, refs_b, h), "grouped enc")
    torch.cuda.synchronize()
    for (a, b, which), C in zip(pairs, outs):
        m, tA, A = As[a]
        n, tB, B = Bs[b]
        if scaling == "fast":
            want = orc.dgemm_mode(A, B, m, n, k, N, orc.FAST_MODE, tA, tB)
        else:
            want = orc.dgemm(A, B, m, n, k, N, tA, tB)
        assert _gpu.same_bits(C.cpu().numpy(), want), (a, b, which)


def test_grouped_encoded_rejects_mismatch_and_accurate_mode(oz):
    import torch

    k, N = 100, 14
    A = _stored(50, k, 1.0, 1)
    B = _stored(k, 60, 1.0, 2)
    ops = [_operand(oz, "A", "N", 50, k, N, A, 50), _operand(oz, "B", "N", 60, k, N, B, k)]
    arr = oz.operands_array(ops)
    _gpu.ok(oz.ozaki2_encode_operands(2, arr), "encode")
    C = torch.zeros((60, 50), dtype=torch.float64, device="cuda")
    bad = oz.problems_array([dict(m=50, n=60, k=k, A=ops[0]["X"], lda=50, B=ops[1]["X"], ldb=k,
                                  C=C, ldc=50, num_moduli=16)])  # encoded with N = 14
    assert oz.ozaki2_dgemm_grouped_encoded(1, bad, oz.encoded_refs(arr, [0]), None) == -107
    assert oz.ozaki2_dgemm_grouped_encoded(1, bad, None, oz.encoded_refs(arr, [1])) == -109
    h = oz.Handle()
    h.set_option(oz.OPT_SCALING, oz.SCALING_ACCURATE)
    assert oz.ozaki2_encode_operands(2, arr, h) == oz.ERROR_MODE
