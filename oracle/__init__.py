"""CPU oracle for Ozaki scheme II (fast mode, Algorithm 2 scaling) -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline and
reference (``--impl reference``) legs may use this package.  It wraps ``ozaki2_oracle.c`` (plain C + OpenMP) through ctypes and shares no
code with the CUDA library.  Matrices are column-major: a rows x cols matrix is a
C-contiguous numpy array of storage shape (cols, rows) with leading dimension rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ozaki2_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SHIFT_NONFINITE = -(2**31)
MODULI = None  # filled from the library by constants()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no architecture-specific flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-frounding-math",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
        ch = ctypes.c_char
        L.orc_num_threads.restype = i32
        L.orc_log2_ru.argtypes = [f32]
        L.orc_log2_ru.restype = f32
        L.orc_alg2_shift.argtypes = [f64, f32]
        L.orc_alg2_shift.restype = i32
        L.orc_constants.argtypes = [i32, P, P, P, P, P]
        L.orc_shifts_a.argtypes = [ch, i32, i32, P, i64, i32, P, P]
        L.orc_shifts_b.argtypes = [ch, i32, i32, P, i64, i32, P, P]
        L.orc_residues_a.argtypes = [ch, i32, i32, P, i64, P, i32, P]
        L.orc_residues_b.argtypes = [ch, i32, i32, P, i64, P, i32, P]
        L.orc_residue_products.argtypes = [i32, i32, i32, i32, P, P, P]
        L.orc_crt.argtypes = [i32, i32, i32, P, P, P, f64, f64, P, i64]
        L.orc_crt_exact.argtypes = [i32, i32, i32, P, P]
        L.orc_words_to_double.argtypes = [i32, P, P]
        L.orc_words_residues.argtypes = [i32, P, i32, P]
        L.orc_dgemm.argtypes = [ch, ch, i32, i32, i32, f64, P, i64, P, i64, f64, P, i64, i32]
        L.orc_dgemm_block.argtypes = [ch, ch, i32, i32, i32, f64, P, i64, P, i64, f64, P,
                                      i32, i32, P, i32, P, P, P, P]
        L.orc_dd_block.argtypes = [ch, ch, i32, P, i64, P, i64, i32, P, i32, P, P, P]
        L.orc_fast_delta.restype = f32
        L.orc_alg1_shift.argtypes = [f64, f64, f32]
        L.orc_alg1_shift.restype = i32
        L.orc_shifts_mode.argtypes = [i32, ch, i32, i32, P, i64, i32, i32, P]
        L.orc_dgemm_mode.argtypes = [ch, ch, i32, i32, i32, f64, P, i64, P, i64, f64, P, i64,
                                     i32, i32]
        L.orc_pprime_fast.argtypes = [i32, P]
        L.orc_accu_shift.argtypes = [i32, i32, i64, f32]
        L.orc_accu_shift.restype = i32
        L.orc_accu_bar.argtypes = [i32, ch, i32, i32, P, i64, P, P, P]
        L.orc_accurate_shifts.argtypes = [ch, ch, i32, i32, i32, P, i64, P, i64, i32, P, P, P, P]
        L.orc_sgemm.argtypes = [ch, ch, i32, i32, i32, f32, P, i64, P, i64, f32, P, i64, i32]
        L.orc_sgemm_block.argtypes = [ch, ch, i32, f32, P, i64, P, i64, f32, P, i32, i32, P, i32,
                                      P, P, P, P]
        L.orc_sgemm_mode.argtypes = [ch, ch, i32, i32, i32, f32, P, i64, P, i64, f32, P, i64,
                                     i32, i32]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _b(c: str) -> bytes:
    return c.encode()


def _ck(rc):
    if rc != 0:
        raise RuntimeError(f"oracle call failed ({rc})")


def num_threads() -> int:
    return lib().orc_num_threads()


# ---------------------------------------------------------------- 256-bit words <-> Python int
def words_to_int(w) -> int:
    v = 0
    for i in range(3, -1, -1):
        v = (v << 64) | int(w[i])
    return v - (1 << 256) if v >> 255 else v


def int_to_words(x: int) -> np.ndarray:
    v = x % (1 << 256)
    return np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)


# ---------------------------------------------------------------- Step 1
def constants(N: int) -> dict:
    """p, q, P'_prop, P and P_i q_i (as Python ints) for N moduli."""
    p = np.zeros(N, np.int32)
    q = np.zeros(N, np.int32)
    pp = ctypes.c_float()
    Pw = np.zeros(4, np.uint64)
    Pqw = np.zeros((N, 4), np.uint64)
    _ck(lib().orc_constants(N, _p(p), _p(q), ctypes.byref(pp), _p(Pw), _p(Pqw)))
    return {"p": [int(x) for x in p], "q": [int(x) for x in q], "pprime": float(pp.value),
            "P": words_to_int(Pw), "Pq": [words_to_int(Pqw[l]) for l in range(N)]}


def alg2_shift(a_norm: float, pprime: float) -> int:
    return lib().orc_alg2_shift(float(a_norm), float(pprime))


def log2_ru(x: float) -> float:
    return lib().orc_log2_ru(float(x))


# ---------------------------------------------------------------- Step 2
def shifts_a(A: np.ndarray, m: int, k: int, N: int, trans: str = "N", lda: int | None = None):
    """(e, norms) for the rows of op(A); A is the storage array of a column-major matrix."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    e = np.zeros(m, np.int32)
    nr = np.zeros(m, np.float64)
    _ck(lib().orc_shifts_a(_b(trans), m, k, _p(A), lda, N, _p(e), _p(nr)))
    return e, nr


def shifts_b(B: np.ndarray, k: int, n: int, N: int, trans: str = "N", ldb: int | None = None):
    B = np.ascontiguousarray(B, dtype=np.float64)
    ldb = ldb if ldb is not None else B.shape[-1]
    f = np.zeros(n, np.int32)
    nr = np.zeros(n, np.float64)
    _ck(lib().orc_shifts_b(_b(trans), k, n, _p(B), ldb, N, _p(f), _p(nr)))
    return f, nr


def residues_a(A, m, k, e, N, trans="N", lda=None) -> np.ndarray:
    """R[l, i, h] = rmod(trunc(2^e_i a_ih), p_l), int8 of shape (N, m, k)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    e = np.ascontiguousarray(e, dtype=np.int32)
    R = np.zeros((N, m, k), np.int8)
    _ck(lib().orc_residues_a(_b(trans), m, k, _p(A), lda, _p(e), N, _p(R)))
    return R


def residues_b(B, k, n, f, N, trans="N", ldb=None) -> np.ndarray:
    """R[l, j, h] = rmod(trunc(2^f_j b_hj), p_l), int8 of shape (N, n, k)."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    ldb = ldb if ldb is not None else B.shape[-1]
    f = np.ascontiguousarray(f, dtype=np.int32)
    R = np.zeros((N, n, k), np.int8)
    _ck(lib().orc_residues_b(_b(trans), k, n, _p(B), ldb, _p(f), N, _p(R)))
    return R


# ---------------------------------------------------------------- Step 3
def residue_products(RA: np.ndarray, RB: np.ndarray) -> np.ndarray:
    """c[l, i, j] = rmod(sum_h RA[l,i,h] RB[l,j,h], p_l), int8 (N, m, n)."""
    N, m, k = RA.shape
    n = RB.shape[1]
    RA = np.ascontiguousarray(RA, dtype=np.int8)
    RB = np.ascontiguousarray(RB, dtype=np.int8)
    c = np.zeros((N, m, n), np.int8)
    _ck(lib().orc_residue_products(N, m, n, k, _p(RA), _p(RB), _p(c)))
    return c


def crt(c: np.ndarray, e, f, alpha=1.0, beta=0.0, Cin=None) -> np.ndarray:
    """Steps 3-4 from product residues; returns C as column-major storage (n, m)."""
    N, m, n = c.shape
    c = np.ascontiguousarray(c, dtype=np.int8)
    C = np.zeros((n, m), np.float64) if Cin is None else np.array(Cin, dtype=np.float64, copy=True)
    _ck(lib().orc_crt(N, m, n, _p(c), _p(np.ascontiguousarray(e, np.int32)),
                      _p(np.ascontiguousarray(f, np.int32)), alpha, beta, _p(C), m))
    return C


def crt_exact(c: np.ndarray) -> np.ndarray:
    """C'' as an object array of Python ints, shape (m, n)."""
    N, m, n = c.shape
    c = np.ascontiguousarray(c, dtype=np.int8)
    w = np.zeros((m * n, 4), np.uint64)
    _ck(lib().orc_crt_exact(N, m, n, _p(c), _p(w)))
    out = np.empty(m * n, dtype=object)
    for t in range(m * n):
        out[t] = words_to_int(w[t])
    return out.reshape(m, n)


def words_to_double(values) -> np.ndarray:
    w = np.stack([int_to_words(int(v)) for v in values]).astype(np.uint64)
    out = np.zeros(len(values), np.float64)
    _ck(lib().orc_words_to_double(len(values), _p(w), _p(out)))
    return out


def int_residues(values, N: int) -> np.ndarray:
    w = np.stack([int_to_words(int(v)) for v in values]).astype(np.uint64)
    out = np.zeros((len(values), N), np.int32)
    _ck(lib().orc_words_residues(len(values), _p(w), N, _p(out)))
    return out


# ---------------------------------------------------------------- original fast mode
FAST_MODE = 1      # Algorithm 1 (Section 2.3)
PROPOSED_MODE = 0  # Algorithm 2 (Section 4)
ACCURATE_MODE = 2  # accurate mode (Section 2.3, eq. mu_accu / nu_accu)
SHIFT_VANISH = -1100


def fast_delta() -> float:
    return lib().orc_fast_delta()


def pprime_fast(N: int) -> float:
    f = ctypes.c_float()
    _ck(lib().orc_pprime_fast(N, ctypes.byref(f)))
    return f.value


def alg1_shift(a_norm: float, a_max: float, pprime_f: float) -> int:
    return lib().orc_alg1_shift(float(a_norm), float(a_max), float(pprime_f))


def shifts_mode(X, lines, length, N, mode, side=0, trans="N", ld=None):
    X = np.ascontiguousarray(X, dtype=np.float64)
    ld = ld if ld is not None else X.shape[-1]
    out = np.zeros(lines, np.int32)
    _ck(lib().orc_shifts_mode(side, _b(trans), lines, length, _p(X), ld, N, mode, _p(out)))
    return out


def dgemm_mode(A, B, m, n, k, N, mode, transA="N", transB="N", alpha=1.0, beta=0.0, Cin=None,
               lda=None, ldb=None) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    C = np.zeros((n, m), np.float64) if Cin is None else np.array(Cin, dtype=np.float64, copy=True)
    _ck(lib().orc_dgemm_mode(_b(transA), _b(transB), m, n, k, alpha, _p(A), lda, _p(B), ldb, beta,
                             _p(C), max(m, 1), N, mode))
    return C


# ---------------------------------------------------------------- whole emulated DGEMM
def dgemm(A, B, m, n, k, N, transA="N", transB="N", alpha=1.0, beta=0.0, Cin=None,
          lda=None, ldb=None) -> np.ndarray:
    """C = alpha op(A) op(B) + beta C, returns column-major storage (n, m)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    C = np.zeros((n, m), np.float64) if Cin is None else np.array(Cin, dtype=np.float64, copy=True)
    _ck(lib().orc_dgemm(_b(transA), _b(transB), m, n, k, alpha, _p(A), lda, _p(B), ldb, beta,
                        _p(C), max(m, 1), N))
    return C


def dgemm_block(A, B, m, n, k, N, I, J, transA="N", transB="N", alpha=1.0, beta=0.0,
                Cin_block=None, e=None, f=None, lda=None, ldb=None) -> np.ndarray:
    """C(I, J) of the emulated DGEMM, as an array of shape (len(J), len(I)) (column-major)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    I = np.ascontiguousarray(I, np.int32)
    J = np.ascontiguousarray(J, np.int32)
    out = np.zeros((len(J), len(I)), np.float64)
    cin = None if Cin_block is None else np.ascontiguousarray(Cin_block, np.float64)
    e = None if e is None else np.ascontiguousarray(e, np.int32)
    f = None if f is None else np.ascontiguousarray(f, np.int32)
    _ck(lib().orc_dgemm_block(_b(transA), _b(transB), m, n, k, alpha, _p(A), lda, _p(B), ldb,
                              beta, _p(cin), N, len(I), _p(I), len(J), _p(J), _p(e), _p(f),
                              _p(out)))
    return out


def dd_block(A, B, k, I, J, transA="N", transB="N", lda=None, ldb=None):
    """Double-double (hi, lo) of (op(A) op(B))(I, J), arrays of shape (len(J), len(I))."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    I = np.ascontiguousarray(I, np.int32)
    J = np.ascontiguousarray(J, np.int32)
    hi = np.zeros((len(J), len(I)), np.float64)
    lo = np.zeros((len(J), len(I)), np.float64)
    _ck(lib().orc_dd_block(_b(transA), _b(transB), k, _p(A), lda, _p(B), ldb, len(I), _p(I),
                           len(J), _p(J), _p(hi), _p(lo)))
    return hi, lo


def max_rel_error(C: np.ndarray, hi: np.ndarray, lo: np.ndarray):
    """Max relative error against a double-double reference; entries whose reference is zero
    are excluded and counted separately.  Returns (max_rel_err, zero_ref_count)."""
    nz = hi != 0
    err = np.abs((C - hi) - lo)
    rel = np.where(nz, err / np.where(nz, np.abs(hi), 1.0), 0.0)
    return float(rel.max(initial=0.0)), int((~nz).sum())


# ---------------------------------------------------------------- accurate mode
def accu_shift(kind: int, E: int, cmax: int, pprime_accu: float) -> int:
    return lib().orc_accu_shift(kind, E, cmax, pprime_accu)


def accu_bar(X, lines, length, side=0, trans="N", ld=None):
    """(bar uint8 (lines, length), E int32 (lines,), kind int32 (lines,)) of accurate mode."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    ld = ld if ld is not None else X.shape[-1]
    bar = np.zeros((max(lines, 1), max(length, 1)), np.uint8)
    E = np.zeros(max(lines, 1), np.int32)
    kind = np.zeros(max(lines, 1), np.int32)
    _ck(lib().orc_accu_bar(side, _b(trans), lines, length, _p(X), ld, _p(bar), _p(E), _p(kind)))
    return bar[:lines, :length], E[:lines], kind[:lines]


def accurate_shifts(A, B, m, n, k, N, transA="N", transB="N", lda=None, ldb=None):
    """(e, f, rowmax, colmax) of accurate mode: shifts of both operands and the row and column
    maxima of C-bar = A-bar B-bar."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    e = np.zeros(max(m, 1), np.int32)
    f = np.zeros(max(n, 1), np.int32)
    rm = np.zeros(max(m, 1), np.int64)
    cm = np.zeros(max(n, 1), np.int64)
    _ck(lib().orc_accurate_shifts(_b(transA), _b(transB), m, n, k, _p(A), lda, _p(B), ldb, N,
                                  _p(e), _p(f), _p(rm), _p(cm)))
    return e[:m], f[:n], rm[:m], cm[:n]


# ---------------------------------------------------------------- SGEMM
def sgemm(A, B, m, n, k, N, transA="N", transB="N", alpha=1.0, beta=0.0, Cin=None, lda=None,
          ldb=None, mode=PROPOSED_MODE) -> np.ndarray:
    """C = alpha op(A) op(B) + beta C in single precision through Ozaki scheme II; float32
    column-major storage (n, m) returned."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    C = np.zeros((n, m), np.float32) if Cin is None else np.array(Cin, dtype=np.float32, copy=True)
    _ck(lib().orc_sgemm_mode(_b(transA), _b(transB), m, n, k, alpha, _p(A), lda, _p(B), ldb,
                             beta, _p(C), max(m, 1), N, mode))
    return C


def sgemm_block(A, B, k, N, I, J, transA="N", transB="N", alpha=1.0, beta=0.0, Cin_block=None,
                e=None, f=None, lda=None, ldb=None) -> np.ndarray:
    """C(I, J) of the emulated SGEMM as float32 of shape (len(J), len(I)); shifts e/f (per row
    of op(A) / column of op(B), full length) are used when given."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    lda = lda if lda is not None else A.shape[-1]
    ldb = ldb if ldb is not None else B.shape[-1]
    I = np.ascontiguousarray(I, np.int32)
    J = np.ascontiguousarray(J, np.int32)
    out = np.zeros((len(J), len(I)), np.float32)
    cin = None if Cin_block is None else np.ascontiguousarray(Cin_block, np.float32)
    e = None if e is None else np.ascontiguousarray(e, np.int32)
    f = None if f is None else np.ascontiguousarray(f, np.int32)
    _ck(lib().orc_sgemm_block(_b(transA), _b(transB), k, alpha, _p(A), lda, _p(B), ldb, beta,
                              _p(cin), N, len(I), _p(I), len(J), _p(J), _p(e), _p(f), _p(out)))
    return out
