"""Thin ctypes binding of libozaki2.so (include/ozaki2.h).

Argument marshalling only: every step of the emulated DGEMM runs in the library's CUDA kernels.
Functions named like the C ABI take the same arguments; device buffers may be given as torch
tensors (their data_ptr is passed) or as integer addresses.  Work is queued on the calling
thread's current torch CUDA stream.  There is no CPU fallback: if the library or an sm_103
GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libozaki2.so")

SUCCESS = 0
STATUS_NONFINITE = 1
STATUS_TIMEOUT = 2
STATUS_RANGE = 4
ROWS_ALIGN_A = 128
ROWS_ALIGN_B = 256
K_ALIGN = 64
SHIFT_NONFINITE = -(2**31)
SHIFT_VANISH = -1100
ACCURATE_MAX_K = 1048575
ERROR_TOO_LARGE = 6
ERROR_MODE = 7
OPT_GEMM_VARIANT = 1
OPT_CHUNK_K = 2
OPT_GRAPH = 3
OPT_SCALING = 4
OPT_WAIT_LIMIT_NS = 5
OPT_GROUP_M = 6
OPT_L2_HINTS = 7
OPT_HOST_COPIES = 8
SCALING_PROPOSED, SCALING_FAST, SCALING_ACCURATE = 0, 1, 2
GEMM_AUTO, GEMM_SINGLE, GEMM_PAIR = 0, 1, 2
NOALLOC_SCRATCH_BYTES = 8 << 20
MAX_TILE_RULES = 16
TILE_WIDTHS = (256, 128, 64)

_lib = None
_lock = threading.Lock()


class Problem(ctypes.Structure):
    """ozaki2_problem: the arguments of one ozaki2_dgemm inside a grouped call."""
    _fields_ = [("transA", ctypes.c_char), ("transB", ctypes.c_char), ("m", ctypes.c_int),
                ("n", ctypes.c_int), ("k", ctypes.c_int), ("alpha", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int), ("beta", ctypes.c_double), ("C", ctypes.c_void_p),
                ("ldc", ctypes.c_int), ("num_moduli", ctypes.c_int)]


class Operand(ctypes.Structure):
    """ozaki2_operand: one operand to encode (side 'A': rows of op(A); 'B': columns of op(B))
    and, after ozaki2_encode_operands, the description of its encoding in `data`."""
    _fields_ = [("side", ctypes.c_char), ("trans", ctypes.c_char), ("lines", ctypes.c_int),
                ("k", ctypes.c_int), ("X", ctypes.c_void_p), ("ld", ctypes.c_int),
                ("num_moduli", ctypes.c_int), ("data", ctypes.c_void_p),
                ("scaling", ctypes.c_int)]


class Ozaki2Error(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {code}: {error_string(code)}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libozaki2.so (built by paper_2606_29129_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2606_29129_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64, f32, ch = (ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                                      ctypes.c_double, ctypes.c_float, ctypes.c_char)
        sig = {
            "ozaki2_create": [ctypes.POINTER(vp)],
            "ozaki2_destroy": [vp],
            "ozaki2_set_stream": [vp, vp],
            "ozaki2_set_workspace": [vp, vp, ctypes.c_size_t],
            "ozaki2_get_status": [vp, ctypes.POINTER(ctypes.c_uint)],
            "ozaki2_constants": [i32, vp, vp, ctypes.POINTER(ctypes.c_float)],
            "ozaki2_dgemm": [ch, ch, i32, i32, i32, f64, vp, i32, vp, i32, f64, vp, i32, i32],
            "ozaki2_dgemm_h": [vp, ch, ch, i32, i32, i32, f64, vp, i32, vp, i32, f64, vp, i32,
                               i32],
            "ozaki2_sgemm": [ch, ch, i32, i32, i32, f32, vp, i32, vp, i32, f32, vp, i32, i32],
            "ozaki2_sgemm_h": [vp, ch, ch, i32, i32, i32, f32, vp, i32, vp, i32, f32, vp, i32,
                               i32],
            "ozaki2_scale_a": [vp, ch, i32, i32, vp, i32, i32, vp],
            "ozaki2_scale_b": [vp, ch, i32, i32, vp, i32, i32, vp],
            "ozaki2_scale_norms": [vp, ch, ch, i32, i32, vp, i32, i32, vp, vp],
            "ozaki2_scale_accurate": [vp, ch, ch, i32, i32, i32, vp, i32, vp, i32, i32, vp, vp,
                                      vp],
            "ozaki2_convert_a": [vp, ch, i32, i32, vp, i32, vp, i32, vp, i32, i32],
            "ozaki2_convert_b": [vp, ch, i32, i32, vp, i32, vp, i32, vp, i32, i32],
            "ozaki2_residue_gemm": [vp, i32, i32, i32, i32, vp, vp, vp],
            "ozaki2_crt": [vp, i32, i32, i32, vp, i32, i64, vp, vp, f64, f64, vp, i32],
            "ozaki2_dgemm_noalloc": [ch, ch, i32, i32, i32, f64, vp, i32, vp, i32, f64, vp, i32,
                                     i32, vp],
            "ozaki2_dgemm_grouped": [vp, i32, vp],
            "ozaki2_set_timing": [vp, i32],
            "ozaki2_set_option": [vp, i32, i32],
            "ozaki2_set_grouped_tiles": [vp, i32, vp, vp, vp, vp],
            "ozaki2_encode_operands": [vp, i32, vp],
            "ozaki2_dgemm_grouped_encoded": [vp, i32, vp, vp, vp],
            "ozaki2_get_timing": [vp, ctypes.POINTER(ctypes.c_float)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = i32
        L.ozaki2_grouped_workspace_size.argtypes = [i32, vp]
        L.ozaki2_grouped_workspace_size.restype = ctypes.c_size_t
        L.ozaki2_grouped_encoded_workspace_size.argtypes = [i32, vp, vp, vp]
        L.ozaki2_grouped_encoded_workspace_size.restype = ctypes.c_size_t
        L.ozaki2_operand_bytes.argtypes = [ch, i32, i32, i32]
        L.ozaki2_operand_bytes.restype = ctypes.c_size_t
        L.ozaki2_workspace_size.argtypes = [i32, i32, i32, i32]
        L.ozaki2_workspace_size.restype = ctypes.c_size_t
        L.ozaki2_error_string.argtypes = [i32]
        L.ozaki2_error_string.restype = ctypes.c_char_p
        _lib = L
        return _lib


def error_string(code: int) -> str:
    return lib().ozaki2_error_string(int(code)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _ch(c: str) -> bytes:
    return c.encode() if isinstance(c, str) else c


def _check(fn: str, rc: int) -> int:
    if rc != SUCCESS:
        raise Ozaki2Error(fn, rc)
    return rc


def _current_stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


class Handle:
    """An ozaki2 handle; each call queues on the current torch stream."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check("ozaki2_create", lib().ozaki2_create(ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            lib().ozaki2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_stream(self):
        _check("ozaki2_set_stream", lib().ozaki2_set_stream(self.h, _current_stream()))
        return self.h

    def set_workspace(self, buf, nbytes: int):
        _check("ozaki2_set_workspace", lib().ozaki2_set_workspace(self.h, _ptr(buf), nbytes))

    def set_option(self, option: int, value: int):
        _check("ozaki2_set_option", lib().ozaki2_set_option(self.h, option, value))

    def set_grouped_tiles(self, rules):
        """Tile configuration of grouped calls by size class: rules is a sequence of
        (n_max, k_max, tile_n, chunk_k); the first rule with n <= n_max and k <= k_max applies
        (chunk_k 0: the handle's OPT_CHUNK_K).  An empty sequence restores the automatic
        choice."""
        rules = list(rules)
        cols = [(ctypes.c_int * max(1, len(rules)))(*(int(r[c]) for r in rules))
                for c in range(4)]
        _check("ozaki2_set_grouped_tiles",
               lib().ozaki2_set_grouped_tiles(self.h, len(rules), *cols))

    def set_timing(self, on: bool = True):
        _check("ozaki2_set_timing", lib().ozaki2_set_timing(self.h, 1 if on else 0))

    def timing(self):
        """Stage milliseconds of the last timed dgemm: (scale, convert, residue_gemm, crt)."""
        ms = (ctypes.c_float * 4)()
        _check("ozaki2_get_timing", lib().ozaki2_get_timing(self.h, ms))
        return tuple(ms)

    def status(self) -> int:
        v = ctypes.c_uint()
        _check("ozaki2_get_status", lib().ozaki2_get_status(self.h, ctypes.byref(v)))
        return v.value


_default = None


def default_handle() -> Handle:
    global _default
    if _default is None:
        _default = Handle()
    return _default


def _h(handle):
    return (handle or default_handle()).sync_stream()


# ---------------------------------------------------------------- C ABI, one wrapper each
def ozaki2_constants(num_moduli: int):
    n = int(num_moduli)
    p = (ctypes.c_int * n)()
    q = (ctypes.c_int * n)()
    f = ctypes.c_float()
    _check("ozaki2_constants", lib().ozaki2_constants(n, p, q, ctypes.byref(f)))
    return list(p), list(q), f.value


def ozaki2_workspace_size(m, n, k, num_moduli) -> int:
    return lib().ozaki2_workspace_size(m, n, k, num_moduli)


def ozaki2_dgemm(transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli,
                 handle: Handle | None = None) -> int:
    return lib().ozaki2_dgemm_h(_h(handle), _ch(transA), _ch(transB), m, n, k, alpha, _ptr(A),
                                lda, _ptr(B), ldb, beta, _ptr(C), ldc, num_moduli)


def ozaki2_sgemm(transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli,
                 handle: Handle | None = None) -> int:
    return lib().ozaki2_sgemm_h(_h(handle), _ch(transA), _ch(transB), m, n, k, alpha, _ptr(A),
                                lda, _ptr(B), ldb, beta, _ptr(C), ldc, num_moduli)


def problems_array(problems):
    """A ctypes array of Problem from dicts with the ozaki2_dgemm argument names (device buffers
    as tensors or addresses)."""
    arr = (Problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = Problem(_ch(p.get("transA", "N")), _ch(p.get("transB", "N")), p["m"], p["n"],
                         p["k"], p.get("alpha", 1.0), _ptr(p["A"]), p["lda"], _ptr(p["B"]),
                         p["ldb"], p.get("beta", 0.0), _ptr(p["C"]), p["ldc"],
                         p["num_moduli"])
    return arr


def ozaki2_dgemm_grouped(count, problems, handle=None) -> int:
    """problems: a ctypes array of Problem (see problems_array)."""
    return lib().ozaki2_dgemm_grouped(_h(handle), count, ctypes.cast(problems, ctypes.c_void_p))


def ozaki2_grouped_workspace_size(count, problems) -> int:
    return lib().ozaki2_grouped_workspace_size(count, ctypes.cast(problems, ctypes.c_void_p))


def ozaki2_operand_bytes(side, lines, k, num_moduli) -> int:
    return lib().ozaki2_operand_bytes(_ch(side), lines, k, num_moduli)


def operands_array(operands):
    """A ctypes array of Operand from dicts with the field names (matrices and data buffers as
    tensors or addresses)."""
    arr = (Operand * len(operands))()
    for i, o in enumerate(operands):
        arr[i] = Operand(_ch(o["side"]), _ch(o.get("trans", "N")), o["lines"], o["k"],
                         _ptr(o["X"]), o["ld"], o["num_moduli"], _ptr(o["data"]), 0)
    return arr


def ozaki2_encode_operands(count, operands, handle=None) -> int:
    """operands: a ctypes array of Operand (see operands_array); its scaling fields are set."""
    return lib().ozaki2_encode_operands(_h(handle), count, ctypes.cast(operands, ctypes.c_void_p))


def encoded_refs(operands, picks):
    """A ctypes array of pointers into `operands` (an Operand array): entry i points at
    operands[picks[i]], or is NULL when picks[i] is None."""
    arr = (ctypes.POINTER(Operand) * len(picks))()
    base = ctypes.addressof(operands)
    size = ctypes.sizeof(Operand)
    for i, j in enumerate(picks):
        if j is not None:
            arr[i] = ctypes.cast(base + j * size, ctypes.POINTER(Operand))
    return arr


def ozaki2_dgemm_grouped_encoded(count, problems, enc_a=None, enc_b=None, handle=None) -> int:
    """problems: a Problem array; enc_a / enc_b: None or pointer arrays (see encoded_refs)."""
    cast = (lambda a: None if a is None else ctypes.cast(a, ctypes.c_void_p))
    return lib().ozaki2_dgemm_grouped_encoded(_h(handle), count,
                                              ctypes.cast(problems, ctypes.c_void_p),
                                              cast(enc_a), cast(enc_b))


def ozaki2_grouped_encoded_workspace_size(count, problems, enc_a=None, enc_b=None) -> int:
    cast = (lambda a: None if a is None else ctypes.cast(a, ctypes.c_void_p))
    return lib().ozaki2_grouped_encoded_workspace_size(count,
                                                       ctypes.cast(problems, ctypes.c_void_p),
                                                       cast(enc_a), cast(enc_b))


def ozaki2_scale_a(transA, m, k, A, lda, num_moduli, shifts, handle=None) -> int:
    return lib().ozaki2_scale_a(_h(handle), _ch(transA), m, k, _ptr(A), lda, num_moduli,
                                _ptr(shifts))


def ozaki2_scale_b(transB, k, n, B, ldb, num_moduli, shifts, handle=None) -> int:
    return lib().ozaki2_scale_b(_h(handle), _ch(transB), k, n, _ptr(B), ldb, num_moduli,
                                _ptr(shifts))


def ozaki2_scale_norms(side, trans, lines, k, X, ld, num_moduli, shifts, norms,
                       handle=None) -> int:
    return lib().ozaki2_scale_norms(_h(handle), _ch(side), _ch(trans), lines, k, _ptr(X), ld,
                                    num_moduli, _ptr(shifts), _ptr(norms))


def ozaki2_scale_accurate(transA, transB, m, n, k, A, lda, B, ldb, num_moduli, e, f, cmax=None,
                          handle=None) -> int:
    return lib().ozaki2_scale_accurate(_h(handle), _ch(transA), _ch(transB), m, n, k, _ptr(A),
                                       lda, _ptr(B), ldb, num_moduli, _ptr(e), _ptr(f),
                                       _ptr(cmax))


def ozaki2_convert_a(transA, m, k, A, lda, shifts, num_moduli, planes, rows_pad, k_pad,
                     handle=None) -> int:
    return lib().ozaki2_convert_a(_h(handle), _ch(transA), m, k, _ptr(A), lda, _ptr(shifts),
                                  num_moduli, _ptr(planes), rows_pad, k_pad)


def ozaki2_convert_b(transB, k, n, B, ldb, shifts, num_moduli, planes, rows_pad, k_pad,
                     handle=None) -> int:
    return lib().ozaki2_convert_b(_h(handle), _ch(transB), k, n, _ptr(B), ldb, _ptr(shifts),
                                  num_moduli, _ptr(planes), rows_pad, k_pad)


def ozaki2_residue_gemm(num_moduli, m_pad, n_pad, k_pad, planes_a, planes_b, residues,
                        handle=None) -> int:
    return lib().ozaki2_residue_gemm(_h(handle), num_moduli, m_pad, n_pad, k_pad,
                                     _ptr(planes_a), _ptr(planes_b), _ptr(residues))


def ozaki2_crt(num_moduli, m, n, residues, ldr, plane_stride, shifts_a, shifts_b, alpha, beta,
               C, ldc, handle=None) -> int:
    return lib().ozaki2_crt(_h(handle), num_moduli, m, n, _ptr(residues), ldr, plane_stride,
                            _ptr(shifts_a), _ptr(shifts_b), alpha, beta, _ptr(C), ldc)


# ---------------------------------------------------------------- torch convenience
def _rowmajor_gemm(name, entry, dtype, A, B, num_moduli, alpha, beta, C, handle):
    import torch

    if A.dtype != dtype or B.dtype != dtype or not A.is_cuda or not B.is_cuda:
        raise TypeError(f"{name} expects {dtype} CUDA tensors")
    A = A.contiguous()
    B = B.contiguous()
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=dtype, device=A.device)
        beta = 0.0
    elif not C.is_contiguous() or tuple(C.shape) != (m, n):
        raise ValueError("C must be a contiguous (m, n) tensor")
    _check(entry.__name__, entry("N", "N", n, m, k, alpha, B, max(n, 1), A, max(k, 1), beta, C,
                                 max(n, 1), num_moduli, handle))
    return C


def dgemm(A, B, num_moduli: int = 16, alpha: float = 1.0, beta: float = 0.0, C=None,
          handle: Handle | None = None):
    """C = alpha A @ B + beta C for row-major float64 CUDA tensors A (m, k), B (k, n).

    Row-major storage of (m, k) is column-major storage of its transpose, so this calls
    ozaki2_dgemm on C^T = B^T A^T.  Returns C (allocated when not given).  The default of 16
    moduli is the smallest count not less accurate than cuBLAS DGEMM at m = n = k = 16384."""
    import torch

    return _rowmajor_gemm("dgemm", ozaki2_dgemm, torch.float64, A, B, num_moduli, alpha, beta, C,
                          handle)


def sgemm(A, B, num_moduli: int = 8, alpha: float = 1.0, beta: float = 0.0, C=None,
          handle: Handle | None = None):
    """The float32 counterpart of dgemm through ozaki2_sgemm (default 8 moduli, the smallest
    count not less accurate than cuBLAS SGEMM at m = n = k = 16384)."""
    import torch

    return _rowmajor_gemm("sgemm", ozaki2_sgemm, torch.float32, A, B, num_moduli, alpha, beta, C,
                          handle)
