"""GB300-native (sm_103a) Ozaki scheme II DGEMM and SGEMM emulation, fast mode with the
scale-invariant scaling of Algorithm 2 (Kawakami & Takahashi); the original fast mode
(Algorithm 1) and accurate mode are selectable per handle.

The compute path lives in libozaki2.so (CUDA kernels for sm_103a behind the C ABI of
include/ozaki2.h); ``ozaki2`` is its ctypes binding, ``autotune`` picks the moduli count from an
accuracy target, ``serve`` is a continuous-batching server over the grouped entry point.
"""
from . import ozaki2  # noqa: F401
from .ozaki2 import Handle, dgemm, sgemm  # noqa: F401
