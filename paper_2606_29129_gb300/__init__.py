"""GB300-native (sm_103a) Ozaki scheme II DGEMM emulation, fast mode with the scale-invariant
scaling of Algorithm 2 (Kawakami & Takahashi).

The compute path lives in libozaki2.so (CUDA kernels for sm_103a behind the C ABI of
include/ozaki2.h); ``ozaki2`` is its ctypes binding.
"""
from . import ozaki2  # noqa: F401
from .ozaki2 import Handle, dgemm  # noqa: F401
