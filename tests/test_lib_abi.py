"""The C-ABI library on a machine without a GPU: it builds, loads, exports every function that
include/*.h declares, and its host-only entry points behave.  No GPU compute is called."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_29129_gb300 import build

    return build.build()


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|size_t|const\s+char\s*\*|void)\s*\**\s*(ozaki2_\w+)\s*\(",
                             text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_path():
    names = declared_functions()
    for required in ["ozaki2_dgemm", "ozaki2_scale_a", "ozaki2_scale_b", "ozaki2_convert_a",
                     "ozaki2_convert_b", "ozaki2_residue_gemm", "ozaki2_crt", "ozaki2_create",
                     "ozaki2_constants"]:
        assert required in names


def test_every_declared_symbol_is_exported(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_library_has_no_driver_dependency(libpath):
    """libcuda is looked up at run time, so the library loads on GPU-less hosts."""
    import subprocess

    out = subprocess.run(["ldd", libpath], capture_output=True, text=True).stdout
    assert "libcuda.so" not in out
    assert "libcudart" not in out


def test_host_constants_agree_with_oracle(libpath, orc):
    """Step 1 computed by the library's host code and, independently, by the oracle."""
    from paper_2606_29129_gb300 import ozaki2

    for N in range(2, 21):
        p, q, pp = ozaki2.ozaki2_constants(N)
        c = orc.constants(N)
        assert p == c["p"] and q == c["q"]
        assert pp == c["pprime"]


def test_argument_checks_without_gpu(libpath):
    from paper_2606_29129_gb300 import ozaki2

    L = ozaki2.lib()
    assert ozaki2.ozaki2_workspace_size(-1, 4, 4, 14) == 0
    assert ozaki2.ozaki2_workspace_size(4, 4, 4, 21) == 0
    assert ozaki2.ozaki2_workspace_size(16384, 16384, 16384, 14) > 14 * 16384 * 16384 * 4
    assert L.ozaki2_constants(1, None, None, None) == -1
    assert L.ozaki2_create(None) == -1
    assert ozaki2.error_string(4) == "no sm_103 GPU available"


def test_gpu_entry_points_fail_loudly_without_gpu(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_29129_gb300 import ozaki2

    h = ctypes.c_void_p()
    assert ozaki2.lib().ozaki2_create(ctypes.byref(h)) == 4   # OZAKI2_ERROR_NO_DEVICE
    rc = ozaki2.lib().ozaki2_dgemm(b"N", b"N", 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 14)
    assert rc == 4
