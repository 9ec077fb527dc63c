"""The C ABI library loads and exports every entry point that include/*.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_2302_09005_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(fv_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(_build.build())


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("fv_batch_create", "fv_patch_update_batch", "fv_halo_fill",
                     "fv_max_eigenvalue_reduce"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_validation_without_gpu(lib):
    lib.fv_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.fv_status_string.restype = ctypes.c_char_p
    h = ctypes.c_void_p(1234)
    # d out of range, s != d + 2: rejected before any CUDA call
    assert lib.fv_batch_create(ctypes.byref(h), 4, 6, None, None) == 1
    assert h.value is None
    assert lib.fv_batch_create(ctypes.byref(h), 3, 4, None, None) == 1
    assert lib.fv_batch_create(None, 3, 5, None, None) == 1
    assert lib.fv_status_string(0) == b"FV_OK"
    assert lib.fv_status_string(7) == b"FV_ERR_BAD_PATCH"
    lib.fv_patch_update_batch.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_int64, ctypes.c_int,
                                                                   ctypes.c_int, ctypes.c_double,
                                                                   ctypes.c_double]
    assert lib.fv_patch_update_batch(None, None, None, None, None, 0, 3, 5, 0.1, 0.1) == 1
