"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no GPU needed, no compute call)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1503_03337_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def library():
    build.build()
    return lbm.load()


def test_header_declares_core_calls():
    names = declared_functions()
    for core in ("lbm_create", "lbm_set_geometry", "lbm_set_params", "lbm_step",
                 "lbm_read_fields", "lbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in sorted(declared_functions()) if not hasattr(library, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert declared_functions() <= set(lbm.SIGNATURES), \
        sorted(declared_functions() - set(lbm.SIGNATURES))


def test_strerror_and_argument_errors(library):
    assert lbm.load().lbm_strerror(lbm.LBM_EINVAL).decode() == "invalid argument"
    out = ctypes.c_void_p()
    # rejected before any CUDA call
    assert library.lbm_create(None, None, ctypes.byref(out)) == lbm.LBM_EINVAL
    bad = lbm.lbm_desc(15, 8, 8, 8, lbm.LBM_STORAGE_F32)
    assert library.lbm_create(ctypes.byref(bad), None, ctypes.byref(out)) == lbm.LBM_EINVAL
    assert b"14, 18 or 26" in library.lbm_last_error()
    bad = lbm.lbm_desc(18, 0, 8, 8, lbm.LBM_STORAGE_F32)
    assert library.lbm_create(ctypes.byref(bad), None, ctypes.byref(out)) == lbm.LBM_EINVAL
    bad = lbm.lbm_desc(18, 8, 8, 8, 9)
    assert library.lbm_create(ctypes.byref(bad), None, ctypes.byref(out)) == lbm.LBM_EINVAL
    big = lbm.lbm_desc(18, 2048, 1024, 1024, lbm.LBM_STORAGE_F16)  # 2^31 cells
    assert library.lbm_create(ctypes.byref(big), None, ctypes.byref(out)) == lbm.LBM_EINVAL
    assert b"2^31" in library.lbm_last_error()
    tall = lbm.lbm_desc(14, 4, 4, 65536, lbm.LBM_STORAGE_F32)  # grid z limit
    assert library.lbm_create(ctypes.byref(tall), None, ctypes.byref(out)) == lbm.LBM_EINVAL
    assert library.lbm_step(None, 1) == lbm.LBM_EINVAL
    library.lbm_destroy(None)
