"""The C-ABI library builds, loads and exports every function that
include/*.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import subprocess

import pytest

from helpers import ROOT, header_functions


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300.build import LIB
    return LIB


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    declared = header_functions()
    assert declared, "no declarations parsed"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    for name in header_functions():
        assert hasattr(L, name), name
    L.fv_last_error.restype = ctypes.c_char_p
    assert L.fv_last_error() == b""


def test_binding_declares_header_functions(libpath):
    from paper_2602_08670_gb300 import fv
    bound = set(fv.exported_symbols())
    for name in header_functions(os.path.join(ROOT, "include", "fv.h")):
        assert name in bound, name


def test_invalid_arguments_rejected_on_host(libpath):
    from paper_2602_08670_gb300 import fv
    L = fv.lib()
    out = ctypes.c_void_p()
    g = fv.fv_grid(0, 8, 1, 1.0, 1.0)
    p = fv.fv_swe_params(9.81, 0.5, 0, 0.0)
    buf = (ctypes.c_float * 3)()
    rc = L.swe_init(ctypes.byref(g), ctypes.byref(p), ctypes.cast(buf, ctypes.c_void_p), 0, None,
                    ctypes.byref(out))
    assert rc == fv.FV_EINVAL
    assert b"grid" in L.fv_last_error()
    assert L.fv_step(None, None) == fv.FV_EINVAL
