"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

from paper_1910_13918_gb300 import build
from paper_1910_13918_gb300 import sllbm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sllbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sllbm_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_bound():
    assert sorted(sllbm.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    lib = sllbm.load()
    for s in range(8):
        assert lib.sllbm_status_string(s)
    # invalid descriptors are rejected on the host, before any CUDA call
    g = sllbm.GridDesc(4, 4, 7, 0.0, 1.0, 0.0, 1.0, 0, 0, 0, 0, (ctypes.c_double * 4)())
    p = sllbm.Params(0, 0.01, 0.8, 2.5, 1.0, 0)
    h = ctypes.c_void_p()
    assert lib.sllbm_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)) == sllbm.ERR_UNSUPPORTED
    g.order = 2
    p.tau = 0.4
    assert lib.sllbm_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)) == sllbm.ERR_ARG
    assert lib.sllbm_create(None, ctypes.byref(p), None, ctypes.byref(h)) == sllbm.ERR_ARG
