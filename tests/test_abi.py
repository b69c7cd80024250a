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
    return sorted(set(re.findall(r"\b(sllbm(?:3d)?_[a-z0-9_]+)\s*\(", text)))


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


def test_host_validation_of_sizes_and_options():
    """Size limits and option combinations are rejected on the host, before any CUDA call."""
    lib = sllbm.load()
    h = ctypes.c_void_p()

    def create(g, p):
        return lib.sllbm_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h))

    ok_grid = lambda: sllbm.GridDesc(4, 4, 2, 0.0, 1.0, 0.0, 1.0, 0, 0, 0, 0, (ctypes.c_double * 4)())
    ok_params = lambda: sllbm.Params(0, 0.01, 0.8, 2.5, 1.0, 0, 1.0, 0)
    g = ok_grid()
    g.nx_cells = (1 << 20) // 2 + 1          # more than 2^20 vertices on an axis
    assert create(g, ok_params()) == sllbm.ERR_UNSUPPORTED
    g = ok_grid()
    g.nx_cells = 0                           # empty grid
    assert create(g, ok_params()) == sllbm.ERR_ARG
    g = ok_grid()
    g.x1 = g.x0                              # degenerate domain
    assert create(g, ok_params()) == sllbm.ERR_ARG
    g = ok_grid()
    g.bc_x = 7
    assert create(g, ok_params()) == sllbm.ERR_ARG
    for field, value, status in (("pr", -1.0, sllbm.ERR_ARG), ("pr", float("nan"), sllbm.ERR_ARG),
                                 ("isothermal", 1, sllbm.ERR_ARG),      # needs cv = 1
                                 ("isothermal", 2, sllbm.ERR_ARG), ("T0", 2.0, sllbm.ERR_ARG),
                                 ("dt", 0.0, sllbm.ERR_ARG), ("cv", 0.5, sllbm.ERR_ARG),
                                 ("velset", 1, sllbm.ERR_UNSUPPORTED),   # D2Q9: isothermal only
                                 ("velset", 2, sllbm.ERR_UNSUPPORTED), ("prec", 9, sllbm.ERR_ARG)):
        p = ok_params()
        setattr(p, field, value)
        assert create(ok_grid(), p) == status, (field, value)
    # the 3D entry point: its own velocity set, FP64 or FP32 (no BF16 storage), checked before
    # any CUDA call
    h3 = ctypes.c_void_p()
    g3 = sllbm.GridDesc3(2, 2, 2, 2, 0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0, 0, 0, 0)
    p3 = lambda **kw: sllbm.Params(kw.get("velset", sllbm.VEL_D3Q125), 0.01, 0.8, kw.get("cv", 2.5), 1.0,
                                   kw.get("prec", sllbm.PREC_F64_PLAIN), kw.get("pr", 1.0),
                                   kw.get("iso", 0))
    create3 = lambda g, p: lib.sllbm3d_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h3))
    assert create3(g3, p3(velset=0)) == sllbm.ERR_UNSUPPORTED
    assert create3(g3, p3(prec=sllbm.PREC_BF16_STORE)) == sllbm.ERR_UNSUPPORTED
    assert create3(g3, p3(pr=0.75)) == sllbm.ERR_UNSUPPORTED
    assert create3(g3, p3(iso=1)) == sllbm.ERR_ARG                 # isothermal needs cv = 3/2
    assert create3(g3, p3(cv=1.0)) == sllbm.ERR_ARG
    g3.nz_cells = 0
    assert create3(g3, p3()) == sllbm.ERR_ARG
    assert create(ok_grid(), p3()) == sllbm.ERR_UNSUPPORTED         # the 2D context refuses D3Q125
    # D2Q9 with the isothermal configuration but a Prandtl number other than 1
    p = sllbm.Params(sllbm.VEL_D2Q9, 0.01, 0.8, 1.0, 1.0, 0, 0.75, 1)
    assert create(ok_grid(), p) == sllbm.ERR_UNSUPPORTED
