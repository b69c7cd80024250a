"""Host-side bookkeeping that needs no GPU: the header's enums and parameter struct against the
Python binding, the update counts of the workloads, and the algorithmic bytes bench.py divides by.
"""
import ctypes
import importlib.util
import os
import re

import pytest

from paper_1910_13918_gb300 import sllbm
from paper_1910_13918_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header():
    return open(os.path.join(ROOT, "include", "sllbm.h")).read()


def _enum_values(text, *names):
    out = {}
    for n in names:
        m = re.search(rf"\b{n}\s*=\s*(\d+)", text)
        assert m, n
        out[n] = int(m.group(1))
    return out


def test_header_enums_match_the_binding():
    e = _enum_values(_header(), "SLLBM_VEL_D2Q25_HERMITE", "SLLBM_VEL_D2Q9", "SLLBM_PREC_F32",
                     "SLLBM_PREC_BF16_STORE", "SLLBM_PREC_F64_PLAIN", "SLLBM_BC_PERIODIC",
                     "SLLBM_BC_ZERO_GRADIENT", "SLLBM_MAP_SINE", "SLLBM_ERR_UNSUPPORTED")
    assert (e["SLLBM_VEL_D2Q25_HERMITE"], e["SLLBM_VEL_D2Q9"]) == (sllbm.VEL_D2Q25, sllbm.VEL_D2Q9)
    assert sllbm.VELSETS == {"d2q25": sllbm.VEL_D2Q25, "d2q9": sllbm.VEL_D2Q9}
    assert (e["SLLBM_PREC_F32"], e["SLLBM_PREC_BF16_STORE"], e["SLLBM_PREC_F64_PLAIN"]) == \
        (sllbm.PREC_F32, sllbm.PREC_BF16_STORE, sllbm.PREC_F64_PLAIN)
    assert (e["SLLBM_BC_PERIODIC"], e["SLLBM_BC_ZERO_GRADIENT"]) == (W.PERIODIC, W.ZERO_GRADIENT)
    assert e["SLLBM_MAP_SINE"] == sllbm.MAP_SINE and e["SLLBM_ERR_UNSUPPORTED"] == sllbm.ERR_UNSUPPORTED


def _struct_fields(name):
    """(field, C type) of a typedef'd struct of the header, arrays as 'double[4]'."""
    text = re.sub(r"/\*.*?\*/", "", _header(), flags=re.S)
    body = re.search(r"typedef struct \{((?:(?!typedef).)*?)\} " + name + ";", text, re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            ctype, names = decl.split(None, 1)
            for n in names.split(","):
                m = re.match(r"\s*(\w+)(?:\[(\d+)\])?", n)
                fields.append((m.group(1), ctype + (f"[{m.group(2)}]" if m.group(2) else "")))
    return fields


def _ctypes_fields(cls):
    names = {ctypes.c_int: "int", ctypes.c_double: "double"}
    out = []
    for n, t in cls._fields_:
        if hasattr(t, "_length_"):
            out.append((n, f"{names[t._type_]}[{t._length_}]"))
        else:
            out.append((n, names[t]))
    return out


def test_structs_match_the_header():
    assert _ctypes_fields(sllbm.Params) == _struct_fields("sllbm_params")
    assert _ctypes_fields(sllbm.GridDesc) == _struct_fields("sllbm_grid_desc")


@pytest.mark.parametrize("w,expect", [
    (W.tgv256(), 1024 * 1024 * 25 * 2),                       # thermal D2Q25: f and g
    (W.tgv_moving(32, 0.05), 32 * 32 * 25),                   # isothermal D2Q25: f only
    (W.tgv_moving(32, 0.05, "d2q9"), 32 * 32 * 9),            # D2Q9: f only
])
def test_updates_per_step(w, expect):
    assert w.updates_per_step == expect


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("w,prec,kernel,expect", [
    (W.tgv256(), "f32", "uniform_fused", 8.0),     # (f, g) pairs: 4 B read + 4 B written each
    (W.tgv256(), "bf16", "uniform_fused", 4.0),
    (W.tgv256(), "f64", "plain_f64", 16.0),
    (W.svi(), "f32", "mapped_fused", 14.0),        # + 12 B record shared by f and g
    (W.tgv_moving(32, 0.05), "f32", "uniform_fused", 16.0),   # one population in pair slots
    (W.tgv_moving(32, 0.05, "d2q9"), "f32", "d2q9", 8.0),     # planar f
    (W.tgv_moving(32, 0.05, "d2q9"), "bf16", "d2q9", 4.0),
])
def test_bench_algorithmic_bytes(w, prec, kernel, expect):
    assert _bench().bytes_per_update(w, prec, kernel) == pytest.approx(expect)
