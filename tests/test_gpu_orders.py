"""Every interpolation order p = 1..4, both node families, both storage types and both grid
kinds against the oracle (FP32 <= 1e-5 after one step, <= 1e-4 after 30 steps; FP64 populations
element by element), including a grid whose tiles are ragged in both directions, zero-gradient
axes, and degenerate grids of one or two cells (which run in the gather kernel).
"""
import dataclasses

import numpy as np
import pytest

from paper_1910_13918_gb300 import workloads as W

from . import helpers as H
from .test_gpu_parity import TOL_1, TOL_100, TOL_F64, gpu_run

pytestmark = pytest.mark.gpu


def _tgv(p, cells_x, cells_y, nodes="glc", bc=(W.PERIODIC, W.PERIODIC)):
    w = W.tgv16()
    w = dataclasses.replace(w, order=p, nodes=nodes, bc_x=bc[0], bc_y=bc[1], seed=20 + p)
    return w.resized(cells_x, cells_y, steps=30)


CASES = {
    "p1": _tgv(1, 36, 21),
    "p2_equidistant": _tgv(2, 17, 11, nodes="equidistant"),
    "p3": _tgv(3, 12, 9),
    "p4_clamped": _tgv(4, 11, 6, bc=(W.ZERO_GRADIENT, W.ZERO_GRADIENT)),
    "tiny_p2_one_cell": _tgv(2, 1, 1),
    "tiny_p4_clamped": _tgv(4, 2, 3, bc=(W.ZERO_GRADIENT, W.ZERO_GRADIENT)),
    "tiny_p3_mixed": _tgv(3, 1, 2, bc=(W.PERIODIC, W.ZERO_GRADIENT)),
    "p3_mapped": dataclasses.replace(W.svi(), order=3).resized(14, 8, steps=30, dt=0.01),
    "p4_mapped": dataclasses.replace(W.svi(), order=4).resized(10, 6, steps=30, dt=0.01),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nsteps,tol", [(1, TOL_1), (30, TOL_100)])
def test_orders_f32(gpu_lib, name, nsteps, tol):
    w = CASES[name]
    s, gpu, _ = gpu_run(w, nsteps, "f32")
    err = H.field_errors(gpu, H.oracle_run(w, nsteps), w.velocity_scale)
    assert max(err.values()) <= tol, (name, s.kernel_name, err)


@pytest.mark.parametrize("name", sorted(CASES))
def test_orders_f64_state(gpu_lib, name):
    w = CASES[name]
    s, _, _ = gpu_run(w, 5, "f64")
    st = s.get_state().cpu().numpy()
    f, g = H.oracle_state(w, 5)
    scale = np.max(np.abs(f))
    assert np.max(np.abs(st[0] - f)) <= TOL_F64 * scale, name
    assert np.max(np.abs(st[1] - g)) <= TOL_F64 * scale, name


@pytest.mark.parametrize("name", ["p1", "p3", "p3_mapped"])
def test_orders_bf16(gpu_lib, name):
    w = CASES[name]
    _, gpu, _ = gpu_run(w, 5, "bf16")
    err = H.field_errors(gpu, H.oracle_run(w, 5), w.velocity_scale)
    assert max(err.values()) <= 2e-2, (name, err)


def test_kernels_selected(gpu_lib):
    """The fused kernels run where they apply: uniform grids in the uniform kernel (the clamped
    grid with a gather fix-up of its boundary vertices), mapped grids in the mapped kernel."""
    from paper_1910_13918_gb300.sllbm import SLLBM
    expect = {"p1": ("uniform_fused", 1), "p3": ("uniform_fused", 1),
              "p4_clamped": ("uniform_fused", 2), "p3_mapped": ("mapped_fused", 1)}
    for name, (kernel, launches) in expect.items():
        s = SLLBM.from_workload(CASES[name], prec="f32")
        s.precompute()
        assert (s.kernel_name, s.launches_per_step) == (kernel, launches), name
