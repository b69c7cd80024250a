"""Prandtl number != 1 (Sec. II.C) on the GPU against the oracle, through the C ABI.

The quasi-equilibrium term runs in every kernel: the fused uniform step (Taylor-Green, Sod with
its boundary fix-up through the gather kernel, Riemann), the fused mapped step (shock-vortex) and
the plain FP64 step.  Tolerances as for Pr = 1: FP32 <= 1e-5 after one step and <= 1e-4 after
100 steps, FP64 populations <= 1e-11 relative to the largest population.
"""
import dataclasses

import numpy as np
import pytest

from paper_1910_13918_gb300 import workloads as W

from . import helpers as H
from .test_gpu_parity import TOL_1, TOL_100, TOL_F64, gpu_run

pytestmark = pytest.mark.gpu

PR = 0.75   # the paper's shock-vortex Prandtl number (Sec. III.E)


def _small(name, pr=PR):
    return dataclasses.replace(H.small_workloads()[name], pr=pr)


@pytest.mark.parametrize("name", ["tgv16", "sod", "riemann", "svi"])
@pytest.mark.parametrize("nsteps,tol", [(1, TOL_1), (100, TOL_100)])
def test_prandtl_parity_f32(gpu_lib, name, nsteps, tol):
    w = _small(name)
    s, gpu, _ = gpu_run(w, nsteps, "f32")
    err = H.field_errors(gpu, H.oracle_run(w, nsteps), w.velocity_scale)
    assert max(err.values()) <= tol, (name, s.kernel_name, err)


@pytest.mark.parametrize("name", ["tgv16", "svi"])
def test_prandtl_parity_f64_state(gpu_lib, name):
    w = _small(name)
    s, _, _ = gpu_run(w, 20, "f64")
    st = s.get_state().cpu().numpy()
    f, g = H.oracle_state(w, 20)
    scale = np.max(np.abs(f))
    assert np.max(np.abs(st[0] - f)) <= TOL_F64 * scale
    assert np.max(np.abs(st[1] - g)) <= TOL_F64 * scale


def test_prandtl_changes_the_flow(gpu_lib):
    """The term is not a no-op: Pr = 0.75 and Pr = 1 differ after 100 steps of the small
    shock-vortex run by far more than the parity tolerance."""
    _, a, _ = gpu_run(_small("svi", PR), 100, "f32")
    _, b, _ = gpu_run(_small("svi", 1.0), 100, "f32")
    assert np.max(np.abs(a[3] - b[3])) > 1e-3


def test_full_size_shock_vortex_prandtl(gpu_lib):
    """The paper's shock-vortex case at Pr = 0.75: one step at sampled vertices against the oracle,
    and 200 FP32 steps against the FP64 step."""
    from .test_gpu_fullsize import _fields, _gpu, _sample
    w = W.svi_pr()
    s = _gpu(w, 1, "f32")
    assert s.kernel_name == "mapped_fused"
    got, _ = _fields(s)
    verts = _sample(w)
    err = H.field_errors(tuple(a[verts] for a in got), H.oracle_step_at(w, verts), w.velocity_scale)
    assert max(err.values()) <= TOL_1, err
    a, ma = _fields(_gpu(w, 200, "f32"))
    b, mb = _fields(_gpu(w, 200, "f64"))
    err = H.field_errors(a, b, w.velocity_scale)
    assert max(err.values()) <= TOL_100, err
    assert abs(ma["mass"] / mb["mass"] - 1) < 1e-6


def test_adjoint_refuses_prandtl(gpu_lib):
    import torch
    from paper_1910_13918_gb300.sllbm import SLLBM, ERR_UNSUPPORTED
    w = _small("tgv16")
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    lam = torch.zeros((2, 25, s.ny, s.nx), dtype=torch.float32, device="cuda")
    out = torch.empty_like(lam)
    mom = torch.ones((4, s.ny, s.nx), dtype=torch.float32, device="cuda")
    st = s.lib.sllbm_adjoint_step(s.h, lam.data_ptr(), out.data_ptr(), mom.data_ptr())
    assert st == ERR_UNSUPPORTED
