"""GPU <-> oracle parity of the forward step through the C ABI (needs a GB300).

Tolerances (per field, see helpers.field_errors): FP32 fused/gather steps <= 1e-5 after one step
and <= 1e-4 after 100 steps; the plain FP64 step <= 1e-11 (same arithmetic, different order);
BF16 storage is reported with a loose bound (8-bit mantissa of the stored deviations).
"""
import numpy as np
import pytest

from paper_1910_13918_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu

TOL_1 = 1e-5
TOL_100 = 1e-4
TOL_F64 = 1e-11


def gpu_run(w, nsteps, prec="f32", perturb=True):
    from paper_1910_13918_gb300.sllbm import SLLBM
    s = SLLBM.from_workload(w, prec=prec)
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=perturb))
    s.step(nsteps)
    m = s.moments()
    out = tuple(m[k].cpu().numpy() for k in ("rho", "u", "v", "T"))
    return s, out, m


@pytest.mark.parametrize("name", ["tgv16", "tgv256", "sod", "riemann", "svi"])
@pytest.mark.parametrize("nsteps,tol", [(1, TOL_1), (100, TOL_100)])
def test_forward_parity_small_f32(gpu_lib, name, nsteps, tol):
    w = H.small_workloads()[name]
    s, gpu, _ = gpu_run(w, nsteps, "f32")
    ref = H.oracle_run(w, nsteps)
    err = H.field_errors(gpu, ref, w.velocity_scale)
    assert max(err.values()) <= tol, (name, s.kernel_name, err)


@pytest.mark.parametrize("name", ["tgv16", "tgv256", "sod", "riemann", "svi"])
@pytest.mark.parametrize("nsteps", [1, 100])
def test_forward_parity_small_f64_state(gpu_lib, name, nsteps):
    """The plain FP64 step reproduces the oracle's populations element by element."""
    w = H.small_workloads()[name]
    s, _, _ = gpu_run(w, nsteps, "f64")
    st = s.get_state().cpu().numpy()
    f, g = H.oracle_state(w, nsteps)
    scale = np.max(np.abs(f))
    assert np.max(np.abs(st[0] - f)) <= TOL_F64 * scale, (name, np.max(np.abs(st[0] - f)))
    assert np.max(np.abs(st[1] - g)) <= TOL_F64 * scale, (name, np.max(np.abs(st[1] - g)))


@pytest.mark.parametrize("name", ["tgv16", "tgv256", "svi"])
def test_bf16_storage_error_reported(gpu_lib, name):
    w = H.small_workloads()[name]
    _, gpu, _ = gpu_run(w, 10, "bf16")
    err = H.field_errors(gpu, H.oracle_run(w, 10), w.velocity_scale)
    assert max(err.values()) < 2e-2, err


def test_vertex_coordinates_and_weights_match_oracle(gpu_lib):
    from paper_1910_13918_gb300.sllbm import SLLBM
    for w in H.small_workloads().values():
        s = SLLBM.from_workload(w)
        s.precompute()
        x, y = (t.cpu().numpy() for t in s.coords())
        grid = H.oracle_grid(w)
        X, Y = grid.coords()
        np.testing.assert_allclose(x, X, atol=1e-14)
        np.testing.assert_allclose(y, Y, atol=1e-14)
        np.testing.assert_allclose(s.vertex_weights().cpu().numpy(), grid.vertex_weights(),
                                   rtol=1e-12, atol=1e-15)


def test_mass_energy_sums_match_oracle(gpu_lib):
    from oracle import sllbm as o
    w = H.small_workloads()["svi"]
    s, _, m = gpu_run(w, 3, "f64")
    grid = H.oracle_grid(w)
    X, Y = grid.coords()
    f, g = o.initial_state(*w.fields(X, Y, perturb=True), w.cv)
    f, g = o.run(f, g, o.Departures(grid, w.dt), w.tau, w.cv, 3)
    M, E = o.mass_energy(f, g, grid.vertex_weights())
    assert abs(m["mass"] / M - 1) < 1e-12 and abs(m["energy"] / E - 1) < 1e-12


def test_uniform_state_fixed_point_f32(gpu_lib):
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = W.tgv256().resized(5, 4)
    s = SLLBM.from_workload(w)
    s.precompute()
    shape = (s.ny, s.nx)
    s.init(np.full(shape, 1.2), np.full(shape, 0.3), np.full(shape, -0.2), np.full(shape, 0.8))
    st0 = s.get_state().clone()
    s.step(5)
    st1 = s.get_state()
    assert float((st1 - st0).abs().max()) < 2e-6
