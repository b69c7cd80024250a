"""The 3D extension (D3Q125 on hexahedral cells, plain FP64 step) on the GPU against the 3D
oracle, through the C ABI: populations element by element after a few steps (<= 1e-11 of the
largest, as for the 2D FP64 step) on a periodic grid, a zero-gradient grid and the isothermal
single-population configuration; and the moments of the state.
"""
import numpy as np
import pytest

from oracle import sllbm as o
from oracle import sllbm3d as o3

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11

CASES = {
    # cells, p, box, periodic, dt, tau, cv, isothermal, steps
    "periodic_p2": ((2, 2, 2), 2, ((0.0, 1.0), (0.0, 0.8), (0.0, 0.6)), True, 0.01, 0.8, 2.5, False, 3),
    "clamped_p3": ((2, 1, 2), 3, ((0.0, 1.0), (0.0, 0.5), (0.0, 0.9)), False, 0.02, 0.7, 2.5, False, 2),
    "isothermal_p2": ((2, 2, 1), 2, ((0.0, 1.0), (0.0, 1.0), (0.0, 0.5)), True, 0.015, 0.9, 1.5, True, 3),
}

# Grids the sum-factorised FP32 step takes (tiles of 32 x 8 x 4 vertices; x vertex count even, at
# least 36 x 12 x 8): ragged tiles on every axis, periodic faces (regions reaching the periodic
# images in the ghost cells) and zero-gradient ones, orders 1 and 2, two populations and the
# isothermal single population.
TILED = {
    "tiled_periodic_p2": ((20, 7, 5), 2, ((0.0, 1.0), (0.0, 0.35), (0.0, 0.25)), True, 0.002, 0.8, 2.5, False, 3),
    "tiled_periodic_p1": ((38, 13, 9), 1, ((0.0, 1.0), (0.0, 0.35), (0.0, 0.25)), True, 0.003, 0.7, 2.5, False, 3),
    "tiled_clamped_p1": ((37, 12, 8), 1, ((0.0, 1.0), (0.0, 0.3), (0.0, 0.2)), False, 0.003, 0.9, 2.5, False, 3),
    "tiled_isothermal_p2": ((18, 6, 4), 2, ((0.0, 1.0), (0.0, 0.35), (0.0, 0.22)), True, 0.002, 0.9, 1.5, True, 3),
}


def _fields(X, Y, Z, box, seed):
    (x0, x1), (y0, y1), (z0, z1) = box
    sx, sy, sz = (2 * np.pi * (X - x0) / (x1 - x0), 2 * np.pi * (Y - y0) / (y1 - y0),
                  2 * np.pi * (Z - z0) / (z1 - z0))
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * np.sin(sx) * np.cos(sy) + 0.02 * np.cos(sz) + 1e-4 * rng.standard_normal(X.shape)
    u = 0.1 * np.sin(sy) + 1e-4 * rng.standard_normal(X.shape)
    v = 0.05 * np.cos(sz)
    w = 0.04 * np.sin(sx)
    T = 1 + 0.05 * np.cos(sx + sz)
    return rho, u, v, w, T


def _oracle(case):
    cells, p, box, periodic, dt, tau, cv, iso, steps = case
    axes = [o.Axis(n, p, lo, hi, periodic) for n, (lo, hi) in zip(cells, box)]
    grid = o3.Grid3(*axes)
    X, Y, Z = grid.coords()
    f, g = o3.initial_state(*_fields(X, Y, Z, box, 3), cv)
    return o3.run(f, g, o3.Departures3(grid, dt), tau, cv, steps, isothermal=iso)


def _gpu(case, prec="f64"):
    from paper_1910_13918_gb300.sllbm import SLLBM3D, BC_PERIODIC, BC_ZERO_GRADIENT
    cells, p, box, periodic, dt, tau, cv, iso, steps = case
    bc = (BC_PERIODIC if periodic else BC_ZERO_GRADIENT,) * 3
    s = SLLBM3D(cells=cells, order=p, box=box, bc=bc, dt=dt, tau=tau, cv=cv, isothermal=iso, prec=prec)
    s.precompute()
    X, Y, Z = (t.cpu().numpy() for t in s.coords())
    s.init(*_fields(X, Y, Z, box, 3))
    s.step(steps)
    return s


@pytest.mark.parametrize("name", list(CASES))
def test_3d_step_parity_f64(gpu_lib, name):
    case = CASES[name]
    s = _gpu(case)
    st = s.get_state().cpu().numpy()
    f, g = _oracle(case)
    assert st.shape == (s.npop, 125) + f.shape[1:]
    scale = np.max(np.abs(f))
    assert np.max(np.abs(st[0] - f)) <= TOL_F64 * scale, np.max(np.abs(st[0] - f))
    if s.npop == 2:
        assert np.max(np.abs(st[1] - g)) <= TOL_F64 * scale
    else:
        assert np.max(np.abs(g)) == 0.0
    m = s.moments()
    rho, u, th = o3.macroscopic(f, g, case[6])
    np.testing.assert_allclose(m["rho"].cpu().numpy(), rho, rtol=1e-12)
    np.testing.assert_allclose(m["u"].cpu().numpy(), u[..., 0], atol=1e-12)
    np.testing.assert_allclose(m["w"].cpu().numpy(), u[..., 2], atol=1e-12)
    np.testing.assert_allclose(m["T"].cpu().numpy(), th, rtol=1e-12)


def test_3d_state_round_trip(gpu_lib):
    s = _gpu(CASES["periodic_p2"])
    st = s.get_state()
    s.step(1)
    after = s.get_state()
    s.set_state(st)
    s.step(1)
    assert np.array_equal(s.get_state().cpu().numpy(), after.cpu().numpy())


@pytest.mark.parametrize("name", list(CASES) + list(TILED))
def test_3d_fused_f32_step_against_oracle(gpu_lib, name):
    """The FP32 steps (deviation pairs): the one-launch gather step on the small grids, the
    sum-factorised step on the TILED ones.  rho, u, v, w, T after the case's steps within the FP32
    tolerance of the 2D step (1e-5, velocities relative to the flow's scale), and populations to
    FP32 precision of the deviations (3e-5 of their largest value)."""
    case = {**CASES, **TILED}[name]
    s = _gpu(case, "f32")
    assert s.kernel_name == ("stream3d" if name in TILED else "gather_f32"), s.kernel_name
    f, g = _oracle(case)
    st = s.get_state().cpu().numpy()
    xi, w = o3.d3q125()
    scale = np.max(np.abs(f - w[:, None, None, None]))
    # the deviations f - w are stored in FP32: a few units of their last place
    assert np.max(np.abs(st[0] - f)) <= 3e-5 * scale, np.max(np.abs(st[0] - f)) / scale
    m = s.moments()
    rho, u, th = o3.macroscopic(f, g, case[6])
    umax = max(float(np.max(np.abs(u))), 1e-3)
    assert np.max(np.abs(m["rho"].cpu().numpy() / rho - 1)) < 1e-5
    assert np.max(np.abs(m["T"].cpu().numpy() / th - 1)) < 1e-5
    for k, name_ in enumerate(("u", "v", "w")):
        assert np.max(np.abs(m[name_].cpu().numpy() - u[..., k])) < 1e-5 * umax, name_


def test_3d_tiled_f32_tracks_f64_over_10_steps(gpu_lib):
    """The sum-factorised FP32 step against the plain FP64 step over 10 steps on the ragged
    periodic p = 2 grid: both populations within the multi-step FP32 tolerance (1e-4 of the
    largest deviation of each population; one step's rounding is a few 1e-6 of it)."""
    case = TILED["tiled_periodic_p2"][:-1] + (10,)
    s32, s64 = _gpu(case, "f32"), _gpu(case, "f64")
    assert s32.kernel_name == "stream3d" and s64.kernel_name == "plain_f64"
    a, b = s32.get_state().cpu().numpy(), s64.get_state().cpu().numpy()
    xi, w = o3.d3q125()
    K = 2 * case[6] - 3
    for pop, ref in ((0, w), (1, K * w)):
        scale = np.max(np.abs(b[pop] - ref[:, None, None, None]))
        err = np.max(np.abs(a[pop] - b[pop]))
        assert err <= 1e-4 * scale, (pop, err / scale)


def test_3d_fused_f32_keeps_mass_and_energy_of_f64(gpu_lib):
    """50 steps on the periodic case: the FP32 step's total mass and energy (sums of rho and
    rho E over the vertices) follow the FP64 step's to FP32 rounding -- the residual correction
    keeps the conserved moments of every collision -- while both carry the scheme's own small
    interpolation loss."""
    case = CASES["periodic_p2"]
    tot = {}
    for prec in ("f64", "f32"):
        s = _gpu(case, prec)
        s.step(50)
        st = s.get_state().cpu().numpy()
        g = st[1] if st.shape[0] == 2 else np.zeros_like(st[0])
        tot[prec] = (float(st[0].sum()), float(o3.total_energy_density(st[0], g).sum()))
    (m64, e64), (m32, e32) = tot["f64"], tot["f32"]
    assert abs(m32 / m64 - 1) < 1e-6 and abs(e32 / e64 - 1) < 1e-6, (m32 / m64 - 1, e32 / e64 - 1)
