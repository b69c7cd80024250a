"""Pins of the 3D oracle (D3Q125 on hexahedral cells), no GPU needed.

Each test checks the oracle against something other than itself: numpy / scipy routines, closed
forms, invariants, and the reduction of a z-uniform 3D flow to the (separately pinned) 2D oracle.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from oracle import sllbm as o
from oracle import sllbm3d as o3

CV = 2.5


def _random_macro(rng, n=4):
    rho = 0.5 + rng.random(n)
    u = 0.3 * rng.standard_normal((n, 3))
    theta = 0.7 + 0.6 * rng.random(n)
    return rho, u, theta


def test_d3q125_tensor_product_and_quadrature_order():
    """Mixed moments sum w xi_x^k xi_y^l xi_z^m equal the standard normal's for k, l, m <= 9
    (products of 1D moments) and the rule fails at order 10 in one axis (825 != 945)."""
    xi, w = o3.d3q125()
    x1, w1 = o.d1q5()
    assert xi.shape == (125, 3) and abs(w.sum() - 1.0) < 1e-14
    for a, b, c in itertools.product(range(5), repeat=3):
        i = 25 * a + 5 * b + c
        assert tuple(xi[i]) == (x1[a], x1[b], x1[c]) and w[i] == w1[a] * w1[b] * w1[c]
    normal = lambda k: 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0
    for k, l, m in itertools.product(range(0, 10, 3), range(0, 10, 2), range(10)):
        terms = w * xi[:, 0] ** k * xi[:, 1] ** l * xi[:, 2] ** m
        assert abs(terms.sum() - normal(k) * normal(l) * normal(m)) < 1e-13 * np.abs(terms).sum()
    assert abs(np.sum(w * xi[:, 2] ** 10) - 825.0) < 1e-8


def test_equilibrium_reproduces_maxwellian_moments_3d():
    """Moments of total order <= 4 of f^eq equal those of rho N(u, theta I) in 3D, whose raw
    moments come from scipy.stats.norm per axis."""
    rng = np.random.default_rng(31)
    rho, u, theta = _random_macro(rng)
    feq = o3.equilibrium_f(rho, u, theta)
    xi, _ = o3.d3q125()
    for v in range(len(rho)):
        sd = math.sqrt(theta[v])
        mom = lambda ax, k: stats.norm(loc=u[v, ax], scale=sd).moment(k) if k else 1.0
        for k, l, m in itertools.product(range(5), repeat=3):
            if k + l + m > 4:
                continue
            disc = np.sum(feq[:, v] * xi[:, 0] ** k * xi[:, 1] ** l * xi[:, 2] ** m)
            ref = rho[v] * mom(0, k) * mom(1, l) * mom(2, m)
            assert abs(disc - ref) < 1e-12 * max(1.0, abs(ref)), (k, l, m)


def test_macroscopic_and_collision_invariants_3d():
    rng = np.random.default_rng(32)
    rho, u, theta = _random_macro(rng)
    f, g = o3.initial_state(rho, u[:, 0], u[:, 1], u[:, 2], theta, CV)
    r2, u2, t2 = o3.macroscopic(f, g, CV)
    np.testing.assert_allclose(r2, rho, atol=1e-13)
    np.testing.assert_allclose(u2, u, atol=1e-13)
    np.testing.assert_allclose(t2, theta, atol=1e-13)
    np.testing.assert_allclose(g.sum(0), (2 * CV - 3) * rho * theta, atol=1e-13)   # internal dof
    fp = f * (1 + 0.05 * rng.standard_normal(f.shape))
    gp = g * (1 + 0.05 * rng.standard_normal(g.shape))
    fs, gs = o3.collide(fp, gp, 0.8, CV)
    xi, _ = o3.d3q125()
    np.testing.assert_allclose(fs.sum(0), fp.sum(0), atol=1e-13)
    for k in range(3):
        np.testing.assert_allclose(xi[:, k] @ fs, xi[:, k] @ fp, atol=1e-13)
    np.testing.assert_allclose(o3.total_energy_density(fs, gs), o3.total_energy_density(fp, gp), atol=1e-13)


def _grid(p, periodic, cells=(2, 2, 2), box=((0.0, 1.0), (0.0, 0.8), (0.0, 0.6))):
    axes = [o.Axis(n, p, lo, hi, periodic) for n, (lo, hi) in zip(cells, box)]
    return o3.Grid3(*axes)


@pytest.mark.parametrize("p", [2, 3])
def test_streaming_exact_for_tensor_polynomials_3d(p):
    """On clamped axes the interpolant of a polynomial of degree <= p per axis is exact at every
    (clamped) departure point."""
    rng = np.random.default_rng(40 + p)
    grid = _grid(p, periodic=False)
    X, Y, Z = grid.coords()
    cx, cy, cz = rng.standard_normal((3, p + 1))
    field = lambda x, y, z: (np.polyval(cx, x) * np.polyval(cy, y) * np.polyval(cz, z))
    F = np.broadcast_to(field(X, Y, Z), (125,) + X.shape).copy()
    dt = 0.031
    out = o3.stream(F, o3.Departures3(grid, dt))
    xi, _ = o3.d3q125()
    for i in range(0, 125, 7):
        xd = np.clip(X - dt * xi[i, 0], 0.0, 1.0)
        yd = np.clip(Y - dt * xi[i, 1], 0.0, 0.8)
        zd = np.clip(Z - dt * xi[i, 2], 0.0, 0.6)
        np.testing.assert_allclose(out[i], field(xd, yd, zd), atol=1e-12)


def test_streaming_exact_shift_by_one_cell_3d():
    """With dt xi_1 = one cell width (all axes share it), the velocity (xi_1, 0, -xi_1) moves the
    field by p vertices in x and -p in z."""
    p = 2
    rng = np.random.default_rng(50)
    grid = _grid(p, periodic=True, cells=(3, 2, 2), box=((0.0, 0.6), (0.0, 0.4), (0.0, 0.4)))
    x1, _ = o.d1q5()
    dt = grid.ax.hc / x1[1]
    F = rng.standard_normal((125, grid.nz, grid.ny, grid.nx))
    out = o3.stream(F, o3.Departures3(grid, dt))
    i = 25 * 1 + 5 * 0 + 3                      # (+small, 0, -small)
    np.testing.assert_allclose(out[i], np.roll(np.roll(F[i], p, axis=2), -p, axis=0), atol=1e-13)
    np.testing.assert_allclose(out[0], F[0], atol=1e-15)


def test_uniform_state_is_fixed_point_3d():
    grid = _grid(2, periodic=True)
    shape = (grid.nz, grid.ny, grid.nx)
    f, g = o3.initial_state(np.full(shape, 1.1), np.full(shape, 0.1), np.full(shape, -0.05),
                            np.full(shape, 0.07), np.full(shape, 0.95), CV)
    f2, g2 = o3.step(f, g, o3.Departures3(grid, 0.017), 0.9, CV)
    np.testing.assert_allclose(f2, f, atol=1e-14)
    np.testing.assert_allclose(g2, g, atol=1e-14)


def test_equilibrium_summed_over_z_is_the_2d_equilibrium():
    """With u_z = 0 the 3D equilibrium summed over the z component is the 2D one at the same
    (rho, u, theta): sum_c w_c He_m(xi_c) = 0 for 1 <= m <= 8 removes every term with a z index."""
    rng = np.random.default_rng(61)
    rho, u, theta = _random_macro(rng, 6)
    u[:, 2] = 0.0
    f3 = o3.equilibrium_f(rho, u, theta).reshape(25, 5, -1).sum(axis=1)
    f2 = o.equilibrium_f(rho, u[:, :2], theta)
    np.testing.assert_allclose(f3, f2, atol=1e-15)


def test_z_uniform_isothermal_flow_reduces_to_the_2d_oracle():
    """An isothermal flow (theta = 1 in the equilibrium, one population) that does not depend on
    z and has u_z = 0 evolves in 3D as in 2D: streaming moves no value along z, and the summed
    equilibrium is the 2D one (previous test), so the 3D populations summed over the z component
    follow the 2D step exactly; (rho, u) agree at every z.  (With the thermal model the two
    differ at the truncation order: the z part of the 3D energy is carried by f's fourth-order
    expansion, the 2D one by g = (2 C_v - 2) theta f^eq.)"""
    p, tau, dt, nsteps = 2, 0.8, 0.02, 3
    ax = o.Axis(3, p, 0.0, 1.0, True)
    ay = o.Axis(2, p, 0.0, 0.7, True)
    az = o.Axis(2, p, 0.0, 0.5, True)
    g3 = o3.Grid3(ax, ay, az)
    g2 = o.Grid(ax, ay)
    X, Y = g2.coords()
    rng = np.random.default_rng(60)
    rho = 1 + 0.05 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y / 0.7) + 0.01 * rng.random(X.shape)
    u = 0.1 * np.cos(2 * np.pi * Y / 0.7)
    v = 0.05 * np.sin(2 * np.pi * X)
    T = np.ones_like(X)
    f2, gg2 = o.initial_state(rho, u, v, T, 1.0)
    f2, gg2 = o.run(f2, gg2, o.Departures(g2, dt), tau, 1.0, nsteps, isothermal=True)
    r2, u2, _ = o.macroscopic(f2, gg2, 1.0)
    ext = lambda A: np.broadcast_to(A, (g3.nz,) + A.shape)
    f3, gg3 = o3.initial_state(ext(rho), ext(u), ext(v), ext(np.zeros_like(u)), ext(T), 1.5)
    f3, gg3 = o3.run(f3, gg3, o3.Departures3(g3, dt), tau, 1.5, nsteps, isothermal=True)
    assert np.max(np.abs(gg3)) == 0.0          # C_v = D/2: no second population
    np.testing.assert_allclose(f3.reshape(25, 5, *f3.shape[1:]).sum(axis=1),
                               np.broadcast_to(f2[:, None], (25, g3.nz) + f2.shape[1:]), atol=1e-14)
    r3, u3, _ = o3.macroscopic(f3, gg3, 1.5)
    for iz in range(g3.nz):
        np.testing.assert_allclose(r3[iz], r2, rtol=1e-13)
        np.testing.assert_allclose(u3[iz, ..., :2], u2, atol=1e-13)
        assert np.max(np.abs(u3[iz, ..., 2])) < 1e-14
