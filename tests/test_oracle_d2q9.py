"""Pins of the oracle's D2Q9 velocity set (the comparison set of Sec. III.A), no GPU needed.

The paper runs the standard D2Q9 set with the same fourth-order equilibrium as D2Q25, isothermal
(theta = 1).  On the three D1Q3 nodes He_3 vanishes and He_4 equals -3 He_2, so the fourth-order
expansion aliases onto lower orders; the tests below check the moments that this aliasing gives
in closed form, worked out by hand from the D1Q3 rule, not by re-evaluating the oracle's tensor
contraction.
"""
import math

import numpy as np
import pytest

from oracle import sllbm as o


def test_d1q3_is_the_three_point_gauss_hermite_rule():
    """Nodes are the roots of He_3 and weights the Gauss-Hermite weights (numpy routine)."""
    xi, w = o.d1q3()
    nodes, weights = np.polynomial.hermite_e.hermegauss(3)
    weights = weights / math.sqrt(2 * math.pi)
    order = np.argsort(xi)
    np.testing.assert_allclose(xi[order], nodes, atol=1e-14)
    np.testing.assert_allclose(w[order], weights, atol=1e-14)
    assert xi[0] == 0.0 and xi[1] > 0 and xi[2] == -xi[1]


def test_d1q3_quadrature_order_five():
    """sum w xi^k equals the standard normal moments for k <= 5 and fails at k = 6 (9 != 15)."""
    xi, w = o.d1q3()
    for k, exact in enumerate([1, 0, 1, 0, 3, 0]):
        assert abs(np.sum(w * xi ** k) - exact) < 1e-14, k
    assert abs(np.sum(w * xi ** 6) - 9.0) < 1e-12


def test_d2q9_tensor_product():
    xi, w = o.d2q9()
    x1, w1 = o.d1q3()
    assert xi.shape == (9, 2)
    for a in range(3):
        for b in range(3):
            i = 3 * a + b
            assert xi[i, 0] == x1[a] and xi[i, 1] == x1[b] and w[i] == w1[a] * w1[b]
    assert abs(w.sum() - 1.0) < 1e-15


def _eq9(rng, n=6):
    rho = 0.5 + rng.random(n)
    u = 0.3 * rng.standard_normal((n, 2))
    return rho, u, o.equilibrium_f(rho, u, np.ones(n), q=9)


def test_d2q9_equilibrium_moments_in_closed_form():
    """At theta = 1 the fourth-order equilibrium on D2Q9 has
    sum f = rho, sum f xi = rho u, sum f xi_x xi_y = rho u_x u_y exactly;
    sum f xi_x^2 = rho (1 + u_x^2 - u_x^4 / 4): the u^4 term of H^(4) aliases onto the second moment
    (sum_a w_a xi_a^2 He_4(xi_a) / 4! = (9 - 18 + 3) / 24 = -1/4 on D1Q3);
    sum f xi_x^3 = 3 rho u_x: the Maxwellian's rho (u_x^3 + 3 u_x) loses its u^3 term, the
    third-order defect that breaks Galilean invariance (Sec. I, III.A)."""
    rng = np.random.default_rng(91)
    rho, u, feq = _eq9(rng)
    xi, _ = o.d2q9()
    mom = lambda wx, wy: np.einsum("i,i...->...", xi[:, 0] ** wx * xi[:, 1] ** wy, feq)
    ux, uy = u[:, 0], u[:, 1]
    np.testing.assert_allclose(mom(0, 0), rho, rtol=1e-14)
    np.testing.assert_allclose(mom(1, 0), rho * ux, atol=1e-14)
    np.testing.assert_allclose(mom(0, 1), rho * uy, atol=1e-14)
    np.testing.assert_allclose(mom(1, 1), rho * ux * uy, atol=1e-14)
    np.testing.assert_allclose(mom(2, 0), rho * (1 + ux ** 2 - ux ** 4 / 4), rtol=1e-13)
    np.testing.assert_allclose(mom(0, 2), rho * (1 + uy ** 2 - uy ** 4 / 4), rtol=1e-13)
    np.testing.assert_allclose(mom(3, 0), 3 * rho * ux, atol=1e-13)
    # the D2Q25 set keeps the third moment of the Maxwellian at theta = 1
    xi25, _ = o.d2q25()
    f25 = o.equilibrium_f(rho, u, np.ones(len(rho)))
    m3 = np.einsum("i,i...->...", xi25[:, 0] ** 3, f25)
    np.testing.assert_allclose(m3, rho * (ux ** 3 + 3 * ux), rtol=1e-12)


def test_d2q9_equilibrium_rest_state_is_the_weights():
    feq = o.equilibrium_f(np.array([1.0]), np.zeros((1, 2)), np.ones(1), q=9)
    _, w = o.d2q9()
    np.testing.assert_allclose(feq[:, 0], w, atol=1e-16)


def test_d2q9_isothermal_collision_conserves_mass_and_momentum():
    rng = np.random.default_rng(92)
    _, w = o.d2q9()
    f = w[:, None] * (1 + 0.1 * rng.standard_normal((9, 8)))
    g = np.zeros_like(f)
    f2, g2 = o.collide(f, g, 0.8, 1.0, isothermal=True)
    xi, _ = o.d2q9()
    for k in range(3):
        c = np.ones(9) if k == 0 else xi[:, k - 1]
        np.testing.assert_allclose(c @ f2, c @ f, atol=1e-14)
    assert np.max(np.abs(g2)) == 0.0
    # the result relaxes towards the D2Q9 equilibrium of the same moments
    rho, u, _ = o.macroscopic(f, g, 1.0)
    feq = o.equilibrium_f(rho, u, np.ones_like(rho), q=9)
    np.testing.assert_allclose(f2, f - (f - feq) / 0.8, atol=1e-15)


@pytest.mark.parametrize("p", [2, 4])
def test_d2q9_streaming_exact_shift_by_one_cell(p):
    """With dt sqrt(3) equal to one cell width, the moving D2Q9 planes shift by p vertices."""
    rng = np.random.default_rng(93 + p)
    ax = o.Axis(5, p, 0.0, 1.0, periodic=True)
    ay = o.Axis(4, p, 0.0, 0.8, periodic=True)
    grid = o.Grid(ax, ay)
    dt = ax.hc / math.sqrt(3.0)
    F = rng.standard_normal((9, grid.ny, grid.nx))
    out = o.stream(F, o.Departures(grid, dt, q=9))
    np.testing.assert_allclose(out[3 * 1 + 0], np.roll(F[3], p, axis=1), atol=1e-13)
    np.testing.assert_allclose(out[3 * 2 + 0], np.roll(F[6], -p, axis=1), atol=1e-13)
    np.testing.assert_allclose(out[0 * 3 + 1], np.roll(F[1], p, axis=0), atol=1e-13)
    np.testing.assert_allclose(out[3 * 1 + 2], np.roll(np.roll(F[5], p, axis=1), -p, axis=0),
                               atol=1e-13)
    np.testing.assert_allclose(out[0], F[0], atol=1e-15)


def test_d2q9_uniform_state_is_fixed_point():
    ax = o.Axis(3, 4, 0.0, 1.0, periodic=True)
    ay = o.Axis(2, 4, 0.0, 1.0, periodic=True)
    grid = o.Grid(ax, ay)
    shape = (grid.ny, grid.nx)
    f, g = o.initial_state(np.full(shape, 1.2), np.full(shape, 0.05), np.full(shape, -0.03),
                           np.ones(shape), 1.0, q=9)
    assert f.shape[0] == 9 and np.max(np.abs(g)) == 0.0
    f2, g2 = o.step(f, g, o.Departures(grid, 0.011, q=9), 0.7, 1.0, isothermal=True)
    np.testing.assert_allclose(f2, f, atol=1e-14)


def test_departures_and_field_must_share_the_velocity_set():
    ax = o.Axis(2, 2, 0.0, 1.0, periodic=True)
    grid = o.Grid(ax, ax)
    with pytest.raises(AssertionError):
        o.stream(np.zeros((25, grid.ny, grid.nx)), o.Departures(grid, 0.01, q=9))
