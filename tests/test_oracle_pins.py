"""Pins of the FP64 oracle against what the paper and mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: a library routine, a closed
form, an invariant, or a textbook/printed value.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import sllbm as o

CV = 2.5


def _random_macro(rng, n=7):
    rho = 0.5 + rng.random(n)
    u = 0.4 * rng.standard_normal((n, 2))
    theta = 0.6 + 0.8 * rng.random(n)
    return rho, u, theta


# --- velocity set (Sec. II.B, Table I) -------------------------------------------------------
def test_d1q5_are_fifth_order_gauss_hermite_nodes():
    """Abscissae are the roots of He_5 and weights the Gauss-Hermite weights (numpy routine)."""
    xi, w = o.d1q5()
    nodes, weights = np.polynomial.hermite_e.hermegauss(5)
    weights = weights / math.sqrt(2 * math.pi)
    order = np.argsort(xi)
    np.testing.assert_allclose(xi[order], nodes, atol=1e-14)
    np.testing.assert_allclose(w[order], weights, atol=1e-14)
    # Table I pairing: index 1/3 the small pair, 2/4 the large pair, +- in that order
    assert xi[1] > 0 and xi[3] == -xi[1] and xi[2] > xi[1] and xi[4] == -xi[2]
    assert abs(w[0] - 8 / 15) < 1e-15


def test_quadrature_order_nine():
    """sum w xi^k equals the standard normal moments for k <= 9 and fails at k = 10 (Q = 9)."""
    xi, w = o.d1q5()
    for k in range(10):
        exact = 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0
        assert abs(np.sum(w * xi ** k) - exact) < 1e-12, k
    assert abs(np.sum(w * xi ** 10) - 825.0) < 1e-9   # != 945 = 9!!


def test_d2q25_tensor_product():
    xi, w = o.d2q25()
    x1, w1 = o.d1q5()
    assert xi.shape == (25, 2)
    for a in range(5):
        for b in range(5):
            i = 5 * a + b
            assert xi[i, 0] == x1[a] and xi[i, 1] == x1[b] and w[i] == w1[a] * w1[b]


# --- equilibrium (Sec. II.A) -----------------------------------------------------------------
def test_equilibrium_reproduces_maxwellian_moments():
    """Moments of total order <= 4 of f^eq equal those of the Maxwell-Boltzmann distribution.

    The Maxwellian rho N(u, theta I) factorises over axes; its raw moments come from
    scipy.stats.norm, independently of the Hermite tensors and coefficients of the oracle.
    A dropped term or wrong sign in a_eq^(n) or H^(n) changes one of these moments.
    """
    rng = np.random.default_rng(1)
    rho, u, theta = _random_macro(rng)
    feq = o.equilibrium_f(rho, u, theta)
    xi, _ = o.d2q25()
    for v in range(len(rho)):
        sd = math.sqrt(theta[v])
        for k in range(5):
            for l in range(5 - k):
                disc = np.sum(feq[:, v] * xi[:, 0] ** k * xi[:, 1] ** l)
                mx = stats.norm(loc=u[v, 0], scale=sd).moment(k) if k else 1.0
                my = stats.norm(loc=u[v, 1], scale=sd).moment(l) if l else 1.0
                assert abs(disc - rho[v] * mx * my) < 1e-12 * max(1.0, abs(rho[v] * mx * my)), (k, l)


def test_hermite_projection_recovers_coefficients():
    """sum_i f_i^eq H^(n)(xi_i) = a_eq^(n) for n <= 4 (Eq. discrete)."""
    import itertools
    rng = np.random.default_rng(2)
    rho, u, theta = _random_macro(rng)
    feq = o.equilibrium_f(rho, u, theta)
    xi, _ = o.d2q25()
    for n in range(5):
        for idx in itertools.product(range(2), repeat=n):
            proj = np.sum(feq * o.hermite(n, idx, xi)[:, None], axis=0)
            np.testing.assert_allclose(proj, o.a_eq(n, idx, rho, u, theta), atol=1e-12)


def test_macroscopic_recovers_equilibrium_state():
    """(rho, u, theta) of (f^eq, g^eq) are the ones it was built from (reading of T)."""
    rng = np.random.default_rng(3)
    rho, u, theta = _random_macro(rng)
    f = o.equilibrium_f(rho, u, theta)
    g = o.equilibrium_g(rho, u, theta, CV)
    r2, u2, t2 = o.macroscopic(f, g, CV)
    np.testing.assert_allclose(r2, rho, atol=1e-13)
    np.testing.assert_allclose(u2, u, atol=1e-13)
    np.testing.assert_allclose(t2, theta, atol=1e-13)
    # internal energy of g: sum g^eq = (2 C_v - D) rho theta
    np.testing.assert_allclose(g.sum(axis=0), (2 * CV - 2) * rho * theta, atol=1e-13)


def test_collision_conserves_mass_momentum_energy():
    rng = np.random.default_rng(4)
    rho, u, theta = _random_macro(rng)
    f = o.equilibrium_f(rho, u, theta) * (1 + 0.05 * rng.standard_normal((25, len(rho))))
    g = o.equilibrium_g(rho, u, theta, CV) * (1 + 0.05 * rng.standard_normal((25, len(rho))))
    fs, gs = o.collide(f, g, 0.77, CV)
    xi, _ = o.d2q25()
    for a, b in ((f, fs), (f * xi[:, :1], fs * xi[:, :1]), (f * xi[:, 1:], fs * xi[:, 1:])):
        np.testing.assert_allclose(a.sum(0), b.sum(0), atol=1e-13)
    np.testing.assert_allclose(o.total_energy_density(f, g), o.total_energy_density(fs, gs),
                               atol=1e-13)
    # tau = 1 lands exactly on the equilibrium of the conserved moments
    f1, g1 = o.collide(f, g, 1.0, CV)
    r, uu, th = o.macroscopic(f, g, CV)
    np.testing.assert_allclose(f1, o.equilibrium_f(r, uu, th), atol=1e-14)


# --- space discretisation (Sec. II.E) --------------------------------------------------------
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_glc_nodes_are_chebyshev_extrema(p):
    ref = np.sort(0.5 * (1 + np.polynomial.chebyshev.chebpts2(p + 1)))
    np.testing.assert_allclose(o.glc_nodes(p), ref, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_interpolation_exact_for_degree_p(p):
    rng = np.random.default_rng(p)
    nodes = o.glc_nodes(p)
    coef = rng.standard_normal(p + 1)
    r = rng.random(50)
    psi = o.lagrange(nodes, r)
    np.testing.assert_allclose(psi.sum(-1), 1.0, atol=1e-14)
    np.testing.assert_allclose(psi @ np.polyval(coef, nodes), np.polyval(coef, r), atol=1e-13)
    np.testing.assert_allclose(o.lagrange(nodes, nodes), np.eye(p + 1), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_streaming_exact_for_tensor_polynomials(p):
    """Pull streaming on zero-gradient axes reproduces any Q_p field at the clamped departure.

    Pins the departure sign (x - dt xi), the cell search, the clamp and the tensor weights.
    """
    rng = np.random.default_rng(10 + p)
    ax = o.Axis(3, p, -1.0, 2.0, periodic=False)
    ay = o.Axis(2, p, 0.0, 1.5, periodic=False)
    grid = o.Grid(ax, ay)
    X, Y = grid.coords()
    cxp, cyp = rng.standard_normal(p + 1), rng.standard_normal(p + 1)
    field = lambda x, y: np.polyval(cxp, x) * np.polyval(cyp, y)
    F = np.stack([field(X, Y)] * 25)
    dt = 0.07
    dep = o.Departures(grid, dt)
    out = o.stream(F, dep)
    xi, _ = o.d2q25()
    for i in range(25):
        xd = np.clip(X - dt * xi[i, 0], -1.0, 2.0)
        yd = np.clip(Y - dt * xi[i, 1], 0.0, 1.5)
        np.testing.assert_allclose(out[i], field(xd, yd), atol=1e-11)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_streaming_exact_shift_by_one_cell(p):
    """With dt xi_a equal to one cell width, streaming is the cyclic shift by p vertices."""
    rng = np.random.default_rng(20 + p)
    ax = o.Axis(5, p, 0.0, 1.0, periodic=True)
    ay = o.Axis(4, p, 0.0, 0.8, periodic=True)         # same cell width as x
    grid = o.Grid(ax, ay)
    x1, _ = o.d1q5()
    dt = ax.hc / x1[1]                      # xi_1 dt = one cell in x
    F = rng.standard_normal((25, grid.ny, grid.nx))
    out = o.stream(F, o.Departures(grid, dt))
    np.testing.assert_allclose(out[5 * 1 + 0], np.roll(F[5], p, axis=1), atol=1e-13)
    np.testing.assert_allclose(out[5 * 3 + 0], np.roll(F[15], -p, axis=1), atol=1e-13)
    np.testing.assert_allclose(out[0 * 5 + 1], np.roll(F[1], p, axis=0), atol=1e-13)
    np.testing.assert_allclose(out[0], F[0], atol=1e-15)      # rest velocity does not move


def test_streaming_exact_shift_by_one_vertex_equidistant():
    """For equidistant p = 2 nodes, dt xi = one vertex spacing shifts by one vertex."""
    rng = np.random.default_rng(5)
    ax = o.Axis(6, 2, 0.0, 3.0, periodic=True, nodes="equidistant")
    ay = o.Axis(3, 2, 0.0, 1.0, periodic=True, nodes="equidistant")
    grid = o.Grid(ax, ay)
    x1, _ = o.d1q5()
    dt = (ax.hc / 2) / x1[2]
    F = rng.standard_normal((25, grid.ny, grid.nx))
    out = o.stream(F, o.Departures(grid, dt))
    np.testing.assert_allclose(out[5 * 2], np.roll(F[10], 1, axis=1), atol=1e-13)


def test_uniform_state_is_fixed_point():
    rng = np.random.default_rng(6)
    ax = o.Axis(3, 3, 0.0, 1.0, periodic=True)
    ay = o.Axis(2, 3, 0.0, 1.0, periodic=True)
    grid = o.Grid(ax, ay)
    shape = (grid.ny, grid.nx)
    f, g = o.initial_state(np.full(shape, 1.3), np.full(shape, 0.2), np.full(shape, -0.1),
                           np.full(shape, 0.9), CV)
    f2, g2 = o.step(f, g, o.Departures(grid, 0.013), 0.8, CV)
    np.testing.assert_allclose(f2, f, atol=1e-14)
    np.testing.assert_allclose(g2, g, atol=1e-14)


@pytest.mark.parametrize("p,expect", [(2, [1 / 6, 2 / 3, 1 / 6]), (1, [0.5, 0.5])])
def test_vertex_weights_closed_form(p, expect):
    """A_v of one cell on [0,1] are the Newton-Cotes weights of its nodes (Simpson for p = 2)."""
    ax = o.Axis(1, p, 0.0, 1.0, periodic=False)
    ay = o.Axis(1, p, 0.0, 1.0, periodic=False)
    A = o.Grid(ax, ay).vertex_weights()
    np.testing.assert_allclose(A, np.outer(expect, expect), atol=1e-15)


def test_sine_map_inverse_and_area():
    m = o.SineMap(0.05)
    rng = np.random.default_rng(7)
    x = 2 * rng.random(200)
    y = rng.random(200)
    xi, eta = m.inverse(x, y)
    fx, fy = m(xi, eta)
    np.testing.assert_allclose(fx, x, atol=1e-13)
    np.testing.assert_allclose(fy, y, atol=1e-13)
    # the map fixes the boundary of [0,2]x[0,1]
    s = np.linspace(0, 1, 11)
    np.testing.assert_allclose(m(np.zeros_like(s), s)[0], 0, atol=1e-15)
    np.testing.assert_allclose(m(2 * np.ones_like(s), s)[0], 2, atol=1e-14)
    np.testing.assert_allclose(m(2 * s, np.ones_like(s))[1], 1, atol=1e-14)
    # integral of |det J| over the reference box is the physical area 2
    grid = o.Grid(o.Axis(6, 2, 0, 2, False), o.Axis(3, 2, 0, 1, True), m)
    assert abs(grid.vertex_weights().sum() - 2.0) < 1e-12


def test_mapped_streaming_identity_map_equals_uniform():
    rng = np.random.default_rng(8)
    ax = o.Axis(4, 2, 0, 2, False)
    ay = o.Axis(3, 2, 0, 1, True)
    F = rng.standard_normal((25, ay.nv, ax.nv))
    a = o.stream(F, o.Departures(o.Grid(ax, ay), 0.03))
    b = o.stream(F, o.Departures(o.Grid(ax, ay, o.SineMap(0.0)), 0.03))
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_mapped_streaming_exact_for_reference_polynomials():
    """On the mapped grid, a Q_p field in reference coordinates is interpolated exactly."""
    rng = np.random.default_rng(9)
    m = o.SineMap(0.05)
    grid = o.Grid(o.Axis(5, 2, 0, 2, False), o.Axis(4, 2, 0, 1, False), m)
    RX, RY = grid.reference_coords()
    c1, c2 = rng.standard_normal(3), rng.standard_normal(3)
    field = lambda a, b: np.polyval(c1, a) * np.polyval(c2, b)
    F = np.stack([field(RX, RY)] * 25)
    dt = 0.02
    out = o.stream(F, o.Departures(grid, dt))
    X, Y = grid.coords()
    xi, _ = o.d2q25()
    for i in (0, 7, 13, 24):
        ex, ey = m.inverse(np.clip(X - dt * xi[i, 0], 0, 2), np.clip(Y - dt * xi[i, 1], 0, 1))
        np.testing.assert_allclose(out[i], field(ex, ey), atol=1e-11)
