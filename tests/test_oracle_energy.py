"""Pin of the oracle's energy diagnostic against the closed form of the total energy.

The total energy density is fixed by the moments of Sec. II (2 rho E = sum f |xi|^2 + sum g) and
the equilibria of Sec. II.A/II.D: sum f^eq |xi|^2 = rho (|u|^2 + D theta) and
sum g^eq = (2 C_v - D) rho theta, so at equilibrium rho E = rho (C_v theta + |u|^2 / 2) with
T0 = R = 1 -- the internal energy C_v T plus the kinetic energy of an ideal gas.  The tests build
equilibrium states from random (rho, u, theta) and compare the oracle's ``total_energy_density``
and ``mass_energy`` with that expression, written from the thermodynamics and not from the
oracle's moment sums; a dropped 1/2, a missing g term or a wrong |xi|^2 fails them.
"""
import numpy as np
import pytest

from oracle import sllbm as o
from oracle import sllbm3d as o3


def _rhoE(rho, u, theta, cv):
    return rho * (cv * theta + 0.5 * np.sum(u * u, axis=-1))


@pytest.mark.parametrize("cv", [2.5, 1.7])
def test_total_energy_density_2d_equilibrium(cv):
    rng = np.random.default_rng(11)
    n = 9
    rho = 0.3 + 1.5 * rng.random(n)
    u = 0.5 * rng.standard_normal((n, 2))
    theta = 0.5 + rng.random(n)
    f = o.equilibrium_f(rho, u, theta)
    g = o.equilibrium_g(rho, u, theta, cv)
    np.testing.assert_allclose(o.total_energy_density(f, g), _rhoE(rho, u, theta, cv), rtol=1e-13)


def test_total_energy_density_3d_equilibrium():
    rng = np.random.default_rng(12)
    n = 5
    cv = 2.5
    rho = 0.3 + 1.5 * rng.random(n)
    u = 0.4 * rng.standard_normal((n, 3))
    theta = 0.5 + rng.random(n)
    f, g = o3.initial_state(rho, u[:, 0], u[:, 1], u[:, 2], theta, cv)
    np.testing.assert_allclose(o3.total_energy_density(f, g), _rhoE(rho, u, theta, cv), rtol=1e-13)


def test_mass_energy_is_the_weighted_sum_of_the_closed_form():
    """M = sum_v A_v rho_v and E = sum_v A_v rho_v (C_v theta_v + |u_v|^2 / 2) on a small grid with
    random equilibrium fields; the vertex weights A_v are the oracle's (pinned separately against
    Newton-Cotes closed forms), the energy per vertex is the thermodynamic expression."""
    rng = np.random.default_rng(13)
    cv = 2.5
    grid = o.Grid(o.Axis(3, 2, 0.0, 1.0, False), o.Axis(2, 2, 0.0, 1.0, True))
    shape = (grid.ny, grid.nx)
    rho = 0.5 + rng.random(shape)
    u = 0.3 * rng.standard_normal(shape + (2,))
    theta = 0.7 + 0.5 * rng.random(shape)
    f = o.equilibrium_f(rho, u, theta)
    g = o.equilibrium_g(rho, u, theta, cv)
    A = grid.vertex_weights()
    M, E = o.mass_energy(f, g, A)
    assert abs(M - float(np.sum(A * rho))) <= 1e-13 * abs(M)
    assert abs(E - float(np.sum(A * _rhoE(rho, u, theta, cv)))) <= 1e-13 * abs(E)
    # and the domain area is what the weights integrate (a constant field)
    assert abs(float(np.sum(A)) - 1.0) < 1e-13
