"""Pins of the oracle's variable-Prandtl and isothermal collisions (Sec. II.C, Sec. III.A).

The quasi-equilibrium exists to relax the heat flux with its own time tau_Pr = (tau - 1/2)/Pr +
1/2 while everything else keeps tau.  Written out, for a collision at one vertex (u is unchanged,
since the collision conserves momentum):
* mass, momentum and total energy are conserved;
* the non-equilibrium stress sum (f - f^eq) xi xi relaxes by 1 - 1/tau;
* the non-equilibrium centred third moment of f, and that of g, relax by 1 - 1/tau_Pr;
* Pr = 1 is plain BGK.
A dropped or extra normalisation of f* (the printed formula has no 1/3!), a wrong sign or a
wrong Hermite tensor breaks the third-moment relaxation.
"""
import numpy as np
import pytest

from oracle import sllbm as o


def _state(seed, n=7):
    """Random near-equilibrium (f, g) on n vertices: equilibrium plus 5 % random deviations."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.3 * rng.random(n)
    u = 0.4 * (rng.random((n, 2)) - 0.5)
    theta = 0.8 + 0.4 * rng.random(n)
    feq = o.equilibrium_f(rho, u, theta)
    cv = 2.5
    geq = (2 * cv - o.D) * theta * feq
    f = feq * (1.0 + 0.05 * rng.standard_normal(feq.shape))
    g = geq * (1.0 + 0.05 * rng.standard_normal(geq.shape))
    return f, g, cv


def _moments(f, g, cv):
    xi, _ = o.d2q25()
    rho = f.sum(0)
    j = np.einsum("in,ik->nk", f, xi)
    e = np.einsum("in,i->n", f, (xi ** 2).sum(1)) + g.sum(0)
    return rho, j, e


@pytest.mark.parametrize("pr", [0.5, 0.75, 2.0])
def test_conserves_mass_momentum_energy(pr):
    f, g, cv = _state(1)
    fn, gn = o.collide(f, g, 0.9, cv, pr)
    for a, b in zip(_moments(f, g, cv), _moments(fn, gn, cv)):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13)


@pytest.mark.parametrize("pr", [0.5, 0.75, 2.0])
def test_stress_relaxes_with_tau_and_heat_flux_with_tau_pr(pr):
    tau = 0.9
    f, g, cv = _state(2)
    rho, u, theta = o.macroscopic(f, g, cv)
    feq = o.equilibrium_f(rho, u, theta)
    geq = (2 * cv - o.D) * theta * feq
    fn, gn = o.collide(f, g, tau, cv, pr)
    xi, _ = o.d2q25()
    stress = lambda F: np.einsum("in,ia,ib->abn", F, xi, xi)
    np.testing.assert_allclose(stress(fn - feq), (1 - 1 / tau) * stress(f - feq), rtol=0, atol=1e-13)
    keep = 1.0 - 1.0 / o.tau_prandtl(tau, pr)
    for new, old, eq in ((fn, f, feq), (gn, g, geq)):
        q_new = o.centered_third_moment(new, u) - o.centered_third_moment(eq, u)
        q_old = o.centered_third_moment(old, u) - o.centered_third_moment(eq, u)
        assert np.max(np.abs(q_old)) > 1e-3            # the test state carries a heat flux
        np.testing.assert_allclose(q_new, keep * q_old, rtol=0, atol=1e-12)


def test_prandtl_one_is_bgk():
    f, g, cv = _state(3)
    fa, ga = o.collide(f, g, 0.9, cv, 1.0)
    rho, u, theta = o.macroscopic(f, g, cv)
    feq = o.equilibrium_f(rho, u, theta)
    geq = (2 * cv - o.D) * theta * feq
    np.testing.assert_allclose(fa, f - (f - feq) / 0.9, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ga, g - (g - geq) / 0.9, rtol=0, atol=1e-15)


def test_equilibrium_has_no_centred_heat_flux():
    """The fourth-order equilibrium reproduces the Maxwellian's moments up to third order, whose
    centred third moment is zero: f^qe of an equilibrium state is zero."""
    rng = np.random.default_rng(4)
    rho = 1.0 + rng.random(5)
    u = 0.5 * (rng.random((5, 2)) - 0.5)
    theta = 0.7 + 0.6 * rng.random(5)
    feq = o.equilibrium_f(rho, u, theta)
    assert np.max(np.abs(o.centered_third_moment(feq, u))) < 1e-14


def test_isothermal_collision_relaxes_kinetic_temperature_to_one():
    """The isothermal configuration (Sec. III.A, one population, C_v = 1): the equilibrium is
    taken at theta = 1, so mass and momentum are kept while the kinetic temperature
    (sum f |xi|^2 - rho |u|^2) / (2 rho) relaxes toward 1 by 1 - 1/tau."""
    f, _, _ = _state(5)
    g = np.zeros_like(f)
    tau = 0.8
    rho, u, theta = o.macroscopic(f, g, 1.0)
    fn, gn = o.collide(f, g, tau, 1.0, isothermal=True)
    rho2, u2, theta2 = o.macroscopic(fn, gn, 1.0)
    np.testing.assert_allclose(rho2, rho, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u2, u, rtol=0, atol=1e-14)
    assert np.max(np.abs(theta - 1.0)) > 1e-2
    np.testing.assert_allclose(theta2 - 1.0, (1 - 1 / tau) * (theta - 1.0), rtol=0, atol=1e-13)
    assert np.max(np.abs(gn)) == 0.0
