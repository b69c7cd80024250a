"""Pins of the oracle's reference adjoint: dot-product identity, conservation and finite differences."""
import numpy as np

from oracle import adjoint as oa
from oracle import sllbm as o
from paper_1910_13918_gb300 import workloads as W


def _small_svi(dt=0.05):
    w = W.svi()
    grid = o.Grid(o.Axis(8, 2, 0, 2, False), o.Axis(4, 2, 0, 1, True), o.SineMap(0.05))
    X, Y = grid.coords()
    return w, grid, X, Y, o.Departures(grid, dt)


def test_adjoint_step_dot_product_identity():
    """<lambda, S'(s) ds> = <S'(s)^T lambda, ds>, S' taken by complex step of the forward step."""
    w, grid, X, Y, dep = _small_svi()
    rng = np.random.default_rng(1)
    f, g = o.initial_state(*w.fields(X, Y), w.cv)
    f = f * (1 + 0.01 * rng.standard_normal(f.shape))
    df, dg = rng.standard_normal(f.shape), rng.standard_normal(g.shape)
    lf, lg = rng.standard_normal(f.shape), rng.standard_normal(g.shape)
    fc, gc = o.step(f + 1e-30j * df, g + 1e-30j * dg, dep, 0.8, w.cv)
    jvp = np.sum(fc.imag / 1e-30 * lf) + np.sum(gc.imag / 1e-30 * lg)
    mf, mg = oa.adjoint_step(f, g, lf, lg, dep, 0.8, w.cv)
    vjp = np.sum(mf * df) + np.sum(mg * dg)
    assert abs(jvp - vjp) < 1e-12 * abs(jvp)


def test_collision_adjoint_preserves_moment_directions():
    """BGK conserves (rho, rho u, rho E), so J_C^T maps the moment covectors to themselves."""
    rng = np.random.default_rng(2)
    xi, _ = o.d2q25()
    n = 5
    rho = 1 + 0.1 * rng.random(n)
    u = 0.3 * rng.standard_normal((n, 2))
    th = 1 + 0.1 * rng.random(n)
    f = o.equilibrium_f(rho, u, th) * (1 + 0.03 * rng.standard_normal((25, n)))
    g = o.equilibrium_g(rho, u, th, 2.5) * (1 + 0.03 * rng.standard_normal((25, n)))
    e2 = (xi ** 2).sum(1)
    for lf, lg in ((np.ones((25, n)), np.zeros((25, n))),
                   (np.repeat(xi[:, :1], n, 1), np.zeros((25, n))),
                   (np.repeat(e2[:, None], n, 1), np.ones((25, n)))):
        mf, mg = oa.collide_vjp(f, g, lf, lg, 0.7, 2.5)
        np.testing.assert_allclose(mf, lf, atol=1e-12)
        np.testing.assert_allclose(mg, lg, atol=1e-12)


def test_rollout_gradient_matches_central_differences():
    w, grid, X, Y, dep = _small_svi()
    rho, u, v, T = w.fields(X, Y)
    weight = grid.vertex_weights() * (X > 1.0)
    J, du, dv = oa.rollout_gradient(rho, u, v, T, dep, 0.8, w.cv, 4, weight)
    rng = np.random.default_rng(3)
    for _ in range(2):
        d1, d2 = rng.standard_normal(u.shape), rng.standard_normal(u.shape)
        eps = 1e-6
        jp = oa.objective(rho, u + eps * d1, v + eps * d2, T, dep, 0.8, w.cv, 4, weight)
        jm = oa.objective(rho, u - eps * d1, v - eps * d2, T, dep, 0.8, w.cv, 4, weight)
        fd = (jp - jm) / (2 * eps)
        ad = np.sum(du * d1) + np.sum(dv * d2)
        assert abs(fd - ad) < 1e-8 * max(1.0, abs(ad)), (fd, ad)
