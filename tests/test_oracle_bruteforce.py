"""One oracle step on tiny periodic grids against a second, slow transcription built from other
routines (no GPU needed).

The second transcription shares no code with the oracle:
* velocity set: numpy's five-point Gauss-Hermite rule, placed in Table I order by value;
* Hermite tensors: H^(n)(xi) = (-1)^n e^{|xi|^2/2} d^n/dxi^n e^{-|xi|^2/2}, differentiated by
  sympy (the Rodrigues form of the probabilists' Hermite tensor, c_s = 1);
* equilibrium coefficients: a^(n) = integral of the Maxwellian rho N(u, theta I) times H^(n),
  by a 6 x 6 Gauss-Hermite rule around u (exact for the degree-4 polynomials);
* support points: numpy's Chebyshev points of the second kind on [0, 1];
* interpolation: scipy's barycentric Lagrange interpolator over the cell's nodes, along x for
  the p + 1 rows of the cell, then along y;
* moments, temperature and BGK written out per vertex in plain Python.
Agreement to 1e-12 pins the oracle's velocity set, tensors, coefficients, departures,
interpolation and collision together (a wrong index, sign or dropped term in any of them shows).
"""
import itertools
import math

import numpy as np
import pytest
from scipy.interpolate import BarycentricInterpolator

sp = pytest.importorskip("sympy")   # not every test machine has it

from oracle import sllbm as o

CV = 2.5


def _velocity_set(n1=5):
    """1D rule in the oracle's order: D1Q5 as in Table I (0, +small, +large, -small, -large),
    D1Q3 as 0, +sqrt3, -sqrt3."""
    nodes, weights = np.polynomial.hermite_e.hermegauss(n1)
    weights = weights / math.sqrt(2 * math.pi)
    order = [2, 3, 4, 1, 0] if n1 == 5 else [1, 2, 0]
    return nodes[order], weights[order]


def _hermite_tensors():
    """{(n, idx): callable H^(n)_idx(x, y)} for n <= 4 from the Rodrigues formula."""
    x, y = sp.symbols("x y")
    G = sp.exp(-(x ** 2 + y ** 2) / 2)
    sym = (x, y)
    out = {}
    for n in range(5):
        for idx in itertools.product(range(2), repeat=n):
            d = G
            for k in idx:
                d = sp.diff(d, sym[k])
            out[n, idx] = sp.lambdify((x, y), sp.expand(sp.simplify((-1) ** n * d / G)), "math")
    return out


H = _hermite_tensors()
GH_Z, GH_W = np.polynomial.hermite_e.hermegauss(6)
GH_W = GH_W / math.sqrt(2 * math.pi)


def _feq(rho, ux, uy, theta, xi1, w1):
    n1 = len(xi1)
    sd = math.sqrt(theta)
    coef = {}
    for (n, idx), h in H.items():
        s = 0.0
        for za, wa in zip(GH_Z, GH_W):
            for zb, wb in zip(GH_Z, GH_W):
                s += wa * wb * h(ux + sd * za, uy + sd * zb)
        coef[n, idx] = rho * s
    f = np.zeros(n1 * n1)
    for a in range(n1):
        for b in range(n1):
            acc = 0.0
            for (n, idx), h in H.items():
                acc += coef[n, idx] * h(xi1[a], xi1[b]) / math.factorial(n)
            f[n1 * a + b] = w1[a] * w1[b] * acc
    return f


def _step(F, G, nodes, n_cells, lengths, dt, tau, xi1, w1, cv=CV, isothermal=False):
    """One step on a periodic grid: F, G are [q][ny][nx] post-collision fields."""
    n1 = len(xi1)
    ny, nx = F.shape[1:]
    p = len(nodes) - 1
    (Lx, Ly), (cx, cy) = lengths, n_cells
    hx, hy = Lx / cx, Ly / cy
    xs = [hx * (j // p + nodes[j % p]) for j in range(nx)]
    ys = [hy * (j // p + nodes[j % p]) for j in range(ny)]
    Fn, Gn = np.zeros_like(F), np.zeros_like(G)
    K = 2 * cv - 2
    vel = [(a, b) for a in range(n1) for b in range(n1)]
    for iy in range(ny):
        for ix in range(nx):
            fpre, gpre = np.zeros(n1 * n1), np.zeros(n1 * n1)
            for a, b in vel:
                i = n1 * a + b
                xd = (xs[ix] - dt * xi1[a]) % Lx
                yd = (ys[iy] - dt * xi1[b]) % Ly
                kx, ky = min(int(xd // hx), cx - 1), min(int(yd // hy), cy - 1)
                rx, ry = xd / hx - kx, yd / hy - ky
                for src, dst in ((F, fpre), (G, gpre)):
                    rows = []
                    for m in range(p + 1):
                        jy = (ky * p + m) % ny
                        vals = [src[i, jy, (kx * p + q) % nx] for q in range(p + 1)]
                        rows.append(float(BarycentricInterpolator(nodes, vals)(rx)))
                    dst[i] = float(BarycentricInterpolator(nodes, rows)(ry))
            rho = fpre.sum()
            jx = sum(fpre[n1 * a + b] * xi1[a] for a, b in vel)
            jy = sum(fpre[n1 * a + b] * xi1[b] for a, b in vel)
            e2 = sum(fpre[n1 * a + b] * (xi1[a] ** 2 + xi1[b] ** 2) for a, b in vel)
            e2 += gpre.sum()
            ux, uy = jx / rho, jy / rho
            theta = 1.0 if isothermal else (e2 - rho * (ux * ux + uy * uy)) / (2 * cv * rho)
            feq = _feq(rho, ux, uy, theta, xi1, w1)
            Fn[:, iy, ix] = fpre - (fpre - feq) / tau
            Gn[:, iy, ix] = gpre - (gpre - K * theta * feq) / tau
    return Fn, Gn


@pytest.mark.parametrize("p,cells", [(2, (2, 2)), (3, (2, 1))])
def test_one_step_matches_an_independent_transcription(p, cells):
    rng = np.random.default_rng(70 + p)
    Lx, Ly = 1.0, 0.8
    ax = o.Axis(cells[0], p, 0.0, Lx, True)
    ay = o.Axis(cells[1], p, 0.0, Ly, True)
    grid = o.Grid(ax, ay)
    X, Y = grid.coords()
    rho = 1 + 0.1 * rng.standard_normal(X.shape) ** 2 * 0.3
    u = 0.1 * rng.standard_normal(X.shape)
    v = 0.1 * rng.standard_normal(X.shape)
    T = 1 + 0.1 * rng.standard_normal(X.shape)
    f, g = o.initial_state(rho, u, v, T, CV)
    # start away from equilibrium so that the step's collision has work to do
    f = f * (1 + 0.02 * rng.standard_normal(f.shape))
    g = g * (1 + 0.02 * rng.standard_normal(g.shape))
    dt, tau = 0.023, 0.85
    f1, g1 = o.step(f, g, o.Departures(grid, dt), tau, CV)

    xi1, w1 = _velocity_set()
    nodes = 0.5 * (1 + np.polynomial.chebyshev.chebpts2(p + 1))
    F2, G2 = _step(f, g, nodes, cells, (Lx, Ly), dt, tau, xi1, w1)
    scale = np.max(np.abs(f1))
    assert np.max(np.abs(f1 - F2)) < 1e-12 * scale
    assert np.max(np.abs(g1 - G2)) < 1e-12 * scale


def test_d2q9_isothermal_step_matches_an_independent_transcription():
    """The same on the D2Q9 set (numpy's three-point rule) with the isothermal equilibrium."""
    p, cells, Lx, Ly = 2, (2, 2), 1.0, 0.8
    rng = np.random.default_rng(77)
    grid = o.Grid(o.Axis(cells[0], p, 0.0, Lx, True), o.Axis(cells[1], p, 0.0, Ly, True))
    X, Y = grid.coords()
    rho = 1 + 0.05 * rng.standard_normal(X.shape)
    u = 0.08 * rng.standard_normal(X.shape)
    v = 0.08 * rng.standard_normal(X.shape)
    f, g = o.initial_state(rho, u, v, np.ones_like(X), 1.0, q=9)
    f = f * (1 + 0.02 * rng.standard_normal(f.shape))
    dt, tau = 0.031, 0.9
    f1, g1 = o.step(f, g, o.Departures(grid, dt, q=9), tau, 1.0, isothermal=True)
    xi1, w1 = _velocity_set(3)
    nodes = 0.5 * (1 + np.polynomial.chebyshev.chebpts2(p + 1))
    F2, _ = _step(f, g, nodes, cells, (Lx, Ly), dt, tau, xi1, w1, cv=1.0, isothermal=True)
    assert np.max(np.abs(f1 - F2)) < 1e-12 * np.max(np.abs(f1))
