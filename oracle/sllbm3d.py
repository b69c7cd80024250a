"""Plain FP64 oracle of the SLLBM step in three dimensions (arXiv:1910.13918): the extension to
D3Q125 on hexahedral cells that the paper names as the next step after its 2D results.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.  The same definitions as the 2D oracle
(``oracle/sllbm.py``), with one more axis: the D3Q125 set is the tensor product of D1Q5 three
times (Sec. II.B), the equilibrium the full fourth-order Hermite contraction over index tuples in
{x, y, z}^n (Sec. II.A), g^eq = (2 C_v - D) theta f^eq with D = 3 (Sec. II.D), the departure
point x - dt xi_i located per axis in a grid of Lagrange cells and the value interpolated with
the tensor product of the three 1D Lagrange bases (Eq. sl_streaming), then BGK (Eq.
streaming_fg, Pr = 1).  The Hermite tensors, the equilibrium coefficients, the 1D velocity set,
the Lagrange basis and the axis geometry are the 2D oracle's own, which are written for any
dimension or per axis.

Arrays: a population field is ``F[i, iz, iy, ix]`` with ``i = 25*a + 5*b + c`` (``a``, ``b``,
``c`` the D1Q5 indices of the x, y, z components); vertex arrays are ``[nz][ny][nx]``.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import sllbm as o

D3 = 3
Q125 = 125


def d3q125():
    """D3Q125 as the tensor product of D1Q5: xi_i = (xi_a, xi_b, xi_c), w_i = w_a w_b w_c."""
    x1, w1 = o.d1q5()
    xi = np.zeros((Q125, D3))
    w = np.zeros(Q125)
    for a, b, c in itertools.product(range(5), repeat=3):
        i = 25 * a + 5 * b + c
        xi[i] = (x1[a], x1[b], x1[c])
        w[i] = w1[a] * w1[b] * w1[c]
    return xi, w


def equilibrium_f(rho, u, theta):
    """f_i^eq = w_i sum_{n=0}^{4} (1/n!) a_eq^(n) : H^(n)(xi_i), the contraction over every index
    tuple in {x, y, z}^n; shape (125,) + vertex shape.  ``u`` has a trailing axis of length 3.
    The coefficients a_eq^(n) do not depend on the velocity and are formed once per call."""
    xi, w = d3q125()
    rho = np.asarray(rho)
    dtype = np.result_type(rho, u, theta, np.float64)
    coeff = {(n, idx): o.a_eq(n, idx, rho, u, theta)
             for n in range(5) for idx in itertools.product(range(D3), repeat=n)}
    out = np.zeros((Q125,) + rho.shape, dtype=dtype)
    for i in range(Q125):
        acc = np.zeros(rho.shape, dtype=dtype)
        for n in range(5):
            s = np.zeros(rho.shape, dtype=dtype)
            for idx in itertools.product(range(D3), repeat=n):
                s = s + coeff[n, idx] * float(o.hermite(n, idx, xi[i]))
            acc = acc + s / math.factorial(n)
        out[i] = w[i] * acc
    return out


def macroscopic(f, g, cv):
    """rho = sum f, rho u = sum f xi, T = (sum f |xi|^2 + sum g - rho |u|^2) / (2 C_v rho)."""
    xi, _ = d3q125()
    rho = np.zeros(f.shape[1:], dtype=f.dtype)
    j = np.zeros(f.shape[1:] + (D3,), dtype=f.dtype)
    e2 = np.zeros(f.shape[1:], dtype=f.dtype)
    for i in range(Q125):
        rho = rho + f[i]
        for k in range(D3):
            j[..., k] = j[..., k] + f[i] * xi[i, k]
        e2 = e2 + f[i] * float(np.sum(xi[i] ** 2)) + g[i]
    u = j / rho[..., None]
    T = (e2 - rho * np.sum(u ** 2, axis=-1)) / (2.0 * cv * rho)
    return rho, u, T / o.T0


def total_energy_density(f, g):
    xi, _ = d3q125()
    e2 = np.zeros(f.shape[1:], dtype=f.dtype)
    for i in range(Q125):
        e2 = e2 + f[i] * float(np.sum(xi[i] ** 2)) + g[i]
    return 0.5 * e2


def collide(f, g, tau, cv, isothermal=False):
    """BGK at the vertices (Eq. streaming_fg, Pr = 1), g^eq = (2 C_v - 3) theta f^eq;
    ``isothermal``: the equilibrium at theta = 1 (the isothermal configuration of Sec. III.A)."""
    rho, u, theta = macroscopic(f, g, cv)
    if isothermal:
        theta = np.ones_like(theta)
    feq = equilibrium_f(rho, u, theta)
    geq = (2.0 * cv - D3) * theta * feq
    return f - (f - feq) / tau, g - (g - geq) / tau


def initial_state(rho, u, v, w, T, cv):
    """Post-collision state at t = 0: the equilibrium of the given fields."""
    uu = np.stack([np.asarray(a, dtype=np.float64) for a in (u, v, w)], axis=-1)
    theta = np.asarray(T, dtype=np.float64) / o.T0
    feq = equilibrium_f(np.asarray(rho, dtype=np.float64), uu, theta)
    return feq, (2.0 * cv - D3) * theta * feq


class Grid3:
    """Tensor-product grid of hexahedral Lagrange cells (uniform in each axis)."""

    def __init__(self, ax: o.Axis, ay: o.Axis, az: o.Axis):
        assert ax.p == ay.p == az.p
        self.ax, self.ay, self.az = ax, ay, az
        self.p = ax.p
        self.nx, self.ny, self.nz = ax.nv, ay.nv, az.nv

    def coords(self):
        """Vertex coordinates, each [nz][ny][nx]."""
        Z, Y, X = np.meshgrid(self.az.vertex_coords(), self.ay.vertex_coords(),
                              self.ax.vertex_coords(), indexing="ij")
        return X, Y, Z


class Departures3:
    """Cell and local coordinate per axis of x_v - dt xi_i for every (velocity, vertex)."""

    def __init__(self, grid: Grid3, dt: float):
        self.grid = grid
        xi, _ = d3q125()
        X, Y, Z = grid.coords()
        self.cells, self.r = [], []
        for i in range(Q125):
            cs, rs = [], []
            for ax, P, k in ((grid.ax, X, 0), (grid.ay, Y, 1), (grid.az, Z, 2)):
                cell, r = ax.locate(ax.fold(P - dt * xi[i, k]))
                cs.append(cell)
                rs.append(r)
            self.cells.append(cs)
            self.r.append(rs)


def stream(F, dep: Departures3):
    """F_pre[i](v) = sum_{a,b,c} psi_a(r_x) psi_b(r_y) psi_c(r_z) F[i](node(a, b, c))."""
    g = dep.grid
    p = g.p
    out = np.zeros_like(F)
    for i in range(Q125):
        (cx, cy, cz), (rx, ry, rz) = dep.cells[i], dep.r[i]
        wx = o.lagrange(g.ax.nodes, rx)
        wy = o.lagrange(g.ay.nodes, ry)
        wz = o.lagrange(g.az.nodes, rz)
        acc = np.zeros(F.shape[1:], dtype=F.dtype)
        for c in range(p + 1):
            jz = g.az.vertex_of(cz, c)
            for b in range(p + 1):
                jy = g.ay.vertex_of(cy, b)
                for a in range(p + 1):
                    jx = g.ax.vertex_of(cx, a)
                    acc = acc + wx[..., a] * wy[..., b] * wz[..., c] * F[i, jz, jy, jx]
        out[i] = acc
    return out


def step(f, g, dep: Departures3, tau, cv, isothermal=False):
    """One step: pull the post-collision populations, then collide at every vertex."""
    return collide(stream(f, dep), stream(g, dep), tau, cv, isothermal)


def run(f, g, dep: Departures3, tau, cv, nsteps, isothermal=False):
    for _ in range(nsteps):
        f, g = step(f, g, dep, tau, cv, isothermal)
    return f, g
