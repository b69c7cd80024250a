"""Plain FP64 oracle of the SLLBM step (arXiv:1910.13918, Sec. II).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.  Every function is the definition the
paper gives, written out with loops over the index sets it names and vectorised over grid
vertices only.  No blocking, fusion, separability trick or closed form is used where the paper
states an explicit sum: in particular the equilibrium is the full Hermite tensor contraction of
Sec. II.A, not a factorised formula.

Arrays
------
A population field is ``F[i, iy, ix]`` with ``i = 5*a + b`` the D2Q25 index (``a`` the D1Q5 index
of the x component, ``b`` of the y component), ``iy`` the vertex row and ``ix`` the vertex column.
The D2Q9 set of the comparison in Sec. III.A is carried the same way (``i = 3*a + b``, D1Q3
indices); a field's velocity set is told by its first axis (25 or 9).
The state of the method is the pair ``(f, g)`` of *post-collision* vertex values (full
populations, not deviations).

Readings of points the paper leaves open (each is also listed in the design notes):
* collide at vertices, store post-collision values, interpolate that field at departure points
  (pull streaming of post-collision populations, Eq. 12 with Eq. 13);
* Prandtl number 1 unless asked otherwise, so the quasi-equilibrium term of Eq. 12 vanishes
  (tau_Pr = tau); for Pr != 1 the quasi-equilibrium f* of Sec. II.C is read with the 1/3! of the
  Hermite normalisation (w_i Q^neq : H^(3)(xi_i) / 3!, whose third moment is Q^neq), and g* as
  the same third-order projection of g's own centred third moment;
* temperature from the moments: T = (sum f|xi|^2 + sum g - rho |u|^2) / (2 C_v rho), T0 = 1;
* zero-gradient boundaries clamp the departure point into the domain; periodic ones wrap it;
* departure points exactly on a cell face belong to the cell on their right, and the upper end of
  a clamped axis belongs to the last cell.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

D = 2          # spatial dimension
Q = 25         # D2Q25 (the default velocity set)
Q9 = 9         # D2Q9, the standard set the paper compares against (Sec. III.A)
T0 = 1.0       # reference temperature; c_s^2 = R*T0 = 1 with R = 1 (Sec. II.A, II.B)


# ---------------------------------------------------------------------------------------------
# Velocity space (Sec. II.B, Table I)
# ---------------------------------------------------------------------------------------------
def d1q5():
    """D1Q5 abscissae and weights in the order of Table I.

    Index 0: 0; indices 1, 3: +-sqrt(5 - sqrt(10)); indices 2, 4: +-sqrt(5 + sqrt(10)).
    Weights 8/15, (7 + 2 sqrt 10)/60, (7 - 2 sqrt 10)/60.
    """
    s10 = math.sqrt(10.0)
    small = math.sqrt(5.0 - s10)
    large = math.sqrt(5.0 + s10)
    xi = np.array([0.0, small, large, -small, -large])
    w = np.array([8.0 / 15.0, (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0,
                  (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0])
    return xi, w


def d2q25():
    """D2Q25 set as the tensor product of D1Q5 (Sec. II.B): xi_i = (xi_a, xi_b), w_i = w_a w_b."""
    x1, w1 = d1q5()
    xi = np.zeros((Q, D))
    w = np.zeros(Q)
    for a in range(5):
        for b in range(5):
            i = 5 * a + b
            xi[i, 0] = x1[a]
            xi[i, 1] = x1[b]
            w[i] = w1[a] * w1[b]
    return xi, w


def d1q3():
    """D1Q3 abscissae and weights (the standard three-point Gauss-Hermite rule, c_s = 1):
    index 0: 0; indices 1, 2: +sqrt(3), -sqrt(3).  Weights 2/3, 1/6, 1/6."""
    s3 = math.sqrt(3.0)
    return np.array([0.0, s3, -s3]), np.array([2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0])


def d2q9():
    """D2Q9 set as the tensor product of D1Q3: i = 3a + b, xi_i = (xi_a, xi_b), w_i = w_a w_b."""
    x1, w1 = d1q3()
    xi = np.zeros((Q9, D))
    w = np.zeros(Q9)
    for a in range(3):
        for b in range(3):
            i = 3 * a + b
            xi[i, 0] = x1[a]
            xi[i, 1] = x1[b]
            w[i] = w1[a] * w1[b]
    return xi, w


def velocity_set(q=Q):
    """(xi, w) of the set with q velocities: 25 (D2Q25, the method's set) or 9 (D2Q9)."""
    if q == Q:
        return d2q25()
    if q == Q9:
        return d2q9()
    raise ValueError(f"no velocity set with {q} velocities")


# ---------------------------------------------------------------------------------------------
# Hermite tensors and equilibrium coefficients (Sec. II.A)
# ---------------------------------------------------------------------------------------------
def _delta(a, b):
    return 1.0 if a == b else 0.0


def hermite(n, idx, xi):
    """Component ``idx`` (a tuple of n axis indices) of the Hermite tensor H^(n) at ``xi``.

    ``xi`` has a trailing axis of length D.  c_s = 1, so H^(n) is the probabilists' Hermite
    tensor of Sec. II.A.  The symmetrised products ("overbrace") are written out: the three
    xi*delta terms of H^(3), the six xi*xi*delta terms and the three delta*delta pairings of H^(4).
    """
    x = lambda k: xi[..., idx[k]]
    d = lambda k, l: _delta(idx[k], idx[l])
    if n == 0:
        return np.ones(xi.shape[:-1])
    if n == 1:
        return x(0)
    if n == 2:
        return x(0) * x(1) - d(0, 1)
    if n == 3:
        return x(0) * x(1) * x(2) - (x(0) * d(1, 2) + x(1) * d(0, 2) + x(2) * d(0, 1))
    if n == 4:
        six = (x(0) * x(1) * d(2, 3) + x(0) * x(2) * d(1, 3) + x(0) * x(3) * d(1, 2)
               + x(1) * x(2) * d(0, 3) + x(1) * x(3) * d(0, 2) + x(2) * x(3) * d(0, 1))
        three = d(0, 1) * d(2, 3) + d(0, 2) * d(1, 3) + d(0, 3) * d(1, 2)
        return x(0) * x(1) * x(2) * x(3) - six + three
    raise ValueError("Hermite order above 4 is not part of the model")


def a_eq(n, idx, rho, u, theta):
    """Component ``idx`` of the equilibrium Hermite coefficient a_eq^(n) (Eq. moments, Sec. II.A).

    ``rho``, ``theta`` have the vertex shape, ``u`` the vertex shape plus a trailing D axis.
    The fourth-order bracket is read as rho[u u u u + T0^2 (theta-1)^2 (three delta pairings)
    + T0 (theta-1) (six delta*u*u terms)].
    """
    q = T0 * (theta - 1.0)
    uu = lambda k: u[..., idx[k]]
    d = lambda k, l: _delta(idx[k], idx[l])
    if n == 0:
        return rho
    if n == 1:
        return rho * uu(0)
    if n == 2:
        return rho * (uu(0) * uu(1) + q * d(0, 1))
    if n == 3:
        return rho * (uu(0) * uu(1) * uu(2)
                      + q * (d(0, 1) * uu(2) + d(0, 2) * uu(1) + d(1, 2) * uu(0)))
    if n == 4:
        pairs = d(0, 1) * d(2, 3) + d(0, 2) * d(1, 3) + d(0, 3) * d(1, 2)
        six = (d(0, 1) * uu(2) * uu(3) + d(0, 2) * uu(1) * uu(3) + d(0, 3) * uu(1) * uu(2)
               + d(1, 2) * uu(0) * uu(3) + d(1, 3) * uu(0) * uu(2) + d(2, 3) * uu(0) * uu(1))
        return rho * (uu(0) * uu(1) * uu(2) * uu(3) + q * q * pairs + q * six)
    raise ValueError("equilibrium coefficients are given up to fourth order")


def equilibrium_f(rho, u, theta, q=Q):
    """Discrete fourth-order equilibrium f_i^eq, shape (q,) + vertex shape.

    f_i^eq = w_i sum_{n=0}^{4} (1/n!) a_eq^(n) : H^(n)(xi_i)    (Eq. equilibrium with Eq. discrete)
    The full contraction runs over every index tuple in {x, y}^n.  The same fourth-order
    expansion serves the D2Q9 set (q = 9), as in the comparison of Sec. III.A.
    """
    xi, w = velocity_set(q)
    rho = np.asarray(rho)
    out = np.zeros((q,) + rho.shape, dtype=np.result_type(rho, u, theta, np.float64))
    for i in range(q):
        acc = np.zeros(rho.shape, dtype=out.dtype)
        for n in range(5):
            # H^(n) at one velocity is a scalar per index tuple; a_eq carries the vertex shape
            s = np.zeros(rho.shape, dtype=out.dtype)
            for idx in itertools.product(range(D), repeat=n):
                s = s + a_eq(n, idx, rho, u, theta) * float(hermite(n, idx, xi[i]))
            acc = acc + s / math.factorial(n)
        out[i] = w[i] * acc
    return out


def equilibrium_g(rho, u, theta, cv, q=Q):
    """Second population equilibrium g_i^eq = (2 C_v - D) theta f_i^eq (Sec. II.D)."""
    return (2.0 * cv - D) * theta * equilibrium_f(rho, u, theta, q)


# ---------------------------------------------------------------------------------------------
# Moments (Sec. II, Eqs. for rho, rho u, 2 rho E)
# ---------------------------------------------------------------------------------------------
def macroscopic(f, g, cv):
    """Density, velocity and theta = T/T0 from the populations.

    rho = sum_i f_i, rho u = sum_i f_i xi_i, 2 rho E = sum_i (f_i |xi_i|^2 + g_i),
    T = (2 rho E - rho |u|^2) / (2 C_v rho)  (gas constant R = 1, T0 = 1).
    Returns (rho, u, theta) with u carrying a trailing D axis.
    """
    xi, _ = velocity_set(f.shape[0])
    rho = np.zeros(f.shape[1:], dtype=f.dtype)
    j = np.zeros(f.shape[1:] + (D,), dtype=f.dtype)
    e2 = np.zeros(f.shape[1:], dtype=f.dtype)
    for i in range(f.shape[0]):
        rho = rho + f[i]
        j[..., 0] = j[..., 0] + f[i] * xi[i, 0]
        j[..., 1] = j[..., 1] + f[i] * xi[i, 1]
        e2 = e2 + f[i] * (xi[i, 0] ** 2 + xi[i, 1] ** 2) + g[i]
    u = j / rho[..., None]
    T = (e2 - rho * (u[..., 0] ** 2 + u[..., 1] ** 2)) / (2.0 * cv * rho)
    return rho, u, T / T0


def total_energy_density(f, g):
    """rho E = (sum f |xi|^2 + sum g) / 2 per vertex (Eq. E)."""
    xi, _ = velocity_set(f.shape[0])
    e2 = np.zeros(f.shape[1:], dtype=f.dtype)
    for i in range(f.shape[0]):
        e2 = e2 + f[i] * (xi[i, 0] ** 2 + xi[i, 1] ** 2) + g[i]
    return 0.5 * e2


# ---------------------------------------------------------------------------------------------
# Collision (Eq. streaming_fg with Pr = 1)
# ---------------------------------------------------------------------------------------------
def centered_third_moment(F, u):
    """Centred third moment Q[a, b, c] = sum_i F_i (xi_i - u)_a (xi_i - u)_b (xi_i - u)_c of a
    population field (the centred heat-flux tensor of Sec. II.C), shape (D, D, D) + vertex shape.
    ``u`` has the vertex shape plus a trailing D axis."""
    xi, _ = velocity_set(F.shape[0])
    out = np.zeros((D, D, D) + F.shape[1:], dtype=F.dtype)
    for i in range(F.shape[0]):
        c = [xi[i, k] - u[..., k] for k in range(D)]
        for a, b, cc in itertools.product(range(D), repeat=3):
            out[a, b, cc] = out[a, b, cc] + F[i] * c[a] * c[b] * c[cc]
    return out


def quasi_equilibrium(Qneq, q=Q):
    """f*_i = w_i Q^neq : H^(3)(xi_i) / 3! (Sec. II.C): the full contraction over the D^3 index
    tuples of the non-equilibrium centred third moment with the third Hermite tensor, weighted by
    the lattice weight.  The 1/3! is the Hermite normalisation of the third-order term (the
    printed formula has no prefactor); with it the third moment of f* is Q^neq."""
    xi, w = velocity_set(q)
    out = np.zeros((q,) + Qneq.shape[3:], dtype=Qneq.dtype)
    for i in range(q):
        acc = np.zeros(Qneq.shape[3:], dtype=Qneq.dtype)
        for idx in itertools.product(range(D), repeat=3):
            acc = acc + Qneq[idx] * hermite(3, idx, xi[i])
        out[i] = w[i] * acc / math.factorial(3)
    return out


def tau_prandtl(tau, pr):
    """tau_Pr = (tau - 1/2) / Pr + 1/2 (Sec. II.D)."""
    return (tau - 0.5) / pr + 0.5


def collide(f, g, tau, cv, pr=1.0, isothermal=False):
    """Collision at the vertices (Eq. streaming_fg):
    f* = f - (f - f^eq)/tau + (1/tau - 1/tau_Pr) f^qe, the same for g with g^eq = (2 C_v - D) theta
    f^eq, where f^qe (g^qe) is the quasi-equilibrium of the non-equilibrium centred third moment
    of f (of g).  With Pr = 1, tau_Pr = tau and the quasi-equilibrium term is zero: plain BGK.
    ``isothermal``: the equilibrium at theta = 1 (the isothermal configuration of Sec. III.A).
    The velocity set is that of the fields (25 or 9 velocities).
    """
    q = f.shape[0]
    rho, u, theta = macroscopic(f, g, cv)
    if isothermal:
        theta = np.ones_like(theta)
    feq = equilibrium_f(rho, u, theta, q)
    geq = (2.0 * cv - D) * theta * feq
    fn, gn = f - (f - feq) / tau, g - (g - geq) / tau
    if pr != 1.0:
        c = 1.0 / tau - 1.0 / tau_prandtl(tau, pr)
        fn = fn + c * quasi_equilibrium(centered_third_moment(f, u) - centered_third_moment(feq, u), q)
        gn = gn + c * quasi_equilibrium(centered_third_moment(g, u) - centered_third_moment(geq, u), q)
    return fn, gn


def initial_state(rho, u, v, T, cv, q=Q):
    """Post-collision state at t = 0: the equilibrium of the given fields (collision keeps it)."""
    uu = np.stack([np.asarray(u, dtype=np.result_type(u, np.float64)),
                   np.asarray(v, dtype=np.result_type(v, np.float64))], axis=-1)
    theta = np.asarray(T) / T0
    feq = equilibrium_f(np.asarray(rho), uu, theta, q)
    return feq, (2.0 * cv - D) * theta * feq


# ---------------------------------------------------------------------------------------------
# Space discretisation (Sec. II.E)
# ---------------------------------------------------------------------------------------------
def glc_nodes(p):
    """Gauss-Lobatto-Chebyshev support points on [0, 1]: x_k = (1 - cos(k pi / p)) / 2."""
    return np.array([0.5 * (1.0 - math.cos(k * math.pi / p)) for k in range(p + 1)])


def equidistant_nodes(p):
    return np.array([k / p for k in range(p + 1)])


def lagrange(nodes, r):
    """Lagrange basis psi_a(r) = prod_{b != a} (r - x_b)/(x_a - x_b); returns shape r.shape+(p+1,)."""
    r = np.asarray(r)
    n = len(nodes)
    out = np.empty(r.shape + (n,), dtype=np.result_type(r, np.float64))
    for a in range(n):
        acc = np.ones(r.shape, dtype=out.dtype)
        for b in range(n):
            if b != a:
                acc = acc * (r - nodes[b]) / (nodes[a] - nodes[b])
        out[..., a] = acc
    return out


class Axis:
    """One axis of a grid of ``n_cells`` cells of order ``p`` on [lo, hi] in reference coordinates.

    Cells share their end vertices (Fig. grid caption).  A periodic axis has n_cells*p vertices
    (the vertex at ``hi`` is the one at ``lo``); a zero-gradient axis has n_cells*p + 1.
    """

    def __init__(self, n_cells, p, lo, hi, periodic, nodes="glc"):
        self.n_cells, self.p, self.lo, self.hi = n_cells, p, float(lo), float(hi)
        self.periodic = bool(periodic)
        self.length = self.hi - self.lo
        self.hc = self.length / n_cells
        self.nodes = glc_nodes(p) if nodes == "glc" else equidistant_nodes(p)
        self.nv = n_cells * p if self.periodic else n_cells * p + 1

    def vertex_coords(self):
        j = np.arange(self.nv)
        cell = j // self.p
        k = j % self.p
        x = self.lo + self.hc * (cell + self.nodes[k])
        if not self.periodic:
            x[-1] = self.hi
        return x

    def fold(self, x):
        """Wrap (periodic) or clamp (zero-gradient) a coordinate into the axis."""
        if self.periodic:
            return self.lo + np.mod(x - self.lo, self.length)
        return np.clip(x, self.lo, self.hi)

    def locate(self, x):
        """Cell index and local coordinate r in [0, 1] of a folded coordinate."""
        s = (x - self.lo) / self.hc
        cell = np.clip(np.floor(s).astype(np.int64), 0, self.n_cells - 1)
        return cell, s - cell

    def vertex_of(self, cell, a):
        j = cell * self.p + a
        return j % self.nv if self.periodic else j


class SineMap:
    """Grid transformation x = xi + a sin(2 pi xi) sin(pi eta), y = eta + a sin(pi xi) sin(2 pi eta).

    The analytic map of the shock-vortex workload (a transformed grid as in Sec. III.E).
    ``a = 0`` is the identity.
    """

    def __init__(self, a):
        self.a = float(a)

    def __call__(self, xi, eta):
        a, pi = self.a, math.pi
        return (xi + a * np.sin(2 * pi * xi) * np.sin(pi * eta),
                eta + a * np.sin(pi * xi) * np.sin(2 * pi * eta))

    def jacobian(self, xi, eta):
        a, pi = self.a, math.pi
        return (1 + 2 * pi * a * np.cos(2 * pi * xi) * np.sin(pi * eta),
                pi * a * np.sin(2 * pi * xi) * np.cos(pi * eta),
                pi * a * np.cos(pi * xi) * np.sin(2 * pi * eta),
                1 + 2 * pi * a * np.sin(pi * xi) * np.cos(2 * pi * eta))

    def inverse(self, x, y, tol=1e-13, max_iter=100):
        """Newton iteration for the reference point of a physical point, started at (x, y)."""
        xi = np.array(x, dtype=np.float64, copy=True)
        eta = np.array(y, dtype=np.float64, copy=True)
        for _ in range(max_iter):
            fx, fy = self(xi, eta)
            rx, ry = fx - x, fy - y
            if np.max(np.abs(rx), initial=0.0) < tol and np.max(np.abs(ry), initial=0.0) < tol:
                return xi, eta
            j11, j12, j21, j22 = self.jacobian(xi, eta)
            det = j11 * j22 - j12 * j21
            xi = xi - (j22 * rx - j12 * ry) / det
            eta = eta - (-j21 * rx + j11 * ry) / det
        raise RuntimeError("Newton inversion of the grid map did not converge")


class Grid:
    """Tensor-product grid of Lagrange cells, optionally transformed by ``mapping``."""

    def __init__(self, ax: Axis, ay: Axis, mapping: SineMap | None = None):
        self.ax, self.ay, self.mapping = ax, ay, mapping
        self.nx, self.ny = ax.nv, ay.nv
        self.p = ax.p
        assert ax.p == ay.p

    def reference_coords(self):
        """Reference coordinates of every vertex, each of shape (ny, nx)."""
        X, Y = np.meshgrid(self.ax.vertex_coords(), self.ay.vertex_coords())
        return X, Y

    def coords(self):
        """Physical coordinates of every vertex, each of shape (ny, nx)."""
        X, Y = self.reference_coords()
        if self.mapping is None:
            return X, Y
        return self.mapping(X, Y)

    def vertex_weights(self):
        """A_v = integral of the shape function of vertex v over the domain (with |det J|).

        Gauss-Legendre quadrature with p + 3 points per axis and cell, summed over the cells that
        contain the vertex.  sum_v A_v rho_v is then the integral of the interpolant of rho.
        """
        ax, ay, p = self.ax, self.ay, self.p
        gp, gw = np.polynomial.legendre.leggauss(p + 3)
        gp = 0.5 * (gp + 1.0)
        gw = 0.5 * gw
        psi = lagrange(ax.nodes, gp)                     # (nq, p+1)
        A = np.zeros((self.ny, self.nx))
        for cy in range(ay.n_cells):
            for cx in range(ax.n_cells):
                for qy in range(len(gp)):
                    for qx in range(len(gp)):
                        xi = ax.lo + ax.hc * (cx + gp[qx])
                        eta = ay.lo + ay.hc * (cy + gp[qy])
                        if self.mapping is None:
                            det = 1.0
                        else:
                            j11, j12, j21, j22 = self.mapping.jacobian(xi, eta)
                            det = abs(j11 * j22 - j12 * j21)
                        wq = gw[qx] * gw[qy] * det * ax.hc * ay.hc
                        for b in range(p + 1):
                            for a in range(p + 1):
                                A[ay.vertex_of(cy, b), ax.vertex_of(cx, a)] += \
                                    wq * psi[qx, a] * psi[qy, b]
        return A


class Departures:
    """Departure cells and reference coordinates of every (velocity, vertex) pair.

    x_d = x_v - dt xi_i (Eq. streaming_fg), folded into the domain per axis, then located in a
    cell.  On a transformed grid the fold is done on the physical point and the reference point
    is found by Newton inversion of the map.  ``vertices`` optionally restricts the computation
    to a flat list of vertex indices (row-major, iy * nx + ix).  ``q`` picks the velocity set.
    """

    def __init__(self, grid: Grid, dt: float, vertices=None, q=Q):
        self.grid = grid
        self.dt = float(dt)
        self.q = q
        xi, _ = velocity_set(q)
        X, Y = grid.coords()
        RX, RY = grid.reference_coords()
        X, Y, RX, RY = (A.reshape(-1) for A in (X, Y, RX, RY))
        if vertices is not None:
            vertices = np.asarray(vertices)
            X, Y, RX, RY = X[vertices], Y[vertices], RX[vertices], RY[vertices]
        self.vertices = vertices
        ax, ay = grid.ax, grid.ay
        self.cx, self.cy, self.rx, self.ry = [], [], [], []
        for i in range(q):
            if grid.mapping is None:
                xd = ax.fold(X - self.dt * xi[i, 0])
                yd = ay.fold(Y - self.dt * xi[i, 1])
                ex, ey = xd, yd
            else:
                # physical domain equals the reference box; fold there, then invert the map
                xd = ax.fold(X - self.dt * xi[i, 0])
                yd = ay.fold(Y - self.dt * xi[i, 1])
                ex, ey = grid.mapping.inverse(xd, yd)
                ex, ey = ax.fold(ex), ay.fold(ey)
            cx, rx = ax.locate(ex)
            cy, ry = ay.locate(ey)
            self.cx.append(cx)
            self.cy.append(cy)
            self.rx.append(rx)
            self.ry.append(ry)


def stream(F, dep: Departures):
    """Pull streaming (Eq. sl_streaming): F_pre[i](v) = sum_{a,b} psi_a(r) psi_b(s) F[i](node(a,b)).

    ``F`` is the post-collision field of the previous step, shape (q, ny, nx).  Returns the values
    at the departure points for every vertex (shape (q, ny, nx)), or for the vertex subset of
    ``dep`` (shape (q, len(subset))).
    """
    grid = dep.grid
    ax, ay, p = grid.ax, grid.ay, grid.p
    assert F.shape[0] == dep.q, "field and departures belong to different velocity sets"
    shape = (grid.ny, grid.nx) if dep.vertices is None else (len(dep.vertices),)
    out = np.zeros((dep.q,) + shape, dtype=F.dtype)
    for i in range(dep.q):
        wx = lagrange(ax.nodes, dep.rx[i])
        wy = lagrange(ay.nodes, dep.ry[i])
        acc = np.zeros(dep.rx[i].shape, dtype=F.dtype)
        for b in range(p + 1):
            jy = ay.vertex_of(dep.cy[i], b)
            for a in range(p + 1):
                jx = ax.vertex_of(dep.cx[i], a)
                acc = acc + wx[:, a] * wy[:, b] * F[i, jy, jx]
        out[i] = acc.reshape(shape)
    return out


def step(f, g, dep: Departures, tau, cv, pr=1.0, isothermal=False):
    """One SLLBM time step: pull the post-collision populations, then collide at every vertex."""
    fpre = stream(f, dep)
    gpre = stream(g, dep)
    return collide(fpre, gpre, tau, cv, pr, isothermal)


def run(f, g, dep: Departures, tau, cv, nsteps, pr=1.0, isothermal=False):
    for _ in range(nsteps):
        f, g = step(f, g, dep, tau, cv, pr, isothermal)
    return f, g


def mass_energy(f, g, A):
    """Global mass M = sum_v A_v rho_v and energy sum_v A_v rho E_v (mass check of Sec. III.E)."""
    rho = f.sum(axis=0)
    return float(np.sum(A * rho)), float(np.sum(A * total_energy_density(f, g)))
