"""Seeded synthetic workloads shaped like the test cases of arXiv:1910.13918 (Sec. III).

This module is the input generator shared by the CUDA path, the tests, the benchmark and the
oracle.  It holds grid sizes, time steps, relaxation times and initial macroscopic fields as
functions of vertex coordinates -- and none of the method's arithmetic (no velocity set,
equilibrium, interpolation or collision).  Each side evaluates the initial fields on its own
vertex coordinates.

Parameter recipe (readings of the paper where it is silent):
* time step from CFL 0.5 on the mean vertex spacing h = L / (cells * p) with respect to the
  largest D2Q25 speed |c|max = sqrt(2 (5 + sqrt 10)) = 4.0404 (Euclidean);
* Taylor-Green vortex: U0 = Ma (c_s = 1), nu = U0 * 2 pi / Re, tau = nu / dt + 1/2 (Sec. II.D),
  p = 1 + (rho U0^2 / 4)(cos 2x + cos 2y), rho = 1, T = p / rho;
* Sod (Sec. III.C) and 2D Riemann (Sec. III.D) use the paper's relaxation times 1.518 and
  1.94815; T = p / rho with R = 1;
* shock-vortex (Sec. III.E): region A (x < 0.5) rho = 1, P = 1/gamma, u = 1.2 (Ma_A = 1.2 with
  c_A = 1); region B from the Rankine-Hugoniot relations; an isentropic vortex of radius 0.075,
  Ma_v = 0.25, with the radial-equilibrium exponent Ma_v^2; nu from Re = c_A R / nu = 75 (the
  paper's 400 diverges at the time step these 200 steps need, see svi());
* gamma = 1.4 everywhere, so C_v = R / (gamma - 1) = 2.5.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4
CV = 1.0 / (GAMMA - 1.0)             # 2.5
C_MAX = math.sqrt(2.0 * (5.0 + math.sqrt(10.0)))  # largest D2Q25 speed, 4.0404

PERIODIC = 0
ZERO_GRADIENT = 1


@dataclasses.dataclass
class Workload:
    name: str
    nx_cells: int
    ny_cells: int
    order: int
    x0: float
    x1: float
    y0: float
    y1: float
    bc_x: int
    bc_y: int
    dt: float
    tau: float
    steps: int
    kind: str                      # which initial field generator
    map_a: float = 0.0             # sine-map amplitude (0: uniform grid)
    cv: float = CV
    pr: float = 1.0                # Prandtl number (1: plain BGK, Sec. II.C)
    isothermal: bool = False       # theta = 1 in the equilibrium (Sec. III.A); needs cv = 1
    velset: str = "d2q25"          # "d2q25", or "d2q9" (the comparison set of Sec. III.A)
    nodes: str = "glc"
    seed: int = 0
    extra: dict = dataclasses.field(default_factory=dict)

    # vertex counts: periodic axes have cells * p vertices, zero-gradient ones cells * p + 1
    @property
    def nx(self):
        return self.nx_cells * self.order + (0 if self.bc_x == PERIODIC else 1)

    @property
    def ny(self):
        return self.ny_cells * self.order + (0 if self.bc_y == PERIODIC else 1)

    @property
    def n_vertices(self):
        return self.nx * self.ny

    @property
    def updates_per_step(self):
        return self.n_vertices * self.n_velocities * self.n_populations

    @property
    def n_velocities(self):
        return 9 if self.velset == "d2q9" else 25

    @property
    def n_populations(self):
        return 1 if self.cv == 1.0 else 2

    @property
    def velocity_scale(self):
        """Characteristic speed of the flow: the scale velocity errors are reported against.

        Taylor-Green: U0; Sod: sound speed of the left state; Riemann: largest state speed;
        shock-vortex: inflow speed.  (Flows that start at rest have no velocity to be relative to.)
        """
        if self.kind == "tgv":
            return self.extra["U0"]
        if self.kind == "sod":
            return math.sqrt(GAMMA * 1.0 / 1.0)
        if self.kind == "riemann":
            states = self.extra.get("states", RIEMANN_STATES)
            return max(math.hypot(st[1], st[2]) for st in states.values())
        if self.kind == "svi":
            return self.extra["Ma_A"]
        if self.kind == "sdp":
            return self.extra["U"]
        if self.kind == "tgvm":
            return self.extra["u_v"]
        return 1.0

    def fields(self, x, y, perturb=False):
        """Initial (rho, u, v, T) on vertex coordinates x, y (arrays of equal shape, float64)."""
        rho, u, v, T = _GENERATORS[self.kind](self, np.asarray(x, np.float64),
                                              np.asarray(y, np.float64))
        if perturb:
            rng = np.random.default_rng(20191031 + self.seed)
            rho = rho * (1.0 + 1e-4 * rng.standard_normal(rho.shape))
            umax = max(float(np.max(np.abs(u))), float(np.max(np.abs(v))), 1e-3)
            u = u + 1e-4 * umax * rng.standard_normal(u.shape)
            v = v + 1e-4 * umax * rng.standard_normal(v.shape)
            T = T * (1.0 + 1e-4 * rng.standard_normal(T.shape))
        return rho, u, v, T

    def resized(self, nx_cells, ny_cells, steps=None, dt=None, keep_tau=False):
        """Same physics on another grid; the time step follows the CFL rule unless given.

        The viscosity is kept (tau follows dt) unless ``keep_tau``: the Sod and 2D Riemann cases
        fix tau itself, as the paper does (Sec. III.C, III.D)."""
        w = dataclasses.replace(self, nx_cells=nx_cells, ny_cells=ny_cells)
        if dt is None:
            dt = cfl_dt(w)
        ratio = dt / self.dt
        nu = (self.tau - 0.5) * self.dt
        w.dt = dt
        w.tau = self.tau if keep_tau else nu / dt + 0.5
        w.steps = steps if steps is not None else max(1, int(round(self.steps / ratio)))
        return w


def cfl_dt(w: Workload, cfl=0.5):
    hx = (w.x1 - w.x0) / (w.nx_cells * w.order)
    hy = (w.y1 - w.y0) / (w.ny_cells * w.order)
    return cfl * min(hx, hy) / C_MAX


# ---------------------------------------------------------------------------------------------
# initial fields
# ---------------------------------------------------------------------------------------------
def _tgv(w, x, y):
    U0 = w.extra["U0"]
    rho = np.ones_like(x)
    u = U0 * np.sin(x) * np.cos(y)
    v = -U0 * np.cos(x) * np.sin(y)
    p = 1.0 + rho * U0 ** 2 / 4.0 * (np.cos(2 * x) + np.cos(2 * y))
    return rho, u, v, p / rho


def _sod(w, x, y):
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(x)
    return rho, z.copy(), z.copy(), p / rho


RIEMANN_STATES = {  # (rho, u, v, p) per quadrant, interfaces at x = y = 0.8
    "NE": (1.5, 0.0, 0.0, 1.5),
    "NW": (0.5323, 1.206, 0.0, 0.3),
    "SW": (0.138, 1.206, 1.206, 0.029),
    "SE": (0.5323, 0.0, 1.206, 0.3),
}


# The 2D Riemann states of the paper's Table III (Lax-Liu), quadrants split at x = y = 0.5.
RIEMANN_STATES_PAPER = {
    "NW": (1.0, 0.7276, 0.0, 1.0),
    "NE": (0.5313, 0.0, 0.0, 0.4),
    "SW": (0.8, 0.0, 0.0, 1.0),
    "SE": (1.0, 0.0, 0.7276, 1.0),
}


def _riemann(w, x, y):
    states = w.extra.get("states", RIEMANN_STATES)
    split = w.extra.get("split", 0.8)
    east = x >= split
    north = y >= split
    out = [np.zeros_like(x) for _ in range(4)]
    for key, mask in (("NE", east & north), ("NW", ~east & north),
                      ("SW", ~east & ~north), ("SE", east & ~north)):
        st = states[key]
        for k in range(4):
            out[k] = np.where(mask, st[k], out[k])
    rho, u, v, p = out
    return rho, u, v, p / rho


def rankine_hugoniot(mach, gamma=GAMMA):
    """Density ratio, pressure ratio and downstream Mach number of a normal shock."""
    m2 = mach * mach
    rho_ratio = (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)
    p_ratio = 1 + 2 * gamma / (gamma + 1) * (m2 - 1)
    mach_b = math.sqrt(((gamma - 1) * m2 + 2) / (2 * gamma * m2 - (gamma - 1)))
    return rho_ratio, p_ratio, mach_b


def _svi(w, x, y):
    g = GAMMA
    ex = w.extra
    ma_a, ma_v, radius = ex["Ma_A"], ex["Ma_v"], ex["radius"]
    xc, yc, xs = ex["xc"], ex["yc"], ex["x_shock"]
    rho_r, p_r, _ = rankine_hugoniot(ma_a)
    pA = 1.0 / g
    uA = ma_a * 1.0                        # c_A = sqrt(gamma pA / rhoA) = 1
    region_a = x < xs
    rho = np.where(region_a, 1.0, rho_r)
    p = np.where(region_a, pA, pA * p_r)
    u = np.where(region_a, uA, uA / rho_r)
    v = np.zeros_like(x)
    # isentropic vortex in region A
    dx, dy = x - xc, y - yc
    r2 = (dx * dx + dy * dy) / radius ** 2
    env = np.exp(0.5 * (1.0 - r2))
    base = 1.0 - 0.5 * (g - 1) * ma_v ** 2 * np.exp(1.0 - r2)
    rho_v = base ** (1.0 / (g - 1))
    p_v = pA * base ** (g / (g - 1))
    rho = np.where(region_a, rho_v, rho)
    p = np.where(region_a, p_v, p)
    u = np.where(region_a, uA - ma_v * env * dy / radius, u)
    v = np.where(region_a, ma_v * env * dx / radius, v)
    return rho, u, v, p / rho


def _sdp(w, x, y):
    rho = sdp_density(w, x, y, 0.0)
    return rho, np.full_like(x, w.extra["U"]), np.zeros_like(x), 1.0 / rho   # P = 1


def sdp_density(w: Workload, x, y, t):
    """Exact density of the smooth density propagation at lattice time t: the initial wave
    1 + 0.2 sin(pi x) sin(pi y) carried along x with the uniform speed U."""
    return 1.0 + 0.2 * np.sin(np.pi * (x - w.extra["U"] * t)) * np.sin(np.pi * y)


def _tgvm(w, x, y):
    u, v, rho = tgvm_reference(w, x, y, 0.0)
    return rho, u, v, np.ones_like(x)


def tgvm_reference(w: Workload, x, y, t):
    """Moving Taylor-Green vortex (Sec. III.A) at lattice time t: velocity (u, v) and density
    rho = 1 + p' (isothermal, c_s = 1), the vortex carried along x with u_h and decaying with
    exp(-2 nu t)."""
    uv, uh, nu = w.extra["u_v"], w.extra["u_h"], w.extra["nu"]
    xs = x - uh * t
    d = np.exp(-2.0 * nu * t)
    u = uh + uv * np.sin(xs) * np.cos(y) * d
    v = -uv * np.cos(xs) * np.sin(y) * d
    rho = 1.0 + uv ** 2 / 4.0 * (np.cos(2.0 * xs) + np.cos(2.0 * y)) * d * d
    return u, v, rho


_GENERATORS = {"tgv": _tgv, "sod": _sod, "riemann": _riemann, "svi": _svi, "sdp": _sdp,
               "tgvm": _tgvm}


def svi_envelope(w: Workload, x, y):
    ex = w.extra
    r2 = ((x - ex["xc"]) ** 2 + (y - ex["yc"]) ** 2) / ex["radius"] ** 2
    return np.exp(0.5 * (1.0 - r2))


def svi_directions(w: Workload, x, y, count=16):
    """Seeded random control directions (du, dv) for finite-difference checks of the gradient."""
    env = svi_envelope(w, x, y)
    out = []
    for s in range(count):
        rng = np.random.default_rng(s)
        out.append((rng.standard_normal(x.shape) * env, rng.standard_normal(x.shape) * env))
    return out


# ---------------------------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------------------------
def _tgv_workload(name, cells, p, ma, re, steps, seed):
    L = 2 * math.pi
    w = Workload(name, cells, cells, p, 0.0, L, 0.0, L, PERIODIC, PERIODIC, 1.0, 1.0, steps,
                 "tgv", seed=seed, extra={"U0": ma})
    w.dt = cfl_dt(w)
    nu = ma * L / re
    w.tau = nu / w.dt + 0.5
    return w


def tgv16():
    """Taylor-Green vortex, 16x16 cells, p = 2 (32x32 vertices), Ma 0.1, Re 100, 100 steps."""
    return _tgv_workload("tgv16_p2", 16, 2, 0.1, 100.0, 100, 1)


def tgv256():
    """Taylor-Green vortex, 256x256 cells, p = 4 (1024x1024 vertices), Ma 0.3, Re 1000."""
    return _tgv_workload("tgv256_p4", 256, 4, 0.3, 1000.0, 1000, 2)


def sod():
    """Sod tube strip [0,1]x[0,4/4096], 4096x4 cells, p = 2, tau 1.518, t = 0.2."""
    w = Workload("sod4096_p2", 4096, 4, 2, 0.0, 1.0, 0.0, 4.0 / 4096, ZERO_GRADIENT, PERIODIC,
                 1.0, 1.518, 1, "sod", seed=3)
    n = int(round(0.2 / cfl_dt(w)))
    w.dt = 0.2 / n
    w.steps = n
    return w


def riemann():
    """2D Riemann problem [0,1]^2, 1024x1024 cells, p = 3, tau 1.94815, t = 0.3."""
    w = Workload("riemann1024_p3", 1024, 1024, 3, 0.0, 1.0, 0.0, 1.0, ZERO_GRADIENT,
                 ZERO_GRADIENT, 1.0, 1.94815, 1, "riemann", seed=4)
    n = int(round(0.3 / cfl_dt(w)))
    w.dt = 0.3 / n
    w.steps = n
    return w


def riemann_paper():
    """The same 1024x1024-cell p = 3 grid with the milder quadrant states of Table III."""
    w = riemann()
    w.name = "riemann1024_p3_tableIII"
    w.kind = "riemann"
    w.extra = {"states": RIEMANN_STATES_PAPER, "split": 0.5}
    w.seed = 6
    return w


def riemann_nodes(nodes="glc", cells=128):
    """The 2D Riemann run of Sec. III.D as printed: 128 x 128 cells of order p = 4 on [0,1]^2
    (513 x 513 vertices), the Table III states, tau = 1.94815, t_end = 0.25 after 2091 steps,
    zero-gradient boundaries; ``nodes`` "glc" or "equidistant" for the comparison of support
    points (the paper's equidistant run diverged shortly after 200 steps)."""
    w = Workload(f"riemann{cells}_p4_{nodes}", cells, cells, 4, 0.0, 1.0, 0.0, 1.0, ZERO_GRADIENT,
                 ZERO_GRADIENT, 0.25 / 2091, 1.94815, 2091, "riemann", nodes=nodes, seed=9,
                 extra={"states": RIEMANN_STATES_PAPER, "split": 0.5})
    w.dt *= 128.0 / cells
    w.steps = int(round(0.25 / w.dt))
    return w


def svi():
    """Shock-vortex interaction on the sine-mapped grid [0,2]x[0,1], 512x256 cells, p = 2.

    dt = 3e-3 lets the acoustic signal of the vortex reach x > 1.5 within the 200 steps (t = 0.6).
    At that step the paper's Re = c_A R / nu = 400 (and 200) leaves tau = 0.56 (0.63) and the
    run diverges within 40 (60) steps in FP64 as well as FP32; Re = 100 (tau = 0.75) stays
    bounded from the smooth fields but diverges within 80 steps once they carry the 1e-4 seeded
    perturbation of the parity tests; Re = 75 (tau = 0.83) stays bounded with it and is used."""
    radius = 0.075
    nu = 1.0 * radius / 75.0
    dt = 3.0e-3
    return Workload("svi512x256_p2_mapped", 512, 256, 2, 0.0, 2.0, 0.0, 1.0, ZERO_GRADIENT,
                    PERIODIC, dt, nu / dt + 0.5, 200, "svi", map_a=0.05, seed=5,
                    extra={"Ma_A": 1.2, "Ma_v": 0.25, "radius": radius, "xc": 0.25, "yc": 0.5,
                           "x_shock": 0.5, "x_objective": 1.5, "checkpoint_every": 20})


def svi_pr():
    """The shock-vortex workload at the paper's Prandtl number 0.75 (Sec. III.E, Sec. II.C)."""
    w = svi()
    w.name = "svi512x256_p2_mapped_pr075"
    w.pr = 0.75
    return w


def tgv_moving(points=32, ma_h=0.05, velset="d2q25"):
    """Isothermal moving Taylor-Green vortex (Sec. III.A) on [0, 2 pi]^2, p = 4, points x points
    vertices: Ma_v = 0.01 (u_v = 0.01, c_s = 1), horizontal Mach number Ma_h, Re = u_v 2 pi / nu
    = 10, compared at the time the vortex speed has decayed to 0.1 u_v.  The paper's time steps
    (0.0008 at 16 points, halved per refinement) are in its unit of time, where u_v = 1: in
    lattice units dt = 0.0008 / u_v = 0.08 at 16 points, and the end time 1.83 is 183.
    ``velset`` "d2q9" runs the comparison set of the same study."""
    uv = 0.01
    nu = uv * 2.0 * math.pi / 10.0
    t_end = math.log(10.0) / (2.0 * nu)          # exp(-2 nu t) = 0.1
    steps0 = int(round(t_end / 0.08))
    steps = steps0 * (points // 16)
    dt = t_end / steps
    L = 2.0 * math.pi
    tag = "" if velset == "d2q25" else f"_{velset}"
    return Workload(f"tgvm{points}_p4_mah{ma_h:g}{tag}", points // 4, points // 4, 4, 0.0, L, 0.0, L,
                    PERIODIC, PERIODIC, dt, nu / dt + 0.5, steps, "tgvm", cv=1.0, isothermal=True,
                    velset=velset, seed=8, extra={"u_v": uv, "u_h": ma_h, "nu": nu, "t_end": t_end})


def sdp(points=16, step_factor=1):
    """Smooth density propagation (Sec. III.B, Table II) on [-1,1]^2, periodic, p = 4, with
    points x points vertices (points / 4 cells per axis).

    Reading of the paper's units: the speed is U = Ma c_s = 0.2 (c_s = 1), so the wave crosses
    the domain once (the paper's t = 2 at unit speed) in lattice time 2 / U = 10.  The paper's
    1105 steps at 16 x 16 points match dt = 0.5 h_min / |c|max with the smallest GLC spacing
    h_min = 0.5 (1 - cos(pi / 4)) / 2 = 0.0732 (10 / 0.00906 = 1104); the step count doubles
    with each doubling of the resolution.  nu = 1e-10, so tau = nu / dt + 1/2 is 1/2 to 1e-8.
    P = 1, so T = 1 / rho."""
    cells = points // 4
    steps = 1105 * (points // 16) * step_factor
    U, t_end, nu = 0.2, 10.0, 1e-10
    dt = t_end / steps
    return Workload(f"sdp{points}_p4", cells, cells, 4, -1.0, 1.0, -1.0, 1.0, PERIODIC, PERIODIC,
                    dt, nu / dt + 0.5, steps, "sdp", seed=7, extra={"U": U, "t_end": t_end})


# ---------------------------------------------------------------------------------------------
# 3D (the extension the paper names as its next step: D3Q125 on hexahedral cells)
# ---------------------------------------------------------------------------------------------
C_MAX_3D = math.sqrt(3.0 * (5.0 + math.sqrt(10.0)))   # largest D3Q125 speed, 4.9487


@dataclasses.dataclass
class Workload3:
    name: str
    cells: tuple
    order: int
    box: tuple                     # ((x0, x1), (y0, y1), (z0, z1))
    periodic: bool
    dt: float
    tau: float
    steps: int
    cv: float = CV
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def shape(self):               # (nz, ny, nx) vertices
        n = [c * self.order + (0 if self.periodic else 1) for c in self.cells]
        return (n[2], n[1], n[0])

    @property
    def n_vertices(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    @property
    def n_populations(self):
        return 1 if self.cv == 1.5 else 2

    @property
    def updates_per_step(self):
        return self.n_vertices * 125 * self.n_populations

    def fields(self, x, y, z):
        """The 3D Taylor-Green vortex: u = U0 sin x cos y cos z, v = -U0 cos x sin y cos z, w = 0,
        p = 1 + (U0^2 / 16)(cos 2x + cos 2y)(cos 2z + 2), rho = 1, T = p / rho."""
        U0 = self.extra["U0"]
        x, y, z = (np.asarray(a, np.float64) for a in (x, y, z))
        u = U0 * np.sin(x) * np.cos(y) * np.cos(z)
        v = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
        w = np.zeros_like(x)
        p = 1.0 + U0 ** 2 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
        return np.ones_like(x), u, v, w, p


def tgv3d(cells=64, order=2, ma=0.1, re=1600.0, steps=100):
    """3D Taylor-Green vortex on the periodic box [0, 2 pi]^3, cells^3 hexahedral cells of order
    p: U0 = Ma c_s, nu = U0 / Re (unit length), dt from CFL 0.5 on the vertex spacing with
    respect to the largest D3Q125 speed."""
    L = 2.0 * math.pi
    h = L / (cells * order)
    dt = 0.5 * h / C_MAX_3D
    nu = ma / re
    return Workload3(f"tgv3d{cells}_p{order}", (cells, cells, cells), order, ((0.0, L),) * 3, True,
                     dt, nu / dt + 0.5, steps, extra={"U0": ma})


def _named(w, name):
    w.name = name
    return w


ALL = {"tgv16": tgv16, "tgv256": tgv256, "sod": sod, "riemann": riemann,
       "riemann_paper": riemann_paper,
       # the same Table III problem on 512 x 512 cells (p = 3): a profiling case of the
       # headline kernel with a state (2 x 472 MB) still larger than L2
       "riemann_paper512": lambda: _named(riemann_paper().resized(512, 512, keep_tau=True),
                                          "riemann512_p3_tableIII"),
       "riemann_glc": riemann_nodes,
       "riemann_equidistant": lambda: riemann_nodes("equidistant"), "svi": svi, "svi_pr": svi_pr, "sdp": sdp,
       "tgv_moving": tgv_moving,
       # the moving vortex on 2048 x 2048 vertices (state larger than L2), both velocity sets
       "tgvm2048": lambda: tgv_moving(2048, 0.05), "tgvm2048_d2q9": lambda: tgv_moving(2048, 0.05, "d2q9")}
