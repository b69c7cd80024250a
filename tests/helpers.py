"""Shared test plumbing: build the oracle and the GPU side of one workload from the same seeds.

The two sides share only the workload description and its seeded field generator; each evaluates
the initial fields on its own vertex coordinates.
"""
from __future__ import annotations

import os

import numpy as np

from oracle import sllbm as o
from paper_1910_13918_gb300 import workloads as W


def oracle_grid(w: W.Workload):
    ax = o.Axis(w.nx_cells, w.order, w.x0, w.x1, w.bc_x == W.PERIODIC, w.nodes)
    ay = o.Axis(w.ny_cells, w.order, w.y0, w.y1, w.bc_y == W.PERIODIC, w.nodes)
    return o.Grid(ax, ay, o.SineMap(w.map_a) if w.map_a else None)


def oracle_state(w: W.Workload, nsteps, perturb=True):
    """Oracle post-collision populations (f, g) after nsteps, each (25, ny, nx) float64."""
    grid = oracle_grid(w)
    X, Y = grid.coords()
    q = w.n_velocities
    f, g = o.initial_state(*w.fields(X, Y, perturb=perturb), w.cv, q)
    return o.run(f, g, o.Departures(grid, w.dt, q=q), w.tau, w.cv, nsteps, w.pr, w.isothermal)


def oracle_run(w: W.Workload, nsteps, perturb=True):
    """(rho, u, v, theta) of the oracle after nsteps, each (ny, nx) float64."""
    f, g = oracle_state(w, nsteps, perturb)
    rho, u, th = o.macroscopic(f, g, w.cv)
    return rho, u[..., 0], u[..., 1], th


class SparseField:
    """Population field known only on a set of vertices, indexable like F[i, jy, jx]."""

    def __init__(self, nx, keys, values):
        self.nx = nx
        order = np.argsort(keys)
        self.keys = keys[order]
        self.values = values[:, order]

    def __getitem__(self, idx):
        i, jy, jx = idx
        k = np.asarray(jy) * self.nx + np.asarray(jx)
        pos = np.searchsorted(self.keys, k)
        assert np.all(self.keys[pos] == k), "stencil vertex outside the sampled support"
        return self.values[i][pos]

    @property
    def dtype(self):
        return self.values.dtype

    @property
    def shape(self):
        """Leading (velocity) axis only: the vertex axes are sparse."""
        return self.values.shape[:1]


def oracle_step_at(w: W.Workload, vertices, perturb=True):
    """Oracle (rho, u, v, theta) after ONE step at the given flat vertex indices only.

    The initial equilibrium is evaluated only on the vertices the stencils of those departure
    points touch, so full-size grids stay cheap.
    """
    grid = oracle_grid(w)
    X, Y = grid.coords()
    q = w.n_velocities
    dep = o.Departures(grid, w.dt, vertices, q=q)
    keys = []
    for i in range(q):
        for b in range(grid.p + 1):
            jy = grid.ay.vertex_of(dep.cy[i], b)
            for a in range(grid.p + 1):
                jx = grid.ax.vertex_of(dep.cx[i], a)
                keys.append(jy * grid.nx + jx)
    keys = np.unique(np.concatenate(keys))
    fields = w.fields(X, Y, perturb=perturb)
    sub = [np.asarray(F).reshape(-1)[keys] for F in fields]
    f0, g0 = o.initial_state(*sub, w.cv, q)
    fpre = o.stream(SparseField(grid.nx, keys, f0), dep)
    gpre = o.stream(SparseField(grid.nx, keys, g0), dep)
    f1, g1 = o.collide(fpre, gpre, w.tau, w.cv, w.pr, w.isothermal)
    rho, u, th = o.macroscopic(f1, g1, w.cv)
    return rho, u[..., 0], u[..., 1], th


def field_errors(gpu, ref, velocity_scale=0.0):
    """Max relative error per field: rho and T pointwise relative; u and v relative to the larger
    of max |u_ref| and the workload's characteristic speed (a flow starting at rest has no
    velocity of its own to be relative to)."""
    rho_g, u_g, v_g, t_g = (np.asarray(a, dtype=np.float64) for a in gpu)
    rho_r, u_r, v_r, t_r = (np.asarray(a, dtype=np.float64) for a in ref)
    umax = max(np.max(np.abs(u_r)), np.max(np.abs(v_r)), velocity_scale, 1e-12)
    return {
        "rho": float(np.max(np.abs(rho_g - rho_r) / np.abs(rho_r))),
        "u": float(np.max(np.abs(u_g - u_r)) / umax),
        "v": float(np.max(np.abs(v_g - v_r)) / umax),
        "T": float(np.max(np.abs(t_g - t_r) / np.abs(t_r))),
    }


def small_workloads():
    """Reduced-size versions of the five workloads: several tiles and ragged tails."""
    return {
        "tgv16": W.tgv16(),
        "tgv256": W.tgv256().resized(9, 7, steps=100),
        "sod": _sod_small(),
        "riemann": W.riemann_paper().resized(20, 21, steps=100, keep_tau=True),
        "svi": _svi_small(),
    }


def _sod_small():
    w = W.sod().resized(64, 2, steps=100, keep_tau=True)
    w.y1 = w.y0 + (w.x1 - w.x0) / 64 * 2
    return w


def _svi_small():
    w = W.svi().resized(24, 12, steps=100, dt=0.01)
    return w


def table2():
    """The paper's smooth-density-propagation errors (Sec. III.B, Table II), tests/golden."""
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "sdp_table2.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, err, _ = line.split()
                out[int(n)] = float(err)
    return out


def sdp_error(w: W.Workload, rho, x, y):
    """max |rho - rho_exact| at the end of a smooth-density-propagation run."""
    return float(np.max(np.abs(rho - W.sdp_density(w, x, y, w.extra["t_end"]))))
