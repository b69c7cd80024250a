"""Reference adjoint of the SLLBM step in float64.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.  The paper has no adjoint; this is the
plain transpose of the discrete step of ``oracle.sllbm`` built two ways that share nothing with
the CUDA path:

* the collision Jacobian J_C (a dense 50 x 50 matrix per vertex) is obtained column by column by
  complex-step differentiation of ``oracle.sllbm.collide`` (exact to rounding: no subtraction),
  and applied transposed;
* the interpolation operator is applied transposed by an explicit scatter (``np.add.at``) over the
  same stencils the forward pull gathers from.

Step map:  s_{n+1} = C(S s_n),  so  lambda_n = S^T J_C(S s_n)^T lambda_{n+1}.
"""
from __future__ import annotations

import numpy as np

from . import sllbm as o

H_CS = 1e-30  # complex-step size


def collide_vjp(fpre, gpre, lam_f, lam_g, tau, cv):
    """J_C(q)^T lambda at every vertex, with q = (fpre, gpre) the pre-collision populations."""
    Qn = o.Q
    mu_f = np.zeros_like(fpre)
    mu_g = np.zeros_like(gpre)
    for pop in range(2):
        for i in range(Qn):
            fc = fpre.astype(np.complex128)
            gc = gpre.astype(np.complex128)
            if pop == 0:
                fc[i] = fc[i] + 1j * H_CS
            else:
                gc[i] = gc[i] + 1j * H_CS
            cf, cg = o.collide(fc, gc, tau, cv)
            col = np.sum(cf.imag / H_CS * lam_f, axis=0) + np.sum(cg.imag / H_CS * lam_g, axis=0)
            if pop == 0:
                mu_f[i] = col
            else:
                mu_g[i] = col
    return mu_f, mu_g


def stream_transpose(L, dep: o.Departures):
    """Transpose of ``oracle.sllbm.stream`` by scatter: out[i](node) += psi_a psi_b L[i](v)."""
    grid = dep.grid
    assert dep.vertices is None
    ax, ay, p = grid.ax, grid.ay, grid.p
    out = np.zeros_like(L)
    for i in range(o.Q):
        wx = o.lagrange(ax.nodes, dep.rx[i])
        wy = o.lagrange(ay.nodes, dep.ry[i])
        src = L[i].reshape(-1)
        for b in range(p + 1):
            jy = ay.vertex_of(dep.cy[i], b)
            for a in range(p + 1):
                jx = ax.vertex_of(dep.cx[i], a)
                np.add.at(out[i], (jy, jx), wx[:, a] * wy[:, b] * src)
    return out


def adjoint_step(f, g, lam_f, lam_g, dep, tau, cv):
    """lambda_n from lambda_{n+1}, given the state s_n = (f, g) the step started from."""
    fpre = o.stream(f, dep)
    gpre = o.stream(g, dep)
    mu_f, mu_g = collide_vjp(fpre, gpre, lam_f, lam_g, tau, cv)
    return stream_transpose(mu_f, dep), stream_transpose(mu_g, dep)


def init_vjp(rho0, u0, v0, T0, lam_f, lam_g, cv):
    """Gradient of <lambda, s_0(rho0, u0, v0, T0)> with respect to u0 and v0 (per vertex)."""
    out = []
    for comp in range(2):
        u = np.asarray(u0, dtype=np.complex128).copy()
        v = np.asarray(v0, dtype=np.complex128).copy()
        if comp == 0:
            u = u + 1j * H_CS
        else:
            v = v + 1j * H_CS
        f, g = o.initial_state(np.asarray(rho0, dtype=np.complex128), u, v,
                               np.asarray(T0, dtype=np.complex128), cv)
        out.append(np.sum(f.imag / H_CS * lam_f, axis=0) + np.sum(g.imag / H_CS * lam_g, axis=0))
    return out[0], out[1]


def rollout_gradient(rho0, u0, v0, T0, dep, tau, cv, nsteps, weight):
    """Value and gradient of J = sum_v weight_v rho_v(t_N) with respect to (u0, v0).

    Stores every intermediate state (no checkpointing is needed at oracle sizes).
    """
    f, g = o.initial_state(rho0, u0, v0, T0, cv)
    states = [(f, g)]
    for _ in range(nsteps):
        f, g = o.step(f, g, dep, tau, cv)
        states.append((f, g))
    J = float(np.sum(weight * f.sum(axis=0)))
    lam_f = np.broadcast_to(weight, f.shape).copy()
    lam_g = np.zeros_like(g)
    for n in range(nsteps - 1, -1, -1):
        fs, gs = states[n]
        lam_f, lam_g = adjoint_step(fs, gs, lam_f, lam_g, dep, tau, cv)
    du, dv = init_vjp(rho0, u0, v0, T0, lam_f, lam_g, cv)
    return J, du, dv


def objective(rho0, u0, v0, T0, dep, tau, cv, nsteps, weight):
    f, g = o.initial_state(rho0, u0, v0, T0, cv)
    f, g = o.run(f, g, dep, tau, cv, nsteps)
    return float(np.sum(weight * f.sum(axis=0)))
