"""Exact solution of the Riemann problem for the 1D Euler equations of an ideal gas.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.  Used to validate the oracle on the Sod
shock tube (Sec. III.C); it is not part of the SLLBM.  Written from the gas-dynamics relations:
the star-region pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, with f_K the shock
(Rankine-Hugoniot) branch for p > p_K and the rarefaction (isentropic) branch otherwise,
solved by Newton's method; the solution is then sampled along x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_branch(p, rho_k, p_k, c_k, gamma):
    if p > p_k:  # shock
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        root = math.sqrt(A / (p + B))
        return (p - p_k) * root, root * (1.0 - 0.5 * (p - p_k) / (B + p))
    ratio = p / p_k  # rarefaction
    f = 2.0 * c_k / (gamma - 1.0) * (ratio ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
    df = 1.0 / (rho_k * c_k) * ratio ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    """Pressure and velocity of the star region between the two nonlinear waves."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _f_branch(p, rl, pl, cl, gamma)
        fr, dfr = _f_branch(p, rr, pr, cr, gamma)
        g = fl + fr + (ur - ul)
        p_new = max(1e-14, p - g / (dfl + dfr))
        if abs(p_new - p) < 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f_branch(p, rl, pl, cl, gamma)
    fr, _ = _f_branch(p, rr, pr, cr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, gamma, s):
    """Density, velocity and pressure at similarity coordinates s = (x - x0) / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    ps, us = star_state(left, right, gamma)
    g = gamma
    s = np.asarray(s, dtype=np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    for k, sk in np.ndenumerate(s):
        if sk <= us:  # left of the contact
            if ps > pl:  # left shock
                shock = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if sk <= shock:
                    rho[k], u[k], p[k] = rl, ul, pl
                else:
                    r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                    rho[k], u[k], p[k] = r, us, ps
            else:  # left rarefaction
                head = ul - cl
                c_star = cl * (ps / pl) ** ((g - 1) / (2 * g))
                tail = us - c_star
                if sk <= head:
                    rho[k], u[k], p[k] = rl, ul, pl
                elif sk >= tail:
                    rho[k], u[k], p[k] = rl * (ps / pl) ** (1 / g), us, ps
                else:
                    uu = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + sk)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - sk))
                    rho[k] = rl * (c / cl) ** (2 / (g - 1))
                    u[k] = uu
                    p[k] = pl * (c / cl) ** (2 * g / (g - 1))
        else:  # right of the contact
            if ps > pr:  # right shock
                shock = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if sk >= shock:
                    rho[k], u[k], p[k] = rr, ur, pr
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    rho[k], u[k], p[k] = r, us, ps
            else:  # right rarefaction
                head = ur + cr
                c_star = cr * (ps / pr) ** ((g - 1) / (2 * g))
                tail = us + c_star
                if sk >= head:
                    rho[k], u[k], p[k] = rr, ur, pr
                elif sk <= tail:
                    rho[k], u[k], p[k] = rr * (ps / pr) ** (1 / g), us, ps
                else:
                    uu = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + sk)
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - sk))
                    rho[k] = rr * (c / cr) ** (2 / (g - 1))
                    u[k] = uu
                    p[k] = pr * (c / cr) ** (2 * g / (g - 1))
    return rho, u, p
