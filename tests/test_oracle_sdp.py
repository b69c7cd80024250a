"""The oracle on the paper's smooth density propagation (Sec. III.B, Table II).

The printed errors of Table II bound the scheme from above: the oracle, which runs the same
method on the same grid for the same number of steps, must carry the density wave across the
domain at least that accurately.  A dropped or mis-signed term (in the equilibrium, the departure
points or the interpolation) moves the wave at the wrong speed or damps it, which the bound
catches: a wave that stood still would be off by up to 0.4.
"""
from paper_1910_13918_gb300 import workloads as W

from . import helpers as H


def test_oracle_smooth_density_propagation_16x16_within_table2():
    w = W.sdp(16)
    rho, _, _, _ = H.oracle_run(w, w.steps, perturb=False)
    X, Y = H.oracle_grid(w).coords()
    err = H.sdp_error(w, rho, X, Y)
    assert err < H.table2()[16], err
    # the exact solution itself is not the initial field shifted by a wrong amount
    assert H.sdp_error(w, W.sdp_density(w, X, Y, 0.5 * w.extra["t_end"]), X, Y) > 0.3
