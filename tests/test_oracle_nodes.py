"""Support points of the cell interpolation: equidistant versus Gauss-Lobatto-Chebyshev (Sec. II.E).

The paper uses Gauss-Lobatto-Chebyshev points because equidistant interpolation is stable for
low orders only; at p = 4 its 2D Riemann run with equidistant nodes diverged shortly after 200
steps while the Gauss-Lobatto-Chebyshev run stayed stable (Sec. III.D).  The streaming step is a
linear map of the stored field, so its stability shows in the spectral radius of that map:
built here column by column from the oracle's own streaming (the departure points and Lagrange
weights of Eq. sl_streaming) on a periodic axis, for the departure shifts a time step can give.
The equidistant p = 4 map amplifies some mode by far more than one per step -- the Runge
phenomenon of equidistant high-order interpolation -- while the Gauss-Lobatto-Chebyshev map stays
at one to within a few parts in 10^4; at p <= 2 the two node families coincide.
"""
import numpy as np
import pytest

from oracle import sllbm as o


def _streaming_radius(nodes, p, shift_cells, cells=8):
    """Largest |eigenvalue| of the periodic 1D streaming map of the velocity with x component
    +sqrt(5 + sqrt 10) and y component 0 when its departure lies shift_cells cells upwind."""
    ax = o.Axis(cells, p, 0.0, 1.0, True, nodes)
    ay = o.Axis(2, p, 0.0, 1.0, True, nodes)
    grid = o.Grid(ax, ay)
    xi, _ = o.d1q5()
    dt = shift_cells * ax.hc / xi[2]
    dep = o.Departures(grid, dt)
    i = 5 * 2 + 0                     # a = 2 (large positive x component), b = 0 (rest in y)
    n = grid.nx
    M = np.zeros((n, n))
    for j in range(n):
        F = np.zeros((25, grid.ny, n))
        F[i, :, j] = 1.0
        M[:, j] = o.stream(F, dep)[i, 0, :]
    return float(np.max(np.abs(np.linalg.eigvals(M))))


SHIFTS = np.linspace(0.02, 0.98, 13)


def test_equidistant_order4_streaming_amplifies():
    r = max(_streaming_radius("equidistant", 4, s) for s in SHIFTS)
    assert r > 1.3, r


def test_glc_order4_streaming_is_neutral():
    r = max(_streaming_radius("glc", 4, s) for s in SHIFTS)
    assert r < 1.001, r


@pytest.mark.parametrize("p", [1, 2])
def test_low_orders_coincide(p):
    """GLC and equidistant points are the same set for p <= 2: identical maps."""
    for s in (0.13, 0.5, 0.87):
        assert abs(_streaming_radius("glc", p, s) - _streaming_radius("equidistant", p, s)) < 1e-12
        assert _streaming_radius("glc", p, s) <= 1.0 + 1e-12
