"""GPU adjoint (C ABI) against the oracle's FP64 reference adjoint and finite differences."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oa
from oracle import sllbm as o
from paper_1910_13918_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu

TOL_ADJ = 1e-4


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _small_cases():
    return {"svi_mapped": H.small_workloads()["svi"],
            "tgv_uniform": W.tgv256().resized(6, 5),
            "sod_uniform": H.small_workloads()["sod"],
            # several 32 x 32 tiles of the one-pass S^T with ragged edges, clamped on both axes
            "riemann_uniform": W.riemann_paper().resized(14, 12, keep_tau=True),
            # 4 times the CFL time step: transposed-stencil halo 5 (over 4), the one-pass S^T
            # compiled for halo 8
            "tgv_mid_uniform": _far(W.tgv256().resized(6, 5), 4.0),
            # 16 times the CFL time step: departure points about 8 nodes away, halo 9, beyond the
            # one-pass S^T, so the adjoint takes the two-pass S^T over the (f, g) pairs
            "tgv_far_uniform": _far(W.tgv256().resized(6, 5), 16.0)}


def _far(w, factor):
    return w.resized(w.nx_cells, w.ny_cells, steps=w.steps, dt=factor * W.cfl_dt(w))


@pytest.mark.parametrize("name", ["svi_mapped", "tgv_uniform", "sod_uniform", "riemann_uniform",
                                  "tgv_mid_uniform", "tgv_far_uniform"])
def test_adjoint_step_matches_oracle(gpu_lib, name):
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = _small_cases()[name]
    n0 = 3
    # oracle: state after n0 steps, then one adjoint step of a seeded random lambda
    grid = H.oracle_grid(w)
    X, Y = grid.coords()
    dep = o.Departures(grid, w.dt)
    f, g = o.initial_state(*w.fields(X, Y, perturb=True), w.cv)
    f, g = o.run(f, g, dep, w.tau, w.cv, n0)
    rng = np.random.default_rng(7)
    lam = rng.standard_normal((2, 25, grid.ny, grid.nx))
    ref_f, ref_g = oa.adjoint_step(f, g, lam[0], lam[1], dep, w.tau, w.cv)
    # GPU: same fields and steps on its own, then step once for the moments, then the adjoint
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    s.step(n0 + 1)
    mom = torch.empty((4, s.ny, s.nx), dtype=torch.float32, device="cuda")
    s.moments_into(mom)
    lam_in = torch.as_tensor(lam, dtype=torch.float32, device="cuda").contiguous()
    lam_out = torch.empty_like(lam_in)
    s.adjoint_step(lam_in, lam_out, mom)
    out = lam_out.cpu().numpy()
    assert _rel(out[0], ref_f) < TOL_ADJ and _rel(out[1], ref_g) < TOL_ADJ, \
        (_rel(out[0], ref_f), _rel(out[1], ref_g))


def test_checkpointed_rollout_gradient_matches_oracle(gpu_lib):
    """dJ/du0, dJ/dv0 of J = sum_{x > 1} A_v rho_v(t_N) on a small mapped shock-vortex grid."""
    from paper_1910_13918_gb300.autograd import rollout
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = H.small_workloads()["svi"]
    nsteps, k = 10, 4
    grid = H.oracle_grid(w)
    X, Y = grid.coords()
    rho0, u0, v0, T0 = w.fields(X, Y)
    weight = grid.vertex_weights() * (X > 1.0)
    J_ref, du_ref, dv_ref = oa.rollout_gradient(rho0, u0, v0, T0, o.Departures(grid, w.dt),
                                                w.tau, w.cv, nsteps, weight)
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    r, u, v, T = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in w.fields(x, y))
    u.requires_grad_(True)
    v.requires_grad_(True)
    A = s.vertex_weights()
    xt = torch.as_tensor(x, device="cuda")
    rho = rollout(s, u, v, r, T, nsteps, k)
    J = (A * (xt > 1.0) * rho).sum()
    J.backward()
    assert abs(float(J.detach()) / J_ref - 1) < 1e-5
    assert _rel(u.grad.cpu().numpy(), du_ref) < TOL_ADJ, _rel(u.grad.cpu().numpy(), du_ref)
    assert _rel(v.grad.cpu().numpy(), dv_ref) < TOL_ADJ, _rel(v.grad.cpu().numpy(), dv_ref)
