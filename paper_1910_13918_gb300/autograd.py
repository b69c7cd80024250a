"""Checkpointed adjoint of an SLLBM rollout behind ``torch.autograd.Function``.

Forward: initial equilibrium of (rho0, u0, v0, T0) (Sec. II.A, II.D), ``nsteps`` fused steps, and
the final density field.  Backward: the hand-written adjoint of the C library, run in reverse over
segments of ``k`` steps.  Only every k-th state is kept; each segment is recomputed forward once
by steps that also write the per-step moments (rho, u, v, theta) the collision Jacobian needs
(the step kernels' own epilogue, no separate moments pass), then the adjoint steps walk back
through it.  The paper has no adjoint; this is its discrete transpose.
"""
from __future__ import annotations

import torch

from .sllbm import SLLBM


class SLLBMRollout(torch.autograd.Function):
    """rho_final = SLLBMRollout.apply(u0, v0, sim, rho0, T0, nsteps, k).

    ``u0``, ``v0``: float64 CUDA tensors of shape (ny, nx), the differentiated initial velocity.
    ``rho0``, ``T0``: float64 tensors held fixed.  Returns rho after ``nsteps`` (float64, (ny, nx)).
    """

    @staticmethod
    def forward(ctx, u0, v0, sim: SLLBM, rho0, T0, nsteps: int, k: int):
        with torch.cuda.stream(sim._stream):
            sim.init(rho0, u0, v0, T0)
            checkpoints = {0: sim.get_state().clone()}
            for n in range(nsteps):
                sim.step(1)
                if (n + 1) % k == 0 and n + 1 < nsteps:
                    checkpoints[n + 1] = sim.get_state().clone()
            rho = sim.moments(sums=False)["rho"].double()
        ctx.sim, ctx.nsteps, ctx.k, ctx.checkpoints = sim, nsteps, k, checkpoints
        ctx.save_for_backward(u0, v0, rho0, T0)
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        sim, nsteps, k, checkpoints = ctx.sim, ctx.nsteps, ctx.k, ctx.checkpoints
        u0, v0, rho0, T0 = ctx.saved_tensors
        ny, nx = sim.ny, sim.nx
        with torch.cuda.stream(sim._stream):
            lam = torch.zeros((2, 25, ny, nx), dtype=torch.float32, device=sim.device)
            lam[0] = grad_rho.float().reshape(1, ny, nx)   # d rho / d f_i = 1, d rho / d g_i = 0
            lam_out = torch.empty_like(lam)
            moments = torch.empty((k, 4, ny, nx), dtype=torch.float32, device=sim.device)
            for start in reversed(range(0, nsteps, k)):
                end = min(start + k, nsteps)
                sim.set_state(checkpoints[start])
                for j in range(end - start):
                    sim.step_moments(moments[j])          # the moments step start + j + 1 used
                for j in reversed(range(end - start)):
                    sim.adjoint_step(lam, lam_out, moments[j])
                    lam, lam_out = lam_out, lam
            du, dv = sim.init_vjp(rho0, u0, v0, T0, lam)
        return du.double(), dv.double(), None, None, None, None, None


def rollout(sim: SLLBM, u0, v0, rho0, T0, nsteps: int, k: int = 20):
    return SLLBMRollout.apply(u0, v0, sim, rho0, T0, nsteps, k)
