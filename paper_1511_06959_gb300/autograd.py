"""torch.autograd.Function over the checkpointed discrete adjoint.

Jbar(w0, theta) is the time-averaged pressure loss of each box (Eq. e:pressure_loss)
after N RK4 steps with the time-constant source s = sum_m theta_m phi_m on the
x-momentum equation, shared by all boxes (section "Unsteady adjoint": the source
sensitivity dJ = -int int w_hat ds, here in its discrete form).  Forward runs the
primal and keeps the planned checkpoints; backward runs the reverse sweep in the CUDA
library and returns dL/dw0 and dL/dtheta.  PyTorch only holds memory; every step is a
kernel of the library.
"""
from __future__ import annotations

import torch

from . import api


class SourceProblem:
    """A batch of periodic boxes, the source shapes phi[nphi][nz][ny][nx] and the sweep
    settings (steps, checkpoint schedule, added adjoint viscosity coefficient)."""

    def __init__(self, solver: api.Solver, phi: torch.Tensor, nsteps: int,
                 schedule: int = api.NS_CKPT_ALL, param: int = 0, lam_coef: float = 0.0,
                 tau: float = 0.0):
        if phi.dtype != torch.float64 or not phi.is_cuda:
            raise ValueError("phi must be a float64 CUDA tensor")
        self.S = solver
        self.phi = phi.reshape(phi.shape[0], -1).contiguous()
        if self.phi.shape[1] != solver.cells:
            raise ValueError("phi must hold one value per cell")
        self.opts = solver.run_opts(nsteps, schedule, param, lam_coef, tau)
        self.arena = torch.empty(solver.arena_bytes(self.opts), dtype=torch.uint8, device=phi.device)

    def source(self, theta: torch.Tensor) -> torch.Tensor:
        """s[b][1] = sum_m theta_m phi_m for every box, zero elsewhere (ns_combine)."""
        S = self.S
        s = torch.zeros(S.shape, dtype=torch.float64, device=self.phi.device)
        th = theta.detach().to(torch.float64).contiguous()
        for b in range(S.batch):
            S.combine(th, self.phi, s[b, 1])
        return s

    def __call__(self, w0: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
        return PressureLoss.apply(w0, theta, self)


class PressureLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w0, theta, problem: SourceProblem):
        S = problem.S
        w = w0.detach().contiguous()
        if w.dtype != torch.float64 or tuple(w.shape) != S.shape:
            raise ValueError(f"w0 must be float64 of shape {S.shape}")
        s = problem.source(theta)
        J = torch.empty(S.batch, dtype=torch.float64, device=w.device)
        S.forward_run(w, problem.opts, problem.arena, J, s)
        ctx.problem = problem
        ctx.generation = S.sweep_generation()   # this loss's trajectory
        ctx.keep = (w, s)            # the reverse sweep reads w0 and s again
        return J

    @staticmethod
    def backward(ctx, gJ):
        problem = ctx.problem
        S = problem.S
        w, s = ctx.keep
        if S.sweep_generation() != ctx.generation:
            raise RuntimeError(
                "PressureLoss.backward: the solver's checkpoints no longer hold this loss's "
                "trajectory (another forward ran on the same solver, or this one was already "
                "reversed); run backward before the next forward, or use one solver per loss")
        lam0 = torch.empty_like(w)
        sbar = torch.empty_like(w)
        S.backward_run(lam0, sbar)
        seed = gJ.detach().to(torch.float64).contiguous()
        S.scale_boxes(seed, lam0)
        S.scale_boxes(seed, sbar)
        gtheta = torch.empty(problem.phi.shape[0], dtype=torch.float64, device=w.device)
        S.dot_boxes(sbar, 1, problem.phi, gtheta)
        return lam0, gtheta, None
