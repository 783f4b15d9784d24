"""torch.autograd bindings of the DUGKS forward run and its adjoint.

Argument marshalling only: the forward steps run in the library's kernels
(``dugks_step``) and the backward pass in its hand-written adjoint kernels
with checkpointed recomputation (``dugks_adjoint_run``).  All tensors are
FP64 CUDA tensors on the current device and stream.

* :class:`T3S3Run` -- ``fhatN = T3S3Run.apply(fhat0, tau, uw, problem, nsteps, every)``
  with ``tau`` a 0-d tensor and ``uw`` a (4, 2) tensor of wall velocities
  (west, east, south, north); gradients flow to ``fhat0``, ``tau`` and ``uw``.
* :class:`Equilibrium` -- ``fhat0 = Equilibrium.apply(rho, ux, uy, problem)``,
  the equilibrium initialisation (gradients to rho, ux, uy).

``problem`` is a :class:`Problem` (mesh, velocity set, dt, wall kinds).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import (Solver, dugks_adjoint_equilibrium, dugks_adjoint_run, dugks_get_state,
               dugks_set_equilibrium)


@dataclass
class Problem:
    nx: int
    ny: int
    dx: float
    dy: float
    xi: np.ndarray
    W: np.ndarray
    RT: float
    dt: float
    kinds: tuple          # boundary kind per side (west, east, south, north)

    def solver(self, tau: float, uw) -> Solver:
        uw = np.asarray(uw, dtype=np.float64).reshape(4, 2)
        bc = [(int(k), float(uw[s, 0]), float(uw[s, 1])) for s, k in enumerate(self.kinds)]
        return Solver(self.nx, self.ny, self.dx, self.dy, self.xi, self.W, self.RT, float(tau),
                      self.dt, bc, stream=torch.cuda.current_stream())


class T3S3Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fhat0, tau, uw, problem: Problem, nsteps: int, every: int):
        solver = problem.solver(float(tau), uw.detach().cpu().numpy())
        f0 = fhat0.detach().contiguous()
        solver.set_state(f0)
        solver.step(int(nsteps))
        out = torch.empty_like(f0)
        dugks_get_state(solver.ctx, out)
        ctx.solver, ctx.nsteps, ctx.every = solver, int(nsteps), int(every)
        ctx.save_for_backward(f0)
        return out

    @staticmethod
    def backward(ctx, grad):
        (f0,) = ctx.saved_tensors
        lam0 = torch.empty_like(f0)
        dtau, duw = dugks_adjoint_run(ctx.solver.ctx, f0, ctx.nsteps, ctx.every,
                                      grad.contiguous(), lam0)
        dev = f0.device
        return (lam0, torch.tensor(dtau, dtype=torch.float64, device=dev),
                torch.tensor(duw, dtype=torch.float64, device=dev), None, None, None)


class Equilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, ux, uy, problem: Problem):
        solver = problem.solver(1.0, np.zeros((4, 2)))
        r, u, v = (t.detach().contiguous() for t in (rho, ux, uy))
        dugks_set_equilibrium(solver.ctx, r, u, v)
        out = torch.empty((len(problem.W), problem.ny, problem.nx), dtype=torch.float64,
                          device=rho.device)
        dugks_get_state(solver.ctx, out)
        ctx.solver = solver
        ctx.save_for_backward(r, u, v)
        return out

    @staticmethod
    def backward(ctx, grad):
        r, u, v = ctx.saved_tensors
        dr, du, dv = torch.empty_like(r), torch.empty_like(u), torch.empty_like(v)
        dugks_adjoint_equilibrium(ctx.solver.ctx, r, u, v, grad.contiguous(), dr, du, dv)
        return dr, du, dv, None
