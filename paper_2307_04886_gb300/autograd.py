"""torch.autograd.Function for x = A(t)^-1 M u0 with A(t) = M + t L
(Eq. (smoothing)), solved by the GPU multigrid library.

forward : b = M u0 (gmg_mass), x = A(t)^-1 b (gmg_solve);
backward: lambda = A(t)^-1 g with the same hierarchy (A is symmetric: the
          adjoint system is the primal one) at the forward's own t (the
          shared solver is moved back to it if another forward changed it),
          then gmg_grad gives
          dloss/du0 = M lambda and dloss/dt = -lambda^T L x.
Only argument marshalling happens here; every step runs in libgmg's kernels.
"""
from __future__ import annotations

import torch


class MultigridSmooth(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, u0, solver, tol: float = 1e-12):
        tv = float(t)
        if tv != solver.t:
            solver.set_t(tv)
        b = solver.mass(u0.contiguous())
        x = torch.zeros_like(b)
        solver.solve(b, x, tol=tol)
        ctx.solver, ctx.tol, ctx.t = solver, tol, tv
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        # the adjoint system is A(t) of THIS forward: another forward on the
        # same solver may have moved it to a different t since
        if solver.t != ctx.t:
            solver.set_t(ctx.t)
        lam = torch.zeros_like(x)
        solver.solve(g.contiguous(), lam, tol=ctx.tol)
        g_u0, dldt, _ = solver.grad(lam, x)
        return dldt.reshape(()), g_u0, None, None


def smooth(t, u0, solver, tol: float = 1e-12):
    """x = (M + t L)^-1 M u0, differentiable in t and u0."""
    return MultigridSmooth.apply(t, u0, solver, tol)
