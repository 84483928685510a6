"""Reverse mode through a rollout: d(outlet flux)/d(eps per cell).

``OutletFlux`` is a ``torch.autograd.Function``.  Its forward sets eps, runs
``nsteps`` steps of the porous LBM from rest and returns the outlet flux
J = sum over the plane x = x_out of eps*rho*u_x (Eq. 1moment) at the last step,
keeping a checkpoint of the state every ``every`` steps.  Its backward walks
the segments newest first: for each, one library call (vans_adjoint_segment,
a CUDA graph replayed per segment) restores the checkpoint, recomputes the
segment's states with the same step kernel (so they are bit-identical to the
forward ones), then applies the hand-written adjoint step kernel to them in
reverse, accumulating dJ/deps; a final kernel adds the initial condition
f = w eps and the transposed grad-eps stencil.
"""
from __future__ import annotations

import torch

from ._binding import Solver


class OutletFlux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, solver: Solver, nsteps: int, every: int, x_out: int):
        solver.set_eps(eps.detach().contiguous().view(-1))
        ckpts = []
        done = 0
        while done < nsteps:
            ckpts.append(solver.get_state())
            n = min(every, nsteps - done)
            solver.step(n)
            done += n
        final = solver.get_state()
        J = solver.flux(x_out, state=final)
        ctx.solver = solver
        ctx.meta = (nsteps, every, x_out)
        ctx.ckpts = ckpts
        ctx.final = final
        ctx.shape = eps.shape
        return J.view(())

    @staticmethod
    def backward(ctx, gJ):
        solver: Solver = ctx.solver
        nsteps, every, x_out = ctx.meta
        lam_a = solver.new_state()
        lam_b = solver.new_state()
        grad = torch.empty(solver.grad_floats(), dtype=torch.float32, device=solver.device)
        solver.flux_seed(x_out, lam_a, grad, state=ctx.final)
        seg = torch.zeros((every + 1, solver.state_floats), dtype=torch.float32,
                          device=solver.device)
        for s in reversed(range(len(ctx.ckpts))):
            start = s * every
            length = min(every, nsteps - start)
            # checkpoint -> recompute -> reverse sweep, one captured graph per segment shape
            solver.adjoint_segment(ctx.ckpts[s], seg, length, lam_a, lam_b, grad)
        dJ = solver.grad_finalize(lam_a, grad)
        return (dJ.view(ctx.shape) * gJ), None, None, None, None


def outlet_flux(eps, solver: Solver, nsteps: int, every: int = 100, x_out: int | None = None):
    """J(eps) with a gradient; x_out defaults to the last plane, nx - 1.  The
    reverse step runs in the precision set by ``solver.set_adjoint_precision``
    (32 by default; 64 for FP64 per-cell arithmetic on long rollouts)."""
    if x_out is None:
        x_out = solver.params.nx - 1
    return OutletFlux.apply(eps, solver, int(nsteps), int(every), int(x_out))
