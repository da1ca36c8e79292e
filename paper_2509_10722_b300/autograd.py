"""PyTorch autograd for the unrolled PMP map (c, w) -> x after a fixed number of iterations.

`solve_x(problem, c, w, iters)` runs `iters` iterations from the zero state on the GPU (the
C ABI) and returns x; its backward is the library's hand-written adjoint (`num_adjoint`):
transposed gathers over R and the prox Jacobians, run backwards through the iterations
from checkpoints.  Each iteration's rho is the one the forward run takes (the map is
differentiated with the rho schedule held fixed).  `total_utility` builds
sum_j U_j(x_j) on top, so torch adds the direct dependence of U on w.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class PMPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, w, problem, iters, checkpoint_every):
        problem.set_capacity(c.detach().double().cpu().numpy())
        problem.set_weights(w.detach().double().cpu().numpy())
        problem.reset()
        problem.solve(int(iters), 0.0)
        x, _, _ = problem.get(prices=False)
        ctx.problem = problem
        ctx.iters = int(iters)
        ctx.kc = int(checkpoint_every)
        ctx.save_for_backward(c, w)
        return torch.as_tensor(x, dtype=torch.float64, device=c.device)

    @staticmethod
    def backward(ctx, xbar):
        c, w = ctx.saved_tensors
        p = ctx.problem
        p.set_capacity(c.detach().double().cpu().numpy())
        p.set_weights(w.detach().double().cpu().numpy())
        cg, wg, _ = p.adjoint(ctx.iters, ctx.kc, xbar=xbar.detach().double().cpu().numpy(),
                              objective=False)
        return (torch.as_tensor(cg, dtype=c.dtype, device=c.device),
                torch.as_tensor(wg, dtype=w.dtype, device=w.device), None, None, None)


def solve_x(problem, c, w, iters, checkpoint_every=50):
    """x after `iters` PMP iterations from zero for capacities c [m] and weights w [n]
    (float64 tensors); differentiable in c and w."""
    return PMPSolve.apply(c, w, problem, iters, checkpoint_every)


def total_utility(problem, utype, c, w, iters, checkpoint_every=50):
    """sum_j U_j(x_j) (w log x for utype 0, w x for 1, -w / x for 2) at the x of `iters`
    iterations."""
    x = solve_x(problem, c, w, iters, checkpoint_every)
    t = np.asarray(utype)
    is_log = torch.as_tensor(t == 0, device=x.device)
    is_a2 = torch.as_tensor(t == 2, device=x.device)
    safe = torch.where(is_log | is_a2, x, torch.ones_like(x))
    return torch.where(is_log, w * torch.log(safe),
                       torch.where(is_a2, -w / safe, w * x)).sum()
