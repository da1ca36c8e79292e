"""PyTorch autograd for the unrolled PMP map (c, w) -> x after a fixed number of iterations.

`solve_x(problem, c, w, iters)` runs `iters` iterations from the zero state on the GPU
(`num_adjoint_forward`: c and w are handed over as device arrays, checkpoints are kept in
the handle) and returns x; its backward is the library's hand-written adjoint
(`num_adjoint_backward`: transposed gathers over R and the prox Jacobians, run backwards
through the iterations from the kept checkpoints, cotangent and gradients as device
arrays), so the forward map runs once per forward call.  `total_utility` is the total
utility sum_j U_j(x_j) of the same map, evaluated and differentiated by the library as
well (its direct dependence on w included).  Each iteration's rho is the one the forward
run takes: the map is differentiated with the rho schedule held fixed.  This module only
moves tensors to and from the library; it does no arithmetic of its own.
"""
from __future__ import annotations

import torch

from . import capi


def _device_f64(t):
    return t.detach().to(device="cuda", dtype=torch.float64).contiguous()


def _forward(problem, c, w, iters, checkpoint_every):
    problem.set_capacity_device(_device_f64(c))
    problem.set_weights_device(_device_f64(w))
    problem.adjoint_forward(int(iters), int(checkpoint_every))
    token = object()
    problem._adjoint_token = token  # which forward the handle's kept checkpoints belong to
    return token


def _backward(ctx, xbar, ubar):
    c, w = ctx.saved_tensors
    p = ctx.problem
    if getattr(p, "_adjoint_token", None) is not ctx.token:
        # another forward ran on this handle since: run this one again
        ctx.token = _forward(p, c, w, ctx.iters, ctx.kc)
    cg = torch.empty(p.m, dtype=torch.float64, device="cuda")
    wg = torch.empty(p.n, dtype=torch.float64, device="cuda")
    p.adjoint_backward(xbar=xbar, ubar=ubar, c_grad=cg, w_grad=wg)
    return cg.to(device=c.device, dtype=c.dtype), wg.to(device=w.device, dtype=w.dtype)


class PMPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, w, problem, iters, checkpoint_every):
        ctx.problem, ctx.iters, ctx.kc = problem, int(iters), int(checkpoint_every)
        ctx.token = _forward(problem, c, w, iters, checkpoint_every)
        ctx.save_for_backward(c, w)
        x = torch.empty(problem.n, dtype=torch.float64, device="cuda")
        problem.get_device(x=x)
        return x.to(device=c.device)

    @staticmethod
    def backward(ctx, xbar):
        gc, gw = _backward(ctx, _device_f64(xbar), 0.0)
        return gc, gw, None, None, None


class PMPTotalUtility(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, w, problem, iters, checkpoint_every):
        ctx.problem, ctx.iters, ctx.kc = problem, int(iters), int(checkpoint_every)
        ctx.token = _forward(problem, c, w, iters, checkpoint_every)
        ctx.save_for_backward(c, w)
        info = problem.get_device()  # the library's FP64 sum of U_j(x_j) at the final rates
        return torch.tensor(info["objective"], dtype=torch.float64, device=c.device)

    @staticmethod
    def backward(ctx, gJ):
        gc, gw = _backward(ctx, None, float(gJ))
        return gc, gw, None, None, None


def solve_x(problem, c, w, iters, checkpoint_every=50):
    """x after `iters` PMP iterations from zero for capacities c [m] and weights w [n]
    (float64 tensors, caller order); differentiable in c and w."""
    return PMPSolve.apply(c, w, problem, iters, checkpoint_every)


def total_utility(problem, c, w, iters, checkpoint_every=50):
    """sum_j U_j(x_j) (w log x, w x or -w / x, by the handle's utility types) at the x of
    `iters` iterations; differentiable in c and w."""
    return PMPTotalUtility.apply(c, w, problem, iters, checkpoint_every)
