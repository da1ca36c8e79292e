"""CPU reference gradient of unrolled PMP -- TEST INFRASTRUCTURE ONLY.

The literal per-terminal ADMM of Sec. III-D..G (the same steps as pmp_oracle.c: stream
prox, link averages, over-relaxation, z projection, u update, residual balancing with a
GIVEN list of rho decisions, then the dual rescale) written with plain PyTorch CPU
operations in float64, so that torch.autograd differentiates the K-step map (c, w) -> x_K
exactly (the rho schedule is an input, not differentiated).  Used to check the GPU adjoint.
Pinned by tests/test_oracle_adjoint_ref.py: its x equals the C oracle's, and its gradients
equal central finite differences of the C oracle.
"""
from __future__ import annotations

import numpy as np
import torch


def _segment_sum(values, index, size):
    out = torch.zeros(size, dtype=values.dtype)
    return out.index_add(0, index, values)


def _alpha2_root(S, L, w, rho):
    """Positive root of rho L x^3 - rho S x^2 - w (U = -w / x): bisection without
    gradient, then one Newton step with it, whose derivative at the root is the implicit
    derivative -f_theta / f_x."""
    with torch.no_grad():
        a = torch.zeros_like(S)
        b = torch.clamp(S, min=0.0) / L + torch.pow(w / (rho * L), 1.0 / 3.0)
        for _ in range(200):
            mid = 0.5 * (a + b)
            f = rho * L * mid ** 3 - rho * S * mid ** 2 - w
            b = torch.where(f > 0, mid, b)
            a = torch.where(f > 0, a, mid)
        x0 = 0.5 * (a + b)
    f = rho * L * x0 ** 3 - rho * S * x0 ** 2 - w
    fx = 3.0 * rho * L * x0 ** 2 - 2.0 * rho * S * x0
    return x0 - f / fx


def unrolled_x(inst, iters, c, w, decisions, rho0=1.0, alpha=1.6, period=50):
    """x after `iters` literal PMP iterations from zero; c [m], w [n] float64 tensors (may
    require grad); decisions = the rho decision (+1, 0, -1) at each update point."""
    n, m = int(inst["n"]), int(inst["m"])
    ptr = np.asarray(inst["route_ptr"], np.int64)
    nnz = int(ptr[-1])
    J = nnz + m
    lengths = np.diff(ptr)
    stream_of = torch.as_tensor(np.repeat(np.arange(n), lengths))
    link_of = torch.as_tensor(np.concatenate([np.asarray(inst["route_links"], np.int64),
                                              np.arange(m)]))
    L = torch.as_tensor(lengths, dtype=torch.float64)
    cnt = _segment_sum(torch.ones(J, dtype=torch.float64), link_of, m)
    is_log = torch.as_tensor(np.asarray(inst["utype"]) == 0)
    is_a2 = torch.as_tensor(np.asarray(inst["utype"]) == 2)
    lo = torch.as_tensor(np.asarray(inst["lo"], np.float64))
    hi = torch.as_tensor(np.asarray(inst["hi"], np.float64))
    p = torch.zeros(J, dtype=torch.float64)
    z = torch.zeros(J, dtype=torch.float64)
    u = torch.zeros(J, dtype=torch.float64)
    rho = float(rho0)
    n_up = 0
    x = torch.zeros(n, dtype=torch.float64)
    for k in range(1, iters + 1):
        zeta = z - u
        S = _segment_sum(zeta[:nnz], stream_of, n)
        D = S * S + 4.0 * w * L / rho
        sq = torch.sqrt(D)
        x_log = torch.where(S >= 0, (S + sq) / (2.0 * L), (2.0 * w / rho) / (sq - S))
        x_lin = (S + w / rho) / L
        x_a2 = _alpha2_root(S, L, w, rho)
        x = torch.clamp(torch.where(is_log, x_log, torch.where(is_a2, x_a2, x_lin)), min=lo, max=hi)
        p = torch.cat([x[stream_of], torch.maximum(zeta[nnz:], -c)])
        pplus = alpha * p + (1.0 - alpha) * z
        v = pplus + u
        z = v - (_segment_sum(v, link_of, m) / cnt)[link_of]
        u = u + pplus - z
        if period > 0 and k % period == 0 and k < iters:
            dec = int(decisions[n_up]) if n_up < len(decisions) else 0
            n_up += 1
            rho_new = rho * 1.1 if dec > 0 else (rho / 1.1 if dec < 0 else rho)
            u = u * (rho / rho_new)
            rho = rho_new
    return x


def gradients(inst, iters, decisions, xbar=None, objective=True, **kw):
    """(dJ/dc, dJ/dw, J) for J = xbar . x_K + [objective] sum_j U_j(x_K,j)."""
    c = torch.tensor(np.asarray(inst["c"], np.float64), requires_grad=True)
    w = torch.tensor(np.asarray(inst["w"], np.float64), requires_grad=True)
    x = unrolled_x(inst, iters, c, w, decisions, **kw)
    J = torch.zeros((), dtype=torch.float64)
    if xbar is not None:
        J = J + torch.dot(torch.as_tensor(np.asarray(xbar, np.float64)), x)
    if objective:
        t = np.asarray(inst["utype"])
        is_log = torch.as_tensor(t == 0)
        is_a2 = torch.as_tensor(t == 2)
        safe = torch.where(is_log | is_a2, x, torch.ones_like(x))
        J = J + torch.where(is_log, w * torch.log(safe),
                            torch.where(is_a2, -w / safe, w * x)).sum()
    J.backward()
    # autograd leaves the gradient of an input unset when J does not depend on it (e.g. c
    # after one iteration, before any capacity has entered x): that gradient is zero
    gc = c.grad.numpy().copy() if c.grad is not None else np.zeros(c.shape)
    gw = w.grad.numpy().copy() if w.grad is not None else np.zeros(w.shape)
    return gc, gw, float(J.detach())
