"""Helpers of the GPU tests: run the CUDA path through the C ABI, run the oracle, compare."""
from __future__ import annotations

import numpy as np

import oracle

PREC = {"fp32": 0, "fp64": 1, "plain": 2}


def run_gpu(inst, iters, precision="fp64", eps=0.0, schedule_decisions=None, device=False,
            **params):
    """Solve through the C ABI; schedule_decisions forces the rho decisions, other keyword
    arguments are num_params fields (schedule = kernel schedule)."""
    from paper_2509_10722_b300 import capi
    params.setdefault("history", max(int(iters), 1))
    with capi.Problem(inst, device=device, precision=PREC[precision], **params) as p:
        if schedule_decisions is not None:
            p.set_rho_schedule(schedule_decisions)
        status, done = p.solve(iters, eps)
        x, lam, info = p.get()
        hist = p.history()
    return dict(x=x, lam=lam, info=info, hist=hist, status=status, iters=done)


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def max_abs_rel(a, b, floor):
    """max |a - b| / max(|b|, floor * max|b|): elementwise error with a floor."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    scale = np.maximum(np.abs(b), floor * max(np.max(np.abs(b)), 1e-300))
    return float(np.max(np.abs(a - b) / scale))


def compare(gpu, ref, tol, floor=1e-3):
    """Relative-norm and floored elementwise errors of x and prices; returns a dict."""
    return dict(x=rel(gpu["x"], ref["x"]), lam=rel(gpu["lam"], ref["lam"]),
                x_el=max_abs_rel(gpu["x"], ref["x"], floor),
                lam_el=max_abs_rel(gpu["lam"], ref["lam"], floor), tol=tol)


def oracle_run(inst, iters, eps=0.0, **kw):
    return oracle.solve(inst, iters, eps_abs=eps, **kw)


def decisions_from_hist(hist, period=50):
    """The rho decision (+1, 0, -1) taken at each update point of a run, read off the rho
    column of its residual history (rho of iteration k+1 against iteration k)."""
    rho = hist[:, 2]
    out = []
    for k in range(period, rho.size, period):
        r = rho[k] / rho[k - 1]
        out.append(1 if r > 1.0 + 1e-12 else (-1 if r < 1.0 - 1e-12 else 0))
    return np.array(out, dtype=np.int8)
