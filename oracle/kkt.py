"""KKT diagnostics of a NUM candidate (x, lambda) -- TEST INFRASTRUCTURE ONLY (numpy, FP64).

The conditions are those of the NUM problem of Sec. II (maximize sum U_j(x_j) subject to
R x <= c and the box), with link prices lambda >= 0 and path prices pi = R' lambda
(Sec. VI-B): primal feasibility, dual feasibility, complementary slackness, stationarity
(w_j / x_j = pi_j for an interior log stream) and the duality gap against the dual function
    g(lambda) = sum_j max_{x in box_j} (U_j(x) - pi_j x) + lambda' c.
Every quantity is written from its definition; the only library steps are numpy sums.
"""
from __future__ import annotations

import numpy as np

LOG = 0
ALPHA2 = 2


def link_loads(inst, x):
    """(R x)_l: the total rate of the streams that use link l."""
    lengths = np.diff(inst["route_ptr"])
    xs = np.repeat(np.asarray(x, dtype=np.float64), lengths)
    return np.bincount(inst["route_links"], weights=xs, minlength=inst["m"])


def path_prices(inst, lam):
    """pi_j = sum over the links of route j of lambda_l (Sec. VI-B)."""
    vals = np.asarray(lam, dtype=np.float64)[inst["route_links"]]
    return np.add.reduceat(vals, inst["route_ptr"][:-1])


def utility(inst, x):
    """sum_j U_j(x_j) with U = w log x (type 0), w x (type 1) or -w / x (type 2, alpha = 2
    fairness), in FP64."""
    x = np.asarray(x, dtype=np.float64)
    w = inst["w"]
    t = inst["utype"]
    with np.errstate(divide="ignore"):
        xs = np.where(t == 1, 1.0, x)
        return float(np.sum(np.where(t == LOG, w * np.log(xs),
                                     np.where(t == ALPHA2, -w / xs, w * x))))


def dual_value(inst, lam):
    """g(lambda) for lambda >= 0 (negative entries are clipped to zero first)."""
    lam = np.maximum(np.asarray(lam, dtype=np.float64), 0.0)
    pi = path_prices(inst, lam)
    w, lo, hi = inst["w"], inst["lo"], inst["hi"]
    t = inst["utype"]
    is_log = t == LOG
    is_a2 = t == ALPHA2
    with np.errstate(divide="ignore", invalid="ignore"):
        xl = np.where(pi > 0, w / np.where(pi > 0, pi, 1.0), hi)      # argmax w log x - pi x
        xa = np.where(pi > 0, np.sqrt(w / np.where(pi > 0, pi, 1.0)), hi)  # of -w/x - pi x
    xl = np.clip(xl, lo, hi)
    xa = np.clip(xa, lo, hi)
    with np.errstate(divide="ignore"):
        vlog = w * np.log(np.where(is_log, xl, 1.0)) - pi * xl
        va2 = -w / np.where(is_a2, xa, 1.0) - pi * xa
    xlin = np.where(w > pi, hi, lo)
    vlin = (w - pi) * xlin
    return float(np.sum(np.where(is_log, vlog, np.where(is_a2, va2, vlin))) + lam @ inst["c"])


def diagnostics(inst, x, lam, bound_tol=1e-9):
    """Scaled KKT violations of (x, lambda); all are zero at an exact optimum.

    feas      max_l (R x - c)_+ / c_l
    box       max_j distance of x_j outside [lo_j, hi_j]
    dual_neg  max_l (-lambda_l)_+
    comp      max_l |lambda_l (c_l - (R x)_l)| / max(1, lambda_l c_l)
    stat      max over interior log streams of |w/x - pi| / (w/x);  over streams at a bound,
              the violated sign condition scaled the same way
    gap       (g(lambda) - U(x)) / max(1, |U(x)|)
    """
    x = np.asarray(x, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    c = inst["c"]
    w, lo, hi = inst["w"], inst["lo"], inst["hi"]
    rx = link_loads(inst, x)
    pi = path_prices(inst, np.maximum(lam, 0.0))
    t = inst["utype"]
    span = np.maximum(hi - lo, 1e-300)
    at_lo = x <= lo + bound_tol * span
    at_hi = x >= hi - bound_tol * span
    with np.errstate(divide="ignore", invalid="ignore"):
        xp = np.where(x > 0, x, np.nan)
        grad = np.where(t == LOG, w / xp, np.where(t == ALPHA2, w / (xp * xp), w))   # U'(x)
    # stationarity of max U(x) - pi x over the box: U' = pi inside, U' <= pi at lo, >= pi at hi
    scale = np.maximum(np.abs(grad), 1e-300)
    viol = np.where(at_lo & ~at_hi, np.maximum(grad - pi, 0.0),
                    np.where(at_hi & ~at_lo, np.maximum(pi - grad, 0.0), np.abs(grad - pi)))
    viol = np.where(np.isnan(viol), 0.0, viol) / scale
    u = utility(inst, x)
    g = dual_value(inst, lam)
    return dict(
        feas=float(np.max(np.maximum(rx - c, 0.0) / c)),
        box=float(np.max(np.maximum(np.maximum(lo - x, x - hi), 0.0))),
        dual_neg=float(np.max(np.maximum(-lam, 0.0))),
        comp=float(np.max(np.abs(lam * (c - rx)) / np.maximum(1.0, np.abs(lam) * c))),
        stat=float(np.max(viol)) if viol.size else 0.0,
        gap=float((g - u) / max(1.0, abs(u))),
        utility=u,
        dual=g,
    )
