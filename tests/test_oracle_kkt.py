"""Pins of the KKT checker `oracle/kkt.py` on points known to be wrong (no GPU).

The checker is what judges converged points at sizes the oracle cannot reach, so it must
also report violations, not only read zero at an optimum.  Each pin below perturbs the
optimum of the four-stream example of Sec. III-A (c = 1, w = 1, log utilities: x* = (1, 1/3,
2/3, 2/3), lambda* = (1, 3/2, 3/2), path prices pi* = R' lambda* = (1, 3, 3/2, 3/2), Sec.
VI-B) or of a one-link network in a way whose violations follow by hand from the
conditions of Sec. II, and checks every figure the checker returns.

`test_planted_kkt_mistake_is_caught` then rebuilds the checker from its source with one
mistake planted (a lenient bound test, a masked stationarity term, a dropped slackness
term, a rescaled feasibility, a wrong dual function) and requires some pin to fail.
"""
from __future__ import annotations

import math
import os
import types

import numpy as np
import pytest

from oracle import kkt as KKT

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "kkt.py")

X_OPT = np.array([1.0, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0])
LAM_OPT = np.array([1.0, 1.5, 1.5])
# U(x*) = log 1 + log(1/3) + 2 log(2/3)
U_OPT = math.log(1.0 / 3.0) + 2.0 * math.log(2.0 / 3.0)


def _four(c=1.0):
    return dict(n=4, m=3, route_ptr=np.array([0, 1, 3, 4, 5], np.int64),
                route_links=np.array([0, 1, 2, 1, 2], np.int32), c=np.full(3, c),
                utype=np.zeros(4, np.uint8), w=np.ones(4), lo=np.zeros(4), hi=np.full(4, 1e3))


def _one_link(utype, w, hi, c=10.0):
    """One link shared by streams with the given utility types, weights and upper bounds."""
    n = len(w)
    return dict(n=n, m=1, route_ptr=np.arange(n + 1, dtype=np.int64),
                route_links=np.zeros(n, np.int32), c=np.array([c]),
                utype=np.asarray(utype, np.uint8), w=np.asarray(w, float), lo=np.zeros(n),
                hi=np.asarray(hi, float))


def _near(a, b, tol=1e-12):
    return abs(a - b) <= tol * max(1.0, abs(b))


def pin_optimum_reads_zero(k):
    d = k.diagnostics(_four(), X_OPT, LAM_OPT)
    ok = all(abs(d[q]) < 1e-14 for q in ("feas", "box", "dual_neg", "comp", "stat", "gap"))
    return ok and _near(d["utility"], U_OPT), d


def pin_rates_scaled(k):
    """x = 1.1 x*: every link carries 1.1 c, so feas = 0.1, comp = lambda * 0.1 c /
    max(1, lambda c) = 0.1 on every link, and w / x = pi* / 1.1 gives stat = 0.1.  With
    c = 2 (x = 2.2 x*) the same relative figures hold: 0.2 over 2 is again 0.1."""
    for c in (1.0, 2.0):
        d = k.diagnostics(_four(c), 1.1 * c * X_OPT, LAM_OPT / c)
        if not (_near(d["feas"], 0.1) and _near(d["comp"], 0.1) and _near(d["stat"], 0.1)
                and d["box"] == 0.0 and d["dual_neg"] == 0.0):
            return False, (c, d)
    return True, "ok"


def pin_prices_scaled(k):
    """lambda = 1.2 lambda* at x*: pi = 1.2 w / x, so stat = 0.2; the links stay tight, so
    feas = comp = 0.  The dual function is g = sum_j (-log pi_j - 1) + lambda'c
    = -4 log 1.2 + U(x*) - 4 + 4.8, so gap = (0.8 - 4 log 1.2) / |U(x*)|."""
    d = k.diagnostics(_four(), X_OPT, 1.2 * LAM_OPT)
    gap = (0.8 - 4.0 * math.log(1.2)) / abs(U_OPT)
    ok = (_near(d["stat"], 0.2) and d["feas"] < 1e-15 and d["comp"] < 1e-15
          and _near(d["gap"], gap) and _near(d["dual"], U_OPT + 0.8 - 4.0 * math.log(1.2)))
    return ok, d


def pin_gap_at_unit_prices(k):
    """lambda = (1, 1, 1): pi = (1, 2, 1, 1), g = -(log 2) - 4 + 3, gap = (g - U) / |U|."""
    d = k.diagnostics(_four(), X_OPT, np.ones(3))
    g = -math.log(2.0) - 1.0
    return _near(d["dual"], g) and _near(d["gap"], (g - U_OPT) / abs(U_OPT)), d


def pin_interior_stream_moved(k):
    """Stream 3 (x* = 2/3, pi* = 3/2) moved by delta: stat = |1 - 1.5 (2/3 + delta)| =
    1.5 delta, link 2 then carries 1 + delta (feas = delta, comp = 1.5 delta / 1.5)."""
    for delta in (1e-2, -3e-3):
        x = X_OPT.copy()
        x[2] += delta
        d = k.diagnostics(_four(), x, LAM_OPT)
        if not (_near(d["stat"], 1.5 * abs(delta), 1e-9)
                and _near(d["feas"], max(delta, 0.0), 1e-9)
                and _near(d["comp"], abs(delta), 1e-9)):
            return False, (delta, d)
    return True, "ok"


def pin_bounds(k):
    """One link, lambda = 1 (pi = 1).  A log stream (w = 1) held at its upper bound 2 has
    U'(2) = 1/2 < pi, which the bound does not excuse: stat = (1 - 1/2) / (1/2) = 1.  One
    at hi = 0.5 (U' = 2 >= pi) is optimal there: stat = 0.  A linear stream (w = 3) at
    x = 0 has w > pi, so it should grow: stat = (3 - 1) / 3; at its upper bound it is
    optimal.  A log stream at x = 1 + 1e-6 of hi = 1e3 is interior: stat = |1/x - 1| x."""
    cases = [
        ([0], [1.0], [2.0], [2.0], 1.0),
        ([0], [1.0], [0.5], [0.5], 0.0),
        ([1], [3.0], [5.0], [0.0], 2.0 / 3.0),
        ([1], [3.0], [5.0], [5.0], 0.0),
        ([0], [1.0], [1e3], [1.0 + 1e-6], 1e-6),
    ]
    for ut, w, hi, x, stat in cases:
        d = k.diagnostics(_one_link(ut, w, hi), np.array(x), np.array([1.0]))
        if not _near(d["stat"], stat, 1e-9):
            return False, (ut, w, hi, x, d["stat"], stat)
    return True, "ok"


def pin_sign_and_box(k):
    """A negative price is reported as dual_neg; a rate outside its box as box."""
    lam = LAM_OPT.copy()
    lam[1] = -0.3
    d = k.diagnostics(_four(), X_OPT, lam)
    x = X_OPT.copy()
    x[0] = -0.25
    with np.errstate(invalid="ignore"):  # log of a negative rate: the utility is NaN there
        e = k.diagnostics(_four(), x, LAM_OPT)
    x2 = X_OPT.copy()
    x2[3] = 1e3 + 2.0
    f = k.diagnostics(_four(), x2, LAM_OPT)
    ok = _near(d["dual_neg"], 0.3) and _near(e["box"], 0.25) and _near(f["box"], 2.0)
    return ok, (d["dual_neg"], e["box"], f["box"])


def pin_alpha2_stationarity(k):
    """U = -w / x (alpha = 2): U' = w / x^2.  One link, lambda = 1, w = 4: the optimum is
    x = 2; at x = 2.5 stat = |4/6.25 - 1| / (4/6.25)."""
    inst = _one_link([2], [4.0], [1e3])
    d0 = k.diagnostics(inst, np.array([2.0]), np.array([1.0]))
    d1 = k.diagnostics(inst, np.array([2.5]), np.array([1.0]))
    g = 4.0 / 6.25
    return d0["stat"] < 1e-15 and _near(d1["stat"], abs(g - 1.0) / g), (d0["stat"], d1["stat"])


KKT_PINS = [pin_optimum_reads_zero, pin_rates_scaled, pin_prices_scaled, pin_gap_at_unit_prices,
            pin_interior_stream_moved, pin_bounds, pin_sign_and_box, pin_alpha2_stationarity]

# (what the mistake is, the text of kkt.py it replaces, the replacement)
KKT_PLANTS = {
    "lenient bound test": ("def diagnostics(inst, x, lam, bound_tol=1e-9):",
                           "def diagnostics(inst, x, lam, bound_tol=1e-1):"),
    "interior stationarity masked": ("np.abs(grad - pi)))", "0.0 * np.abs(grad - pi)))"),
    "upper-bound sign test dropped": ("np.maximum(pi - grad, 0.0)", "0.0 * (pi - grad)"),
    "complementary slackness dropped": ("comp=float(np.max(np.abs(lam * (c - rx))",
                                        "comp=float(np.max(0.0 * np.abs(lam * (c - rx))"),
    "feasibility over a fixed scale": ("np.maximum(rx - c, 0.0) / c)", "np.maximum(rx - c, 0.0) / (c * c))"),
    "feasibility divided away": ("feas=float(np.max(np.maximum(rx - c, 0.0) / c)),",
                                 "feas=float(np.max(np.maximum(rx - c, 0.0) / c)) * 1e-6,"),
    "stationarity scaled by pi": ("scale = np.maximum(np.abs(grad), 1e-300)",
                                  "scale = np.maximum(np.abs(grad) + 10.0 * np.abs(pi), 1e-300)"),
    "dual function without lambda'c": ("+ lam @ inst[\"c\"])", ")"),
    "path prices from the first link only": ("np.add.reduceat(vals, inst[\"route_ptr\"][:-1])",
                                             "vals[inst[\"route_ptr\"][:-1]]"),
    "negative prices not reported": ("dual_neg=float(np.max(np.maximum(-lam, 0.0))),",
                                     "dual_neg=0.0,"),
}


def _planted(name):
    old, new = KKT_PLANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"plant target not found once in kkt.py: {old!r}"
    mod = types.ModuleType(f"kkt_planted_{abs(hash(name))}")
    exec(compile(src.replace(old, new), SRC, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("pin", KKT_PINS, ids=[p.__name__ for p in KKT_PINS])
def test_kkt_pin(pin):
    ok, detail = pin(KKT)
    assert ok, detail


@pytest.mark.parametrize("name", sorted(KKT_PLANTS))
def test_planted_kkt_mistake_is_caught(name):
    k = _planted(name)
    caught = []
    for pin in KKT_PINS:
        try:
            ok, _ = pin(k)
        except Exception:  # a crash on a broken checker counts as caught
            ok = False
        if not ok:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted checker mistake: {name}"
