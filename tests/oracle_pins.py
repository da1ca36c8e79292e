"""Pins of the FP64 oracle: checks against what the paper and the mathematics fix, each
written independently of the oracle's own formulas.

Every pin is a function `pin_*(plant=0) -> (ok, detail)`.  `plant` selects an oracle build
with one planted mistake; `test_oracle_pins.py` requires every pin to pass on the real
oracle, `test_oracle_planted.py` requires every planted variant to fail at least one pin.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
from scipy import optimize

import oracle
from oracle import kkt
from paper_2509_10722_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _inst(route_lists, m, c, w, utype, lo=None, hi=None):
    n = len(route_lists)
    ptr = np.zeros(n + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in route_lists])
    links = np.array([l for r in route_lists for l in r], dtype=np.int32)
    return dict(n=n, m=m, route_ptr=ptr, route_links=links, c=np.asarray(c, float),
                utype=np.asarray(utype, np.uint8), w=np.asarray(w, float),
                lo=np.zeros(n) if lo is None else np.asarray(lo, float),
                hi=np.full(n, 1e3) if hi is None else np.asarray(hi, float))


def _close(a, b, rtol, atol=0.0):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if a.shape != b.shape or not np.all(np.isfinite(a)):
        return False
    return bool(np.all(np.abs(a - b) <= atol + rtol * np.abs(b)))


def _solve(inst, plant, eps=1e-11, iters=200_000, **kw):
    return oracle.solve(inst, iters, eps_abs=eps, plant=plant, **kw)


# ---- 1. proximal operators against 1-D bisection (Sec. III-E) -------------------------------

def _bisect_root(dfun, lo, hi, iters=200):
    """Minimizer over [lo, hi] of a convex function with increasing derivative dfun."""
    a, b = lo, hi
    if dfun(b) <= 0.0:
        return b
    if a > 0.0 and dfun(a) >= 0.0:
        return a
    if a <= 0.0:
        a = 0.0
    for _ in range(iters):
        mid = 0.5 * (a + b)
        if dfun(mid) > 0.0:
            b = mid
        else:
            a = mid
        if b - a <= 1e-300:
            break
    return 0.5 * (a + b)


def _prox_cases(rng, count=400):
    for i in range(count):
        L = int(rng.integers(1, 13))
        S = float(rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-6, 3))
        w = float(rng.uniform(0.1, 5.0))
        rho = float(10.0 ** rng.uniform(-3, 3))
        lo = 0.0 if i % 3 else float(rng.uniform(0.0, 1.0))
        hi = float(lo + 10.0 ** rng.uniform(-2, 2))
        yield S, L, w, rho, lo, hi


def pin_prox_log(plant=0):
    """prox of -w log x over the box: the minimizer of -w log x + rho/2 sum (x - zeta_t)^2,
    whose derivative is -w/x + rho (L x - S); found here by bisection."""
    rng = np.random.default_rng(1)
    worst = 0.0
    for S, L, w, rho, lo, hi in _prox_cases(rng):
        ref = _bisect_root(lambda x: (-w / x if x > 0 else -math.inf) + rho * (L * x - S),
                           max(lo, 0.0), hi)
        got = oracle.prox_log(S, L, w, rho, lo, hi, plant=plant)
        err = abs(got - ref) / max(abs(ref), 1e-300)
        worst = max(worst, err if math.isfinite(err) else math.inf)
    return worst < 1e-12, f"max rel err {worst:.3e}"


def pin_prox_linear(plant=0):
    rng = np.random.default_rng(2)
    worst = 0.0
    for S, L, w, rho, lo, hi in _prox_cases(rng):
        ref = _bisect_root(lambda x: -w + rho * (L * x - S), lo, hi)
        if lo > 0.0 or ref > 0.0:
            pass
        got = oracle.prox_linear(S, L, w, rho, lo, hi, plant=plant)
        err = abs(got - ref) / max(abs(ref), 1e-12)
        worst = max(worst, err if math.isfinite(err) else math.inf)
    return worst < 1e-9, f"max rel err {worst:.3e}"


def pin_prox_alpha2(plant=0):
    """prox of U = -w / x: the positive root of rho L x^3 - rho S x^2 - w (numpy.roots, a
    library eigenvalue solve of the companion matrix), clipped to the box."""
    rng = np.random.default_rng(9)
    worst = 0.0
    for S, L, w, rho, lo, hi in _prox_cases(rng, 300):
        r = np.roots([rho * L, -rho * S, 0.0, -w])
        r = r[np.abs(r.imag) <= 1e-9 * np.abs(r)].real
        root = float(r[r > 0].max())
        ref = min(max(root, lo), hi)
        got = oracle.prox_alpha2(S, L, w, rho, lo, hi, plant=plant)
        worst = max(worst, abs(got - ref) / max(abs(ref), 1e-300))
    return worst < 1e-8, f"max rel err {worst:.3e}"


def pin_prox_slack(plant=0):
    """prox of the indicator of {p + c >= 0}: the closest feasible point, found here by
    minimizing (p - zeta)^2 over a dense grid of feasible points."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        c = float(rng.uniform(0.1, 10.0))
        zeta = float(rng.uniform(-20.0, 20.0))
        grid = np.linspace(-c, 40.0, 400_001)
        ref = grid[np.argmin((grid - zeta) ** 2)]
        got = oracle.prox_slack(zeta, c, plant=plant)
        if not (got + c >= -1e-15 and abs(got - ref) <= 1e-4 + 1e-12 * abs(ref)):
            return False, f"zeta={zeta} c={c} got={got} ref={ref}"
    return True, "ok"


# ---- 2. closed-form networks (Sec. II KKT, Sec. VI-B stationarity) --------------------------

def pin_single_link(plant=0):
    """One link of capacity c shared by k log streams: x_j = w_j c / sum w, lambda = sum w / c."""
    rng = np.random.default_rng(4)
    for k in (1, 2, 5, 17):
        w = rng.uniform(0.5, 2.0, size=k)
        c = float(rng.uniform(1.0, 10.0))
        inst = _inst([[0]] * k, 1, [c], w, [0] * k)
        r = _solve(inst, plant)
        if not (_close(r["x"], w * c / w.sum(), 1e-7) and
                _close(r["lam"], [w.sum() / c], 1e-7)):
            return False, f"k={k} x={r['x']} lam={r['lam']}"
    return True, "ok"


def pin_single_link_waterfill(plant=0):
    """Box clipping: c = 10, w = (1, 1, 8), hi = 5.  Unclipped shares (1, 1, 8) put stream 3
    above its box, so it sits at hi = 5 and the two others split the remaining 5:
    x = (2.5, 2.5, 5), lambda = 1/2.5 = 0.4 (stream 3: w/x = 1.6 >= lambda, as required at hi)."""
    inst = _inst([[0], [0], [0]], 1, [10.0], [1.0, 1.0, 8.0], [0, 0, 0], hi=[5.0, 5.0, 5.0])
    r = _solve(inst, plant)
    ok = _close(r["x"], [2.5, 2.5, 5.0], 1e-7) and _close(r["lam"], [0.4], 1e-7)
    return ok, f"x={r['x']} lam={r['lam']}"


def pin_linear_single_link(plant=0):
    """Linear utilities are an LP: link c = 5 shared by w = (1, 2), box [0, 10]: all capacity
    goes to the heavier stream, x = (0, 5); the price equals its weight, lambda = 2."""
    inst = _inst([[0], [0]], 1, [5.0], [1.0, 2.0], [1, 1], hi=[10.0, 10.0])
    r = _solve(inst, plant)
    ok = _close(r["x"], [0.0, 5.0], 1e-6, 1e-7) and _close(r["lam"], [2.0], 1e-6)
    return ok, f"x={r['x']} lam={r['lam']}"


def pin_alpha2_single_link(plant=0):
    """alpha = 2 fairness on one link: w_j / x_j^2 = lambda gives x_j = sqrt(w_j) c / sum
    sqrt(w), lambda = (sum sqrt(w) / c)^2."""
    w = np.array([1.0, 4.0, 0.25, 2.0])
    c = 3.0
    inst = _inst([[0]] * 4, 1, [c], w, [2] * 4)
    r = _solve(inst, plant)
    sw = np.sqrt(w)
    ok = _close(r["x"], sw * c / sw.sum(), 1e-7) and _close(r["lam"], [(sw.sum() / c) ** 2], 1e-7)
    return ok, f"x={r['x']} lam={r['lam']}"


def pin_alpha2_kkt(plant=0):
    """A random instance mixing all three utilities satisfies the KKT conditions."""
    inst = W.random_instance(200, 60, 1, 5, seed=44, frac_log=0.4, frac_alpha2=0.3,
                             box=(0.0, 20.0))
    r = _solve(inst, plant, eps=1e-11)
    d = kkt.diagnostics(inst, r["x"], r["lam"])
    ok = (r["converged"] and d["feas"] < 1e-7 and d["comp"] < 1e-7 and d["stat"] < 1e-6
          and abs(d["gap"]) < 1e-7)
    return ok, str(d)


def pin_four_stream(plant=0):
    """The paper's small example (Sec. III-A), golden values in tests/golden."""
    g = json.load(open(os.path.join(GOLDEN, "four_stream_example.json")))
    inst = dict(n=4, m=3, route_ptr=np.array(g["route_ptr"], np.int64),
                route_links=np.array(g["route_links"], np.int32), c=np.array(g["c"]),
                utype=np.array(g["utype"], np.uint8), w=np.array(g["w"]), lo=np.zeros(4),
                hi=np.full(4, 1e3))
    r = _solve(inst, plant)
    ok = _close(r["x"], g["x"], 1e-8) and _close(r["lam"], g["lambda"], 1e-8)
    return ok, f"x={r['x']} lam={r['lam']}"


def pin_line_network(plant=0):
    g = json.load(open(os.path.join(GOLDEN, "line_network.json")))
    for case in g["cases"]:
        L = case["L"]
        routes = [list(range(L))] + [[l] for l in range(L)]
        inst = _inst(routes, L, [1.0] * L, [1.0] * (L + 1), [0] * (L + 1))
        r = _solve(inst, plant)
        xref = [case["x_long"]] + [case["x_short"]] * L
        if not (_close(r["x"], xref, 1e-7) and _close(r["lam"], [case["lambda"]] * L, 1e-7)):
            return False, f"L={L} x={r['x']} lam={r['lam']}"
    return True, "ok"


# ---- 3. independent solvers on random instances ---------------------------------------------

def _dual_solution(inst):
    """All-log NUM through its dual: minimize g(lambda) over lambda >= 0 with L-BFGS-B,
    x(lambda) = clip(w / pi, lo, hi), gradient c - R x(lambda)."""
    ptr, links = inst["route_ptr"], inst["route_links"]
    lengths = np.diff(ptr)
    w, lo, hi, c, m = inst["w"], inst["lo"], inst["hi"], inst["c"], inst["m"]

    def xs(lam):
        pi = np.add.reduceat(lam[links], ptr[:-1])
        with np.errstate(divide="ignore"):
            return np.clip(np.where(pi > 0, w / np.maximum(pi, 1e-300), hi), lo, hi), pi

    def fg(lam):
        x, pi = xs(lam)
        val = np.sum(w * np.log(x) - pi * x) + lam @ c
        grad = c - np.bincount(links, weights=np.repeat(x, lengths), minlength=m)
        return val, grad

    res = optimize.minimize(fg, np.ones(m), jac=True, method="L-BFGS-B",
                            bounds=[(0.0, None)] * m,
                            options=dict(maxiter=20000, ftol=1e-16, gtol=1e-13, maxcor=50))
    return xs(res.x)[0], res.x


def pin_dual_solver(plant=0):
    """Random all-log instances: the oracle's x equals the dual-ascent x (unique optimum)."""
    for seed in (11, 12):
        inst = W.random_instance(60, 25, 1, 5, seed=seed, frac_log=1.0, box=(0.0, 20.0))
        xd, _ = _dual_solution(inst)
        r = _solve(inst, plant, eps=1e-10)
        if not _close(r["x"], xd, 1e-5, 1e-7):
            return False, f"seed {seed}: max err {np.max(np.abs(r['x'] - xd)):.3e}"
    return True, "ok"


def pin_lp(plant=0):
    """Random all-linear instances are LPs: the oracle's utility equals HiGHS's optimum."""
    for seed in (21, 22):
        inst = W.random_instance(40, 15, 1, 4, seed=seed, frac_log=0.0, box=(0.0, 5.0))
        n, m = inst["n"], inst["m"]
        A = np.zeros((m, n))
        for j in range(n):
            A[inst["route_links"][inst["route_ptr"][j]:inst["route_ptr"][j + 1]], j] = 1.0
        lp = optimize.linprog(-inst["w"], A_ub=A, b_ub=inst["c"],
                              bounds=list(zip(inst["lo"], inst["hi"])), method="highs")
        r = _solve(inst, plant, eps=1e-10)
        d = kkt.diagnostics(inst, r["x"], r["lam"])
        ok = abs(d["utility"] - (-lp.fun)) <= 1e-6 * abs(lp.fun) and d["feas"] < 1e-7
        if not ok:
            return False, f"seed {seed}: oracle {d['utility']} lp {-lp.fun} feas {d['feas']}"
    return True, "ok"


def pin_mixed_slsqp(plant=0):
    """Small mixed log/linear instances: utility equals an SLSQP solve of the primal."""
    for seed in (31, 32):
        inst = W.random_instance(8, 5, 1, 3, seed=seed, frac_log=0.5, box=(0.0, 4.0))
        n, m = inst["n"], inst["m"]
        A = np.zeros((m, n))
        for j in range(n):
            A[inst["route_links"][inst["route_ptr"][j]:inst["route_ptr"][j + 1]], j] = 1.0
        w, is_log = inst["w"], inst["utype"] == 0

        def f(x):
            return -np.sum(np.where(is_log, w * np.log(np.maximum(x, 1e-300)), w * x))

        def g(x):
            return -np.where(is_log, w / np.maximum(x, 1e-300), w)

        best = None
        for start in (0.1, 0.5):
            res = optimize.minimize(f, np.full(n, start), jac=g, method="SLSQP",
                                    bounds=[(1e-9, h) for h in inst["hi"]],
                                    constraints=[dict(type="ineq", fun=lambda x: inst["c"] - A @ x,
                                                      jac=lambda x: -A)],
                                    options=dict(ftol=1e-14, maxiter=2000))
            if best is None or res.fun < best:
                best = res.fun
        r = _solve(inst, plant, eps=1e-10)
        d = kkt.diagnostics(inst, r["x"], r["lam"])
        if not (abs(d["utility"] + best) <= 1e-6 * max(1.0, abs(best)) and d["feas"] < 1e-7):
            return False, f"seed {seed}: oracle {d['utility']} slsqp {-best} feas {d['feas']}"
    return True, "ok"


def pin_bruteforce(plant=0):
    """Two streams, two links (stream 1 on links 0 and 1, stream 2 on link 0), one log and
    one linear utility: dense grid search of the feasible box."""
    inst = _inst([[0, 1], [0]], 2, [3.0, 1.2], [1.0, 0.45], [0, 1], hi=[5.0, 5.0])
    g1 = np.linspace(1e-6, 5.0, 4001)[:, None]
    g2 = np.linspace(0.0, 5.0, 4001)[None, :]
    feas = (g1 + g2 <= 3.0) & (g1 <= 1.2)
    val = np.where(feas, 1.0 * np.log(g1) + 0.45 * g2, -np.inf)
    best = float(val.max())
    r = _solve(inst, plant, eps=1e-11)
    d = kkt.diagnostics(inst, r["x"], r["lam"])
    # the grid optimum is below the true one by at most (max slope) x (grid step)
    ok = (d["feas"] < 1e-8 and best - 1e-9 <= d["utility"] <= best + 2e-3)
    return ok, f"oracle {d['utility']} grid {best}"


def pin_kkt_random(plant=0):
    """Random mixed instance run to a tight tolerance satisfies every KKT condition."""
    inst = W.random_instance(300, 120, 2, 6, seed=41, frac_log=0.5, box=(0.0, 20.0))
    r = _solve(inst, plant, eps=1e-11)
    d = kkt.diagnostics(inst, r["x"], r["lam"])
    ok = (r["converged"] and d["feas"] < 1e-7 and d["box"] == 0.0 and d["dual_neg"] < 1e-7
          and d["comp"] < 1e-7 and d["stat"] < 1e-6 and abs(d["gap"]) < 1e-7)
    return ok, str(d)


def pin_large_rho_start(plant=0):
    """A far-off initial penalty (rho0 = 100) forces many rho decreases and dual rescales;
    the prices must still be the KKT prices of the four-stream example."""
    g = json.load(open(os.path.join(GOLDEN, "four_stream_example.json")))
    inst = dict(n=4, m=3, route_ptr=np.array(g["route_ptr"], np.int64),
                route_links=np.array(g["route_links"], np.int32), c=np.array(g["c"]),
                utype=np.array(g["utype"], np.uint8), w=np.array(g["w"]), lo=np.zeros(4),
                hi=np.full(4, 1e3))
    for rho0 in (100.0, 0.01):
        r = _solve(inst, plant, rho0=rho0, period=10)
        if not (r["converged"] and _close(r["x"], g["x"], 1e-7) and
                _close(r["lam"], g["lambda"], 1e-7)):
            return False, f"rho0={rho0} x={r['x']} lam={r['lam']} iters={r['iters']}"
        if not np.any(r["decisions"] != 0):
            return False, "no rho change happened"
    return True, "ok"


def pin_capacity_switch(plant=0):
    """Warm start after a capacity change (Sec. V-D): converged on c = 3, then switched to
    c = 6, the run converges to the closed form of the new capacity, x = w c / sum w."""
    w = np.array([1.0, 2.0, 0.5])
    inst = _inst([[0]] * 3, 1, [3.0], w, [0, 0, 0])
    r = oracle.solve(inst, 3000, eps_abs=0.0, c_switch=np.array([6.0]), switch_iter=400,
                     plant=plant)
    before = oracle.solve(inst, 400, eps_abs=0.0, plant=plant)
    ok = _close(before["x"], w * 3.0 / w.sum(), 1e-7) and \
        _close(r["x"], w * 6.0 / w.sum(), 1e-7) and \
        _close(r["lam"], [w.sum() / 6.0], 1e-7) and _close(r["slack"], [0.0], 0.0, 1e-6)
    return ok, f"iters {r['iters']} x={r['x']} lam={r['lam']}"


# ---- 4. residuals, stopping test and rho rule (Sec. III-F, III-G) ---------------------------

def _terminal_flows(inst, x, slack):
    """Terminal flows recovered from the NUM variables (Sec. III-D): a traffic terminal of
    stream j carries x_j, the slack terminal of link l carries s_l - c_l.  Returns the flows
    and the link of each terminal, traffic terminals first (stream-major), then slack ones."""
    lengths = np.diff(inst["route_ptr"])
    flows = np.concatenate([np.repeat(x, lengths), slack - inst["c"]])
    links = np.concatenate([inst["route_links"], np.arange(inst["m"])])
    return flows, links


def _link_mean(inst, flows, links):
    cnt = np.bincount(links, minlength=inst["m"]).astype(float)
    return np.bincount(links, weights=flows, minlength=inst["m"]) / cnt


def pin_residuals(plant=0):
    """||r|| and ||s|| recomputed from the recovered x and slack at iterations k-1 and k:
    r = pbar repeated on every terminal, s = rho ((p - pbar) - (p - pbar)_prev)."""
    inst = W.random_instance(50, 20, 1, 5, seed=51, frac_log=0.5, box=(0.0, 20.0))
    for k in (1, 2, 7, 50, 51, 52, 120):
        a = oracle.solve(inst, k, eps_abs=0.0, rho0=3.0, period=50, plant=plant)
        fa, links = _terminal_flows(inst, a["x"], a["slack"])
        pa = _link_mean(inst, fa, links)
        r_ref = math.sqrt(np.sum(pa[links] ** 2))
        if k > 1:
            b = oracle.solve(inst, k - 1, eps_abs=0.0, rho0=3.0, period=50, plant=plant)
            fb, _ = _terminal_flows(inst, b["x"], b["slack"])
            pb = _link_mean(inst, fb, links)
            dev_b = fb - pb[links]
        else:
            dev_b = np.zeros_like(fa)
        rho_k = a["hist"][-1, 2]
        s_ref = rho_k * math.sqrt(np.sum(((fa - pa[links]) - dev_b) ** 2))
        r_got, s_got = a["hist"][-1, 0], a["hist"][-1, 1]
        if not (_close([r_got], [r_ref], 1e-9, 1e-14) and _close([s_got], [s_ref], 1e-9, 1e-14)):
            return False, f"k={k}: r {r_got} vs {r_ref}, s {s_got} vs {s_ref}"
    return True, "ok"


def pin_stop_rule(plant=0):
    """The run stops at the first iteration with ||r|| and ||s|| both below
    eps_abs * sqrt(J), J = nnz + m."""
    inst = W.random_instance(80, 30, 1, 5, seed=61, frac_log=0.5, box=(0.0, 20.0))
    eps = 1e-6
    r = oracle.solve(inst, 100_000, eps_abs=eps, plant=plant)
    tol = eps * math.sqrt(inst["route_links"].size + inst["m"])
    h = r["hist"]
    below = (h[:, 0] < tol) & (h[:, 1] < tol)
    ok = r["converged"] and below[-1] and not np.any(below[:-1])
    return ok, f"iters {r['iters']} last {h[-1, :2]} tol {tol}"


def pin_rho_rule(plant=0):
    """At every update point k = 50 i: rho grows by gamma when ||r|| > mu ||s||, shrinks by
    gamma when ||s|| > mu ||r||, stays otherwise (Eq. rho-update); the next iteration runs
    with the new rho."""
    inst = W.random_instance(120, 40, 1, 6, seed=71, frac_log=0.5, box=(0.0, 20.0))
    for rho0 in (0.05, 1.0, 30.0):
        r = oracle.solve(inst, 600, eps_abs=0.0, rho0=rho0, plant=plant)
        h = r["hist"]
        for k in range(50, 600, 50):
            rn, sn, rho = h[k - 1]
            want = 1.1 if rn > 2.0 * sn else (1 / 1.1 if sn > 2.0 * rn else 1.0)
            if not _close([h[k, 2]], [rho * want], 1e-14):
                return False, f"rho0 {rho0} k {k}: r {rn} s {sn} rho {rho} -> {h[k, 2]}"
        if not np.all(h[1:, 2][np.arange(1, 600) % 50 != 0] == h[:-1, 2][np.arange(1, 600) % 50 != 0]):
            return False, "rho changed off an update point"
    return True, "ok"


def pin_identities(plant=0):
    """ADMM identities of the literal iteration: u is the same on every terminal of a link
    and z sums to zero over every link, after every iteration."""
    inst = W.random_instance(100, 40, 1, 6, seed=81, frac_log=0.5, box=(0.0, 20.0))
    r = oracle.solve(inst, 300, eps_abs=0.0, rho0=2.0, debug=True, plant=plant)
    return r["identity_violation"] < 1e-11, f"violation {r['identity_violation']:.3e}"


PINS = [pin_prox_log, pin_prox_linear, pin_prox_alpha2, pin_prox_slack, pin_single_link,
        pin_alpha2_single_link, pin_alpha2_kkt,
        pin_single_link_waterfill, pin_linear_single_link, pin_four_stream, pin_line_network,
        pin_dual_solver, pin_lp, pin_mixed_slsqp, pin_bruteforce, pin_kkt_random,
        pin_large_rho_start, pin_capacity_switch, pin_residuals, pin_stop_rule, pin_rho_rule,
        pin_identities]

# planted mistakes of pmp_oracle.c (ORACLE_PLANT values) and what each one is
PLANTS = {
    1: "log prox takes the negative root",
    2: "linear prox subtracts w / rho",
    3: "slack prox takes the min",
    4: "link average divides by deg instead of deg + 1",
    5: "over-relaxation weights swapped",
    6: "dual update uses p instead of the relaxed p+",
    7: "dual residual without the rho factor",
    8: "primal residual over slack terminals only",
    9: "residual-balancing branches swapped",
    10: "dual rescale inverted",
    11: "stopping tolerance without sqrt(J)",
    12: "z projection averages over traffic terminals only",
    13: "log prox not clipped to the box",
    14: "alpha = 2 prox with the wrong sign of the S x^2 term",
    15: "dual residual without the previous iterate (p - pbar, not its change)",
    16: "rho updated one iteration late",
    17: "alpha = 2 prox not clipped to the box",
    18: "log prox ignoring the number of terminals of the stream",
}
