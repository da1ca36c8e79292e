"""Property-based parity: random small instances and parameters, the CUDA path against the
oracle.  Each example draws the sizes, route lengths (sometimes with a few routes longer
than 32 links), link distribution (uniform or Zipf), utility mix (log, linear, alpha = 2),
box (uniform, per stream, or fixed rates), rho0, alpha, the rho update period and the
iteration count.

- Single instances: one kernel path per example (FP64 fused, plain FP64, FP32 fused on
  the oracle's rho decisions), compared after the same number of iterations.
- Batches: 1 to 8 such instances in one batch with a random work partition, in FP64 (with
  a stopping tolerance half of the time: every instance must stop at the oracle's
  iteration) or in FP32 on the oracle's decisions.
- Adjoints: dJ/dc and dJ/dw of an FP64 or plain run with a random checkpoint interval,
  for the total utility or a random cotangent on x, against the CPU reference gradient.
- Warm starts: new capacities (some links kept, the others scaled by U[0.2, 1.5]) set
  after k1 iterations, then k2 more, against the oracle switching at the same iteration.
- Many links: 5e5 to 1.2e6 links for 1e3 to 3e4 streams, where the link kernel spreads
  the epilogues of a group's links over its lanes.

FP64 results must match to 1e-9 and FP32 to 1e-4 in relative norm.  Prices are marginal
utilities, of the order of w / x, and an uncongested link's price tends to zero through
rounding noise (e.g. -1e-8 after 45 iterations on one stream and one link); so the norm of
the prices, and of dJ/dc, is floored at 1e-3 of the largest weight per link before
dividing.  The examples are derandomized: every run draws the same ones."""
import numpy as np
import pytest
from hypothesis import HealthCheck, given, settings
from hypothesis import strategies as st

from gpu_util import oracle_run, rel, run_gpu
from oracle import adjoint_ref
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu

FUZZ = dict(deadline=None, derandomize=True, database=None,
            suppress_health_check=[HealthCheck.too_slow, HealthCheck.data_too_large])


def _long_routes(inst, rng, count):
    """Give `count` random streams routes of 33..min(m, 90) distinct links."""
    n, m = int(inst["n"]), int(inst["m"])
    lens = np.diff(inst["route_ptr"])
    longs = rng.choice(n, size=min(count, n), replace=False)
    lens[longs] = rng.integers(33, min(m, 90) + 1, size=longs.size)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    rl = np.concatenate([rng.choice(m, size=int(k), replace=False) for k in lens])
    return dict(inst, route_ptr=rp, route_links=rl.astype(np.int32))


@st.composite
def instances(draw, max_n=3000, max_m=400):
    n = draw(st.integers(1, max_n))
    m = draw(st.integers(1, max_m))
    len_lo = draw(st.integers(1, 4))
    len_hi = draw(st.integers(len_lo, 12))
    zipf = draw(st.booleans())
    frac_log = draw(st.sampled_from([0.0, 0.3, 0.7, 1.0]))
    frac_a2 = draw(st.sampled_from([0.0, 0.0, 0.2])) if frac_log < 1.0 else 0.0
    box_kind = draw(st.sampled_from(["uniform", "per_stream", "fixed"]))
    seed = draw(st.integers(0, 2**31 - 1))
    n_long = draw(st.sampled_from([0, 0, 0, 3])) if m >= 40 else 0

    def box(rng, k):
        lo = rng.uniform(0.0, 0.4, k)
        hi = lo + rng.uniform(0.2, 5.0, k)
        if box_kind == "fixed":
            pin = rng.random(k) < 0.15
            hi[pin] = lo[pin] + 0.05 * (lo[pin] == 0)  # log streams need hi > 0
            lo[pin] = hi[pin]
        return lo, hi

    inst = W.random_instance(n, m, len_lo, len_hi, seed=seed,
                             link_dist="zipf" if zipf else "uniform",
                             c_scale=draw(st.sampled_from([0.1, 1.0])), frac_log=frac_log,
                             frac_alpha2=frac_a2,
                             box=(0.0, 20.0) if box_kind == "uniform" else box)
    if n_long:
        inst = _long_routes(inst, np.random.default_rng(seed + 1), n_long)
    return inst


def solver_params(draw):
    return dict(rho0=draw(st.sampled_from([0.3, 1.0, 4.0])),
                alpha=draw(st.sampled_from([1.0, 1.6, 1.8])),
                period=draw(st.sampled_from([10, 50])))


def gpu_params(params):
    return dict(rho0=params["rho0"], alpha=params["alpha"], rho_period=params["period"])


def price_err(got, ref, inst):
    floor = 1e-3 * float(np.max(inst["w"])) * np.sqrt(np.asarray(ref).size)
    return float(np.linalg.norm(np.asarray(got) - ref) / max(np.linalg.norm(ref), floor))


# ---- single instances ---------------------------------------------------------------------

@st.composite
def cases(draw):
    inst = draw(instances())
    params = solver_params(draw)
    iters = draw(st.integers(1, 260))
    path = draw(st.sampled_from(["fp64_rows", "plain", "fp32_rows"]))
    return inst, params, iters, path


@settings(max_examples=150, **FUZZ)
@given(cases())
def test_random_instances_match_oracle(case):
    inst, params, iters, path = case
    ref = oracle_run(inst, iters, **params)
    kw = gpu_params(params)
    if path == "fp64_rows":
        g = run_gpu(inst, iters, "fp64", **kw)
        tol = 1e-9
    elif path == "plain":
        g = run_gpu(inst, iters, "plain", **kw)
        tol = 1e-9
    else:
        g = run_gpu(inst, iters, "fp32", schedule_decisions=ref["decisions"], **kw)
        tol = 1e-4
    assert g["iters"] == iters
    assert rel(g["x"], ref["x"]) <= tol, (path, rel(g["x"], ref["x"]))
    err = price_err(g["lam"], ref["lam"], inst)
    assert err <= tol, (path, err)


# ---- batches ------------------------------------------------------------------------------

@st.composite
def batch_cases(draw):
    insts = draw(st.lists(instances(max_n=1500, max_m=300), min_size=1, max_size=8))
    params = solver_params(draw)
    iters = draw(st.integers(1, 200))
    precision = draw(st.sampled_from([0, 1]))
    eps = draw(st.sampled_from([0.0, 1e-3])) if precision == 1 else 0.0
    # 0: balanced ranges (one per block, cut at instance boundaries)
    part = (draw(st.sampled_from([0] + [2 ** k for k in range(8, 14)])),
            draw(st.sampled_from([0] + [2 ** k for k in range(5, 11)])),
            draw(st.sampled_from([4, 8, 16, 32])))
    return insts, params, iters, precision, eps, part


@settings(max_examples=60, **FUZZ)
@given(batch_cases())
def test_random_batches_match_oracle(case):
    from paper_2509_10722_b300 import capi
    insts, params, iters, precision, eps, part = case
    refs = [oracle_run(inst, iters, eps=eps, **params) for inst in insts]
    with capi.Batch(insts, precision=precision, history=64, **gpu_params(params)) as b:
        b.set_schedule(*part)
        if precision == 0:
            per = params["period"]
            sched = np.zeros((len(insts), max(iters // per, 1)), dtype=np.int8)
            for i, r in enumerate(refs):
                sched[i, :r["decisions"].size] = r["decisions"]
            b.set_rho_schedules(sched)
        rc, its, status = b.solve(iters, eps)
        xs, ps, _ = b.get()
    tol = 1e-9 if precision == 1 else 1e-4
    for i, (inst, r) in enumerate(zip(insts, refs)):
        assert int(its[i]) == int(r["iters"]), (i, its[i], r["iters"])
        assert rel(xs[i], r["x"]) <= tol, (i, rel(xs[i], r["x"]))
        err = price_err(ps[i], r["lam"], inst)
        assert err <= tol, (i, err)


# ---- adjoints -----------------------------------------------------------------------------

@st.composite
def adjoint_cases(draw):
    inst = draw(instances(max_n=300, max_m=60))
    params = solver_params(draw)
    iters = draw(st.integers(1, 150))
    precision = draw(st.sampled_from([1, 2]))
    kc = draw(st.sampled_from([0, 1, 7, 50]))
    use_xbar = draw(st.booleans())
    return inst, params, iters, precision, kc, use_xbar


@settings(max_examples=40, **FUZZ)
@given(adjoint_cases())
def test_random_adjoints_match_reference(case):
    from paper_2509_10722_b300 import capi
    inst, params, iters, precision, kc, use_xbar = case
    dec = oracle_run(inst, iters, **params)["decisions"]
    xbar = (np.random.default_rng(int(inst["n"]) + iters).standard_normal(int(inst["n"]))
            if use_xbar else None)
    with capi.Problem(inst, precision=precision, history=max(iters, 1),
                      **gpu_params(params)) as p:
        gc, gw, J = p.adjoint(iters, kc, xbar=xbar, objective=not use_xbar)
    rc, rw, rJ = adjoint_ref.gradients(inst, iters, dec, xbar=xbar, objective=not use_xbar,
                                       **params)
    if not use_xbar:  # J is the total utility; with a cotangent, rJ also holds xbar . x
        assert abs(J - rJ) <= 1e-9 * max(abs(rJ), 1.0)
    assert price_err(gc, rc, inst) <= 1e-9, price_err(gc, rc, inst)
    floor = 1e-3 * np.sqrt(rw.size)
    assert np.linalg.norm(gw - rw) / max(np.linalg.norm(rw), floor) <= 1e-9


# ---- warm starts after a capacity change --------------------------------------------------

@st.composite
def switch_cases(draw):
    inst = draw(instances(max_n=1500, max_m=300))
    params = solver_params(draw)
    k1 = draw(st.integers(0, 150))
    k2 = draw(st.integers(1, 150))
    path = draw(st.sampled_from(["fp64_rows", "plain", "fp32_rows"]))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    c = np.asarray(inst["c"], dtype=np.float64)
    keep = rng.random(c.size) < draw(st.sampled_from([0.0, 0.5, 0.9]))
    c_new = np.where(keep, c, c * rng.uniform(0.2, 1.5, c.size))
    return inst, params, k1, k2, path, c_new


@settings(max_examples=50, **FUZZ)
@given(switch_cases())
def test_random_capacity_switches_match_oracle(case):
    """num_set_capacity after k1 iterations, then k2 more, against the oracle whose
    capacities switch at iteration k1 (the warm start of Sec. V-D)."""
    from paper_2509_10722_b300 import capi
    inst, params, k1, k2, path, c_new = case
    if k1 == 0:  # a switch before the first iteration is a cold start on the new network
        ref = oracle_run(dict(inst, c=c_new), k2, **params)
    else:
        ref = oracle_run(inst, k1 + k2, c_switch=c_new, switch_iter=k1, **params)
    precision = {"fp64_rows": 1, "plain": 2, "fp32_rows": 0}[path]
    with capi.Problem(inst, precision=precision, history=k1 + k2, **gpu_params(params)) as p:
        if precision == 0:
            p.set_rho_schedule(ref["decisions"])
        p.solve(k1, 0.0)
        p.set_capacity(c_new)
        p.solve(k2, 0.0)
        x, lam, _ = p.get()
    tol = 1e-4 if precision == 0 else 1e-9
    assert rel(x, ref["x"]) <= tol, (path, rel(x, ref["x"]))
    err = price_err(lam, ref["lam"], inst)
    assert err <= tol, (path, err)


# ---- many links: the link kernel's spread variant ------------------------------------------

@st.composite
def many_link_cases(draw):
    """Half a million links or more, where each link group of a resident grid has many
    links to sum and the link kernel runs the epilogues of 8 consecutive links on a
    group's lanes; few streams, so most links carry none."""
    n = draw(st.integers(1_000, 30_000))
    m = draw(st.integers(500_000, 1_200_000))
    zipf = draw(st.booleans())
    inst = W.random_instance(n, m, 1, draw(st.integers(1, 8)), seed=draw(st.integers(0, 2**31 - 1)),
                             link_dist="zipf" if zipf else "uniform", frac_log=0.7,
                             frac_alpha2=draw(st.sampled_from([0.0, 0.2])), box=(0.0, 20.0))
    iters = draw(st.integers(1, 80))
    path = draw(st.sampled_from(["fp64_rows", "fp32_rows"]))
    return inst, iters, path


@settings(max_examples=10, **FUZZ)
@given(many_link_cases())
def test_random_many_link_instances_match_oracle(case):
    inst, iters, path = case
    ref = oracle_run(inst, iters)
    if path == "fp64_rows":
        g = run_gpu(inst, iters, "fp64")
        tol = 1e-9
    else:
        g = run_gpu(inst, iters, "fp32", schedule_decisions=ref["decisions"])
        tol = 1e-4
    assert rel(g["x"], ref["x"]) <= tol, (path, rel(g["x"], ref["x"]))
    err = price_err(g["lam"], ref["lam"], inst)
    assert err <= tol, (path, err)
