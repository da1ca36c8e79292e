"""Property-based parity: random small instances and parameters, the CUDA path against the
oracle after the same number of iterations.  Each example draws the sizes, route lengths,
link distribution (uniform or Zipf), utility mix (log, linear, alpha = 2), box (uniform,
per stream, or fixed rates), rho0, alpha, the rho update period and the iteration count,
then one kernel path:
FP64 rows, FP64 tiles (with a random tile size), plain FP64, or FP32 rows on the oracle's
rho decisions.  FP64 paths must match to 1e-9 and FP32 to 1e-4 in the relative norms of x
and of the prices.  Prices are marginal utilities, of the order of w / x, and an
uncongested link's price tends to zero through rounding noise (e.g. -1e-8 after 45
iterations on one stream and one link); so the norm of the prices is floored at 1e-3 of
the largest weight per link before dividing."""
import pytest
from hypothesis import HealthCheck, given, settings
from hypothesis import strategies as st

import numpy as np

from gpu_util import oracle_run, rel, run_gpu
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


@st.composite
def cases(draw):
    n = draw(st.integers(1, 3000))
    m = draw(st.integers(1, 400))
    len_lo = draw(st.integers(1, 4))
    len_hi = draw(st.integers(len_lo, 12))
    zipf = draw(st.booleans())
    frac_log = draw(st.sampled_from([0.0, 0.3, 0.7, 1.0]))
    frac_a2 = draw(st.sampled_from([0.0, 0.0, 0.2])) if frac_log < 1.0 else 0.0
    box_kind = draw(st.sampled_from(["uniform", "per_stream", "fixed"]))
    seed = draw(st.integers(0, 2**31 - 1))

    def box(rng, k):
        lo = rng.uniform(0.0, 0.4, k)
        hi = lo + rng.uniform(0.2, 5.0, k)
        if box_kind == "fixed":
            pin = rng.random(k) < 0.15
            hi[pin] = lo[pin] + 0.05 * (lo[pin] == 0)
            lo[pin] = hi[pin]
        return lo, hi

    inst = W.random_instance(n, m, len_lo, len_hi, seed=seed,
                             link_dist="zipf" if zipf else "uniform",
                             c_scale=draw(st.sampled_from([0.1, 1.0])), frac_log=frac_log,
                             frac_alpha2=frac_a2,
                             box=(0.0, 20.0) if box_kind == "uniform" else box)
    params = dict(rho0=draw(st.sampled_from([0.3, 1.0, 4.0])),
                  alpha=draw(st.sampled_from([1.0, 1.6, 1.8])),
                  period=draw(st.sampled_from([10, 50])))
    iters = draw(st.integers(1, 260))
    path = draw(st.sampled_from(["fp64_rows", "fp64_tiles", "plain", "fp32_rows"]))
    tile = draw(st.sampled_from([256, 512, 2048]))
    return inst, params, iters, path, tile


@settings(max_examples=150, deadline=None, derandomize=True, database=None,
          suppress_health_check=[HealthCheck.too_slow, HealthCheck.data_too_large])
@given(cases())
def test_random_instances_match_oracle(case):
    inst, params, iters, path, tile = case
    ref = oracle_run(inst, iters, **params)
    kw = dict(rho0=params["rho0"], alpha=params["alpha"], rho_period=params["period"])
    if path == "fp64_rows":
        g = run_gpu(inst, iters, "fp64", schedule=1, **kw)
        tol = 1e-9
    elif path == "fp64_tiles":
        g = run_gpu(inst, iters, "fp64", schedule=2, tile_items=tile, **kw)
        tol = 1e-9
    elif path == "plain":
        g = run_gpu(inst, iters, "plain", **kw)
        tol = 1e-9
    else:
        g = run_gpu(inst, iters, "fp32", schedule=1, schedule_decisions=ref["decisions"], **kw)
        tol = 1e-4
    assert g["iters"] == iters
    assert rel(g["x"], ref["x"]) <= tol, (path, rel(g["x"], ref["x"]))
    floor = 1e-3 * float(np.max(inst["w"])) * np.sqrt(ref["lam"].size)
    err = np.linalg.norm(g["lam"] - ref["lam"]) / max(np.linalg.norm(ref["lam"]), floor)
    assert err <= tol, (path, err)
