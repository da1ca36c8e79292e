"""Warm starts (Sec. V-D): a capacity change continues from the current iterate exactly as
the oracle does when its capacities switch mid-run; the iterate survives a round trip
through num_get_state / num_set_state bit for bit; warm starts after degradation and after
failures with pruning reach the same solutions as cold starts, in fewer iterations."""
import numpy as np
import pytest

from gpu_util import oracle_run, rel, run_gpu
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def inst():
    return W.random_instance(4000, 600, 2, 8, seed=21, frac_log=0.7, box=(0.0, 20.0))


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-4)])
def test_set_capacity_matches_oracle_switch(inst, precision, tol):
    from paper_2509_10722_b300 import capi
    c2, _ = W.degraded_capacities(inst, seed=5)
    ref = oracle_run(inst, 500, c_switch=c2, switch_iter=300)
    with capi.Problem(inst, precision=precision, history=600) as p:
        if precision == 0:
            p.set_rho_schedule(ref["decisions"])
        p.solve(300, 0.0)
        p.set_capacity(c2)
        p.solve(200, 0.0)
        x, lam, _ = p.get()
    assert rel(x, ref["x"]) <= tol and rel(lam, ref["lam"]) <= tol


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_state_round_trip(inst, precision):
    from paper_2509_10722_b300 import capi
    with capi.Problem(inst, precision=precision) as a:
        a.solve(200, 0.0)
        st = a.get_state()
        a.solve(100, 0.0)
        xa, la, _ = a.get()
    with capi.Problem(inst, precision=precision) as b:
        b.set_state(st)
        b.solve(100, 0.0)
        xb, lb, _ = b.get()
    assert np.array_equal(xa, xb) and np.array_equal(la, lb)


def test_degraded_warm_start(inst):
    from oracle import kkt
    from paper_2509_10722_b300 import capi
    c2, _ = W.degraded_capacities(inst, seed=6)
    eps = 1e-6
    with capi.Problem(inst, precision=1) as p:
        p.solve(100_000, eps)
        p.set_capacity(c2)
        _, warm = p.solve(100_000, eps)
        xw, lw, iw = p.get()
        p.reset()
        _, cold = p.solve(100_000, eps)
        xc, lc, ic = p.get()
    assert warm < cold
    deg = dict(inst, c=c2)
    ref = oracle_run(deg, 100_000, eps=eps)
    u = kkt.utility(deg, ref["x"])
    assert abs(iw["objective"] - u) <= 1e-5 * abs(u) and abs(ic["objective"] - u) <= 1e-5 * abs(u)


def test_pruned_warm_start(inst):
    from oracle import kkt
    from paper_2509_10722_b300 import capi
    failed = W.failed_links(inst, p=0.1, seed=7)
    pr, ks, kl = W.prune(inst, failed)
    eps = 1e-6
    with capi.Problem(inst, precision=1) as p:
        p.solve(100_000, eps)
        st = p.get_state()
    warm_state = {k: st[k][ks] for k in ("x", "Z")}
    warm_state.update({k: st[k][kl] for k in ("pbar", "y", "zs", "Rx", "ps")})
    warm_state["rho"] = st["rho"]
    with capi.Problem(pr, precision=1) as q:
        _, cold = q.solve(100_000, eps)
        _, _, ic = q.get()
        q.set_state(warm_state)
        _, warm = q.solve(100_000, eps)
        _, _, iw = q.get()
    assert warm < cold
    ref = oracle_run(pr, 100_000, eps=eps)
    u = kkt.utility(pr, ref["x"])
    assert abs(iw["objective"] - u) <= 1e-5 * abs(u) and abs(ic["objective"] - u) <= 1e-5 * abs(u)


def test_fp32_then_fp64_reaches_a_tolerance_fp32_cannot():
    """Precision escalation through the state API: FP32 iterates down to eps_abs = 1e-7,
    the state moved into an FP64 handle (num_get_state / num_set_state carry FP64 values
    whatever the handle's precision), then FP64 to 1e-10.  The result passes the same
    stopping test as a solve in FP64 from zero and agrees with the oracle's solution at
    that tolerance."""
    from paper_2509_10722_b300 import capi
    inst = W.workload("c1")
    with capi.Problem(inst, precision=capi.NUM_FUSED_FP32) as p32, \
            capi.Problem(inst, precision=capi.NUM_FUSED_FP64) as p64:
        st, it32 = p32.solve(100_000, 1e-7)
        assert st == 0
        p64.set_state(p32.get_state())
        st, it64 = p64.solve(100_000, 1e-10)
        assert st == 0
        x, lam, info = p64.get()
    assert info["primal"] < info["eps_tol"] and info["dual"] < info["eps_tol"]
    ref = oracle_run(inst, 100_000, eps=1e-10)
    assert ref["converged"]
    assert rel(x, ref["x"]) <= 1e-6 and rel(lam, ref["lam"]) <= 1e-6
