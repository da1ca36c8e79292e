"""Batched solves against the oracle, instance by instance, through the C ABI.

Each instance of a batch must follow its own trajectory: its own rho decisions, stopping
iteration and solution, exactly as if solved alone."""
import numpy as np
import pytest

from gpu_util import oracle_run, rel
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _mixed_batch():
    def box(rng, n):
        lo = rng.uniform(0.0, 0.3, n)
        return lo, lo + rng.uniform(0.5, 4.0, n)
    return [W.random_instance(1, 1, 1, 1, seed=1),
            W.random_instance(5, 3, 1, 3, seed=2),
            W.random_instance(37, 11, 1, 6, seed=3, frac_log=0.0),
            W.random_instance(300, 40, 2, 8, seed=4),
            W.random_instance(1000, 500, 2, 6, seed=5),
            W.random_instance(3000, 200, 1, 6, seed=6, box=box),
            W.random_instance(5000, 5000, 1, 4, seed=7, frac_log=0.5, frac_alpha2=0.5),
            _with_long_routes(W.random_instance(3000, 1000, 1, 6, seed=9), seed=9),
            W.random_instance(20000, 2000, 2, 8, seed=8, link_dist="zipf", frac_log=1.0,
                              c_scale=0.1, w_dist="lognormal", box=(0.0, 10.0))]


def _with_long_routes(inst, seed):
    """2% of the streams get routes of 33..300 links, which the stream kernels sum by
    warps on both the single-instance and the batched path."""
    rng = np.random.default_rng(seed + 100)
    n, m = inst["n"], inst["m"]
    lens = np.diff(inst["route_ptr"])
    longs = rng.choice(n, size=n // 50, replace=False)
    lens[longs] = rng.integers(33, 301, size=longs.size)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    rl = np.concatenate([rng.choice(m, size=int(k), replace=False) for k in lens])
    return dict(inst, route_ptr=rp, route_links=rl.astype(np.int32))


@pytest.fixture(scope="module")
def batch():
    return _mixed_batch()


def _run_batch(insts, iters, precision, eps=0.0, schedules=None, **params):
    from paper_2509_10722_b300 import capi
    params.setdefault("history", 64)
    with capi.Batch(insts, precision=precision, **params) as b:
        if schedules is not None:
            b.set_rho_schedules(schedules)
        rc, it, st = b.solve(iters, eps)
        xs, ps, infos = b.get()
    return dict(rc=rc, iters=it, status=st, x=[x.copy() for x in xs],
                lam=[p.copy() for p in ps], info=infos)


@pytest.mark.parametrize("iters", [1, 60, 300])
def test_batch_fp64_matches_oracle_per_instance(batch, iters):
    g = _run_batch(batch, iters, 1)
    assert list(g["iters"]) == [iters] * len(batch)
    for i, inst in enumerate(batch):
        ref = oracle_run(inst, iters)
        assert rel(g["x"][i], ref["x"]) <= 1e-10, i
        assert rel(g["lam"][i], ref["lam"]) <= 1e-10, i


def test_batch_fp32_matches_oracle_on_its_schedules(batch):
    iters = 300
    refs = [oracle_run(inst, iters) for inst in batch]
    sched = np.zeros((len(batch), iters // 50), dtype=np.int8)
    for i, r in enumerate(refs):
        sched[i, :r["decisions"].size] = r["decisions"]
    g = _run_batch(batch, iters, 0, schedules=sched)
    for i, r in enumerate(refs):
        assert rel(g["x"][i], r["x"]) <= 1e-4, i
        assert rel(g["lam"][i], r["lam"]) <= 1e-4, i


def test_batch_instances_stop_independently(batch):
    """Instances that have a solution stop at the oracle's iteration, each at its own count
    (left out: the per-stream-box instance, whose lower bounds exceed some capacities, so it
    is infeasible and diverges in the oracle too, and the congested Zipf instance, which
    does not reach 1e-6 within the limit)."""
    batch = [batch[i] for i in (0, 1, 2, 3, 4, 6)]
    eps = 1e-6
    g = _run_batch(batch, 100_000, 1, eps=eps)
    assert g["rc"] == 0 and np.all(g["status"] == 0)
    refs = [oracle_run(inst, 100_000, eps=eps) for inst in batch]
    assert list(g["iters"]) == [r["iters"] for r in refs]
    assert len(set(g["iters"])) > 1
    for i, r in enumerate(refs):
        assert rel(g["x"][i], r["x"]) <= 1e-9, i


def test_batch_equals_single_solves(batch):
    """Same rows, same arithmetic: bit-identical to solving each instance alone, including
    the Zipf instance, whose links above 256 streams are summed by whole warps in chunks
    of 2,048 entries on both paths (8 lanes per shorter link, the default partition), and
    the instance whose long routes are summed by warps on both paths."""
    from paper_2509_10722_b300 import capi
    assert np.bincount(batch[-1]["route_links"], minlength=batch[-1]["m"]).max() > 2 * 2048
    g = _run_batch(batch, 200, 0)
    for i, inst in enumerate(batch):
        with capi.Problem(inst, precision=0, history=64) as p:
            p.solve(200, 0.0)
            x, lam, info = p.get()
        assert np.array_equal(g["x"][i], x), i
        assert np.array_equal(g["lam"][i], lam), i
        assert abs(g["info"][i]["objective"] - info["objective"]) <= 1e-12 * max(1.0, abs(info["objective"]))


def test_batch_rejects_cross_instance_routes():
    from paper_2509_10722_b300 import capi
    insts = [W.random_instance(20, 5, 1, 3, seed=11), W.random_instance(20, 5, 1, 3, seed=12)]
    so, lo, st = capi.stack_instances(insts)
    st["route_links"][0] = 7  # stream 0 (instance 0) uses a link of instance 1
    h = capi.ctypes.c_void_p()
    arr = [np.ascontiguousarray(st[k]) for k in ("route_ptr", "route_links", "c", "utype", "w",
                                                  "lo", "hi")]
    rc = capi.library().num_batch_create(capi.ctypes.byref(h), 2, capi._hptr(so), capi._hptr(lo),
                                         *[capi._hptr(a) for a in arr], None, None)
    assert rc == capi.NUM_ERR_INVALID and "another instance" in capi.num_last_error()


def test_c4_recipe_batch_converges():
    """The batched recipe (256 instances, n log-uniform in [1e3, 1e5], m = n / 10, routes of
    2..8 links, degraded capacities), FP32: every instance reaches eps_abs = 1e-4; every
    instance's objective matches the FP64 batch stopped by the same test to 1e-5; and a
    sample of instances (the four smallest and four drawn at random among those below
    2e4 streams) matches the FP64 oracle objective at the same tolerance to 1e-5."""
    from oracle import kkt
    insts = W.batched_instances(256, seed=0)
    g = _run_batch(insts, 50_000, 0, eps=1e-4)
    assert np.all(g["status"] == 0)
    g64 = _run_batch(insts, 50_000, 1, eps=1e-4)
    assert np.all(g64["status"] == 0)
    for i in range(len(insts)):
        o32, o64 = g["info"][i]["objective"], g64["info"][i]["objective"]
        assert abs(o32 - o64) <= 1e-5 * abs(o64), i
    ns = np.array([t["n"] for t in insts])
    order = np.argsort(ns)
    pool = np.flatnonzero((ns < 20_000) & ~np.isin(np.arange(ns.size), order[:4]))
    sample = list(order[:4]) + list(np.random.default_rng(4).choice(pool, 4, replace=False))
    for i in sample:
        ref = oracle_run(insts[i], 100_000, eps=1e-4)
        u = kkt.utility(insts[i], ref["x"])
        assert abs(g["info"][i]["objective"] - u) <= 1e-5 * abs(u), i
        assert int(g64["iters"][i]) == int(ref["iters"]), i  # FP64: the oracle's stop


# ---- the work partition and its autotuner ---------------------------------------------------

PARTITIONS = [(256, 32, 4), (512, 64, 8), (2048, 256, 16), (65536, 8192, 32), (1024, 1024, 8)]


@pytest.mark.parametrize("part", PARTITIONS, ids=[f"{a}-{b}-{c}" for a, b, c in PARTITIONS])
def test_every_partition_matches_oracle(batch, part):
    from paper_2509_10722_b300 import capi
    iters = 120
    with capi.Batch(batch, precision=1, history=64) as b:
        b.set_schedule(*part)
        assert b.schedule() == part
        b.solve(iters, 0.0)
        xs, ps, _ = b.get()
    for i, inst in enumerate(batch):
        ref = oracle_run(inst, iters)
        assert rel(xs[i], ref["x"]) <= 1e-10, (part, i)
        assert rel(ps[i], ref["lam"]) <= 1e-10, (part, i)


def test_item_sizes_do_not_change_the_iterates(batch):
    """With the lanes per link fixed and the rho decisions replayed, the FP32 iterates are
    bit-identical for every item size and for the balanced ranges: the partition only
    regroups the residual sums."""
    from paper_2509_10722_b300 import capi
    iters = 200
    sched = np.zeros((len(batch), iters // 50), dtype=np.int8)
    for i, inst in enumerate(batch):
        d = oracle_run(inst, iters)["decisions"]
        sched[i, :d.size] = d
    out = []
    for part in [(0, 0, 8), (2048, 256, 8), (256, 32, 8), (65536, 8192, 8), (0, 512, 8),
                 (1024, 0, 8)]:
        with capi.Batch(batch, precision=0, history=64) as b:
            b.set_schedule(*part)
            b.set_rho_schedules(sched)
            b.solve(iters, 0.0)
            xs, ps, _ = b.get()
        out.append((np.concatenate(xs), np.concatenate(ps)))
    for x, p in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(p, out[0][1])


def test_autotune_chooses_a_partition_and_resets(batch):
    from paper_2509_10722_b300 import capi
    iters = 150
    with capi.Batch(batch, precision=0, history=64) as b:
        chosen, trials = b.autotune(trial_iters=5)
        assert trials.shape == (30, 4) and np.all(trials[:, 3] > 0)
        assert b.schedule() == chosen
        # stage 1 varied stream_item only (0: balanced ranges), stage 2 link_item and lanes
        assert sorted(set(trials[:6, 0])) == [0, 512, 1024, 2048, 4096, 8192]
        assert len(set(map(tuple, trials[6:, 1:3]))) == 24
        assert chosen[0] == trials[:6][np.argmin(trials[:6, 3]), 0]
        rc, it, _ = b.solve(iters, 0.0)
        assert list(it) == [iters] * len(batch)  # reset: counts start from zero
        xs, ps, infos = b.get()
        assert all(inf["iters"] == iters for inf in infos)
    with capi.Batch(batch, precision=0, history=64) as b2:
        b2.set_schedule(*chosen)
        b2.solve(iters, 0.0)
        xs2, ps2, _ = b2.get()
    for a, c in zip(xs, xs2):
        assert np.array_equal(a, c)
    for a, c in zip(ps, ps2):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("bad", [(128, 256, 8), (3000, 256, 8), (2048, 16, 8), (2048, 16384, 8),
                                 (2048, 256, 2), (2048, 256, 64), (2048, 100, 8)])
def test_bad_partitions_are_rejected(bad):
    from paper_2509_10722_b300 import capi
    with capi.Batch([W.random_instance(50, 10, 1, 3, seed=1)], precision=0) as b:
        with pytest.raises(capi.NumError) as e:
            b.set_schedule(*bad)
        assert e.value.code == capi.NUM_ERR_INVALID
        assert b.schedule() == (0, 0, 8)


# ---- creation from separate instances (num_batch_create_instances) -------------------------

def _create_stacked(insts, precision):
    """A batch through num_batch_create from arrays stacked on the host."""
    import ctypes
    from paper_2509_10722_b300 import capi
    so, lo, st = capi.stack_instances(insts)
    prm = capi.num_default_params(precision=precision, history=64)
    arrs = [np.ascontiguousarray(st[k], dt) for k, dt in
            (("route_ptr", np.int64), ("route_links", np.int32), ("c", np.float64),
             ("utype", np.uint8), ("w", np.float64), ("lo", np.float64), ("hi", np.float64))]
    h = ctypes.c_void_p()
    rc = capi.library().num_batch_create(ctypes.byref(h), len(insts), capi._hptr(so),
                                         capi._hptr(lo), *[capi._hptr(a) for a in arrs],
                                         ctypes.byref(prm), None)
    assert rc == 0, capi.num_last_error()
    return h, int(so[-1]), int(lo[-1])


def test_instances_equal_host_stacked(batch):
    """Stacking on the device gives the same batch as stacking on the host: bit-identical
    iterates after 150 iterations, FP32 and FP64.  Half the instances pass lo = None."""
    from paper_2509_10722_b300 import capi
    insts = [dict(t, lo=None) if i % 2 else t for i, t in enumerate(batch)]
    insts_host = [dict(t, lo=np.zeros(t["n"])) if t["lo"] is None else t for t in insts]
    for precision in (0, 1):
        h, n, m = _create_stacked(insts_host, precision)
        try:
            capi.library().num_batch_solve(h, 150, 0.0, None, None)
            x1, p1 = np.empty(n), np.empty(m)
            assert capi.library().num_batch_get(h, capi._hptr(x1), capi._hptr(p1), None) == 0
        finally:
            capi.library().num_batch_destroy(h)
        with capi.Batch(insts, precision=precision, history=64) as b:
            b.solve(150, 0.0)
            xs, ps, _ = b.get()
        assert np.array_equal(np.concatenate(xs), x1) and np.array_equal(np.concatenate(ps), p1)


@pytest.mark.parametrize("defect,msg", [("link_beyond_own", "another instance"),
                                         ("negative_link", "outside"),
                                         ("route_ptr_start", "route_ptr[0]")])
def test_instances_rejects_bad_instances(batch, defect, msg):
    from paper_2509_10722_b300 import capi
    insts = [dict(t) for t in batch[:4]]
    t = insts[1]
    if defect == "link_beyond_own":
        rl = np.array(t["route_links"]).copy()
        rl[0] = t["m"]  # a link of the next instance once stacked
        t["route_links"] = rl
    elif defect == "negative_link":  # in the first instance, where it stays negative
        t = insts[0]
        rl = np.array(t["route_links"]).copy()
        rl[-1] = -5
        t["route_links"] = rl
    else:
        rp = np.array(t["route_ptr"]).copy()
        rp[0] = 1
        t["route_ptr"] = rp
    with pytest.raises(capi.NumError) as ei:
        capi.Batch(insts, precision=0)
    assert ei.value.code == capi.NUM_ERR_INVALID and msg in str(ei.value)
