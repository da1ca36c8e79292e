"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances: the FP64 paths (fused and plain) within 1e-10 relative (2-norm) of the oracle
after the same iteration count with their own rho decisions; the FP32 fused path within
1e-4 relative after the same iteration count on the oracle's rho schedule.  Integer work
(the device-built CSR) is compared bit for bit.
"""
import numpy as np
import pytest

from gpu_util import compare, oracle_run, rel, run_gpu
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def c1():
    return W.workload("c1")


@pytest.fixture(scope="module")
def c1_oracle(c1):
    return {k: oracle_run(c1, k) for k in (1, 7, 50, 51, 300, 2000)}


def _check_hist(gh, oh, rtol):
    assert gh.shape == oh.shape
    scale = np.max(np.abs(oh[:, :2]))
    assert np.allclose(gh[:, :2], oh[:, :2], rtol=rtol, atol=rtol * 1e-3 * scale)


@pytest.mark.parametrize("precision,reorder", [("fp64", 1), ("plain", 1), ("fp64", 0)])
@pytest.mark.parametrize("iters", [1, 7, 50, 51, 300, 2000])
def test_c1_fp64_paths_match_oracle(c1, c1_oracle, precision, reorder, iters):
    ref = c1_oracle[iters]
    g = run_gpu(c1, iters, precision, reorder=reorder)
    assert g["iters"] == iters
    e = compare(g, ref, FP64_TOL)
    assert e["x"] <= FP64_TOL and e["lam"] <= FP64_TOL, e
    assert e["x_el"] <= 1e-9 and e["lam_el"] <= 1e-9, e
    _check_hist(g["hist"], ref["hist"], 1e-9)
    assert np.array_equal(g["hist"][:, 2], ref["hist"][:, 2])  # identical rho decisions


@pytest.mark.parametrize("iters", [50, 300, 2000])
def test_c1_fp32_matches_oracle_on_its_rho_schedule(c1, c1_oracle, iters):
    ref = c1_oracle[iters]
    g = run_gpu(c1, iters, "fp32", schedule_decisions=ref["decisions"])
    e = compare(g, ref, FP32_TOL)
    assert e["x"] <= FP32_TOL and e["lam"] <= FP32_TOL, e
    assert np.array_equal(g["hist"][:, 2], ref["hist"][:, 2])


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_c1_fp32_own_decisions_objective_matches_oracle(c1, eps):
    """FP32 with its own rho decisions, stopped by the same test as the oracle: the
    objective agrees to 1e-5 relative (at eps = 1e-4 the stopped iterate itself is ~1e-3
    away from the optimum, for the oracle just the same)."""
    from oracle import kkt
    ref = oracle_run(c1, 100_000, eps=eps)
    g = run_gpu(c1, 100_000, "fp32", eps=eps)
    assert g["status"] == 0 and ref["converged"]
    u_ref = kkt.utility(c1, ref["x"])
    assert abs(g["info"]["objective"] - u_ref) <= 1e-5 * abs(u_ref)
    assert abs(g["iters"] - ref["iters"]) <= 5


@pytest.mark.parametrize("precision", ["fp64", "plain", "fp32"])
def test_stopping_iteration_matches_oracle(c1, precision):
    eps = 1e-6 if precision != "fp32" else 1e-4
    ref = oracle_run(c1, 100_000, eps=eps)
    sched = ref["decisions"] if precision == "fp32" else None
    g = run_gpu(c1, 100_000, precision, eps=eps, schedule_decisions=sched)
    assert g["status"] == 0 and ref["converged"]
    if precision == "fp32":
        assert abs(g["iters"] - ref["iters"]) <= 2
    else:
        assert g["iters"] == ref["iters"]
    assert g["info"]["primal"] < g["info"]["eps_tol"] and g["info"]["dual"] < g["info"]["eps_tol"]


# ---- ragged shapes, skew, degenerate rows -------------------------------------------------------

def _cases():
    yield "one_stream_one_link", W.random_instance(1, 1, 1, 1, seed=1), {}
    yield "tiny", W.random_instance(37, 11, 1, 6, seed=2), {}
    yield "links_without_streams", W.random_instance(40, 400, 1, 3, seed=3), {}
    yield "dense_links", W.random_instance(5000, 300, 1, 8, seed=4), {}
    yield "zipf_hot_links", W.random_instance(
        20000, 500, 2, 12, seed=5, link_dist="zipf", frac_log=1.0, c_scale=0.1,
        w_dist="lognormal", box=(0.0, 10.0)), {}
    yield "zipf_chunked_links", W.random_instance(
        60000, 2000, 2, 12, seed=6, link_dist="zipf", frac_log=1.0, c_scale=0.1,
        w_dist="lognormal", box=(0.0, 10.0)), {}
    yield "long_routes", W.random_instance(300, 200, 60, 150, seed=7), {}

    def mix_long(seed):
        """Short routes (1..6 links) with 2% of the streams on 33..400 links: the row stream
        kernel sums those by warps in the same launch as the rest."""
        short = W.random_instance(4000, 1200, 1, 6, seed=seed)
        rng = np.random.default_rng(seed + 100)
        n, m = short["n"], short["m"]
        lens = np.diff(short["route_ptr"])
        longs = rng.choice(n, size=n // 50, replace=False)
        lens[longs] = rng.integers(33, 401, size=longs.size)
        rp = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        rl = np.concatenate([rng.choice(m, size=int(k), replace=False) for k in lens])
        return dict(short, route_ptr=rp, route_links=rl.astype(np.int32))
    yield "mixed_long_routes", mix_long(13), {}
    yield "ragged_tail", W.random_instance(4097, 1025, 1, 10, seed=8), {}
    yield "all_linear", W.random_instance(2000, 300, 1, 6, seed=9, frac_log=0.0), {}
    yield "alpha2_mixed", W.random_instance(3000, 400, 1, 6, seed=12, frac_log=0.4,
                                            frac_alpha2=0.4), {}

    def box(rng, n):
        lo = rng.uniform(0.0, 0.5, n)
        return lo, lo + rng.uniform(0.1, 3.0, n)
    yield "per_stream_box", W.random_instance(3000, 200, 1, 6, seed=10, box=box), {}

    def fixed(rng, n):
        lo = rng.uniform(0.0, 0.3, n)
        hi = lo + rng.uniform(0.1, 3.0, n)
        pin = rng.random(n) < 0.2  # a fifth of the streams have a fixed rate (lo = hi)
        hi[pin] = lo[pin] + 0.05 * (lo[pin] == 0)  # log streams need hi > 0
        lo[pin] = hi[pin]
        return lo, hi
    yield "fixed_rates", W.random_instance(3000, 300, 1, 6, seed=11, frac_log=0.5,
                                           frac_alpha2=0.2, box=fixed), {}


CASES = list(_cases())


@pytest.mark.parametrize("name,inst,params", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision,reorder", [("fp64", 1), ("plain", 1), ("fp64", 0)])
def test_shapes_fp64_match_oracle(name, inst, params, precision, reorder):
    iters = 200
    ref = oracle_run(inst, iters)
    g = run_gpu(inst, iters, precision, reorder=reorder, **params)
    e = compare(g, ref, FP64_TOL)
    assert e["x"] <= FP64_TOL and e["lam"] <= FP64_TOL, e
    assert e["x_el"] <= 1e-9 and e["lam_el"] <= 1e-9, e


@pytest.mark.parametrize("name,inst,params", CASES, ids=[c[0] for c in CASES])
def test_shapes_fp32_match_oracle(name, inst, params):
    iters = 200
    ref = oracle_run(inst, iters)
    g = run_gpu(inst, iters, "fp32", schedule_decisions=ref["decisions"], **params)
    e = compare(g, ref, FP32_TOL)
    assert e["x"] <= FP32_TOL and e["lam"] <= FP32_TOL, e


@pytest.mark.parametrize("name,inst,params", CASES[:6], ids=[c[0] for c in CASES[:6]])
@pytest.mark.parametrize("reorder", [0, 1])
def test_operator_is_bit_exact(name, inst, params, reorder):
    from paper_2509_10722_b300 import capi
    with capi.Problem(inst, reorder=reorder, **params) as p:
        rp, ci = p.operator()
    rp_ref, ci_ref = W.csr_of(inst)
    assert np.array_equal(rp, rp_ref) and np.array_equal(ci, ci_ref)


# ---- determinism, graph vs launches, device inputs ----------------------------------------------

def test_runs_are_bit_identical(c1):
    a = run_gpu(c1, 500, "fp32")
    b = run_gpu(c1, 500, "fp32")
    c = run_gpu(c1, 500, "fp32", use_graph=0)
    d = run_gpu(c1, 500, "fp32", check_every=7)
    for other in (b, c, d):
        assert np.array_equal(a["x"], other["x"]) and np.array_equal(a["lam"], other["lam"])


def test_skewed_runs_are_bit_identical():
    """Zipf links, several split into chunks: which warp takes which chunk from the link
    kernel's queue varies from run to run, the bits must not."""
    inst = CASES[5][1]
    a = run_gpu(inst, 100, "fp32")
    b = run_gpu(inst, 100, "fp32")
    c = run_gpu(inst, 100, "fp32", use_graph=0)
    for other in (b, c):
        assert np.array_equal(a["x"], other["x"]) and np.array_equal(a["lam"], other["lam"])


def test_device_inputs_equal_host_inputs(c1):
    a = run_gpu(c1, 300, "fp32")
    b = run_gpu(c1, 300, "fp32", device=True)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["lam"], b["lam"])


def test_torch_allocator(c1):
    a = run_gpu(c1, 100, "fp64")
    b = run_gpu(c1, 100, "fp64", use_torch_allocator=True)
    assert np.array_equal(a["x"], b["x"])


def test_continue_and_reset(c1):
    from paper_2509_10722_b300 import capi
    whole = run_gpu(c1, 300, "fp64")
    with capi.Problem(c1, precision=1) as p:
        assert p.solve(120, 0.0) == (1, 120)
        assert p.solve(180, 0.0) == (1, 180)
        x, lam, info = p.get()
        assert info["iters"] == 300
        assert np.array_equal(x, whole["x"]) and np.array_equal(lam, whole["lam"])
        p.reset()
        p.solve(300, 0.0)
        x2, lam2, _ = p.get()
        assert np.array_equal(x2, whole["x"])


def test_objective_matches_fp64_utility(c1):
    from oracle import kkt
    g = run_gpu(c1, 400, "fp64")
    assert abs(g["info"]["objective"] - kkt.utility(c1, g["x"])) <= 1e-12 * abs(
        kkt.utility(c1, g["x"]))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_alpha2_objective_and_kkt(precision):
    """U = -w / x streams mixed with log and linear ones: the reported objective is the
    FP64 utility of the returned rates (the FP32 path sums with its FP32 copy of w), and a
    tight FP64 solve satisfies the KKT conditions."""
    from oracle import kkt
    inst = W.random_instance(3000, 400, 1, 6, seed=13, frac_log=0.4, frac_alpha2=0.4,
                             box=(0.0, 20.0))
    eps = 1e-9 if precision == "fp64" else 1e-5
    g = run_gpu(inst, 200_000, precision, eps=eps)
    wi = inst["w"] if precision == "fp64" else inst["w"].astype(np.float32).astype(np.float64)
    u = kkt.utility(dict(inst, w=wi), g["x"])
    assert abs(g["info"]["objective"] - u) <= 1e-12 * abs(u)
    if precision == "fp64":
        d = kkt.diagnostics(inst, g["x"], g["lam"])
        assert d["feas"] < 1e-6 and d["stat"] < 1e-5 and abs(d["gap"]) < 1e-6, d


# ---- the paper's example and closed forms through the GPU path --------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32", "plain"])
def test_alpha2_single_link_closed_form(precision):
    """alpha = 2 fairness on one link: x_j = sqrt(w_j) c / sum sqrt(w), lambda = (sum sqrt(w)
    / c)^2 (w_j / x_j^2 equal to the link price)."""
    w = np.array([1.0, 4.0, 0.25, 2.0])
    c = 3.0
    inst = dict(n=4, m=1, route_ptr=np.arange(5, dtype=np.int64),
                route_links=np.zeros(4, np.int32), c=np.array([c]),
                utype=np.full(4, W.ALPHA2, np.uint8), w=w, lo=np.zeros(4),
                hi=np.full(4, 50.0))
    g = run_gpu(inst, 50_000, precision, eps=1e-6 if precision == "fp32" else 1e-11)
    sw = np.sqrt(w)
    rt = 1e-4 if precision == "fp32" else 1e-7
    assert np.allclose(g["x"], sw * c / sw.sum(), rtol=rt)
    assert np.allclose(g["lam"], [(sw.sum() / c) ** 2], rtol=rt)


def test_four_stream_example_fp32():
    inst = W.four_stream_example()
    g = run_gpu(inst, 10_000, "fp32", eps=1e-5)
    assert np.allclose(g["x"], [1.0, 1 / 3, 2 / 3, 2 / 3], rtol=1e-4)
    assert np.allclose(g["lam"], [1.0, 1.5, 1.5], rtol=1e-4)


def test_profile_times_and_launch_count(c1):
    """Per-kernel CUDA-event times inside replayed graphs, and the launch counter."""
    from paper_2509_10722_b300 import capi
    with capi.Problem(c1, precision=0, profile=1, check_every=10) as p:
        l0 = capi.num_kernel_launches()
        status, done = p.solve(95, 0.0)
        launched = capi.num_kernel_launches() - l0
        ms, runs = p.kernel_times()
    assert done == 95 and list(runs) == [95, 95] and np.all(ms > 0)
    assert launched >= 10 * 10 * 2  # ten replays of ten iterations, two kernels each
    with capi.Problem(c1, precision=2, profile=1, check_every=10) as p:
        p.solve(30, 0.0)
        ms, runs = p.kernel_times()
    assert list(runs) == [30] * 8 and np.all(ms > 0)


@pytest.mark.parametrize("precision,nk", [(0, 2), (2, 8)])
def test_sampled_profile(c1, precision, nk):
    """profile = 2 times the kernels of the first iteration of every replay only (95
    iterations in replays of 10: ten timed launches per kernel), and leaves the iterates
    bit-identical to a run without events."""
    from paper_2509_10722_b300 import capi
    out = []
    for prof in (2, 0):
        with capi.Problem(c1, precision=precision, profile=prof, check_every=10) as p:
            status, done = p.solve(95, 0.0)
            if prof:
                ms, runs = p.kernel_times()
                assert list(runs) == [10] * nk and np.all(ms > 0)
            out.append(p.get()[0])
    assert done == 95 and np.array_equal(out[0], out[1])


def test_sampled_profile_batch(c1):
    from paper_2509_10722_b300 import capi
    insts = [c1, W.random_instance(300, 40, 2, 8, seed=4)]
    with capi.Batch(insts, precision=0, profile=2, check_every=10) as b:
        b.solve(95, 0.0)
        ms, runs = b.kernel_times()
    assert list(runs) == [10, 10] and np.all(ms > 0)


@pytest.mark.parametrize("precision,nk", [(0, 2), (1, 2), (2, 8)])
def test_profile_without_graphs(c1, precision, nk):
    """Per-kernel times with plain launches (use_graph = 0): the events are recorded on the
    stream directly rather than as graph nodes, and the iterates equal the graph path's."""
    from paper_2509_10722_b300 import capi
    out = []
    for g in (0, 1):
        with capi.Problem(c1, precision=precision, profile=1,
                          use_graph=g, check_every=10) as p:
            status, done = p.solve(40, 0.0)
            ms, runs = p.kernel_times()
            x, lam, _ = p.get()
        assert done == 40 and list(runs) == [40] * nk and np.all(ms > 0)
        out.append(x)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("decades", [0, 2, 4])
def test_badly_scaled_instances(decades):
    """Weights and capacities spread over `decades` decades (log-uniform factors): FP32 on
    the oracle's rho decisions stays within the 1e-4 bar (about 2e-6 measured at 4
    decades) and FP64 within 1e-9, after 300 iterations."""
    inst = W.random_instance(3000, 400, 1, 8, seed=100, frac_log=0.7, box=(0.0, 50.0))
    rng = np.random.default_rng(decades)
    inst["w"] = inst["w"] * 10.0 ** rng.uniform(-decades / 2, decades / 2, inst["n"])
    inst["c"] = inst["c"] * 10.0 ** rng.uniform(-decades / 2, decades / 2, inst["m"])
    ref = oracle_run(inst, 300)
    g32 = run_gpu(inst, 300, "fp32", schedule_decisions=ref["decisions"])
    g64 = run_gpu(inst, 300, "fp64")
    assert rel(g32["x"], ref["x"]) <= 1e-4 and rel(g32["lam"], ref["lam"]) <= 1e-4
    assert rel(g64["x"], ref["x"]) <= 1e-9 and rel(g64["lam"], ref["lam"]) <= 1e-9


@pytest.fixture(scope="module")
def many_links():
    """About a million links (not a multiple of 8) for 60,000 streams of 1..6 Zipf-chosen
    links: each link group of a resident grid has many links to sum, so the link kernel
    spreads the epilogues of 8 consecutive links over a group's lanes; most links carry no
    stream, and the hottest carry thousands (summed in chunks by whole warps)."""
    inst = W.random_instance(60_000, 1_000_003, 1, 6, seed=61, link_dist="zipf",
                             frac_log=0.6, frac_alpha2=0.1, box=(0.0, 20.0))
    deg = np.bincount(inst["route_links"], minlength=inst["m"])
    assert deg.max() > 2048 and (deg == 0).mean() > 0.5
    return inst


@pytest.mark.parametrize("precision", ["fp64", "plain"])
def test_many_links_fp64_match_oracle(many_links, precision):
    ref = oracle_run(many_links, 150)
    g = run_gpu(many_links, 150, precision)
    assert rel(g["x"], ref["x"]) <= 1e-9 and rel(g["lam"], ref["lam"]) <= 1e-9


def test_many_links_fp32_match_oracle(many_links):
    ref = oracle_run(many_links, 150)
    g = run_gpu(many_links, 150, "fp32", schedule_decisions=ref["decisions"])
    assert rel(g["x"], ref["x"]) <= 1e-4 and rel(g["lam"], ref["lam"]) <= 1e-4


@pytest.mark.parametrize("m", [500_009, 681_997, 1_048_583])
def test_spread_rounds_cover_every_link(m):
    """Half a million to a million links without any long one: the link kernel runs its
    spread variant without the chunk phase, rounds of 8 links per group dealt out in turn,
    the last round partial by a different amount at each size.  A link left out of every
    round would keep its initial price; element by element against the oracle after 3
    iterations (FP64 1e-10, FP32 1e-4 in norm, ten times that element by element with the
    floor of 1e-3 of the largest value)."""
    inst = W.random_instance(m // 4, m, 1, 4, seed=m % 1000, frac_log=0.7, box=(0.0, 20.0))
    assert np.bincount(inst["route_links"], minlength=m).max() <= 256
    ref = oracle_run(inst, 3)
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
        g = run_gpu(inst, 3, precision)
        e = compare(g, ref, tol)
        assert e["x"] <= tol and e["lam"] <= tol, (precision, e)
        assert e["x_el"] <= 10 * tol and e["lam_el"] <= 10 * tol, (precision, e)


@pytest.mark.parametrize("m,n", [(30_011, 300_007), (120_007, 30_011), (400_009, 700_001)])
def test_grid_rounds_cover_every_stream_and_link(m, n):
    """Below the spread threshold the link kernel runs one group per link, links dealt out
    to a resident grid in turn; the stream kernel deals streams to its threads the same
    way.  Sizes chosen so that both have a partial last round (up to three rounds of
    streams, four of links): element by element against the oracle after 3 iterations."""
    inst = W.random_instance(n, m, 1, 4, seed=(m + n) % 1000, frac_log=0.7, box=(0.0, 20.0))
    ref = oracle_run(inst, 3)
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
        g = run_gpu(inst, 3, precision)
        e = compare(g, ref, tol)
        assert e["x"] <= tol and e["lam"] <= tol, (precision, e)
        assert e["x_el"] <= 10 * tol and e["lam_el"] <= 10 * tol, (precision, e)
