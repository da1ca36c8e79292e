"""The seeded instance generator (no GPU): shapes, ranges, distinct links per route,
reproducibility, and the CSR bookkeeping used to check the device transpose."""
import numpy as np

from paper_2509_10722_b300 import workloads as W


def _check(inst, len_lo, len_hi):
    n, m = inst["n"], inst["m"]
    ptr, links = inst["route_ptr"], inst["route_links"]
    assert ptr.dtype == np.int64 and links.dtype == np.int32
    assert ptr[0] == 0 and ptr[-1] == links.size and np.all(np.diff(ptr) >= 1)
    lengths = np.diff(ptr)
    assert lengths.min() >= len_lo and lengths.max() <= len_hi
    assert links.min() >= 0 and links.max() < m
    for j in range(min(n, 2000)):
        r = links[ptr[j]:ptr[j + 1]]
        assert np.unique(r).size == r.size
    assert np.all(inst["c"] > 0) and np.all(inst["w"] > 0)
    assert np.all(inst["lo"] <= inst["hi"])


def test_c1_recipe():
    inst = W.workload("c1")
    assert inst["n"] == 1000 and inst["m"] == 500
    _check(inst, 2, 6)
    assert np.sum(inst["utype"] == W.LOG) == 500
    assert 1.0 <= inst["c"].min() and inst["c"].max() <= 10.0
    assert 0.5 <= inst["w"].min() and inst["w"].max() <= 2.0
    assert np.all(inst["hi"] == 20.0) and np.all(inst["lo"] == 0.0)


def test_reproducible():
    a = W.workload("c1")
    b = W.workload("c1")
    for k in ("route_ptr", "route_links", "c", "utype", "w"):
        assert np.array_equal(a[k], b[k])
    c = W.workload("c1", seed=1)
    assert not np.array_equal(a["route_links"], c["route_links"])


def test_scaled_c2_statistics():
    inst = W.workload("c2", scale=0.01)       # n = 1e5, m = 1e4
    _check(inst, 1, 10)
    lengths = np.diff(inst["route_ptr"])
    assert abs(lengths.mean() - 5.5) < 0.05
    assert abs(np.mean(inst["utype"] == W.LOG) - 0.7) < 1e-3
    deg = np.bincount(inst["route_links"], minlength=inst["m"])
    assert abs(deg.mean() - 55.0) < 1.0 and deg.max() < 3 * 55


def test_zipf_is_skewed():
    inst = W.workload("c3", scale=0.001)      # n = 2e4, m = 2e3
    _check(inst, 2, 12)
    deg = np.sort(np.bincount(inst["route_links"], minlength=inst["m"]))[::-1]
    # the hottest link is on a large share of the routes; the median link on very few
    assert deg[0] > 0.3 * inst["n"] and np.median(deg) < 20
    assert np.all(inst["utype"] == W.LOG)


def test_long_routes_distinct():
    inst = W.random_instance(50, 200, 60, 120, seed=3)
    _check(inst, 60, 120)


def test_csr_of_matches_dense():
    inst = W.random_instance(37, 11, 1, 6, seed=5)
    row_ptr, col_idx = W.csr_of(inst)
    dense = np.zeros((inst["m"], inst["n"]), dtype=int)
    for j in range(inst["n"]):
        dense[inst["route_links"][inst["route_ptr"][j]:inst["route_ptr"][j + 1]], j] = 1
    for l in range(inst["m"]):
        assert list(col_idx[row_ptr[l]:row_ptr[l + 1]]) == list(np.flatnonzero(dense[l]))


def test_batched_recipe():
    insts = W.batched_instances(count=6, seed=2)
    for inst in insts:
        assert 1000 <= inst["n"] <= 100000
        assert inst["m"] == max(8, inst["n"] // 10)
        _check(inst, 2, 8)


def test_degrade_and_prune_bookkeeping():
    inst = W.random_instance(500, 80, 1, 6, seed=9)
    c2, hit = W.degraded_capacities(inst, p=0.25, factor=0.5, seed=3)
    assert np.allclose(c2[hit], 0.5 * inst["c"][hit]) and np.array_equal(c2[~hit], inst["c"][~hit])
    assert 0.1 < hit.mean() < 0.4
    failed = W.failed_links(inst, p=0.25, seed=4)
    pr, ks, kl = W.prune(inst, failed)
    assert pr["n"] == ks.size and pr["m"] == kl.size == (~failed).sum()
    # every kept stream keeps its whole route (renumbered); no removed stream survives
    for new_j, old_j in enumerate(ks):
        old = inst["route_links"][inst["route_ptr"][old_j]:inst["route_ptr"][old_j + 1]]
        new = pr["route_links"][pr["route_ptr"][new_j]:pr["route_ptr"][new_j + 1]]
        assert not failed[old].any()
        assert np.array_equal(kl[new], old)
    for old_j in np.setdiff1d(np.arange(inst["n"]), ks):
        old = inst["route_links"][inst["route_ptr"][old_j]:inst["route_ptr"][old_j + 1]]
        assert failed[old].any()


def test_hot_links_follow_the_congestion_model():
    """add_hot_links (Sec. V-C): 0.1% of the links each join 10% of the routes; original
    routes stay prefixes, no route repeats a link, the rest of the instance is unchanged."""
    base = W.random_instance(20_000, 5_000, 2, 6, seed=3)
    cong, hot = W.add_hot_links(base, 0.001, 0.10, seed=4)
    assert hot.size == 5 and len(set(hot.tolist())) == 5
    rp0, rl0 = base["route_ptr"], base["route_links"]
    rp1, rl1 = cong["route_ptr"], cong["route_links"]
    assert rp1.size == rp0.size and np.all(np.diff(rp1) >= np.diff(rp0))
    for j in range(base["n"]):
        r0 = rl0[rp0[j]:rp0[j + 1]]
        r1 = rl1[rp1[j]:rp1[j + 1]]
        assert np.array_equal(r1[:r0.size], r0)
        assert len(set(r1.tolist())) == r1.size
        assert set(r1[r0.size:].tolist()) <= set(hot.tolist())
    deg0 = np.bincount(rl0, minlength=base["m"])
    deg1 = np.bincount(rl1, minlength=base["m"])
    # each hot link reaches 10% of the streams (fewer only where a route already had it)
    assert np.all(deg1[hot] >= 2_000) and np.all(deg1[hot] <= 2_000 + deg0[hot])
    others = np.setdiff1d(np.arange(base["m"]), hot)
    assert np.array_equal(deg1[others], deg0[others])
    for k in ("c", "utype", "w", "lo", "hi"):
        assert cong[k] is base[k]
