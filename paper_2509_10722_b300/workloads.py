"""Seeded synthetic NUM instances (the only module shared by the oracle side and the CUDA side).

This module draws random problem data and nothing else: it holds none of the method's
arithmetic (no prox, no averaging, no residuals).  Every instance is a plain dict of numpy
arrays in the layout the C ABI takes:

    n, m          number of traffic streams and of links
    route_ptr     int64[n+1]   CSC column pointer of the 0/1 link-route matrix R (Sec. II)
    route_links   int32[nnz]   link ids of each route, stream-major; no duplicate within a route
    c             float64[m]   link capacities, > 0
    utype         uint8[n]     0 = w log x utility, 1 = w x utility
    w             float64[n]   utility weights, > 0
    lo, hi        float64[n]   box of each stream rate

The five named workloads follow the instance recipes stated for this build (uniform routes
without replacement, Zipf-skewed link choice for the congested case); the paper itself only
says its matrices are random with about ten links per route (Sec. V-B) and that congestion
makes a few links carry a large share of the streams (Sec. V-C).
"""
from __future__ import annotations

import numpy as np

LOG = 0
LINEAR = 1
ALPHA2 = 2  # U = -w / x, alpha = 2 fairness (minimum potential delay)


def _dedupe_routes(rng, route_ptr, links, draw, max_rounds=10_000):
    """Redraw every link id that repeats an earlier id of the same route until none repeats.

    Redrawing a repeated id from the same distribution is rejection sampling, so a route of
    length L drawn this way is a sample of L distinct links (without replacement).
    """
    n = route_ptr.size - 1
    lengths = np.diff(route_ptr)
    nnz = links.size
    if nnz == 0:
        return links
    maxlen = int(lengths.max())
    if maxlen <= 64:
        # first pass over every route, later passes only over the routes that had a repeat
        routes = np.arange(n, dtype=np.int64)
        for _ in range(max_rounds):
            lens = lengths[routes]
            sub_ptr = np.zeros(routes.size + 1, dtype=np.int64)
            np.cumsum(lens, out=sub_ptr[1:])
            total = int(sub_ptr[-1])
            owner = np.repeat(np.arange(routes.size, dtype=np.int64), lens)
            pos = np.arange(total, dtype=np.int64) - sub_ptr[:-1][owner]
            gidx = route_ptr[:-1][routes][owner] + pos   # positions in the full link array
            sub = links[gidx]
            bad = np.zeros(total, dtype=bool)
            for d in range(1, int(lens.max()) if lens.size else 0):
                eq = sub[d:] == sub[:-d]
                eq &= pos[d:] >= d
                bad[d:] |= eq
            idx = np.flatnonzero(bad)
            if idx.size == 0:
                return links
            links[gidx[idx]] = draw(idx.size)
            routes = np.unique(routes[owner[idx]])
        raise RuntimeError("could not draw distinct links for every route")
    route_of = np.repeat(np.arange(n, dtype=np.int64), lengths)
    for _ in range(max_rounds):
        order = np.lexsort((np.arange(nnz), links, route_of))
        sl = links[order]
        sr = route_of[order]
        dup = (sl[1:] == sl[:-1]) & (sr[1:] == sr[:-1])
        idx = order[1:][dup]
        if idx.size == 0:
            return links
        links[idx] = draw(idx.size)
    raise RuntimeError("could not draw distinct links for every route")


def _zipf_sampler(rng, m, s):
    """Truncated Zipf(s) over ranks 1..m by inverse CDF, ranks mapped to link ids by a seeded
    random permutation (so the hot links are spread over the id range)."""
    ranks = np.arange(1, m + 1, dtype=np.float64)
    pmf = ranks ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    perm = rng.permutation(m).astype(np.int32)

    def draw(k):
        u = rng.random(k)
        r = np.searchsorted(cdf, u, side="right")
        np.minimum(r, m - 1, out=r)
        return perm[r]

    return draw


def random_instance(n, m, len_lo, len_hi, *, seed=0, link_dist="uniform", zipf_s=1.1,
                    c_lo=1.0, c_hi=10.0, c_scale=1.0, frac_log=0.5, w_dist="uniform",
                    w_lo=0.5, w_hi=2.0, box=(0.0, 20.0), degrade=None, frac_alpha2=0.0):
    """Draw one NUM instance.

    len_lo..len_hi    route length, uniform over the integers in that range (capped at m)
    link_dist         "uniform" (links uniform without replacement) or "zipf"
    frac_log          fraction of streams with log utility (exact count, random positions)
    frac_alpha2       fraction with U = -w / x (alpha = 2 fairness), taken from the others
    w_dist            "uniform" (U[w_lo, w_hi]) or "lognormal" (LogNormal(0, 0.5))
    box               (lo, hi) applied to every stream, or a callable(rng, n) -> (lo, hi) arrays
    degrade           None or (lo, hi): capacities multiplied by a per-link U[lo, hi] factor
    """
    if n < 1 or m < 1:
        raise ValueError("n and m must be positive")
    rng = np.random.default_rng(seed)
    len_hi = min(len_hi, m)
    len_lo = max(1, min(len_lo, len_hi))
    lengths = rng.integers(len_lo, len_hi + 1, size=n, dtype=np.int64)
    route_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=route_ptr[1:])
    nnz = int(route_ptr[-1])
    if link_dist == "uniform":
        def draw(k):
            return rng.integers(0, m, size=k, dtype=np.int64).astype(np.int32)
    elif link_dist == "zipf":
        draw = _zipf_sampler(rng, m, zipf_s)
    else:
        raise ValueError(link_dist)
    links = draw(nnz).astype(np.int32)
    links = _dedupe_routes(rng, route_ptr, links, draw)
    c = rng.uniform(c_lo, c_hi, size=m) * c_scale
    if degrade is not None:
        c = c * rng.uniform(degrade[0], degrade[1], size=m)
    n_log = int(round(frac_log * n))
    utype = np.full(n, LINEAR, dtype=np.uint8)
    order = rng.permutation(n)
    utype[order[:n_log]] = LOG
    if frac_alpha2 > 0.0:
        n_a2 = min(int(round(frac_alpha2 * n)), n - n_log)
        utype[order[n_log:n_log + n_a2]] = ALPHA2
    if w_dist == "uniform":
        w = rng.uniform(w_lo, w_hi, size=n)
    elif w_dist == "lognormal":
        w = rng.lognormal(0.0, 0.5, size=n)
    else:
        raise ValueError(w_dist)
    if callable(box):
        lo, hi = box(rng, n)
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
    else:
        lo = np.full(n, float(box[0]))
        hi = np.full(n, float(box[1]))
    return dict(n=int(n), m=int(m), route_ptr=route_ptr, route_links=links, c=c,
                utype=utype, w=w, lo=lo, hi=hi)


def add_hot_links(inst, frac_links=0.001, frac_streams=0.10, seed=1):
    """The congestion model of Sec. V-C on top of an instance: pick round(frac_links * m)
    links at random and add each of them to the routes of round(frac_streams * n) streams
    drawn at random (a stream that already uses the link is left as it is).  Every original
    route stays the prefix of its new route; the hot links follow in the order they were
    drawn.  Returns a new instance dict with its own route arrays (the rest is shared) and
    the hot link ids."""
    rng = np.random.default_rng(seed)
    n, m = int(inst["n"]), int(inst["m"])
    route_ptr = np.asarray(inst["route_ptr"], dtype=np.int64)
    links = np.asarray(inst["route_links"], dtype=np.int32)
    k = max(1, int(round(frac_links * m)))
    s = max(1, int(round(frac_streams * n)))
    hot = rng.choice(m, size=k, replace=False).astype(np.int32)
    pair_s = np.concatenate([rng.choice(n, size=s, replace=False) for _ in range(k)])
    pair_l = np.repeat(hot, s)
    lengths = np.diff(route_ptr)
    owner = np.repeat(np.arange(n, dtype=np.int64), lengths)
    is_hot = np.zeros(m, dtype=bool)
    is_hot[hot] = True
    sel = is_hot[links]
    if sel.any():  # (stream, link) pairs the routes already have
        have = owner[sel] * m + links[sel].astype(np.int64)
        keep = ~np.isin(pair_s.astype(np.int64) * m + pair_l, have)
        pair_s, pair_l = pair_s[keep], pair_l[keep]
    order = np.argsort(pair_s, kind="stable")
    ps, pl = pair_s[order].astype(np.int64), pair_l[order]
    extra = np.bincount(ps, minlength=n)
    new_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths + extra, out=new_ptr[1:])
    out = np.empty(int(new_ptr[-1]), dtype=np.int32)
    out[new_ptr[owner] + (np.arange(links.size, dtype=np.int64) - route_ptr[owner])] = links
    rank = np.arange(ps.size, dtype=np.int64) - np.searchsorted(ps, ps, side="left")
    out[new_ptr[ps] + lengths[ps] + rank] = pl
    cong = dict(inst)
    cong["route_ptr"] = new_ptr
    cong["route_links"] = out
    return cong, hot


def congestion_pair(scale=1.0, seed=0):
    """The uncongested and congested networks of Sec. V-C at the size of its degree
    histograms (m = 1e6 links, n = 5e5 streams): routes of U{5..15} uniform links (mean
    10), c ~ U[1,10], 70% log / 30% linear, w ~ U[0.5,2], box [0, 50]; the congested one
    adds 0.1% of the links to 10% of the streams each.  `scale` shrinks n and m together."""
    n = max(1, int(round(500_000 * scale)))
    m = max(1, int(round(1_000_000 * scale)))
    base = random_instance(n, m, 5, 15, seed=seed, frac_log=0.7, box=(0.0, 50.0))
    cong, hot = add_hot_links(base, 0.001, 0.10, seed=seed + 1)
    return base, cong, hot


# ---------------------------------------------------------------------------------------------
# The named workloads.  Sizes, distributions and boxes are the ones the instance recipes state;
# C4 (batched) and C5 (differentiation) are listed for completeness of the recipe table.

WORKLOADS = {
    # small FP64 parity case: 2,000 iterations
    "c1": dict(n=1_000, m=500, len_lo=2, len_hi=6, frac_log=0.5, box=(0.0, 20.0), seed=0),
    # headline: n = 1e7 streams, m = 1e6 links, about 5.5e7 nonzeros
    "c2": dict(n=10_000_000, m=1_000_000, len_lo=1, len_hi=10, frac_log=0.7,
               box=(0.0, 50.0), seed=0),
    # congested, skewed: Zipf(1.1) link choice, capacities scaled by 0.1, all log utilities
    "c3": dict(n=20_000_000, m=2_000_000, len_lo=2, len_hi=12, link_dist="zipf",
               zipf_s=1.1, c_scale=0.1, frac_log=1.0, w_dist="lognormal",
               box=(0.0, 10.0), seed=0),
    # differentiation case (forward solve only is used here)
    "c5": dict(n=1_000_000, m=100_000, len_lo=2, len_hi=8, frac_log=1.0,
               box=(0.0, 20.0), seed=0),
}

WORKLOAD_ITERS = {"c1": 2000}


def workload(name, seed=None, scale=None):
    """Instance for a named workload.  `scale` (> 0) multiplies n and m together, keeping
    route lengths and distributions: below 1 for CPU-sized stand-ins of a large case, above
    1 for larger instances of the same recipe."""
    spec = dict(WORKLOADS[name])
    if seed is not None:
        spec["seed"] = seed
    if scale is not None:
        spec["n"] = max(1, int(round(spec["n"] * scale)))
        spec["m"] = max(1, int(round(spec["m"] * scale)))
    n = spec.pop("n")
    m = spec.pop("m")
    lo = spec.pop("len_lo")
    hi = spec.pop("len_hi")
    return random_instance(n, m, lo, hi, **spec)


def batched_instances(count=256, seed=0, congested=False):
    """Batched-solve recipe: `count` independent instances, n log-uniform in [1e3, 1e5],
    m = n/10, routes of 2..8 uniform links, capacities U[1,10] times a per-link U[0.3,1]
    degradation factor, 70% log utilities, box [0, 20].  congested=True draws the links of
    every route from a truncated Zipf(1.1) instead (a few links carry most streams), the
    congestion scenario of the batched recipe."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(1e3), np.log(1e5), size=count)).astype(np.int64)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for n, s in zip(ns, seeds):
        m = max(8, int(n) // 10)
        out.append(random_instance(int(n), m, 2, 8, seed=int(s), frac_log=0.7,
                                   box=(0.0, 20.0), degrade=(0.3, 1.0),
                                   link_dist="zipf" if congested else "uniform"))
    return out


def degraded_capacities(inst, p=0.25, factor=0.5, seed=1):
    """Capacity degradation of Sec. V-D: every link independently keeps its capacity, or
    with probability p has it multiplied by `factor`."""
    rng = np.random.default_rng(seed)
    hit = rng.random(inst["m"]) < p
    return np.where(hit, inst["c"] * factor, inst["c"]), hit


def failed_links(inst, p=0.25, seed=2):
    """Link failures of Sec. V-D: every link fails independently with probability p."""
    rng = np.random.default_rng(seed)
    return rng.random(inst["m"]) < p


def prune(inst, failed):
    """The instance left after link failures (Sec. V-D): failed links leave R, and so does
    every stream whose route uses one of them.  Returns (pruned instance, kept stream ids,
    kept link ids), ids in the original numbering, in increasing order."""
    failed = np.asarray(failed, dtype=bool)
    lengths = np.diff(inst["route_ptr"])
    route_of = np.repeat(np.arange(inst["n"]), lengths)
    dead_stream = np.zeros(inst["n"], dtype=bool)
    np.logical_or.at(dead_stream, route_of, failed[inst["route_links"]])
    keep_s = np.flatnonzero(~dead_stream)
    keep_l = np.flatnonzero(~failed)
    if keep_s.size == 0 or keep_l.size == 0:
        raise ValueError("no stream or no link survives")
    new_link = np.full(inst["m"], -1, dtype=np.int64)
    new_link[keep_l] = np.arange(keep_l.size)
    keep_entry = ~dead_stream[route_of]
    route_ptr = np.zeros(keep_s.size + 1, dtype=np.int64)
    np.cumsum(lengths[keep_s], out=route_ptr[1:])
    out = dict(n=int(keep_s.size), m=int(keep_l.size), route_ptr=route_ptr,
               route_links=new_link[inst["route_links"][keep_entry]].astype(np.int32),
               c=inst["c"][keep_l], utype=inst["utype"][keep_s], w=inst["w"][keep_s],
               lo=inst["lo"][keep_s], hi=inst["hi"][keep_s])
    return out, keep_s, keep_l


def four_stream_example():
    """The four-stream, three-link network of the paper's small example (Sec. III-A):
    R = [[1,0,0,0],[0,1,1,0],[0,1,0,1]].  The paper gives only the structure; capacities 1,
    weights 1 and log utilities are this fixture's choice."""
    route_ptr = np.array([0, 1, 3, 4, 5], dtype=np.int64)
    route_links = np.array([0, 1, 2, 1, 2], dtype=np.int32)
    n, m = 4, 3
    return dict(n=n, m=m, route_ptr=route_ptr, route_links=route_links,
                c=np.ones(m), utype=np.zeros(n, dtype=np.uint8), w=np.ones(n),
                lo=np.zeros(n), hi=np.full(n, 1e3))


def instance_bytes(inst):
    """Bytes the C ABI copies host-to-device for one instance."""
    return sum(int(inst[k].nbytes) for k in ("route_ptr", "route_links", "c", "utype", "w",
                                            "lo", "hi"))


def csr_of(inst):
    """Row-major (link-major) copy of R: (row_ptr int64[m+1], col_idx int32[nnz]) with each
    row's stream ids ascending.  Pure index bookkeeping used to check the device transpose."""
    n, m = inst["n"], inst["m"]
    lengths = np.diff(inst["route_ptr"])
    stream_of = np.repeat(np.arange(n, dtype=np.int32), lengths)
    order = np.argsort(inst["route_links"], kind="stable")
    col_idx = stream_of[order]
    counts = np.bincount(inst["route_links"], minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, col_idx.astype(np.int32)
