"""The C ABI without a GPU: the library loads, exports every symbol include/num_pmp.h
declares, and rejects malformed calls on the host before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_10722_b300 import build as B


@pytest.fixture(scope="module")
def capi():
    B.build()
    from paper_2509_10722_b300 import capi as C
    return C


def _declared():
    text = open(os.path.join(B.INCLUDE, "num_pmp.h")).read()
    return sorted(set(re.findall(r"NUM_API\s+[\w\s\*]*?\b(num_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(capi):
    names = _declared()
    assert len(names) == 41
    lib = ctypes.CDLL(capi.library_path())
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(capi.EXPORTED)


def test_debug_build_exports_the_same_symbols(capi):
    """The debug build (gather bounds checks compiled in) has the same C ABI."""
    path = B.build(debug=True)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_and_defaults(capi):
    assert capi.num_strerror(0) == "ok"
    assert "invalid" in capi.num_strerror(-1)
    assert capi.num_strerror(12345) == "unknown status code"
    p = capi.num_default_params()
    assert (p.rho0, p.alpha, p.mu, p.gamma, p.eps_abs) == (1.0, 1.6, 2.0, 1.1, 1e-4)
    assert (p.rho_period, p.precision, p.check_every, p.use_graph) == (50, 0, 50, 1)


def _tiny():
    return dict(n=2, m=1, route_ptr=np.array([0, 1, 2]), route_links=np.array([0, 0]),
                c=np.ones(1), utype=np.zeros(2), w=np.ones(2), lo=None, hi=np.ones(2))


def _create(capi, params=None, **over):
    a = _tiny()
    a.update(over)
    return capi.num_create(a["n"], a["m"], a["route_ptr"], a["route_links"], a["c"],
                           a["utype"], a["w"], a["lo"], a["hi"], params)


@pytest.mark.parametrize("over,msg", [
    (dict(n=0, route_ptr=np.array([0]), utype=np.zeros(0), w=np.zeros(0), hi=np.zeros(0)),
     "n and m"),
    (dict(m=0, c=np.zeros(0)), "n and m"),
    (dict(route_ptr=np.array([1, 2, 3])), "route_ptr[0]"),
    (dict(route_ptr=np.array([0, 1, 1])), "empty"),
])
def test_host_rejections(capi, over, msg):
    with pytest.raises(capi.NumError) as ei:
        _create(capi, **over)
    assert ei.value.code == capi.NUM_ERR_INVALID and msg in str(ei.value)


def test_size_limit_rejected_before_allocation(capi):
    """route_ptr[n] beyond the 32-bit index range: rejected from route_ptr alone, through
    the raw entry point (route_links is never read)."""
    rp = np.array([0, 1, 2**31], dtype=np.int64)
    rl = np.zeros(2, np.int32)
    c, w, hi = np.ones(1), np.ones(2), np.ones(2)
    ut = np.zeros(2, np.uint8)
    h = ctypes.c_void_p()
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    rc = capi.library().num_create(ctypes.byref(h), 2, 1, ptr(rp), ptr(rl), ptr(c), ptr(ut),
                                   ptr(w), None, ptr(hi), None, None)
    assert rc == capi.NUM_ERR_INVALID and "2^31" in capi.num_last_error() and not h.value


@pytest.mark.parametrize("field,value", [("alpha", 2.5), ("rho0", -1.0), ("mu", 0.5),
                                         ("gamma", 0.9), ("precision", 7), ("check_every", 0),
                                         ("history", -1),
                                         ("rho_period", -5), ("profile", 3),
                                         ("profile", -1)])
def test_bad_params(capi, field, value):
    p = capi.num_default_params(**{field: value})
    with pytest.raises(capi.NumError) as ei:
        _create(capi, params=p)
    assert ei.value.code == capi.NUM_ERR_INVALID


def test_failing_allocator_reports_oom(capi):
    calls = []

    def alloc(ctx, nbytes, stream):
        calls.append(nbytes)
        return None

    def release(ctx, ptr, nbytes, stream):
        raise AssertionError("nothing was allocated")

    a = capi.num_allocator(capi.ALLOC_FN(alloc), capi.RELEASE_FN(release), None)
    p = capi.num_default_params(allocator=ctypes.pointer(a))
    with pytest.raises(capi.NumError) as ei:
        _create(capi, params=p)
    assert ei.value.code == capi.NUM_ERR_OOM and len(calls) == 1


def test_allocator_blocks_are_aligned_to_16_bytes(capi):
    """The kernels read 16-byte pairs: a block the caller's allocator returns off a 16-byte
    boundary is handed back at once and asked again 16 bytes larger; every block is
    released with the address and size the allocator saw."""
    live = {}
    calls = []
    counter = [0]
    fake = [0x10000]

    def alloc(ctx, nbytes, stream):
        counter[0] += 1
        if counter[0] == 9:
            return None
        fake[0] += 1 << 20
        ptr = fake[0] + (8 if counter[0] % 2 else 0)  # every other block misaligned
        live[ptr] = nbytes
        calls.append((ptr, nbytes))
        return ptr

    def release(ctx, ptr, nbytes, stream):
        assert live.pop(ptr) == nbytes

    a = capi.num_allocator(capi.ALLOC_FN(alloc), capi.RELEASE_FN(release), None)
    p = capi.num_default_params(allocator=ctypes.pointer(a))
    with pytest.raises(capi.NumError) as ei:
        _create(capi, params=p)
    assert ei.value.code == capi.NUM_ERR_OOM and counter[0] == 9 and not live
    for i, (ptr, nbytes) in enumerate(calls):
        if ptr % 16:
            assert calls[i + 1][1] == nbytes + 16


def test_allocator_failing_midway_releases_everything(capi):
    """The k-th allocation fails: every earlier block is handed back, none twice."""
    live = {}
    counter = [0]
    fake = [0x10000]

    def alloc(ctx, nbytes, stream):
        counter[0] += 1
        if counter[0] == 6:
            return None
        fake[0] += 1 << 20
        live[fake[0]] = nbytes
        return fake[0]

    def release(ctx, ptr, nbytes, stream):
        assert live.pop(ptr) == nbytes

    a = capi.num_allocator(capi.ALLOC_FN(alloc), capi.RELEASE_FN(release), None)
    p = capi.num_default_params(allocator=ctypes.pointer(a))
    with pytest.raises(capi.NumError) as ei:
        _create(capi, params=p)
    assert ei.value.code == capi.NUM_ERR_OOM and counter[0] == 6 and not live


def test_null_handle_calls(capi):
    with pytest.raises(capi.NumError):
        capi.num_solve(None, 10)
    with pytest.raises(capi.NumError):
        capi.num_reset(None)
    capi.num_destroy(None)
    lib = capi.library()
    assert lib.num_batch_set_persistent(None, 1, 0) == capi.NUM_ERR_INVALID
    assert lib.num_batch_reset(None) == capi.NUM_ERR_INVALID
    assert "wait between blocks" in capi.num_strerror(capi.NUM_ERR_TIMEOUT)


@pytest.mark.parametrize("so,lo,msg", [([0], [0], "count"), ([1, 2], [0, 1], "must be 0"),
                                       ([0, 0], [0, 1], "stream"), ([0, 1], [0, 0], "stream")])
def test_batch_host_rejections(capi, so, lo, msg):
    so = np.array(so, np.int64)
    lo = np.array(lo, np.int64)
    h = ctypes.c_void_p()
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    rp = np.array([0, 1], np.int64)
    rl = np.zeros(1, np.int32)
    one = np.ones(1)
    ut = np.zeros(1, np.uint8)
    rc = capi.library().num_batch_create(ctypes.byref(h), len(so) - 1, ptr(so), ptr(lo), ptr(rp),
                                         ptr(rl), ptr(one), ptr(ut), ptr(one), None, ptr(one),
                                         None, None)
    assert rc == capi.NUM_ERR_INVALID and not h.value


def _instance(capi, keep, n=2, m=1, rp0=0, links=None):
    rp = np.array([rp0] + list(range(1, n + 1)), np.int64)
    rl = np.zeros(n, np.int32) if links is None else np.array(links, np.int32)
    arrs = [rp, rl, np.ones(m), np.zeros(n, np.uint8), np.ones(n), np.ones(n)]
    keep.extend(arrs)
    p = [ctypes.c_void_p(a.ctypes.data) for a in arrs]
    return capi.num_instance(n, m, p[0], p[1], p[2], p[3], p[4], None, p[5])


@pytest.mark.parametrize("case,msg", [("count", "count"), ("empty_n", "n, m >= 1"),
                                      ("null", "NULL"), ("rp0", "route_ptr[0]"),
                                      ("empty_route", "empty route")])
def test_batch_instances_host_rejections(capi, case, msg):
    """num_batch_create_instances checks sizes, pointers and route offsets of every
    instance on the host, before any CUDA call."""
    keep = []
    insts = (capi.num_instance * 2)(_instance(capi, keep), _instance(capi, keep))
    count = 2
    if case == "count":
        count = 0
    elif case == "empty_n":
        insts[1].n = 0
    elif case == "null":
        insts[0].w = None
    elif case == "rp0":
        insts[1] = _instance(capi, keep, rp0=1)
    else:
        rp = np.array([0, 1, 1], np.int64)  # route_ptr[n] = 1 < n = 2
        keep.append(rp)
        insts[1].route_ptr = ctypes.c_void_p(rp.ctypes.data)
    h = ctypes.c_void_p()
    rc = capi.library().num_batch_create_instances(ctypes.byref(h), count, insts, None, None)
    assert rc == capi.NUM_ERR_INVALID and msg in capi.num_last_error() and not h.value


def test_batch_binding_checks_array_sizes(capi):
    """The binding refuses an instance whose arrays do not match its n and m before it
    calls the library."""
    from paper_2509_10722_b300 import workloads as W
    t = W.random_instance(20, 5, 1, 3, seed=1)
    bad = dict(t, c=np.ones(4))
    with pytest.raises(ValueError):
        capi.Batch([t, bad])
