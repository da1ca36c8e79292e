"""Thin Python binding of the C ABI in include/num_pmp.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no arithmetic of
its own: arrays are checked for dtype / length and passed by pointer, status codes become
`NumError` exceptions.  The shared library is loaded from the package's `lib/` folder; if
it is missing the import of this module fails loudly (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

# the in-tree library; NUM_PMP_LIBRARY may name another build of it (the debug build,
# lib/libnum_pmp_debug.so, whose kernels check every gathered index)
_LIB_PATH = os.environ.get("NUM_PMP_LIBRARY") or os.path.join(
    os.path.dirname(os.path.abspath(__file__)), "lib", "libnum_pmp.so")

NUM_OK = 0
NUM_NOT_CONVERGED = 1
NUM_ERR_INVALID = -1
NUM_ERR_OOM = -2
NUM_ERR_CUDA = -3
NUM_ERR_NUMERIC = -4
NUM_ERR_STATE = -5
NUM_ERR_TIMEOUT = -6

NUM_LOG = 0
NUM_LINEAR = 1
NUM_ALPHA2 = 2

NUM_FUSED_FP32 = 0
NUM_FUSED_FP64 = 1
NUM_PLAIN_FP64 = 2


INFO = dict(primal=0, dual=1, eps_tol=2, rho=3, objective=4, iters=5, status=6, J=7)
NUM_INFO_LEN = 8

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                              ctypes.c_void_p)


class num_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


class num_params(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("alpha", ctypes.c_double), ("mu", ctypes.c_double),
                ("gamma", ctypes.c_double), ("eps_abs", ctypes.c_double),
                ("rho_period", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("check_every", ctypes.c_int32),
                ("history", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("reorder", ctypes.c_int32),
                ("profile", ctypes.c_int32),
                ("allocator", ctypes.POINTER(num_allocator))]


class num_instance(ctypes.Structure):
    """One instance of a batch (host arrays, its own link ids)."""
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("route_ptr", ctypes.c_void_p), ("route_links", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("utype", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p)]


class BatchSchedule(ctypes.Structure):
    """num_batch_schedule: work partition of a batch's kernels."""
    _fields_ = [("stream_item", ctypes.c_int32), ("link_item", ctypes.c_int32),
                ("link_lanes", ctypes.c_int32)]

    def as_tuple(self):
        return (self.stream_item, self.link_item, self.link_lanes)


class NumError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{num_strerror(code)} ({code}): {message}")
        self.code = code


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -m paper_2509_10722_b300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    pp = ctypes.POINTER(num_params)
    sig = {
        "num_default_params": (None, [pp]),
        "num_create": (ctypes.c_int, [ctypes.POINTER(P), i64, i64, P, P, P, P, P, P, P, pp, P]),
        "num_create_device": (ctypes.c_int, [ctypes.POINTER(P), i64, i64, P, P, P, P, P, P, P,
                                             pp, P]),
        "num_set_rho_schedule": (ctypes.c_int, [P, P, i64]),
        "num_solve": (ctypes.c_int, [P, i64, d, ctypes.POINTER(i64)]),
        "num_get": (ctypes.c_int, [P, P, P, P]),
        "num_get_device": (ctypes.c_int, [P, P, P, P]),
        "num_get_history": (ctypes.c_int, [P, P, i64, ctypes.POINTER(i64)]),
        "num_get_operator": (ctypes.c_int, [P, P, P]),
        "num_reset": (ctypes.c_int, [P]),
        "num_set_capacity": (ctypes.c_int, [P, P]),
        "num_set_weights": (ctypes.c_int, [P, P]),
        "num_adjoint": (ctypes.c_int, [P, i64, i32, P, i32, P, P, ctypes.POINTER(d)]),
        "num_adjoint_forward": (ctypes.c_int, [P, i64, i32]),
        "num_adjoint_backward": (ctypes.c_int, [P, P, d, P, P]),
        "num_adjoint_release": (ctypes.c_int, [P]),
        "num_set_capacity_device": (ctypes.c_int, [P, P]),
        "num_set_weights_device": (ctypes.c_int, [P, P]),
        "num_get_state": (ctypes.c_int, [P, P, P, P, P, P, P, P, ctypes.POINTER(d)]),
        "num_set_state": (ctypes.c_int, [P, P, P, P, P, P, P, P, d]),
        "num_iteration_bytes": (ctypes.c_int, [P, P]),
        "num_get_kernel_times": (ctypes.c_int, [P, P, P, i32, ctypes.POINTER(i32)]),
        "num_kernel_launches": (ctypes.c_int64, []),
        "num_objective_noalloc": (ctypes.c_int, [i64, P, P, P, P, P]),
        "num_measure_gather_rate": (ctypes.c_int, [i64, i64, i32, i32, ctypes.POINTER(d)]),
        "num_measure_scatter_rate": (ctypes.c_int, [i64, i64, i32, i32, ctypes.POINTER(d)]),
        "num_batch_create": (ctypes.c_int, [ctypes.POINTER(P), i32, P, P, P, P, P, P, P, P, P,
                                            pp, P]),
        "num_batch_create_instances": (ctypes.c_int, [ctypes.POINTER(P), i32,
                                                      ctypes.POINTER(num_instance), pp, P]),
        "num_batch_set_rho_schedules": (ctypes.c_int, [P, P, i64]),
        "num_batch_solve": (ctypes.c_int, [P, i64, d, P, P]),
        "num_batch_get": (ctypes.c_int, [P, P, P, P]),
        "num_batch_get_kernel_times": (ctypes.c_int, [P, P, P, i32, ctypes.POINTER(i32)]),
        "num_batch_get_schedule": (ctypes.c_int, [P, ctypes.POINTER(BatchSchedule)]),
        "num_batch_set_schedule": (ctypes.c_int, [P, ctypes.POINTER(BatchSchedule)]),
        "num_batch_autotune": (ctypes.c_int, [P, i32, ctypes.POINTER(BatchSchedule), P, i32,
                                              ctypes.POINTER(i32)]),
        "num_batch_set_persistent": (ctypes.c_int, [P, i32, i64]),
        "num_batch_reset": (ctypes.c_int, [P]),
        "num_batch_destroy": (None, [P]),
        "num_destroy": (None, [P]),
        "num_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "num_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("num_default_params", "num_create", "num_create_device", "num_set_rho_schedule",
            "num_solve", "num_get", "num_get_device", "num_get_history", "num_get_operator",
            "num_reset", "num_set_capacity", "num_set_weights", "num_adjoint",
            "num_adjoint_forward", "num_adjoint_backward", "num_adjoint_release",
            "num_set_capacity_device", "num_set_weights_device",
            "num_get_state", "num_set_state",
            "num_iteration_bytes", "num_get_kernel_times", "num_kernel_launches",
            "num_objective_noalloc", "num_measure_gather_rate", "num_measure_scatter_rate",
            "num_destroy", "num_strerror",
            "num_last_error",
            "num_batch_create", "num_batch_create_instances", "num_batch_set_rho_schedules",
            "num_batch_solve",
            "num_batch_get", "num_batch_get_kernel_times", "num_batch_get_schedule",
            "num_batch_set_schedule", "num_batch_autotune", "num_batch_set_persistent",
            "num_batch_reset", "num_batch_destroy")


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib


def library_path():
    return _LIB_PATH


def num_strerror(code):
    return _lib.num_strerror(int(code)).decode()


def num_last_error():
    return _lib.num_last_error().decode()


def _check(rc):
    if rc < 0:
        raise NumError(rc, num_last_error())
    return rc


def num_default_params(**overrides):
    p = num_params()
    _lib.num_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _host(a, dtype, n, name):
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.shape != (n,):
        raise ValueError(f"{name} must have shape ({n},), got {a.shape}")
    return a


def _hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def num_create(n, m, route_ptr, route_links, c, utype, w, lo, hi, params=None, stream=None):
    """Create a handle from host arrays (numpy); returns the handle (a c_void_p)."""
    n, m = int(n), int(m)
    rp = _host(route_ptr, np.int64, n + 1, "route_ptr")
    nnz = int(rp[-1]) if rp[0] == 0 and rp[-1] >= 0 else 0
    rl = np.ascontiguousarray(route_links, dtype=np.int32)
    if rl.size < nnz:
        raise ValueError("route_links shorter than route_ptr[n]")
    args = [rp, rl, _host(c, np.float64, m, "c"), _host(utype, np.uint8, n, "utype"),
            _host(w, np.float64, n, "w"),
            None if lo is None else _host(lo, np.float64, n, "lo"), _host(hi, np.float64, n, "hi")]
    h = ctypes.c_void_p()
    keep = params
    _check(_lib.num_create(ctypes.byref(h), n, m, *[_hptr(a) for a in args],
                           None if params is None else ctypes.byref(params),
                           ctypes.c_void_p(stream) if stream else None))
    del keep
    return h


def _dptr(t, dtype_name, n, name):
    import torch
    want = getattr(torch, dtype_name)
    if t is None:
        return None
    if not t.is_cuda or t.dtype != want or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype_name} tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def num_create_device(n, m, route_ptr, route_links, c, utype, w, lo, hi, params=None,
                      stream=None):
    """Create a handle from device arrays (torch CUDA tensors, same layout)."""
    n, m = int(n), int(m)
    nnz = int(route_links.numel())
    ptrs = [_dptr(route_ptr, "int64", n + 1, "route_ptr"),
            _dptr(route_links, "int32", nnz, "route_links"), _dptr(c, "float64", m, "c"),
            _dptr(utype, "uint8", n, "utype"), _dptr(w, "float64", n, "w"),
            _dptr(lo, "float64", n, "lo"), _dptr(hi, "float64", n, "hi")]
    h = ctypes.c_void_p()
    _check(_lib.num_create_device(ctypes.byref(h), n, m, *ptrs,
                                  None if params is None else ctypes.byref(params),
                                  ctypes.c_void_p(stream) if stream else None))
    return h


def num_set_rho_schedule(h, decisions):
    d = np.ascontiguousarray(decisions, dtype=np.int8)
    _check(_lib.num_set_rho_schedule(h, _hptr(d) if d.size else None, d.size))


def num_solve(h, max_iters, eps_abs=-1.0):
    """Returns (status, iterations run): status NUM_OK or NUM_NOT_CONVERGED."""
    it = ctypes.c_int64(0)
    rc = _check(_lib.num_solve(h, int(max_iters), float(eps_abs), ctypes.byref(it)))
    return rc, int(it.value)


def num_get(h, n, m, x=True, prices=True, out_x=None, out_prices=None):
    """Host copies: returns (x[n] or None, prices[m] or None, info dict).  out_x / out_prices
    (float64 numpy arrays of n / m values, e.g. views of pinned memory) receive the copies
    instead of new arrays."""
    xa = (out_x if out_x is not None else np.empty(n)) if x else None
    pa = (out_prices if out_prices is not None else np.empty(m)) if prices else None
    for a, k, name in ((xa, n, "out_x"), (pa, m, "out_prices")):
        if a is not None and (a.dtype != np.float64 or a.size != k or not a.flags.c_contiguous):
            raise ValueError(f"{name} must be a contiguous float64 array of {k} values")
    info = np.zeros(NUM_INFO_LEN)
    _check(_lib.num_get(h, _hptr(xa), _hptr(pa), _hptr(info)))
    return xa, pa, {k: float(info[i]) for k, i in INFO.items()}


def num_get_device(h, x=None, prices=None, n=None, m=None):
    """Write x / prices into float64 CUDA tensors (either may be None); returns info dict.
    The library writes n values to x and m to prices: pass n and m to have the tensor
    sizes checked (a smaller tensor would be overrun)."""
    info = np.zeros(NUM_INFO_LEN)
    xp = None if x is None else _dptr(x, "float64", x.numel() if n is None else int(n), "x")
    pp = None if prices is None else _dptr(prices, "float64",
                                           prices.numel() if m is None else int(m), "prices")
    _check(_lib.num_get_device(h, xp, pp, _hptr(info)))
    return {k: float(info[i]) for k, i in INFO.items()}


def num_get_history(h, max_rows):
    buf = np.zeros((max(int(max_rows), 0), 3))
    rows = ctypes.c_int64(0)
    _check(_lib.num_get_history(h, _hptr(buf) if max_rows else None, int(max_rows),
                                ctypes.byref(rows)))
    return buf[:rows.value]


def num_get_operator(h, m, nnz):
    rp = np.zeros(m + 1, dtype=np.int64)
    ci = np.zeros(nnz, dtype=np.int32)
    _check(_lib.num_get_operator(h, _hptr(rp), _hptr(ci)))
    return rp, ci


def num_reset(h):
    _check(_lib.num_reset(h))


STATE_FIELDS = ("x", "Z", "pbar", "y", "zs", "Rx", "ps")


def num_set_capacity(h, m, c):
    _check(_lib.num_set_capacity(h, _hptr(_host(c, np.float64, int(m), "c"))))


def num_set_weights(h, n, w):
    _check(_lib.num_set_weights(h, _hptr(_host(w, np.float64, int(n), "w"))))


def num_adjoint(h, n, m, iters, checkpoint_every=50, xbar=None, objective=True):
    """Gradients of `iters` unrolled iterations from the zero state: returns
    (dJ/dc [m], dJ/dw [n], U) for J = xbar . x (+ sum_j U_j(x_j) if objective), with U the
    total utility sum_j U_j(x_j) at the final rates."""
    cg = np.empty(int(m))
    wg = np.empty(int(n))
    xb = None if xbar is None else _host(xbar, np.float64, int(n), "xbar")
    obj = ctypes.c_double(0.0)
    _check(_lib.num_adjoint(h, int(iters), int(checkpoint_every), _hptr(xb),
                            1 if objective else 0, _hptr(cg), _hptr(wg), ctypes.byref(obj)))
    return cg, wg, obj.value


def num_set_capacity_device(h, m, c):
    """c: contiguous float64 CUDA tensor of m values."""
    _check(_lib.num_set_capacity_device(h, _dptr(c, "float64", int(m), "c")))


def num_set_weights_device(h, n, w):
    """w: contiguous float64 CUDA tensor of n values (caller order)."""
    _check(_lib.num_set_weights_device(h, _dptr(w, "float64", int(n), "w")))


def num_adjoint_forward(h, iters, checkpoint_every=50):
    _check(_lib.num_adjoint_forward(h, int(iters), int(checkpoint_every)))


def num_adjoint_backward(h, n, m, xbar=None, ubar=0.0, c_grad=None, w_grad=None):
    """Device tensors: xbar [n] (or None), c_grad [m], w_grad [n] (float64, CUDA)."""
    _check(_lib.num_adjoint_backward(h, _dptr(xbar, "float64", int(n), "xbar"), float(ubar),
                                     _dptr(c_grad, "float64", int(m), "c_grad"),
                                     _dptr(w_grad, "float64", int(n), "w_grad")))


def num_adjoint_release(h):
    _check(_lib.num_adjoint_release(h))


def num_get_state(h, n, m):
    """The iterate as a dict of FP64 arrays (streams in the caller's order) plus rho."""
    st = {k: np.empty(n if k in ("x", "Z") else m) for k in STATE_FIELDS}
    rho = ctypes.c_double(0.0)
    _check(_lib.num_get_state(h, *[_hptr(st[k]) for k in STATE_FIELDS], ctypes.byref(rho)))
    st["rho"] = rho.value
    return st


def num_set_state(h, n, m, state):
    """Start a fresh run from `state` (dict as from num_get_state; missing arrays kept)."""
    arrs = []
    for k in STATE_FIELDS:
        a = state.get(k)
        arrs.append(None if a is None else _host(a, np.float64, n if k in ("x", "Z") else m, k))
    _check(_lib.num_set_state(h, *[_hptr(a) for a in arrs], float(state["rho"])))


def num_iteration_bytes(h):
    out = np.zeros(2)
    _check(_lib.num_iteration_bytes(h, _hptr(out)))
    return float(out[0]), float(out[1])


def num_get_kernel_times(h, max_kernels=8):
    """Per-kernel (total ms, launches that did work) of the profiled iterations."""
    ms = np.zeros(max_kernels)
    cnt = np.zeros(max_kernels, dtype=np.int64)
    nk = ctypes.c_int32(0)
    _check(_lib.num_get_kernel_times(h, _hptr(ms), _hptr(cnt), max_kernels, ctypes.byref(nk)))
    k = min(nk.value, max_kernels)
    return ms[:k], cnt[:k]


def num_kernel_launches():
    return int(_lib.num_kernel_launches())


def num_objective_noalloc(n, x, utype, w, objective, stream=None):
    """sum_j U_j(x_j) of CUDA tensors x (float64), utype (uint8), w (float64) into the
    CUDA float64 tensor `objective` (first element), allocating nothing."""
    n = int(n)
    _check(_lib.num_objective_noalloc(n, _dptr(x, "float64", n, "x"),
                                      _dptr(utype, "uint8", n, "utype"),
                                      _dptr(w, "float64", n, "w"),
                                      _dptr(objective, "float64", max(objective.numel(), 1),
                                            "objective"),
                                      ctypes.c_void_p(stream) if stream else None))


def num_measure_gather_rate(count, vec_len, vec_bytes, repeats=5):
    """Uniformly random 4- or 8-byte reads per second from a vector of vec_len elements."""
    out = ctypes.c_double(0.0)
    _check(_lib.num_measure_gather_rate(int(count), int(vec_len), int(vec_bytes), int(repeats),
                                        ctypes.byref(out)))
    return out.value


def num_measure_scatter_rate(count, vec_len, vec_bytes, repeats=5):
    """Uniformly random 4- or 8-byte stores per second to a vector of vec_len elements."""
    out = ctypes.c_double(0.0)
    _check(_lib.num_measure_scatter_rate(int(count), int(vec_len), int(vec_bytes),
                                         int(repeats), ctypes.byref(out)))
    return out.value


def num_destroy(h):
    _lib.num_destroy(h)


def stack_instances(insts):
    """Stack instance dicts block-diagonally: returns (stream_off, link_off, stacked dict)
    with global link ids (pure index bookkeeping for num_batch_create).  Each output array
    is allocated once and filled slice by slice."""
    k = len(insts)
    so = np.zeros(k + 1, dtype=np.int64)
    lo = np.zeros(k + 1, dtype=np.int64)
    eo = np.zeros(k + 1, dtype=np.int64)
    for i, t in enumerate(insts):
        so[i + 1] = so[i] + int(t["n"])
        lo[i + 1] = lo[i] + int(t["m"])
        eo[i + 1] = eo[i] + int(t["route_ptr"][-1])
    if lo[-1] >= 2**31:
        raise ValueError("the stacked problem has 2^31 or more links")
    route_ptr = np.empty(int(so[-1]) + 1, dtype=np.int64)
    route_ptr[0] = 0
    route_links = np.empty(int(eo[-1]), dtype=np.int32)
    for i, t in enumerate(insts):
        np.add(np.asarray(t["route_ptr"][1:], np.int64), eo[i],
               out=route_ptr[so[i] + 1:so[i + 1] + 1])
        np.add(np.asarray(t["route_links"], np.int32), np.int32(lo[i]),
               out=route_links[eo[i]:eo[i + 1]])
    cat = {key: np.concatenate([np.asarray(t[key]) for t in insts])
           for key in ("c", "utype", "w", "lo", "hi")}
    stacked = dict(n=int(so[-1]), m=int(lo[-1]), route_ptr=route_ptr, route_links=route_links,
                   **cat)
    return so, lo, stacked


class Batch:
    """Owner of a num_batch over a list of instance dicts (see workloads.py)."""

    def __init__(self, insts, stream=None, **params):
        """The instances are passed one by one (num_batch_create_instances): the library
        stacks them on the device, so nothing is concatenated on the host."""
        self.count = len(insts)
        self.so = np.zeros(self.count + 1, dtype=np.int64)
        self.lo = np.zeros(self.count + 1, dtype=np.int64)
        np.cumsum([int(t["n"]) for t in insts], out=self.so[1:])
        np.cumsum([int(t["m"]) for t in insts], out=self.lo[1:])
        self.n, self.m = int(self.so[-1]), int(self.lo[-1])
        self.params = num_default_params(**params)
        keep = []  # the arrays must stay alive during the call

        def arr(a, dtype, size, name):
            a = np.ascontiguousarray(a, dtype=dtype)
            if a.shape != (size,):
                raise ValueError(f"{name} must have {size} elements, got {a.shape}")
            keep.append(a)
            return a.ctypes.data

        table = (num_instance * self.count)()
        for i, t in enumerate(insts):
            n, m = int(t["n"]), int(t["m"])
            rp = arr(t["route_ptr"], np.int64, n + 1, "route_ptr")
            nnz = int(keep[-1][-1]) if keep[-1][0] == 0 else 0
            rl = np.ascontiguousarray(t["route_links"], dtype=np.int32)
            if rl.size < nnz:
                raise ValueError("route_links shorter than route_ptr[n]")
            keep.append(rl)
            lo = t.get("lo")
            table[i] = num_instance(n, m, rp, rl.ctypes.data, arr(t["c"], np.float64, m, "c"),
                                    arr(t["utype"], np.uint8, n, "utype"),
                                    arr(t["w"], np.float64, n, "w"),
                                    None if lo is None else arr(lo, np.float64, n, "lo"),
                                    arr(t["hi"], np.float64, n, "hi"))
        h = ctypes.c_void_p()
        _check(_lib.num_batch_create_instances(ctypes.byref(h), self.count, table,
                                               ctypes.byref(self.params),
                                               ctypes.c_void_p(stream) if stream else None))
        del keep
        self.h = h

    def set_rho_schedules(self, decisions):
        """decisions: int8 array (count, len)."""
        d = np.ascontiguousarray(decisions, dtype=np.int8)
        _check(_lib.num_batch_set_rho_schedules(self.h, _hptr(d) if d.size else None,
                                                d.shape[1] if d.ndim == 2 else 0))

    def solve(self, max_iters, eps_abs=-1.0):
        it = np.zeros(self.count, dtype=np.int64)
        stt = np.zeros(self.count, dtype=np.int32)
        rc = _check(_lib.num_batch_solve(self.h, int(max_iters), float(eps_abs), _hptr(it),
                                         _hptr(stt)))
        return rc, it, stt

    def get(self, out_x=None, out_prices=None):
        """Per-instance lists of x and prices, and an info dict per instance.  out_x /
        out_prices (contiguous float64 arrays of the total n / m, e.g. views of pinned
        memory) receive the stacked results instead of new arrays; the lists are views."""
        x = np.empty(self.n) if out_x is None else out_x
        p = np.empty(self.m) if out_prices is None else out_prices
        for a, k, name in ((x, self.n, "out_x"), (p, self.m, "out_prices")):
            if a.dtype != np.float64 or a.size != k or not a.flags.c_contiguous:
                raise ValueError(f"{name} must be a contiguous float64 array of {k} values")
        info = np.zeros((self.count, NUM_INFO_LEN))
        _check(_lib.num_batch_get(self.h, _hptr(x), _hptr(p), _hptr(info)))
        xs = [x[self.so[i]:self.so[i + 1]] for i in range(self.count)]
        ps = [p[self.lo[i]:self.lo[i + 1]] for i in range(self.count)]
        infos = [{k: float(info[i, j]) for k, j in INFO.items()} for i in range(self.count)]
        return xs, ps, infos

    def kernel_times(self):
        ms = np.zeros(2)
        cnt = np.zeros(2, dtype=np.int64)
        nk = ctypes.c_int32(0)
        _check(_lib.num_batch_get_kernel_times(self.h, _hptr(ms), _hptr(cnt), 2, ctypes.byref(nk)))
        return ms, cnt

    def schedule(self):
        """(stream_item, link_item, link_lanes) in use."""
        out = BatchSchedule()
        _check(_lib.num_batch_get_schedule(self.h, ctypes.byref(out)))
        return out.as_tuple()

    def set_schedule(self, stream_item, link_item, link_lanes):
        s = BatchSchedule(int(stream_item), int(link_item), int(link_lanes))
        _check(_lib.num_batch_set_schedule(self.h, ctypes.byref(s)))

    def autotune(self, trial_iters=20):
        """Run the autotuner; returns (chosen (stream_item, link_item, link_lanes), trials)
        with trials an array of rows (stream_item, link_item, link_lanes, ms)."""
        out = BatchSchedule()
        trials = np.zeros((64, 4))
        nt = ctypes.c_int32(0)
        _check(_lib.num_batch_autotune(self.h, int(trial_iters), ctypes.byref(out), _hptr(trials),
                                       64, ctypes.byref(nt)))
        return out.as_tuple(), trials[:min(nt.value, 64)]

    def set_persistent(self, enable=True, wait_polls=0):
        """Persistent form of solve (one cooperative launch per check_every iterations,
        a team of blocks per instance); wait_polls bounds each wait between blocks."""
        _check(_lib.num_batch_set_persistent(self.h, int(bool(enable)), int(wait_polls)))

    def reset(self):
        _check(_lib.num_batch_reset(self.h))

    def close(self):
        if getattr(self, "h", None) is not None:
            _lib.num_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def torch_allocator():
    """A num_allocator that takes device memory from PyTorch's caching allocator (the
    returned object must stay alive as long as the handles that use it)."""
    import torch

    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
        except Exception:
            return None

    def _release(ctx, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    a = num_allocator(ALLOC_FN(_alloc), RELEASE_FN(_release), None)
    return a


class Problem:
    """Owner of one handle: `Problem(inst, **params)` with an instance dict as made by
    `workloads.py`; `device=True` copies the instance to torch CUDA tensors first and uses
    num_create_device."""

    def __init__(self, inst, device=False, stream=None, use_torch_allocator=False, **params):
        self.n, self.m = int(inst["n"]), int(inst["m"])
        self.nnz = int(np.asarray(inst["route_ptr"])[-1])
        self._alloc = torch_allocator() if use_torch_allocator else None
        if self._alloc is not None:
            params["allocator"] = ctypes.pointer(self._alloc)
        self.params = num_default_params(**params)
        self.h = None
        if device:
            import torch
            dev = {k: torch.as_tensor(np.ascontiguousarray(inst[k])).cuda()
                   for k in ("route_ptr", "route_links", "c", "utype", "w", "lo", "hi")}
            self.h = num_create_device(self.n, self.m, dev["route_ptr"], dev["route_links"],
                                       dev["c"], dev["utype"], dev["w"], dev["lo"], dev["hi"],
                                       self.params, stream)
        else:
            self.h = num_create(self.n, self.m, inst["route_ptr"], inst["route_links"],
                                inst["c"], inst["utype"], inst["w"], inst["lo"], inst["hi"],
                                self.params, stream)

    def solve(self, max_iters, eps_abs=-1.0):
        return num_solve(self.h, max_iters, eps_abs)

    def get(self, x=True, prices=True):
        return num_get(self.h, self.n, self.m, x, prices)

    def get_device(self, x=None, prices=None):
        """x / prices into float64 CUDA tensors of n / m values; returns the info dict."""
        return num_get_device(self.h, x, prices, self.n, self.m)

    def history(self, max_rows=None):
        return num_get_history(self.h, self.params.history if max_rows is None else max_rows)

    def operator(self):
        return num_get_operator(self.h, self.m, self.nnz)

    def set_rho_schedule(self, decisions):
        num_set_rho_schedule(self.h, decisions)

    def reset(self):
        num_reset(self.h)

    def set_capacity(self, c):
        num_set_capacity(self.h, self.m, c)

    def set_weights(self, w):
        num_set_weights(self.h, self.n, w)

    def adjoint(self, iters, checkpoint_every=50, xbar=None, objective=True):
        return num_adjoint(self.h, self.n, self.m, iters, checkpoint_every, xbar, objective)

    def set_capacity_device(self, c):
        num_set_capacity_device(self.h, self.m, c)

    def set_weights_device(self, w):
        num_set_weights_device(self.h, self.n, w)

    def adjoint_forward(self, iters, checkpoint_every=50):
        num_adjoint_forward(self.h, iters, checkpoint_every)

    def adjoint_backward(self, xbar=None, ubar=0.0, c_grad=None, w_grad=None):
        num_adjoint_backward(self.h, self.n, self.m, xbar, ubar, c_grad, w_grad)

    def adjoint_release(self):
        num_adjoint_release(self.h)

    def get_state(self):
        return num_get_state(self.h, self.n, self.m)

    def set_state(self, state):
        num_set_state(self.h, self.n, self.m, state)

    def iteration_bytes(self):
        return num_iteration_bytes(self.h)

    def kernel_times(self):
        return num_get_kernel_times(self.h)

    def close(self):
        if self.h is not None:
            num_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
