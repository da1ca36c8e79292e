"""FP64 CPU oracle of proximal message passing for NUM -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this package.  It shares no code with the CUDA path: the solver is the plain C file
`pmp_oracle.c` (a literal per-terminal ADMM, Sec. III) compiled with gcc and called through
ctypes; `kkt.py` evaluates the KKT conditions of Sec. II / VI-B with numpy.

Parity status: every function here is pinned by `tests/test_oracle_*.py` (prox against
bisection, closed-form networks, independent dual and LP solvers, residual definitions
recomputed from the recovered primal variables, and planted-mistake variants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs = {}


class _Params(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("mu", ctypes.c_double), ("gamma", ctypes.c_double),
                ("eps_abs", ctypes.c_double), ("period", ctypes.c_int64),
                ("max_iters", ctypes.c_int64), ("debug", ctypes.c_int32),
                ("switch_iter", ctypes.c_int64), ("c_switch", ctypes.c_void_p)]


def lib_path(plant=0):
    name = "libpmp_oracle.so" if not plant else f"libpmp_oracle_plant{plant}.so"
    return os.path.join(_BUILD, name)


def build(plant=0, force=False):
    """Compile the oracle (gcc -O2, single thread).  `plant` > 0 builds a variant with one
    planted mistake, used only by the tests that show the pins catch such mistakes."""
    out = lib_path(plant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    if plant:
        cmd.insert(1, f"-DORACLE_PLANT={int(plant)}")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(plant=0):
    with _lock:
        if plant not in _libs:
            lib = ctypes.CDLL(build(plant))
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
            P = ctypes.c_void_p
            lib.oracle_prox_log.restype = d
            lib.oracle_prox_log.argtypes = [d, d, d, d, d, d]
            lib.oracle_prox_linear.restype = d
            lib.oracle_prox_linear.argtypes = [d, d, d, d, d, d]
            lib.oracle_prox_alpha2.restype = d
            lib.oracle_prox_alpha2.argtypes = [d, d, d, d, d, d]
            lib.oracle_prox_slack.restype = d
            lib.oracle_prox_slack.argtypes = [d, d]
            lib.oracle_solve.restype = ctypes.c_int
            lib.oracle_solve.argtypes = [i64, i64, P, P, P, P, P, P, P,
                                         ctypes.POINTER(_Params), P, i64, P, P, P, P, P,
                                         ctypes.POINTER(i64), ctypes.POINTER(i32),
                                         ctypes.POINTER(d)]
            _libs[plant] = lib
        return _libs[plant]


def prox_log(S, L, w, rho, lo, hi, plant=0):
    return _lib(plant).oracle_prox_log(S, L, w, rho, lo, hi)


def prox_linear(S, L, w, rho, lo, hi, plant=0):
    return _lib(plant).oracle_prox_linear(S, L, w, rho, lo, hi)


def prox_alpha2(S, L, w, rho, lo, hi, plant=0):
    return _lib(plant).oracle_prox_alpha2(S, L, w, rho, lo, hi)


def prox_slack(zeta, c, plant=0):
    return _lib(plant).oracle_prox_slack(zeta, c)


DEFAULTS = dict(rho0=1.0, alpha=1.6, mu=2.0, gamma=1.1, eps_abs=1e-4, period=50)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def solve(inst, max_iters, *, eps_abs=None, rho0=None, alpha=None, mu=None, gamma=None,
          period=None, rho_replay=None, debug=False, plant=0, c_switch=None, switch_iter=0):
    """Run the literal PMP of Sec. III on `inst` (see workloads.py for the layout).

    c_switch / switch_iter: after `switch_iter` iterations the capacities become c_switch
    and the run continues from its current iterate (the warm start of Sec. V-D).

    Returns a dict: x[n], slack[m], lam[m] (prices rho u), hist[k, 3] = (||r||, ||s||, rho)
    per iteration, decisions (rho decision at each update point), iters, converged,
    identity_violation (debug only).  eps_abs <= 0 runs exactly max_iters iterations.
    """
    prm = dict(DEFAULTS)
    for k, v in dict(eps_abs=eps_abs, rho0=rho0, alpha=alpha, mu=mu, gamma=gamma,
                     period=period).items():
        if v is not None:
            prm[k] = v
    n, m = int(inst["n"]), int(inst["m"])
    rp = np.ascontiguousarray(inst["route_ptr"], dtype=np.int64)
    rl = np.ascontiguousarray(inst["route_links"], dtype=np.int32)
    c = np.ascontiguousarray(inst["c"], dtype=np.float64)
    ut = np.ascontiguousarray(inst["utype"], dtype=np.uint8)
    w = np.ascontiguousarray(inst["w"], dtype=np.float64)
    lo = np.ascontiguousarray(inst["lo"], dtype=np.float64)
    hi = np.ascontiguousarray(inst["hi"], dtype=np.float64)
    x = np.zeros(n)
    slack = np.zeros(m)
    lam = np.zeros(m)
    hist = np.zeros((max(int(max_iters), 1), 3))
    ndec = max(int(max_iters) // max(int(prm["period"]), 1), 1)
    dec = np.zeros(ndec, dtype=np.int8)
    iters = ctypes.c_int64(0)
    conv = ctypes.c_int32(0)
    viol = ctypes.c_double(0.0)
    cs = None if c_switch is None else np.ascontiguousarray(c_switch, dtype=np.float64)
    p = _Params(prm["rho0"], prm["alpha"], prm["mu"], prm["gamma"], prm["eps_abs"],
                int(prm["period"]), int(max_iters), 1 if debug else 0,
                int(switch_iter) if cs is not None else 0,
                None if cs is None else cs.ctypes.data)
    if rho_replay is not None:
        rr = np.ascontiguousarray(rho_replay, dtype=np.int8)
        rr_ptr, rr_len = _ptr(rr), rr.size
    else:
        rr, rr_ptr, rr_len = None, None, 0
    rc = _lib(plant).oracle_solve(n, m, _ptr(rp), _ptr(rl), _ptr(c), _ptr(ut), _ptr(w),
                                  _ptr(lo), _ptr(hi), ctypes.byref(p), rr_ptr, rr_len,
                                  _ptr(x), _ptr(slack), _ptr(lam), _ptr(hist), _ptr(dec),
                                  ctypes.byref(iters), ctypes.byref(conv), ctypes.byref(viol))
    if rc != 0:
        raise ValueError("oracle_solve rejected the instance")
    k = int(iters.value)
    nd = k // int(prm["period"]) if prm["period"] > 0 else 0
    if conv.value and prm["period"] > 0 and k % int(prm["period"]) == 0:
        nd -= 1  # the stopping test passed before the update point of the last iteration
    return dict(x=x, slack=slack, lam=lam, hist=hist[:k].copy(), decisions=dec[:max(nd, 0)].copy(),
                iters=k, converged=bool(conv.value), identity_violation=float(viol.value),
                params=prm)
