"""The CPU reference gradient (oracle/adjoint_ref.py) against the C oracle: the same x
after the same iterations, and gradients equal to central finite differences of the C
oracle's utility with the rho decisions held fixed (no GPU)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint_ref, kkt
from paper_2509_10722_b300 import workloads as W


@pytest.fixture(scope="module", params=["log_linear", "with_alpha2"])
def inst(request):
    a2 = 0.3 if request.param == "with_alpha2" else 0.0
    return W.random_instance(40, 12, 1, 4, seed=31, frac_log=0.5, frac_alpha2=a2,
                             box=(0.0, 20.0))


def test_reference_forward_equals_oracle(inst):
    iters = 120
    ref = oracle.solve(inst, iters, eps_abs=0.0)
    c = torch.tensor(inst["c"])
    w = torch.tensor(inst["w"])
    x = adjoint_ref.unrolled_x(inst, iters, c, w, ref["decisions"]).numpy()
    assert np.max(np.abs(x - ref["x"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["x"])))


def _J(inst, iters, dec, c=None, w=None):
    t = dict(inst)
    if c is not None:
        t["c"] = c
    if w is not None:
        t["w"] = w
    r = oracle.solve(t, iters, eps_abs=0.0, rho_replay=dec)
    return kkt.utility(t, r["x"])


def test_reference_gradient_equals_finite_differences(inst):
    # steps of 1e-6 relative: at 1e-4 a clip of some stream switches inside +-h
    iters = 120
    dec = oracle.solve(inst, iters, eps_abs=0.0)["decisions"]
    gc, gw, J = adjoint_ref.gradients(inst, iters, dec)
    assert abs(J - _J(inst, iters, dec)) <= 1e-12 * abs(J)
    rng = np.random.default_rng(0)
    for l in rng.choice(inst["m"], 5, replace=False):
        h = 1e-6 * inst["c"][l]
        cp, cm = inst["c"].copy(), inst["c"].copy()
        cp[l] += h
        cm[l] -= h
        fd = (_J(inst, iters, dec, c=cp) - _J(inst, iters, dec, c=cm)) / (2 * h)
        assert abs(fd - gc[l]) <= 1e-6 * max(1.0, abs(gc[l])), (l, fd, gc[l])
    for j in rng.choice(inst["n"], 5, replace=False):
        h = 1e-6 * inst["w"][j]
        wp, wm = inst["w"].copy(), inst["w"].copy()
        wp[j] += h
        wm[j] -= h
        fd = (_J(inst, iters, dec, w=wp) - _J(inst, iters, dec, w=wm)) / (2 * h)
        assert abs(fd - gw[j]) <= 1e-6 * max(1.0, abs(gw[j])), (j, fd, gw[j])
