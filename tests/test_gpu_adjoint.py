"""The GPU adjoint (num_adjoint) against the CPU reference gradient (plain PyTorch autograd
through the literal per-terminal ADMM, itself pinned against finite differences of the C
oracle) and against finite differences of the GPU forward, with the rho decisions fixed."""
import numpy as np
import pytest

from gpu_util import oracle_run, rel
from oracle import adjoint_ref
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return W.random_instance(300, 60, 1, 6, seed=41, frac_log=0.7, box=(0.0, 20.0))


@pytest.fixture(scope="module")
def small_a2():
    return W.random_instance(300, 60, 1, 6, seed=42, frac_log=0.4, frac_alpha2=0.4,
                             box=(0.0, 20.0))


@pytest.fixture(scope="module")
def slice_c5():
    # a 10^3-stream slice of the differentiation recipe: routes of 2..8 links, log
    # utilities, w ~ U[0.5, 2], box [0, 20], m = n / 10
    return W.random_instance(1000, 100, 2, 8, seed=5, frac_log=1.0, box=(0.0, 20.0))


def _gpu_adjoint(inst, iters, precision, kc=50, xbar=None, objective=True, sched=None):
    from paper_2509_10722_b300 import capi
    with capi.Problem(inst, precision=precision, history=max(iters, 1)) as p:
        if sched is not None:
            p.set_rho_schedule(sched)
        return p.adjoint(iters, kc, xbar=xbar, objective=objective)


@pytest.mark.parametrize("precision,tol", [(1, 1e-9), (2, 1e-9)])
def test_fp64_adjoint_equals_reference(small, precision, tol):
    iters = 120
    dec = oracle_run(small, iters)["decisions"]
    gc, gw, J = _gpu_adjoint(small, iters, precision)
    rc, rw, rJ = adjoint_ref.gradients(small, iters, dec)
    assert abs(J - rJ) <= 1e-12 * abs(rJ)
    assert rel(gc, rc) <= tol and rel(gw, rw) <= tol


@pytest.mark.parametrize("precision,tol", [(1, 1e-9), (0, 1e-3)])
def test_alpha2_adjoint_equals_reference(small_a2, precision, tol):
    iters = 120
    dec = oracle_run(small_a2, iters)["decisions"]
    gc, gw, J = _gpu_adjoint(small_a2, iters, precision, sched=dec)
    rc, rw, rJ = adjoint_ref.gradients(small_a2, iters, dec)
    assert abs(J - rJ) <= max(tol, 1e-12) * abs(rJ)
    assert rel(gc, rc) <= tol and rel(gw, rw) <= tol


@pytest.fixture(scope="module")
def skewed():
    """Zipf link choice: the hottest link has 3,342 streams (two chunks of 2,048 entries)
    and 14 links have more than 256, so the backward link pass takes its chunk path."""
    inst = W.random_instance(6000, 30, 1, 4, seed=43, link_dist="zipf", frac_log=0.7,
                             box=(0.0, 20.0))
    deg = np.bincount(inst["route_links"], minlength=inst["m"])
    assert deg.max() > 2048 and (deg > 256).sum() > 5
    return inst


@pytest.mark.parametrize("precision,tol", [(1, 1e-9), (0, 1e-3)])
def test_skewed_adjoint_equals_reference(skewed, precision, tol):
    iters = 120
    dec = oracle_run(skewed, iters)["decisions"]
    gc, gw, J = _gpu_adjoint(skewed, iters, precision, sched=dec)
    rc, rw, rJ = adjoint_ref.gradients(skewed, iters, dec)
    assert abs(J - rJ) <= max(tol, 1e-12) * abs(rJ)
    assert rel(gc, rc) <= tol and rel(gw, rw) <= tol


def test_vjp_equals_reference(small):
    iters = 120
    dec = oracle_run(small, iters)["decisions"]
    xbar = np.random.default_rng(3).standard_normal(small["n"])
    gc, gw, _ = _gpu_adjoint(small, iters, 1, xbar=xbar, objective=False)
    rc, rw, _ = adjoint_ref.gradients(small, iters, dec, xbar=xbar, objective=False)
    assert rel(gc, rc) <= 1e-9 and rel(gw, rw) <= 1e-9


def test_fp32_adjoint_near_reference(small):
    iters = 120
    dec = oracle_run(small, iters)["decisions"]
    gc, gw, _ = _gpu_adjoint(small, iters, 0, sched=dec)
    rc, rw, _ = adjoint_ref.gradients(small, iters, dec)
    assert rel(gc, rc) <= 1e-3 and rel(gw, rw) <= 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpointing_does_not_change_the_result(small, precision):
    a = _gpu_adjoint(small, 130, precision, kc=0)
    b = _gpu_adjoint(small, 130, precision, kc=7)
    c = _gpu_adjoint(small, 130, precision, kc=50)
    for other in (b, c):
        assert np.array_equal(a[0], other[0]) and np.array_equal(a[1], other[1])


def test_adjoint_equals_gpu_finite_differences(small):
    """Central differences (step 1e-4, FP64) of the GPU forward's utility, rho decisions
    fixed to the unperturbed run's."""
    from oracle import kkt
    from paper_2509_10722_b300 import capi
    iters = 120
    dec = oracle_run(small, iters)["decisions"]
    gc, gw, _ = _gpu_adjoint(small, iters, 1)

    def J(c, w):
        with capi.Problem(small, precision=1) as p:
            p.set_rho_schedule(dec)
            p.set_capacity(c)
            p.set_weights(w)
            p.solve(iters, 0.0)
            x, _, _ = p.get(prices=False)
        return kkt.utility(dict(small, w=w), x)

    rng = np.random.default_rng(1)
    for l in rng.choice(small["m"], 4, replace=False):
        h = 1e-4
        cp, cm = small["c"].copy(), small["c"].copy()
        cp[l] += h
        cm[l] -= h
        fd = (J(cp, small["w"]) - J(cm, small["w"])) / (2 * h)
        assert abs(fd - gc[l]) <= 1e-5 * max(1.0, abs(gc[l])), (l, fd, gc[l])
    for j in rng.choice(small["n"], 4, replace=False):
        h = 1e-4
        wp, wm = small["w"].copy(), small["w"].copy()
        wp[j] += h
        wm[j] -= h
        fd = (J(small["c"], wp) - J(small["c"], wm)) / (2 * h)
        assert abs(fd - gw[j]) <= 1e-5 * max(1.0, abs(gw[j])), (j, fd, gw[j])


def test_c5_slice_500_iterations(slice_c5):
    """The differentiation recipe: 500 unrolled iterations, checkpoints every 50, FP64
    against the CPU reference gradient; FP32 on the same rho schedule close to it."""
    iters = 500
    dec = oracle_run(slice_c5, iters)["decisions"]
    rc, rw, _ = adjoint_ref.gradients(slice_c5, iters, dec)
    gc, gw, _ = _gpu_adjoint(slice_c5, iters, 1, kc=50)
    assert rel(gc, rc) <= 1e-8 and rel(gw, rw) <= 1e-8
    fc, fw, _ = _gpu_adjoint(slice_c5, iters, 0, kc=50, sched=dec)
    assert rel(fc, rc) <= 1e-2 and rel(fw, rw) <= 1e-2


def test_autograd_function(small):
    import torch
    from paper_2509_10722_b300 import autograd, capi
    iters = 120
    c = torch.tensor(small["c"], requires_grad=True)
    w = torch.tensor(small["w"], requires_grad=True)
    with capi.Problem(small, precision=1) as p:
        J = autograd.total_utility(p, small["utype"], c, w, iters)
        J.backward()
        gc, gw, J2 = p.adjoint(iters, 50)
    assert abs(float(J.detach()) - J2) <= 1e-12 * abs(J2)
    assert rel(c.grad.numpy(), gc) <= 1e-12 and rel(w.grad.numpy(), gw) <= 1e-12


def test_c5_full_size_fp32_gradients_track_fp64():
    """Full differentiation recipe (n = 1e6, m = 1e5, 500 iterations, checkpoints every
    50): FP32 gradients within 1e-4 of the FP64 ones (5e-7 measured)."""
    inst = W.workload("c5")
    c32, w32, _ = _gpu_adjoint(inst, 500, 0, kc=50)
    c64, w64, _ = _gpu_adjoint(inst, 500, 1, kc=50)
    assert rel(c32, c64) <= 1e-4 and rel(w32, w64) <= 1e-4
