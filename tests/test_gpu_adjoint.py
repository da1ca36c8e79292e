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
    # FP32 iterates and cotangents against the FP64 reference gradient
    assert rel(gc, rc) <= 1e-4 and rel(gw, rw) <= 1e-4


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
    against the CPU reference gradient; FP32 on the same rho schedule within 1e-4."""
    iters = 500
    dec = oracle_run(slice_c5, iters)["decisions"]
    rc, rw, _ = adjoint_ref.gradients(slice_c5, iters, dec)
    gc, gw, _ = _gpu_adjoint(slice_c5, iters, 1, kc=50)
    assert rel(gc, rc) <= 1e-8 and rel(gw, rw) <= 1e-8
    fc, fw, _ = _gpu_adjoint(slice_c5, iters, 0, kc=50, sched=dec)
    assert rel(fc, rc) <= 1e-4 and rel(fw, rw) <= 1e-4


def test_autograd_function(small):
    """total_utility and solve_x through torch autograd equal num_adjoint (host entry), and
    the torch path runs the forward map once: its launches are the forward, the recomputed
    segments and the backward sweep, with no second forward from zero."""
    import torch
    from paper_2509_10722_b300 import autograd, capi
    iters, kc = 120, 50
    c = torch.tensor(small["c"], requires_grad=True)
    w = torch.tensor(small["w"], requires_grad=True)
    with capi.Problem(small, precision=1) as p:
        l0 = capi.num_kernel_launches()
        J = autograd.total_utility(p, c, w, iters, kc)
        J.backward()
        launched = capi.num_kernel_launches() - l0
        gc, gw, J2 = p.adjoint(iters, kc)
    assert abs(float(J.detach()) - J2) <= 1e-12 * abs(J2)
    assert rel(c.grad.numpy(), gc) <= 1e-12 and rel(w.grad.numpy(), gw) <= 1e-12
    # forward 2 x 120, recompute of the first two segments 2 x 100, backward 2 x 120, plus
    # a few setup kernels; a second forward from zero would add another 240
    assert launched <= 2 * iters + 2 * (iters - kc + 30) + 2 * iters + 40, launched
    # solve_x: a vector-Jacobian product against the host entry with the same cotangent
    xbar = np.random.default_rng(7).standard_normal(small["n"])
    c2 = torch.tensor(small["c"], requires_grad=True)
    w2 = torch.tensor(small["w"], requires_grad=True)
    with capi.Problem(small, precision=1) as p:
        x = autograd.solve_x(p, c2, w2, iters, kc)
        (x * torch.tensor(xbar)).sum().backward()
        hc, hw, _ = p.adjoint(iters, kc, xbar=xbar, objective=False)
    assert rel(c2.grad.numpy(), hc) <= 1e-12 and rel(w2.grad.numpy(), hw) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_device_entries_equal_host_entry(small, precision):
    """num_adjoint_forward + num_adjoint_backward (device arrays) give the host entry's
    gradients bit for bit, twice in a row from one forward; a utility cotangent ubar
    scales them; changed capacities or a missing forward are refused."""
    import torch
    from paper_2509_10722_b300 import capi
    iters, kc = 130, 50
    xbar = np.random.default_rng(9).standard_normal(small["n"])
    with capi.Problem(small, precision=precision) as p:
        hc, hw, _ = p.adjoint(iters, kc, xbar=xbar, objective=True)
        with pytest.raises(capi.NumError) as e0:
            p.adjoint_backward(ubar=1.0, c_grad=torch.empty(p.m, dtype=torch.float64,
                                                            device="cuda"))
        assert e0.value.code == capi.NUM_ERR_STATE
        p.adjoint_forward(iters, kc)
        xb = torch.tensor(xbar, device="cuda")
        outs = []
        for ubar in (1.0, 1.0, 2.5):
            cg = torch.empty(p.m, dtype=torch.float64, device="cuda")
            wg = torch.empty(p.n, dtype=torch.float64, device="cuda")
            p.adjoint_backward(xbar=xb if ubar == 1.0 else None, ubar=ubar, c_grad=cg,
                               w_grad=wg)
            outs.append((cg.cpu().numpy(), wg.cpu().numpy()))
        assert np.array_equal(outs[0][0], hc) and np.array_equal(outs[0][1], hw)
        assert np.array_equal(outs[1][0], hc) and np.array_equal(outs[1][1], hw)
        # the utility part alone, scaled by 2.5, against the host entry's
        uc, uw, _ = p.adjoint(iters, kc, objective=True)
        tol = 1e-12 if precision == 1 else 1e-6
        assert rel(outs[2][0], 2.5 * uc) <= tol and rel(outs[2][1], 2.5 * uw) <= tol
        p.adjoint_forward(iters, kc)
        p.set_capacity_device(torch.tensor(small["c"] * 1.01, device="cuda"))
        with pytest.raises(capi.NumError) as e1:
            p.adjoint_backward(ubar=1.0, w_grad=torch.empty(p.n, dtype=torch.float64,
                                                            device="cuda"))
        assert e1.value.code == capi.NUM_ERR_STATE
        p.adjoint_release()


def test_device_setters(small):
    """Device-array setters equal the host ones (same iterates after a solve) and refuse
    non-positive or non-finite values without changing anything."""
    import torch
    from paper_2509_10722_b300 import capi
    c = small["c"] * np.linspace(0.5, 1.5, small["m"])
    w = small["w"] * np.linspace(1.5, 0.5, small["n"])
    out = []
    for dev in (False, True):
        with capi.Problem(small, precision=1) as p:
            if dev:
                p.set_capacity_device(torch.tensor(c, device="cuda"))
                p.set_weights_device(torch.tensor(w, device="cuda"))
            else:
                p.set_capacity(c)
                p.set_weights(w)
            p.solve(200, 0.0)
            out.append(p.get()[0])
            for bad in (0.0, -1.0, np.nan, np.inf):
                cb = torch.tensor(c, device="cuda")
                cb[3] = bad
                with pytest.raises(capi.NumError) as e:
                    p.set_capacity_device(cb)
                assert e.value.code == capi.NUM_ERR_INVALID
                wb = torch.tensor(w, device="cuda")
                wb[5] = bad
                with pytest.raises(capi.NumError) as e:
                    p.set_weights_device(wb)
                assert e.value.code == capi.NUM_ERR_INVALID
            p.solve(10, 0.0)
            out.append(p.get()[0])
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[3])


def test_c5_full_size_fp32_gradients_track_fp64():
    """Full differentiation recipe (n = 1e6, m = 1e5, 500 iterations, checkpoints every
    50): FP32 gradients within 1e-4 of the FP64 ones (5e-7 measured)."""
    inst = W.workload("c5")
    c32, w32, _ = _gpu_adjoint(inst, 500, 0, kc=50)
    c64, w64, _ = _gpu_adjoint(inst, 500, 1, kc=50)
    assert rel(c32, c64) <= 1e-4 and rel(w32, w64) <= 1e-4
