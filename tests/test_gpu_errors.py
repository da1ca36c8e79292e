"""Malformed instances are rejected by the device-side validation (NUM_ERR_INVALID with a
message naming the defect), from host and from device arrays; a handle stays usable."""
import numpy as np
import pytest

from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _base():
    return W.random_instance(50, 20, 1, 5, seed=3)


def _mutations():
    yield "duplicate", "twice", lambda i: i["route_links"].__setitem__(
        slice(int(i["route_ptr"][_long(i)]) + 1, int(i["route_ptr"][_long(i)]) + 2),
        i["route_links"][int(i["route_ptr"][_long(i)])])
    yield "link_id_high", "outside", lambda i: i["route_links"].__setitem__(3, 20)
    yield "link_id_negative", "outside", lambda i: i["route_links"].__setitem__(5, -1)
    yield "capacity_zero", "capacity", lambda i: i["c"].__setitem__(4, 0.0)
    yield "capacity_nan", "capacity", lambda i: i["c"].__setitem__(4, np.nan)
    yield "weight_negative", "weight", lambda i: i["w"].__setitem__(7, -1.0)
    yield "weight_inf", "weight", lambda i: i["w"].__setitem__(7, np.inf)
    yield "utype", "utility type", lambda i: i["utype"].__setitem__(2, 3)
    yield "box_inverted", "box", lambda i: (i["lo"].__setitem__(9, 5.0), i["hi"].__setitem__(9, 1.0))
    yield "box_nan", "box", lambda i: i["hi"].__setitem__(9, np.nan)
    yield "log_hi_zero", "box", lambda i: (i["utype"].__setitem__(11, 0), i["hi"].__setitem__(11, 0.0),
                                           i["lo"].__setitem__(11, 0.0))


def _long(inst):
    return int(np.flatnonzero(np.diff(inst["route_ptr"]) >= 2)[0])


MUT = list(_mutations())


@pytest.mark.parametrize("name,msg,mut", MUT, ids=[m[0] for m in MUT])
@pytest.mark.parametrize("device", [False, True])
def test_invalid_instance(name, msg, mut, device):
    from paper_2509_10722_b300 import capi
    inst = _base()
    mut(inst)
    with pytest.raises(capi.NumError) as ei:
        capi.Problem(inst, device=device)
    assert ei.value.code == capi.NUM_ERR_INVALID
    assert msg in str(ei.value)


def test_valid_after_rejection():
    from paper_2509_10722_b300 import capi
    bad = _base()
    bad["c"][0] = -1.0
    with pytest.raises(capi.NumError):
        capi.Problem(bad)
    with capi.Problem(_base()) as p:
        status, done = p.solve(20, 0.0)
        assert (status, done) == (1, 20)


def test_bad_solve_arguments():
    from paper_2509_10722_b300 import capi
    with capi.Problem(_base()) as p:
        with pytest.raises(capi.NumError):
            p.solve(-1)
        with pytest.raises(capi.NumError):
            p.set_rho_schedule([0, 2, 0])
        assert p.solve(0, 0.0) == (1, 0)


def test_get_device_checks_tensor_sizes():
    """A device output smaller than the handle's n (or m) is refused on the host, before
    the library could write past its end."""
    import torch
    from paper_2509_10722_b300 import capi
    with capi.Problem(_base()) as p:
        p.solve(5, 0.0)
        with pytest.raises(ValueError):
            p.get_device(x=torch.empty(p.n - 1, dtype=torch.float64, device="cuda"))
        with pytest.raises(ValueError):
            p.get_device(prices=torch.empty(p.m + 1, dtype=torch.float64, device="cuda"))
        x = torch.empty(p.n, dtype=torch.float64, device="cuda")
        info = p.get_device(x=x)
        assert np.allclose(x.cpu().numpy(), p.get()[0]) and info["iters"] == 5
