"""num_objective_noalloc: the utility reduction for callers that cannot allocate device
memory (allocation locked by a host framework, real-time loops that may not synchronize
through cudaMalloc, fixed memory budgets).  It keeps its partial sums in a static device
array of the library instead of allocating, so this test checks, through the C ABI, that
two calls in a row give the same number as the objective num_get reports for the same
rates and as an FP64 host sum of the utilities, and that sizes beyond the array's limit
are refused.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,a2", [(20_000, 2_000, 0.0), (1_000, 500, 0.0), (5_000, 800, 0.3)])
def test_noalloc_objective_matches_num_get(n, m, a2):
    import torch

    from paper_2509_10722_b300 import capi
    inst = W.random_instance(n, m, 1, 8, seed=17, frac_log=0.6 - a2, frac_alpha2=a2,
                             box=(0.0, 20.0))
    # the FP64 path keeps the caller's FP64 weights, so both sides sum the same doubles
    with capi.Problem(inst, precision=capi.NUM_FUSED_FP64) as p:
        p.solve(300, 0.0)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        info = capi.num_get_device(p.h, x, None, n=p.n)
    ut = torch.as_tensor(inst["utype"]).cuda()
    w = torch.as_tensor(inst["w"]).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    capi.num_objective_noalloc(n, x, ut, w, out[0:1])
    capi.num_objective_noalloc(n, x, ut, w, out[1:2])
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = info["objective"]
    assert np.all(np.abs(got - ref) <= 1e-12 * abs(ref)), (got, ref)
    assert got[0] == got[1]
    # and the FP64 host sum of the same rates, written from Sec. II's definition
    from oracle import kkt
    host = kkt.utility(inst, x.cpu().numpy())
    assert np.all(np.abs(got - host) <= 1e-12 * abs(host)), (got, host)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    from paper_2509_10722_b300 import capi
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    u = torch.zeros(1, dtype=torch.uint8, device="cuda")
    n_too_big = 33_554_432 + 1
    rc = capi.library().num_objective_noalloc(n_too_big, t.data_ptr(), u.data_ptr(),
                                              t.data_ptr(), t.data_ptr(), None)
    assert rc == capi.NUM_ERR_INVALID
    assert "no-allocation maximum" in capi.num_last_error()
