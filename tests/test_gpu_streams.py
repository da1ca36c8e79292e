"""Stream ordering of the C ABI: device inputs produced by work that the caller queued on
its own stream are read only after that work, and the results are complete when the call
returns.  (Host arrays are read when the call is made, like any host argument.)"""
import numpy as np
import pytest

from gpu_util import oracle_run, rel
from paper_2509_10722_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_create_device_waits_for_the_callers_stream():
    """route_ptr and the other device inputs are filled by copies queued on the caller's
    stream behind a long chain of kernels; num_create_device on that stream must read
    the filled arrays (before, route_ptr holds -1 everywhere)."""
    import torch
    from paper_2509_10722_b300 import capi
    inst = W.random_instance(20000, 2000, 1, 8, seed=31, frac_log=0.7, box=(0.0, 20.0))
    keys = ("route_ptr", "route_links", "c", "utype", "w", "lo", "hi")
    src = {k: torch.as_tensor(np.ascontiguousarray(inst[k])).cuda() for k in keys}
    dst = {k: torch.full_like(src[k], -1 if src[k].dtype != torch.uint8 else 7) for k in keys}
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = torch.randn(4096, 4096, device="cuda")
        for _ in range(20):  # keep the stream busy for a while
            a = a @ a
            a = a / a.norm()
        for k in keys:
            dst[k].copy_(src[k])
    prm = capi.num_default_params(precision=capi.NUM_FUSED_FP64)
    h = capi.num_create_device(inst["n"], inst["m"], dst["route_ptr"], dst["route_links"],
                               dst["c"], dst["utype"], dst["w"], dst["lo"], dst["hi"], prm,
                               s.cuda_stream)
    try:
        capi.num_solve(h, 200, 0.0)
        x, lam, _ = capi.num_get(h, inst["n"], inst["m"])
    finally:
        capi.num_destroy(h)
    ref = oracle_run(inst, 200)
    assert rel(x, ref["x"]) <= 1e-10 and rel(lam, ref["lam"]) <= 1e-10


def test_get_device_is_ordered_on_the_handles_stream():
    """num_get_device writes on the handle's stream: a copy queued after it on that stream
    sees the exported values."""
    import torch
    from paper_2509_10722_b300 import capi
    inst = W.random_instance(5000, 500, 1, 8, seed=32, frac_log=0.7, box=(0.0, 20.0))
    s = torch.cuda.Stream()
    with capi.Problem(inst, stream=s.cuda_stream, precision=capi.NUM_FUSED_FP64) as p:
        p.solve(100, 0.0)
        x_dev = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        p.get_device(x=x_dev)
        with torch.cuda.stream(s):
            out = x_dev.clone()
        s.synchronize()
        x_host = p.get()[0]
    assert np.array_equal(out.cpu().numpy(), x_host)


def test_separate_handles_from_two_threads():
    """Two handles driven from two host threads at once (the binding releases the
    interpreter lock during library calls): each result matches the oracle."""
    import threading
    from paper_2509_10722_b300 import capi
    insts = [W.random_instance(4000, 600, 1, 8, seed=71 + i, frac_log=0.6, box=(0.0, 20.0))
             for i in range(2)]
    out = [None, None]
    errors = []

    def work(i):
        try:
            with capi.Problem(insts[i], precision=capi.NUM_FUSED_FP64) as p:
                for _ in range(4):
                    p.solve(50, 0.0)
                out[i] = p.get()[:2]
        except Exception as exc:  # reported below, on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in range(2):
        ref = oracle_run(insts[i], 200)
        assert rel(out[i][0], ref["x"]) <= 1e-10 and rel(out[i][1], ref["lam"]) <= 1e-10
