"""The persistent form of the batched solve (num_batch_set_persistent), through the C ABI.

One cooperative launch runs many iterations; each instance has a team of blocks that
meet at bounded barriers.  Checked here: the iterates equal the default form's (two
launches per iteration) under the same rho decisions, bit for bit, including an instance
whose long links are summed in chunks and one with long routes; every instance against
the oracle; stopping per instance; the full 256-instance recipe; the timeout status when
the waits are given a single poll (no wait of the kernel is unbounded, so the launch ends
and the host reads the status); more instances than resident blocks, packed several to
a block."""
import numpy as np
import pytest

from gpu_util import oracle_run, rel
from paper_2509_10722_b300 import workloads as W
from test_gpu_batch import _mixed_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    return _mixed_batch()


def _run(insts, iters, precision, eps=0.0, schedules=None, persistent=True, wait_polls=0,
         **params):
    from paper_2509_10722_b300 import capi
    params.setdefault("history", 64)
    with capi.Batch(insts, precision=precision, **params) as b:
        if persistent:
            b.set_persistent(True, wait_polls)
        if schedules is not None:
            b.set_rho_schedules(schedules)
        rc, it, st = b.solve(iters, eps)
        xs, ps, infos = b.get()
    return dict(rc=rc, iters=it, status=st, x=[x.copy() for x in xs],
                lam=[p.copy() for p in ps], info=infos)


@pytest.mark.parametrize("precision,check_every", [(0, 50), (1, 50), (0, 7)])
def test_persistent_iterates_equal_the_default_form(batch, precision, check_every):
    """Fixed iteration count: the rho decisions follow from the residual sums, whose FP64
    grouping differs between the forms, so both runs are given the same decisions."""
    iters = 300
    sched = np.tile(np.array([1, 0, -1, 1, 1, 0], dtype=np.int8), (len(batch), 1))
    a = _run(batch, iters, precision, schedules=sched, persistent=False, check_every=check_every)
    p = _run(batch, iters, precision, schedules=sched, persistent=True, check_every=check_every)
    assert list(p["iters"]) == [iters] * len(batch)
    for i in range(len(batch)):
        assert np.array_equal(a["x"][i], p["x"][i]), i
        assert np.array_equal(a["lam"][i], p["lam"][i]), i


def test_persistent_fp64_matches_oracle_per_instance(batch):
    iters = 200
    g = _run(batch, iters, 1)
    for i, inst in enumerate(batch):
        ref = oracle_run(inst, iters)
        assert rel(g["x"][i], ref["x"]) <= 1e-10, i
        assert rel(g["lam"][i], ref["lam"]) <= 1e-10, i


def test_persistent_instances_stop_independently(batch):
    """As in the default form: instances with a solution stop at the oracle's iteration."""
    batch = [batch[i] for i in (0, 1, 2, 3, 4, 6)]
    eps = 1e-6
    g = _run(batch, 100_000, 1, eps=eps, check_every=64)
    assert g["rc"] == 0 and np.all(g["status"] == 0)
    refs = [oracle_run(inst, 100_000, eps=eps) for inst in batch]
    assert list(g["iters"]) == [r["iters"] for r in refs]
    assert len(set(g["iters"])) > 1
    for i, r in enumerate(refs):
        assert rel(g["x"][i], r["x"]) <= 1e-9, i


def test_persistent_full_recipe_matches_default_form():
    """The 256-instance batched recipe to eps_abs = 1e-4 (FP32): every instance converges
    in both forms, at the same iteration give or take one (residual sums grouped
    differently), with objectives within 1e-6 relative."""
    insts = W.batched_instances(256, seed=0)
    a = _run(insts, 50_000, 0, eps=1e-4, persistent=False)
    p = _run(insts, 50_000, 0, eps=1e-4, persistent=True)
    assert a["rc"] == 0 and p["rc"] == 0
    assert np.all(np.abs(a["iters"] - p["iters"]) <= 1)
    for i in range(len(insts)):
        oa, op = a["info"][i]["objective"], p["info"][i]["objective"]
        assert abs(oa - op) <= 1e-6 * abs(oa), i


def test_persistent_wait_limit_returns_timeout():
    """One poll per wait: a block that reaches a team barrier before its team mates gives up
    at once, records it and returns, and so do its mates; the solve reports
    NUM_ERR_TIMEOUT, refuses to continue, and after num_batch_reset runs normally again."""
    from paper_2509_10722_b300 import capi
    insts = [W.random_instance(60_000, 6_000, 2, 8, seed=21),
             W.random_instance(40_000, 4_000, 2, 8, seed=22)]
    with capi.Batch(insts, precision=0) as b:
        b.set_persistent(True, wait_polls=1)
        with pytest.raises(capi.NumError) as e:
            b.solve(200, 0.0)
        assert e.value.code == capi.NUM_ERR_TIMEOUT
        assert "ran out" in capi.num_last_error()
        with pytest.raises(capi.NumError) as e2:
            b.solve(10, 0.0)
        assert e2.value.code == capi.NUM_ERR_STATE
        b.reset()
        b.set_persistent(True, wait_polls=0)
        b.solve(120, 0.0)
        xs, ps, _ = b.get()
        x_after = [x.copy() for x in xs]
    ref = _run(insts, 120, 0, persistent=False)
    for i in range(2):
        # same iterates unless the residual sums took a different rho decision at 50 / 100
        assert rel(x_after[i], ref["x"][i]) <= 1e-4, i


def test_persistent_packs_more_instances_than_resident_blocks():
    """3,000 small instances, more than the GPU holds resident blocks of the kernel: they
    are packed several to a block, and the iterates equal the default form's."""
    insts = [W.random_instance(int(n), 3, 1, 2, seed=s)
             for s, n in enumerate(np.random.default_rng(5).integers(2, 40, 3000))]
    sched = np.zeros((len(insts), 2), dtype=np.int8)
    a = _run(insts, 100, 0, schedules=sched, persistent=False)
    p = _run(insts, 100, 0, schedules=sched, persistent=True)
    assert list(p["iters"]) == [100] * len(insts)
    for i in range(len(insts)):
        assert np.array_equal(a["x"][i], p["x"][i]), i
