"""The debug build (libnum_pmp_debug.so, kernels compiled with PMP_DEBUG_BOUNDS): every
gathered index is checked against the length of the vector it indexes.  Run in a child
process that loads that library, over every kernel family, it must record no index out of
range (a solve would return NUM_ERR_STATE) and give bit-identical results to the release
build, since the checks leave valid indices alone."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, sys.argv[2])
import numpy as np
from paper_2509_10722_b300 import capi, workloads as W
out = {}
c1 = W.workload("c1")
zipf = W.random_instance(20000, 500, 2, 12, seed=5, link_dist="zipf", frac_log=0.6,
                         frac_alpha2=0.2, c_scale=0.1, box=(0.0, 10.0))
for name, inst in (("c1", c1), ("zipf", zipf)):
    for prec in (0, 1, 2):
        with capi.Problem(inst, precision=prec) as p:
            st, it = p.solve(300, 0.0)
            assert st in (0, 1), st
            x, lam, _ = p.get()
        out[f"{name}_{prec}_x"] = x
        out[f"{name}_{prec}_lam"] = lam
with capi.Batch([c1, zipf], precision=0) as b:
    rc, it, stt = b.solve(300, 0.0)
    xs, ps, _ = b.get()
out["batch_x"] = np.concatenate(xs)
with capi.Problem(zipf, precision=0) as p:
    cg, wg, J = p.adjoint(100, 25)
out["adj_c"] = cg
out["adj_w"] = wg
np.savez(sys.argv[1], **out)
'''


def _run(lib, out):
    env = dict(os.environ)
    if lib:
        env["NUM_PMP_LIBRARY"] = lib
    else:
        env.pop("NUM_PMP_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT, out, ROOT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_debug_build_finds_no_out_of_range_gather_and_matches_release(tmp_path):
    from paper_2509_10722_b300 import build as B
    debug = B.build(debug=True)
    got = _run(debug, str(tmp_path / "debug.npz"))
    ref = _run(None, str(tmp_path / "release.npz"))
    assert sorted(got.files) == sorted(ref.files)
    for k in ref.files:
        assert np.array_equal(got[k], ref[k]), k
