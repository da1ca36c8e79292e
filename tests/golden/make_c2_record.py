"""Write the oracle's record of the n = 1e7, m = 1e6 headline instance solved to eps_abs = 1e-4.

This script calls only the FP64 CPU oracle (`oracle/`) and the seeded instance generator;
nothing in it comes from the CUDA path.  It runs the literal per-terminal ADMM of Sec. III
(with the residual balancing and over-relaxation of Sec. III-G) on the whole instance until
the stopping test of Sec. III-F passes (||r|| and ||s|| below eps_abs sqrt(J)), which takes
on the order of two hours on one host core, and writes

  c2_oracle_record.json   iteration count, rho decisions, residuals at the stop, objective
                          sum U_j(x_j) (Sec. II), KKT diagnostics, SHA-256 of the full x and
                          prices, the sample recipe, wall time
  c2_oracle_record.npz    the residual history (||r||, ||s||, rho) of every iteration and a
                          seeded sample of 100,000 stream rates x_j and 100,000 prices
                          lambda_l (= rho u_l, Sec. III-C), FP64

Usage:  python tests/golden/make_c2_record.py [--full-out PATH.npz] [--out-dir DIR]
(--full-out also keeps the full x and prices, which are too large to commit.)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import kkt  # noqa: E402
from paper_2509_10722_b300 import workloads as W  # noqa: E402

EPS_ABS = 1e-4
MAX_ITERS = 6000
SAMPLE = 100_000
SAMPLE_SEED = 20250910


def sample_indices(n, m, k=SAMPLE, seed=SAMPLE_SEED):
    """The sampled stream and link ids (sorted, distinct), reproducible from the seed."""
    rng = np.random.default_rng(seed)
    xi = np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)
    li = np.sort(rng.choice(m, size=min(k, m), replace=False)).astype(np.int64)
    return xi, li


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--full-out", default=None)
    ap.add_argument("--out-dir", default=HERE)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="n and m times this factor (below 1 only to try the script out)")
    a = ap.parse_args()
    t0 = time.time()
    inst = W.workload("c2", scale=a.scale if a.scale != 1.0 else None)
    t_gen = time.time() - t0
    t1 = time.time()
    res = oracle.solve(inst, MAX_ITERS, eps_abs=EPS_ABS)
    t_solve = time.time() - t1
    x, lam = res["x"], res["lam"]
    if a.full_out:
        np.savez(a.full_out, x=x, lam=lam, slack=res["slack"], hist=res["hist"],
                 decisions=res["decisions"])
    xi, li = sample_indices(inst["n"], inst["m"])
    d = kkt.diagnostics(inst, x, lam)
    nnz = int(inst["route_ptr"][-1])
    J = nnz + inst["m"]
    hist = res["hist"]
    rec = dict(
        source=("FP64 CPU oracle (literal per-terminal ADMM, Sec. III, III-F, III-G) on the "
                "headline workload c2 of workloads.py (n = 1e7, m = 1e6, seed 0), run until "
                "||r|| and ||s|| < eps_abs sqrt(J); written by tests/golden/make_c2_record.py"),
        n=int(inst["n"]), m=int(inst["m"]), nnz=nnz, J=int(J), eps_abs=EPS_ABS,
        params=res["params"], iters=int(res["iters"]), converged=bool(res["converged"]),
        decisions=[int(v) for v in res["decisions"]],
        r_norm=float(hist[-1, 0]), s_norm=float(hist[-1, 1]), rho=float(hist[-1, 2]),
        tol=float(EPS_ABS * np.sqrt(J)),
        objective=kkt.utility(inst, x),
        kkt={k: float(v) for k, v in d.items()},
        sha256_x=hashlib.sha256(np.ascontiguousarray(x, dtype=np.float64).tobytes()).hexdigest(),
        sha256_lam=hashlib.sha256(np.ascontiguousarray(lam, dtype=np.float64).tobytes()).hexdigest(),
        sample=dict(k=SAMPLE, seed=SAMPLE_SEED,
                    recipe="numpy default_rng(seed).choice(n, k, replace=False), then "
                           "choice(m, k, replace=False), each sorted"),
        seconds=dict(generate=round(t_gen, 1), solve=round(t_solve, 1)),
    )
    np.savez_compressed(os.path.join(a.out_dir, "c2_oracle_record.npz"), hist=hist,
                        x_idx=xi.astype(np.int32), x=x[xi], lam_idx=li.astype(np.int32),
                        lam=lam[li])
    with open(os.path.join(a.out_dir, "c2_oracle_record.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps({k: rec[k] for k in ("iters", "converged", "objective", "r_norm",
                                          "s_norm", "rho", "seconds")}))


if __name__ == "__main__":
    main()
