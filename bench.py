#!/usr/bin/env python
"""Benchmark of the PMP solver: iterations/s and time to the 1e-4 residual tolerance on the
n = 1e7 streams, m = 1e6 links instance, FP32 fused path vs the plain FP64 GPU path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one whole solve from inputs already resident in HBM: num_create_device (input
validation and the device CSR build), num_solve to eps_abs = 1e-4 (Sec. III-F), and
num_get_device (x, prices, FP64 objective).  `value` = iterations of the timed steps per
second of device time (CUDA events on the solver's stream).  Prints one JSON line.

--impl reference times the FP64 CPU oracle (a literal per-terminal ADMM, single thread) on
the same instance, as the slow reference arm.  With N > 1 (torchrun) every rank solves an
independent instance (replicas; no collective in the data path).
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import hashlib
import io
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_10722_b300 import workloads as W  # noqa: E402

METRIC = "PMP iters/s & time-to-1e-4 KKT residual, n=1e7 m=1e6, vs FP64 plain path"
WORKLOAD_TEXT = {
    "c2": ("n=1e7 streams, m=1e6 links, route length U{1..10} over uniform links without "
           "replacement (nnz~5.5e7), c~U[1,10], 70% log / 30% linear, w~U[0.5,2], box [0,50], "
           "eps_abs=1e-4 (||r||,||s|| < eps_abs*sqrt(nnz+m)), rho0=1, alpha=1.6, mu=2, "
           "gamma=1.1, rho period 50"),
    "c3": ("n=2e7 streams, m=2e6 links, route length U{2..12}, Zipf(1.1) link choice, "
           "c~0.1*U[1,10], all log, w~LogNormal(0,0.5), box [0,10], eps_abs=1e-4"),
}
PRECISION = {"fp32": 0, "fp64": 1, "plain": 2}
KERNEL_NAMES = {0: ["stream (SpMV-transpose + prox)", "link (SpMV + link update + finalize)"],
                2: ["plain SpMV-transpose", "plain stream prox", "plain SpMV", "plain link update",
                    "plain reduce 1", "plain reduce 2", "plain reduce 3", "plain finalize"]}


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOAD_TEXT) + ["c4"])
    ap.add_argument("--scale", type=float, default=None, help="shrink n and m (testing only)")
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--max-iters", type=int, default=50_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-reorder", action="store_true",
                    help="keep the caller's stream order (measures the first-link ordering)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--ref-iters", type=int, default=1, help="oracle iterations per reference step")
    ap.add_argument("--scenario", choices=["none", "warmstart", "adjoint", "congestion", "scaling"],
                    default="none",
                    help="warmstart: degradation and failure re-solves of Sec. V-D; "
                         "adjoint: gradients of 500 unrolled iterations on c5")
    ap.add_argument("--congested", action="store_true",
                    help="c4: Zipf(1.1) link choice in every instance (congestion scenario)")
    ap.add_argument("--no-seq", action="store_true",
                    help="c4: skip the two sequential legs (for profiling the batch kernels)")
    ap.add_argument("--tune-iters", type=int, default=10,
                    help="c4: timed iterations per candidate partition of the autotuner")
    ap.add_argument("--record-traffic", metavar="CSV", default=None,
                    help="write profiles/traffic.json from an ncu CSV (TRAFFIC_CMD) and exit")
    return ap.parse_args()


# ---- distributed plumbing (replicas) -------------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        return self._reduce(v, "max")

    def sum(self, v):
        return self._reduce(v, "sum")

    def _reduce(self, v, op):
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---- clocks during the timed region ---------------------------------------------------------------

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling the clocks every 200 ms while it runs; its lines are read from
    a pipe by a thread, so nothing is written to disk."""

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.reader = None

    def start(self):
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={CLOCK_QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.reader = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout),
                                       daemon=True)
        self.reader.start()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=5)
        return parse_clocks("".join(self.lines))


def parse_clocks(text):
    """Summary of `nvidia-smi --query-gpu=CLOCK_QUERY --format=csv,noheader,nounits`
    samples: median SM clock, max SM clock, and the throttle reasons seen active."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in csv.reader(io.StringIO(text)):
        if len(r) < 9:
            continue
        try:
            sm.append(float(r[1]))
            smax.append(float(r[2]))
        except ValueError:
            continue
        for name, val in zip(names, r[5:9]):
            if val.strip().lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
            "reasons": sorted(reasons), "samples": len(sm)}


class Measured:
    """SM clocks sampled and library kernels counted over a region of a scenario run."""

    def __init__(self, torch, capi):
        self.sampler = ClockSampler(torch.cuda.current_device())
        self.capi = capi
        self.clocks, self.launches = None, 0

    def start(self):
        self.sampler.start()
        self.l0 = self.capi.num_kernel_launches()
        return self

    def stop(self):
        self.launches = int(self.capi.num_kernel_launches() - self.l0)
        self.clocks = self.sampler.stop()


# ---- helpers --------------------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    return 6400.0, "of fallback (6.4 TB/s)"


ROW_SOURCES = ("rows.cu", "pmp_rows.cuh", "pmp_device.cuh", "pmp_internal.cuh")
TRAFFIC_CMD = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none "
               "--print-units base -k regex:\"k_(stream|link)_rows\" -s 200 -c 2 --csv "
               "--log-file traffic.csv python bench.py --steps 1 --warmup 0 "
               "--no-fp64 --no-e2e --no-cpu-baseline")


def row_sources_sha():
    """First 16 hex digits of sha256 over the sources the row kernels are compiled from."""
    h = hashlib.sha256()
    for f in ROW_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2509_10722_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(kernel_key):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on the current
    kernel sources (profiles/traffic.json holds the source hash it was taken on)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel_key)
    if not rec:
        return None
    return rec if rec.get("source_sha") == row_sources_sha() else None


_UNIT = {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9}


def record_traffic(csv_path, workload, out_path=None):
    """Write profiles/traffic.json from the CSV of an ncu capture of the row kernels (the
    capture command is TRAFFIC_CMD): mean DRAM bytes per launch of each kernel."""
    import csv
    sums = {}
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        name = row["Kernel Name"]
        kern = "k_stream_rows" if "k_stream_rows" in name else (
            "k_link_rows" if "k_link_rows" in name else None)
        metric = row["Metric Name"]
        if kern is None or metric not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        v = float(row["Metric Value"].replace(",", "")) * _UNIT[row["Metric Unit"].lower()]
        d = sums.setdefault(kern, {"launches": set(), "read": 0.0, "write": 0.0})
        d["launches"].add(row["ID"])
        d["read" if metric.endswith("read.sum") else "write"] += v
    out = {"_about": "DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of "
                     "the fused row kernels on the full solve, from one ncu capture; "
                     "source_sha = first 16 hex digits of sha256 over csrc/" +
                     ", csrc/".join(ROW_SOURCES) + " when captured. Command: " + TRAFFIC_CMD}
    sha = row_sources_sha()
    for kern, d in sorted(sums.items()):
        k = len(d["launches"])
        out[f"{workload}:{kern}"] = {
            "dram_bytes_per_launch": int(round((d["read"] + d["write"]) / k)),
            "read": int(round(d["read"] / k)), "write": int(round(d["write"] / k)),
            "launches": k, "source_sha": sha}
    with open(out_path or os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    return out


def to_device(inst, torch):
    return {k: torch.as_tensor(np.ascontiguousarray(inst[k])).cuda()
            for k in ("route_ptr", "route_links", "c", "utype", "w", "lo", "hi")}


def pinned_copy(inst, torch):
    out = {}
    for k in ("route_ptr", "route_links", "c", "utype", "w", "lo", "hi"):
        a = np.ascontiguousarray(inst[k])
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
        t.numpy()[...] = a
        out[k] = t.numpy()
    return out


class Solver:
    """One whole solve per call, on a fixed torch stream, inputs resident on the device."""

    def __init__(self, capi, torch, dev_inst, n, m, precision, eps, max_iters, stream,
                 reorder=1):
        self.capi, self.torch = capi, torch
        self.d = dev_inst
        self.n, self.m = n, m
        self.eps, self.max_iters = eps, max_iters
        self.stream = stream
        self.alloc = capi.torch_allocator()
        self.params = capi.num_default_params(precision=precision, profile=2, reorder=reorder,
                                              allocator=ctypes.pointer(self.alloc))
        self.x = torch.empty(n, dtype=torch.float64, device="cuda")
        self.p = torch.empty(m, dtype=torch.float64, device="cuda")
        self.kernel_ms = None
        self.kernel_runs = None
        self.bytes = None
        self.phase_ms = np.zeros(3)  # create, solve, get (CUDA events on the stream)

    def step(self):
        c, d, torch = self.capi, self.d, self.torch
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(self.stream)
        h = c.num_create_device(self.n, self.m, d["route_ptr"], d["route_links"], d["c"],
                                d["utype"], d["w"], d["lo"], d["hi"], self.params,
                                self.stream.cuda_stream)
        try:
            ev[1].record(self.stream)
            status, iters = c.num_solve(h, self.max_iters, self.eps)
            ev[2].record(self.stream)
            info = c.num_get_device(h, self.x, self.p, self.n, self.m)
            ev[3].record(self.stream)
            ev[3].synchronize()
            self.phase_ms += [ev[q].elapsed_time(ev[q + 1]) for q in range(3)]
            ms, runs = c.num_get_kernel_times(h)
            if self.kernel_ms is None:
                self.kernel_ms, self.kernel_runs = np.zeros_like(ms), np.zeros_like(runs)
                self.bytes = c.num_iteration_bytes(h)
            self.kernel_ms += ms
            self.kernel_runs += runs
        finally:
            c.num_destroy(h)
        return status, iters, info

    def reset_kernel_times(self):
        self.kernel_ms = None
        self.kernel_runs = None
        self.phase_ms = np.zeros(3)


def timed(solver, torch, steps):
    """Run `steps` solves between CUDA events on the solver's stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters, infos = 0, []
    e0.record(solver.stream)
    for _ in range(steps):
        status, it, info = solver.step()
        iters += it
        infos.append((status, it, info))
    e1.record(solver.stream)
    e1.synchronize()
    return e0.elapsed_time(e1), iters, infos


# ---- arms --------------------------------------------------------------------------------------------

GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "c2_oracle_record")


def error_vs_oracle(x, lam, objective, iters):
    """A c2 result against the FP64 oracle's own run of the same instance to the same
    tolerance (the record in tests/golden, written by tests/golden/make_c2_record.py with
    the oracle alone): the seeded samples of rates and prices, the objective and the
    stopping iteration.  None if the record is absent."""
    if not (os.path.exists(GOLDEN_C2 + ".json") and os.path.exists(GOLDEN_C2 + ".npz")):
        return None
    rec = json.load(open(GOLDEN_C2 + ".json"))
    z = np.load(GOLDEN_C2 + ".npz")
    out = {}
    for name, got, idx, ref in (("x", x, z["x_idx"], z["x"]), ("prices", lam, z["lam_idx"], z["lam"])):
        d = np.asarray(got, dtype=np.float64)[idx] - ref
        scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
        out[f"{name}_rel"] = float(np.linalg.norm(d) / np.linalg.norm(ref))
        out[f"{name}_el_max"] = float(np.max(np.abs(d) / scale))
    out["objective_rel"] = abs(objective - rec["objective"]) / abs(rec["objective"])
    out["iters"] = int(iters)
    out["oracle_iters"] = int(rec["iters"])
    out["sample"] = (f"{len(z['x_idx'])} stream rates and {len(z['lam_idx'])} prices at seeded "
                     f"positions; elementwise errors floored at 1e-3 of the largest value")
    out["record"] = "tests/golden/c2_oracle_record.json"
    return out


def workload_config(args, n, m, nnz):
    """The workload of a line, the same in both arms (what is run, not how)."""
    return {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
            "scale": args.scale, "n": int(n), "m": int(m), "nnz": int(nnz),
            "l2": "no flush: every iteration moves ~0.8 GB, far more than the 126 MB L2"}


def run_reference(args, dist):
    """The FP64 CPU oracle as the reference arm (rank 0 only).  Each oracle call builds its
    per-terminal link lists before iterating; that setup is measured once in the warm-up
    (t(1 iteration) - (t(2) - t(1))) and taken off each timed step, so the value is the
    oracle's iteration rate, as the repo arm's cpu_baseline reports it."""
    if dist.rank != 0:
        return
    import oracle
    inst = W.workload(args.workload, scale=args.scale)
    k = max(args.ref_iters, 1)
    t0 = time.perf_counter()
    oracle.solve(inst, 1, eps_abs=0.0)
    t1 = time.perf_counter()
    oracle.solve(inst, 2, eps_abs=0.0)
    t2 = time.perf_counter()
    setup = max((t1 - t0) - ((t2 - t1) - (t1 - t0)), 0.0)
    for _ in range(max(args.warmup - 2, 0)):
        oracle.solve(inst, k, eps_abs=0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(inst, k, eps_abs=0.0)
    dt = time.perf_counter() - t0
    value = args.steps * k / max(dt - args.steps * setup, 1e-9)
    sample = (f"{k} oracle iteration(s) per step on the full {args.workload} instance, single "
              f"thread, the oracle's setup ({setup:.2f} s per call, measured in the warm-up) "
              f"taken off each step")
    nnz = int(inst["route_ptr"][-1])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, inst["n"], inst["m"], nnz),
            "step": f"oracle.solve of {k} iteration(s)", "parallelism": "cpu, 1 thread",
            "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args, inst):
    """Oracle iterations/s on the same instance: (t(k) - t(1)) / (k - 1) per iteration."""
    import oracle
    k = max(args.cpu_iters, 2)
    t0 = time.perf_counter()
    oracle.solve(inst, 1, eps_abs=0.0)
    t1 = time.perf_counter()
    oracle.solve(inst, k, eps_abs=0.0)
    t2 = time.perf_counter()
    per_it = ((t2 - t1) - (t1 - t0)) / (k - 1)
    return {"value": 1.0 / per_it, "unit": "iterations/s", "cores": 1, "kind": "oracle",
            "sample": f"{k - 1} oracle iterations on the full instance (difference of a "
                      f"{k}-iteration and a 1-iteration run, single thread)"}


def gather_roofline(capi, n, m, nnz, per_launch_ms, iter_ms):
    """The kernels against the ceiling that bounds them: each pass makes nnz reads at
    positions set by the routes (link kernel: x, 4 bytes, from the n-vector; stream kernel:
    (pbar, y), 8 bytes, from the m-vector).  The ceiling is this GPU's rate of uniformly
    random reads of the same element size from a vector of the same length, measured now
    (num_measure_gather_rate, outside the timed region).  The streams are ordered by their
    first link, which makes some reads adjacent, so a kernel can come out a little above 1."""
    rate = {4: capi.num_measure_gather_rate(nnz, n, 4, 5),
            8: capi.num_measure_gather_rate(nnz, m, 8, 5)}
    kern = {}
    bound_ms = 0.0
    for q, (vb, what) in enumerate([(8, "(pbar, y) pairs, 8 B, from the m-vector"),
                                    (4, "x, 4 B, from the n-vector")]):
        b = nnz / rate[vb] * 1e3
        bound_ms += b
        kern[KERNEL_NAMES[0][q]] = {"reads": nnz, "gathers": what,
                                    "achieved_g_per_s": nnz / (per_launch_ms[q] / 1e3) / 1e9,
                                    "ceiling_g_per_s": rate[vb] / 1e9,
                                    "frac": b / float(per_launch_ms[q])}
    return {"bound": "random L2 reads (one 32-byte sector each)", "unit": "G reads/s",
            "kernels": kern,
            "iteration": {"bound_ms": bound_ms, "ms": iter_ms, "frac": bound_ms / iter_ms},
            "measured_by": "num_measure_gather_rate: nnz uniformly random reads of the same "
                           "element size and vector length, 4 in flight per thread, full "
                           "occupancy, 5 timed passes after 1 warm-up"}


def run_ours(args, dist):
    import torch
    dist.init("nccl")
    torch.cuda.set_device(dist.local)
    from paper_2509_10722_b300 import capi
    inst = W.workload(args.workload, seed=dist.rank if dist.world > 1 else None, scale=args.scale)
    n, m, nnz = inst["n"], inst["m"], int(inst["route_ptr"][-1])
    dev = to_device(inst, torch)
    stream = torch.cuda.Stream()
    fp32 = Solver(capi, torch, dev, n, m, PRECISION["fp32"], args.eps, args.max_iters, stream,
                  reorder=0 if args.no_reorder else 1)
    for _ in range(args.warmup):
        fp32.step()
    fp32.reset_kernel_times()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    launches0 = capi.num_kernel_launches()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms, iters, infos = timed(fp32, torch, args.steps)
    clocks = sampler.stop()
    launches = capi.num_kernel_launches() - launches0
    torch.cuda.synchronize()
    dist.barrier()
    ms_max = dist.max(ms)
    iters_all = dist.sum(iters)
    value = iters_all / (ms_max / 1e3)
    statuses = [s for s, _, _ in infos]
    it_per_solve = [it for _, it, _ in infos]
    info = infos[-1][2]
    x32 = fp32.x.double().cpu().numpy()
    p32 = fp32.p.double().cpu().numpy()
    ev_oracle = (error_vs_oracle(x32, p32, info["objective"], it_per_solve[-1])
                 if args.workload == "c2" and args.scale is None and dist.rank == 0 else None)

    # per-kernel device times measured by events inside the timed solves
    kms, kruns = fp32.kernel_ms, fp32.kernel_runs
    per_launch_ms = kms / np.maximum(kruns, 1)
    dom = int(np.argmax(kms))
    bytes_per_launch = fp32.bytes[dom]
    achieved = bytes_per_launch / (per_launch_ms[dom] / 1e3) / 1e9
    peak, peak_note = measured_peaks()
    kernel_key = ["k_stream_rows", "k_link_rows"][dom]
    # the committed capture is of the full-size workload only
    trec = traffic_record(f"{args.workload}:{kernel_key}") if args.scale is None else None
    iter_bytes = float(sum(fp32.bytes))
    iter_ms = float(np.sum(per_launch_ms))
    roofline = {"bound": "hbm", "kernel": KERNEL_NAMES[0][dom], "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_note": peak_note,
                "traffic": None if trec is None else trec["dram_bytes_per_launch"],
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "launch_ms": float(per_launch_ms[dom]),
                "launch_timing": "CUDA events on the solver's stream around the kernels of "
                                 "the first iteration of every replay of 50 iterations "
                                 "(profile = 2), over the timed solves",
                "share": float(kms[dom] / kms.sum()),
                "iteration": {"bytes": iter_bytes, "ms": iter_ms,
                              "achieved_gbs": iter_bytes / (iter_ms / 1e3) / 1e9,
                              "frac": iter_bytes / (iter_ms / 1e3) / 1e9 / peak,
                              "frac_of_8tbs": iter_bytes / (iter_ms / 1e3) / 1e9 / 8000.0},
                "kernels": {KERNEL_NAMES[0][q]: {"ms_per_launch": float(per_launch_ms[q]),
                                                 "timed_launches": int(kruns[q]),
                                                 "bytes_per_launch": float(fp32.bytes[q]),
                                                 "gbs": float(fp32.bytes[q] / (per_launch_ms[q] / 1e3) / 1e9)}
                            for q in range(len(kms))}}

    gather = gather_roofline(capi, n, m, nnz, per_launch_ms, iter_ms)

    line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args, n, m, nnz),
            "step": "num_create_device + num_solve(eps_abs=1e-4) + num_get_device",
            "parallelism": "single GPU" if dist.world == 1 else f"{dist.world} replicas",
            "precision": "FP32 iterates, FP64 residual sums / stopping test / rho",
            "time_to_tol_s": ms_max / args.steps / 1e3,
            "phases_ms_per_step": {
                "create (validation, stream ordering, CSR build, tables)":
                    float(fp32.phase_ms[0] / args.steps),
                "solve (num_solve to the stopping test)": float(fp32.phase_ms[1] / args.steps),
                "get (FP64 export, objective)": float(fp32.phase_ms[2] / args.steps)},
            "iters_to_tol": it_per_solve[-1], "converged": all(s == 0 for s in statuses),
            "error_vs_oracle": ev_oracle,
            "final_residuals": {"primal": info["primal"], "dual": info["dual"],
                                "eps_tol": info["eps_tol"]},
            "objective": info["objective"],
            "roofline": roofline, "gather_roofline": gather, "gpu_launches": int(launches),
            "clocks": clocks}

    if not args.no_fp64:
        plain = Solver(capi, torch, dev, n, m, PRECISION["plain"], args.eps, args.max_iters,
                       stream)
        plain.step()
        plain.reset_kernel_times()
        pms, pit, pinfos = timed(plain, torch, 1)
        x64 = plain.x.cpu().numpy()
        p64 = plain.p.cpu().numpy()
        pk = plain.kernel_ms / np.maximum(plain.kernel_runs, 1)
        line["fp64_plain"] = {
            "iters_per_s": pit / (pms / 1e3), "time_to_tol_s": pms / 1e3, "iters_to_tol": pit,
            "converged": pinfos[0][0] == 0, "objective": pinfos[0][2]["objective"],
            "iteration_ms": float(np.sum(pk)),
            "kernels_ms_per_launch": {KERNEL_NAMES[2][q]: float(pk[q]) for q in range(len(pk))}}
        line["speedup_vs_fp64_plain"] = {
            "iters_per_s": value / dist.world / (pit / (pms / 1e3)),
            "time_to_tol": (pms / 1e3) / (ms_max / args.steps / 1e3)}
        o32, o64 = info["objective"], pinfos[0][2]["objective"]
        line["parity_vs_fp64_plain"] = {
            "objective_rel": abs(o32 - o64) / abs(o64),
            "x_rel": float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64)),
            "prices_rel": float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64))}
        del plain

    if not args.no_e2e:
        host = pinned_copy(inst, torch)
        # device memory from PyTorch's caching allocator, as in the device-resident leg
        e2e_alloc = capi.torch_allocator()
        e2e_params = capi.num_default_params(precision=0, allocator=ctypes.pointer(e2e_alloc))
        # results land in pinned host memory (a device-to-host copy at full speed)
        xh = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        ph = torch.empty(m, dtype=torch.float64, pin_memory=True).numpy()
        t_e2e, it_e2e = 0.0, 0
        for rep in range(1 + args.steps):
            t0 = time.perf_counter()
            h = capi.num_create(n, m, host["route_ptr"], host["route_links"], host["c"],
                                host["utype"], host["w"], host["lo"], host["hi"], e2e_params,
                                stream.cuda_stream)
            st, it = capi.num_solve(h, args.max_iters, args.eps)
            capi.num_get(h, n, m, out_x=xh, out_prices=ph)
            capi.num_destroy(h)
            dt = time.perf_counter() - t0
            if rep > 0:
                t_e2e += dt
                it_e2e += it
        line["e2e"] = {"value": dist.sum(it_e2e) / dist.max(t_e2e), "unit": "iterations/s",
                       "h2d_bytes_per_step": W.instance_bytes(inst),
                       "d2h_bytes_per_step": 8 * (n + m) + 8 * 8,
                       "time_to_tol_s": t_e2e / args.steps,
                       "path": "num_create (pinned host arrays, PyTorch caching allocator) + "
                               "num_solve + num_get (pinned host) + num_destroy, wall clock"}

    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, inst)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


def run_batched(args):
    """The batched recipe: 256 independent instances (n log-uniform in [1e3, 1e5], m = n/10,
    routes of 2..8 links, capacities degraded by U[0.3, 1], 70% log) solved to eps_abs =
    1e-4 as one batch, against the same 256 instances solved one after the other with the
    single-instance FP32 path and with the plain FP64 path.  Each leg includes creation from
    host arrays, the solve and the host copy of the results; CUDA events on one stream.
    The batch runs with the partition chosen by num_batch_autotune (headline: that partition
    set with num_batch_set_schedule, as a caller that tuned once would), and is also timed
    with the tuning inside the step and with the default partition."""
    import torch
    from paper_2509_10722_b300 import capi
    # the instances' arrays live in pinned host memory (as the single-instance e2e leg's),
    # for every leg alike
    insts = [dict(t, **pinned_copy(t, torch))
             for t in W.batched_instances(256, seed=0, congested=args.congested)]
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    n_all = int(sum(int(t["n"]) for t in insts))
    m_all = int(sum(int(t["m"]) for t in insts))
    # the results land in pinned host memory (a device-to-host copy at full speed)
    xh = torch.empty(n_all, dtype=torch.float64, pin_memory=True).numpy()
    ph = torch.empty(m_all, dtype=torch.float64, pin_memory=True).numpy()

    def batch_leg(mode="default", part=None, precision=0, keep=None):
        tune = None
        with capi.Batch(insts, stream=sp, precision=precision, profile=2) as b:
            if mode == "autotune":
                tune = b.autotune(trial_iters=args.tune_iters)
            elif mode in ("pinned", "persistent"):
                b.set_schedule(*part)
            if mode == "persistent":
                b.set_persistent(True)
            rc, it, st = b.solve(args.max_iters, args.eps)
            xs, ps, infos = b.get(out_x=xh, out_prices=ph)
            ms, runs = b.kernel_times()
            if keep is not None:
                keep["x"] = [x.copy() for x in xs]
                keep["obj"] = np.array([inf["objective"] for inf in infos])
                keep["iters"] = it.copy()
        return int(it.sum()), st, ms, runs, tune

    def seq_leg(precision):
        tot = 0
        for inst in insts:
            with capi.Problem(inst, stream=sp, precision=precision) as p:
                _, it = p.solve(args.max_iters, args.eps)
                p.get()
            tot += it
        return tot

    def timed_leg(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = [fn() for _ in range(reps)]
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps, out[-1]

    def kern(kms, kruns):
        return {"stream": float(kms[0] / max(kruns[0], 1)), "link": float(kms[1] / max(kruns[1], 1)),
                "timed_launches": int(kruns[0])}

    for _ in range(args.warmup):
        batch_leg("autotune")
    if not args.no_seq:
        seq_leg(0)
    t_a, (it_a, st_a, kms_a, kruns_a, tune) = timed_leg(lambda: batch_leg("autotune"), args.steps)
    chosen, trials = tune
    t_d, (it_d, st_d, kms_d, kruns_d, _) = timed_leg(lambda: batch_leg("default"), args.steps)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = capi.num_kernel_launches()
    t_f, (it_f, st_f, kms_f, kruns_f, _) = timed_leg(lambda: batch_leg("pinned", chosen), args.steps)
    launches = (capi.num_kernel_launches() - launches0) // max(args.steps, 1)
    clocks = sampler.stop()
    # the persistent form (one cooperative launch per 50 iterations, a team of blocks per
    # instance) on the same partition
    t_q, (it_q, st_q, _, _, _) = timed_leg(lambda: batch_leg("persistent", chosen), args.steps)
    # precision: the same batch in FP64 (default partition, untimed) against the FP32 run
    r32, r64 = {}, {}
    batch_leg("pinned", chosen, 0, r32)  # also gives the per-instance iteration counts
    batch_leg("default", None, 1, r64)
    obj_rel = np.abs(r32["obj"] - r64["obj"]) / np.maximum(np.abs(r64["obj"]), 1e-300)
    x_rel = [float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
             for a, b in zip(r32["x"], r64["x"])]
    if args.no_seq:
        t_s = t_p = float("nan")
        it_s = it_p = 0
    else:
        t_s, it_s = timed_leg(lambda: seq_leg(0), 1)
        t_p, it_p = timed_leg(lambda: seq_leg(2), 1)
    n_tot = int(sum(t["n"] for t in insts))
    m_tot = int(sum(t["m"] for t in insts))
    nnz_tot = int(sum(int(t["route_ptr"][-1]) for t in insts))
    st1, st2 = trials[:6], trials[6:]
    # Both kernels against their ceilings.  The sampled launches spread over the whole run,
    # tail included, where few instances still run; so the work of an average launch is
    # each instance's work weighted by its iterations, over the launches of the run.
    pk = [float(kms_f[q] / max(kruns_f[q], 1)) for q in range(2)]
    its = np.asarray(r32["iters"], dtype=np.float64)
    launches_run = float(its.max())
    ns = np.array([t["n"] for t in insts], dtype=np.float64)
    ms_ = np.array([t["m"] for t in insts], dtype=np.float64)
    nnzs = np.array([int(t["route_ptr"][-1]) for t in insts], dtype=np.float64)
    reads = float((its * nnzs).sum() / launches_run)
    rate = {4: capi.num_measure_gather_rate(nnz_tot, n_tot, 4, 5),
            8: capi.num_measure_gather_rate(nnz_tot, m_tot, 8, 5)}
    gk = {}
    for q, vb in enumerate((8, 4)):
        gk[["stream", "link"][q]] = {"reads_per_launch": reads,
                                     "achieved_g_per_s": reads / (pk[q] / 1e3) / 1e9,
                                     "ceiling_g_per_s": rate[vb] / 1e9,
                                     "frac": reads / rate[vb] * 1e3 / pk[q]}
    gather = {"bound": "random L2 reads (one 32-byte sector each)", "unit": "G reads/s",
              "kernels": gk, "note": "reads per launch = sum over instances of iterations x "
                                     "nnz, over the launches of the run"}
    # algorithmic bytes of the batch kernels: the single-instance formulas (FP32, uniform
    # box [0, 20]: no per-stream box arrays), weighted the same way
    b_stream = float((its * (4.0 * (ns + 1) + 4.0 * nnzs + 20.0 * ns + 8.0 * ms_)).sum()
                     / launches_run)
    b_link = float((its * (4.0 * (ms_ + 1) + 4.0 * nnzs + 4.0 * ns + 44.0 * ms_)).sum()
                   / launches_run)
    peak, peak_note = measured_peaks()
    dom = int(np.argmax(pk))
    bytes_dom = [b_stream, b_link][dom]
    roofline = {"bound": "hbm", "kernel": ["stream", "link"][dom],
                "achieved": bytes_dom / (pk[dom] / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": bytes_dom / (pk[dom] / 1e3) / 1e9 / peak, "peak_note": peak_note,
                "traffic": None, "algorithmic_bytes_per_launch": bytes_dom,
                "launch_ms": pk[dom],
                "launch_timing": "CUDA events around the kernels of the first iteration of "
                                 "every replay of 50 iterations (profile = 2), over the timed "
                                 "batch solves"}
    line = {"metric": "batched PMP: 256 instances to eps_abs 1e-4, aggregate iterations/s",
            "value": it_f / (t_f / 1e3), "unit": "iterations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_f,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "c4: 256 instances, n log-uniform in [1e3, 1e5], m = n/10, "
                                   "routes U{2..8}, c ~ U[1,10] x U[0.3,1], 70% log, box [0,20]"
                                   + (", Zipf(1.1) link choice (congested)" if args.congested
                                      else ", uniform links"),
                       "total_n": n_tot, "total_nnz": nnz_tot,
                       "step": "num_batch_create_instances (pinned host arrays of each "
                               "instance) + num_batch_set_schedule (the autotuned partition) + "
                               "num_batch_solve + num_batch_get (into pinned host memory); the "
                               "sequential legs create from the same pinned arrays"},
            "converged": int(np.sum(st_f == 0)), "batch_ms": t_f,
            "with_autotune_ms": t_a, "autotune_ms": t_a - t_f,
            "autotune": {"chosen": {"stream_item": int(chosen[0]), "link_item": int(chosen[1]),
                                    "link_lanes": int(chosen[2])},
                         "trial_iters": args.tune_iters, "candidates": int(len(trials)),
                         "stream_kernel_ms": {f"{int(r[0])}": round(float(r[3]), 4) for r in st1},
                         "link_kernel_ms_best": float(st2[:, 3].min()),
                         "link_kernel_ms_worst": float(st2[:, 3].max())},
            "default_partition_ms": t_d, "pinned_tuned_partition_ms": t_f,
            "persistent_ms": t_q, "persistent_converged": int(np.sum(st_q == 0)),
            "sequential_fp32_ms": t_s, "sequential_plain_fp64_ms": t_p,
            "speedup_vs_sequential_fp32": t_s / t_f, "speedup_vs_sequential_plain_fp64": t_p / t_f,
            "iterations": {"batch": it_f, "batch_default_partition": it_d,
                           "batch_persistent": it_q,
                           "batch_with_autotune": it_a, "sequential_fp32": int(it_s),
                           "sequential_plain_fp64": int(it_p)},
            "fp32_vs_fp64_batch": {"objective_rel_max": float(obj_rel.max()),
                                   "objective_rel_median": float(np.median(obj_rel)),
                                   "x_rel_max": float(max(x_rel)),
                                   "note": "per instance, both stopped by the same test at "
                                           "eps_abs 1e-4"},
            "kernels_ms_per_launch": {"autotuned": kern(kms_a, kruns_a),
                                      "default_partition": kern(kms_d, kruns_d),
                                      "pinned": kern(kms_f, kruns_f)},
            "roofline": roofline, "gather_roofline": gather, "gpu_launches": int(launches),
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_congestion(args):
    """The congestion experiment of Sec. V-C: the same network without and with 0.1% of its
    links each added to 10% of the streams (m = 1e6 links, n = 5e5 streams, routes of
    U{5..15} links), solved to eps_abs = 1e-4 in FP32 from zero.  The paper reports about
    1,000 iterations uncongested and a few hundred more congested."""
    import torch
    from paper_2509_10722_b300 import capi
    base, cong, hot = W.congestion_pair(scale=args.scale or 1.0)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    out = {}
    meas = Measured(torch, capi).start()
    for name, inst in (("uncongested", base), ("congested", cong)):
        deg = np.bincount(inst["route_links"], minlength=inst["m"])
        with capi.Problem(inst, stream=sp, precision=0) as p:
            p.solve(args.max_iters, args.eps)  # warm-up run of the same solve
            p.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, it = p.solve(args.max_iters, args.eps)
            e1.record(stream)
            e1.synchronize()
            x, lam, info = p.get()
        out[name] = {"iterations": int(it), "converged": st == 0,
                     "solve_ms": e0.elapsed_time(e1),
                     "ms_per_iteration": e0.elapsed_time(e1) / max(int(it), 1),
                     "nnz": int(inst["route_ptr"][-1]), "max_link_degree": int(deg.max()),
                     "objective": info["objective"]}
    meas.stop()
    u, c = out["uncongested"], out["congested"]
    line = {"metric": "iterations to eps_abs 1e-4 with and without congestion (Sec. V-C)",
            "value": c["iterations"] - u["iterations"], "unit": "extra iterations",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "m = 1e6 links, n = 5e5 streams, routes U{5..15} uniform "
                                   "links, c ~ U[1,10], 70% log, box [0,50]; congested: "
                                   "0.1% of links each on 10% of the streams",
                       "eps_abs": args.eps, "scale": args.scale},
            "paper": "about 1,000 iterations uncongested, a few hundred more congested",
            **out, "gpu_launches": meas.launches, "clocks": meas.clocks}
    print(json.dumps(line), flush=True)


def run_scaling(args):
    """The scaling experiment of Sec. V-B: random networks of m links and n = m / 2
    streams whose routes average 10 links (U{5..15} uniform links; c ~ U[1,10], 70% log,
    box [0, 50]), m = 1e5, 1e6, 1e7, each solved in FP32 to eps_abs = 1e-4 from device
    arrays.  Times by CUDA events on the solver's stream: the whole step (create + solve +
    FP64 export) and the solve alone.  The paper reports the largest of these networks
    (m = 1e7, n = 5e6) solved in 1,847 s on one A100 (its precision and stopping point not
    stated): context, not a target."""
    import torch
    from paper_2509_10722_b300 import capi
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    out = {}
    meas = Measured(torch, capi).start()
    for m in (100_000, 1_000_000, 10_000_000):
        inst = W.random_instance(m // 2, m, 5, 15, seed=0, frac_log=0.7, box=(0.0, 50.0))
        dev = to_device(inst, torch)
        prm = capi.num_default_params(precision=0)
        rows = []
        for rep in range(1 + args.steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            h = capi.num_create_device(inst["n"], m, dev["route_ptr"], dev["route_links"],
                                       dev["c"], dev["utype"], dev["w"], dev["lo"], dev["hi"],
                                       prm, sp)
            ev[1].record(stream)
            st, it = capi.num_solve(h, args.max_iters, args.eps)
            info = capi.num_get_device(h, None, None)
            ev[2].record(stream)
            ev[2].synchronize()
            capi.num_destroy(h)
            if rep > 0:
                rows.append((ev[0].elapsed_time(ev[2]), ev[1].elapsed_time(ev[2]), it, st))
        step_ms = float(np.median([r[0] for r in rows]))
        solve_ms = float(np.median([r[1] for r in rows]))
        out[f"m={m:.0e}"] = {"n": inst["n"], "m": m, "nnz": int(inst["route_ptr"][-1]),
                             "iterations": int(rows[-1][2]), "converged": rows[-1][3] == 0,
                             "step_ms": step_ms, "solve_and_export_ms": solve_ms,
                             "ms_per_iteration": solve_ms / max(rows[-1][2], 1),
                             "objective": info["objective"]}
        del dev
    meas.stop()
    big = out["m=1e+07"]
    line = {"metric": "time to eps_abs 1e-4 on the scaling networks of Sec. V-B",
            "value": big["step_ms"] / 1e3, "unit": "s (m = 1e7, n = 5e6)",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "m links, n = m/2 streams, routes U{5..15} uniform links, "
                                   "c ~ U[1,10], 70% log / 30% linear, w ~ U[0.5,2], box [0,50]",
                       "eps_abs": args.eps, "steps": args.steps},
            "paper": "m = 1e7, n = 5e6 solved in 1,847 s on one A100-SXM4 (precision and "
                     "stopping point not stated)",
            **out, "gpu_launches": meas.launches, "clocks": meas.clocks}
    print(json.dumps(line), flush=True)


def run_warmstart(args):
    """Re-solves after the perturbations of Sec. V-D on the solved c2 instance, FP32:
    degradation (each link has a 25% chance of a 50% capacity cut), warm (continue from the
    solution) vs cold (from zero); failure (each link fails with probability 25%, failed
    links and the streams that use them are pruned), warm (the solution restricted to what
    survives) vs cold.  Solve times by CUDA events on the solver's stream."""
    import torch
    from paper_2509_10722_b300 import capi
    inst = W.workload(args.workload, scale=args.scale)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    def timed_solve(p):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status, it = p.solve(args.max_iters, args.eps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), it, status

    out = {}
    meas = Measured(torch, capi).start()
    with capi.Problem(inst, stream=sp, precision=0) as p:
        t0, it0, _ = timed_solve(p)
        base_state = p.get_state()
        c2, hit = W.degraded_capacities(inst)
        p.set_capacity(c2)
        tw, iw, sw = timed_solve(p)
        p.reset()
        tc, ic, sc = timed_solve(p)
        out["degrade"] = {"links_degraded": int(hit.sum()), "warm_ms": tw, "warm_iters": iw,
                          "cold_ms": tc, "cold_iters": ic, "speedup_time": tc / tw,
                          "speedup_iters": ic / max(iw, 1), "converged": sw == 0 and sc == 0}
    failed = W.failed_links(inst)
    pr, ks, kl = W.prune(inst, failed)
    warm = {k: base_state[k][ks] for k in ("x", "Z")}
    warm.update({k: base_state[k][kl] for k in ("pbar", "y", "zs", "Rx", "ps")})
    warm["rho"] = base_state["rho"]
    with capi.Problem(pr, stream=sp, precision=0) as q:
        tc, ic, sc = timed_solve(q)
        q.set_state(warm)
        tw, iw, sw = timed_solve(q)
    meas.stop()
    out["fail_prune"] = {"links_failed": int(failed.sum()), "streams_left": pr["n"],
                         "links_left": pr["m"], "warm_ms": tw, "warm_iters": iw, "cold_ms": tc,
                         "cold_iters": ic, "speedup_time": tc / tw,
                         "speedup_iters": ic / max(iw, 1), "converged": sw == 0 and sc == 0}
    line = {"metric": "warm-start re-solve speedup after degradation / failure (Sec. V-D)",
            "value": out["degrade"]["speedup_time"], "unit": "x (cold time / warm time)",
            "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                       "scale": args.scale, "base_solve_ms": t0, "base_iters": it0},
            "paper": {"degrade": "about 5x", "fail_prune": "about 10x (pruned vs full cold)"},
            **out, "gpu_launches": meas.launches, "clocks": meas.clocks}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """The differentiation recipe (c5: n = 1e6, m = 1e5, routes of 2..8 links, log
    utilities, box [0, 20]): d(sum U(x_500))/dc and /dw through 500 unrolled iterations with
    checkpoints every 50, FP32 and FP64, timed with CUDA events against the plain forward
    solve of the same 500 iterations; FP32 gradients compared with FP64 ones."""
    import torch
    from paper_2509_10722_b300 import capi
    inst = W.workload("c5", scale=args.scale)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    iters, kc = 500, 50
    out = {}
    grads = {}
    meas = Measured(torch, capi).start()
    for name, prec in (("fp32", 0), ("fp64", 1)):
        with capi.Problem(inst, stream=sp, precision=prec) as p:
            p.adjoint(iters, kc)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cg, wg, J = p.adjoint(iters, kc)
            e1.record(stream)
            e1.synchronize()
            t_adj = e0.elapsed_time(e1)
            # one segment (checkpoint_every = 0): the forward run tapes every iteration
            e0.record(stream)
            cg1, wg1, J1 = p.adjoint(iters, 0)
            e1.record(stream)
            e1.synchronize()
            t_one = e0.elapsed_time(e1)
            p.reset()
            e0.record(stream)
            p.solve(iters, 0.0)
            e1.record(stream)
            e1.synchronize()
            t_fwd = e0.elapsed_time(e1)
            # the split entries (what the torch Function calls): the forward that keeps its
            # checkpoints, then the backward sweep from them (device arrays)
            cgd = torch.empty(p.m, dtype=torch.float64, device="cuda")
            wgd = torch.empty(p.n, dtype=torch.float64, device="cuda")
            e0.record(stream)
            p.adjoint_forward(iters, kc)
            e1.record(stream)
            e1.synchronize()
            t_kf = e0.elapsed_time(e1)
            e0.record(stream)
            p.adjoint_backward(ubar=1.0, c_grad=cgd, w_grad=wgd)
            e1.record(stream)
            e1.synchronize()
            t_kb = e0.elapsed_time(e1)
            split_equal = bool(np.array_equal(cgd.cpu().numpy(), cg) and
                               np.array_equal(wgd.cpu().numpy(), wg))
            # the sweep alone: one kept segment (checkpoint_every = 0), so the backward
            # recomputes nothing; against the random-read ceiling of its two gather passes
            # ((Abar, Bbar) pairs from the n-vector, Rx_bar from the m-vector)
            p.adjoint_forward(iters, 0)
            e0.record(stream)
            p.adjoint_backward(ubar=1.0, c_grad=cgd, w_grad=wgd)
            e1.record(stream)
            e1.synchronize()
            t_sweep = e0.elapsed_time(e1)
            nnz = int(inst["route_ptr"][-1])
            # one 32-byte sector per read whatever the element size; the probe reads 4 or
            # 8 bytes (an FP64 pair is 16: measured as 8-byte reads of the same vector)
            r_pair = capi.num_measure_gather_rate(nnz, p.n, 8, 3)
            r_one = capi.num_measure_gather_rate(nnz, p.m, 4 if prec == 0 else 8, 3)
            sweep_bound_ms = iters * (nnz / r_pair + nnz / r_one) * 1e3
            # the torch path: total_utility forward and backward (after one untimed call:
            # the first autograd call of a process sets up torch's engine)
            from paper_2509_10722_b300 import autograd
            ct = torch.tensor(inst["c"], device="cuda", requires_grad=True)
            wt = torch.tensor(inst["w"], device="cuda", requires_grad=True)
            with torch.cuda.stream(stream):
                autograd.total_utility(p, ct, wt, iters, kc).backward()
                ct.grad = None
                wt.grad = None
            with torch.cuda.stream(stream):
                e0.record(stream)
                Jt = autograd.total_utility(p, ct, wt, iters, kc)
                Jt.backward()
                e1.record(stream)
            e1.synchronize()
            t_torch = e0.elapsed_time(e1)
            torch_equal = bool(np.array_equal(ct.grad.cpu().numpy(), cg) and
                               np.array_equal(wt.grad.cpu().numpy(), wg))
            p.adjoint_release()
        grads[name] = (cg, wg)
        out[name] = {"adjoint_ms": t_adj, "forward_ms": t_fwd, "ratio": t_adj / t_fwd,
                     "objective": J, "one_segment_ms": t_one,
                     "one_segment_ratio": t_one / t_fwd,
                     "one_segment_equal": bool(np.array_equal(cg, cg1) and
                                               np.array_equal(wg, wg1)),
                     "kept_forward_ms": t_kf, "backward_ms": t_kb,
                     "backward_ratio": t_kb / t_fwd, "split_equal": split_equal,
                     "sweep_ms": t_sweep, "sweep_bound_ms": sweep_bound_ms,
                     "sweep_frac_of_gather_ceiling": sweep_bound_ms / t_sweep,
                     "torch_forward_backward_ms": t_torch,
                     "torch_ratio": t_torch / t_fwd, "torch_equal": torch_equal}
    meas.stop()
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    line = {"metric": "adjoint of 500 unrolled PMP iterations (dJ/dc, dJ/dw), c5",
            "value": out["fp32"]["adjoint_ms"], "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c5: n=1e6, m=1e5, routes U{2..8}, log utilities, "
                                   "w~U[0.5,2], box [0,20]", "iters": iters,
                       "checkpoint_every": kc, "scale": args.scale},
            **out,
            "fp32_vs_fp64": {"dc_rel": rel(grads["fp32"][0], grads["fp64"][0]),
                             "dw_rel": rel(grads["fp32"][1], grads["fp64"][1])},
            "gpu_launches": meas.launches, "clocks": meas.clocks}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.record_traffic:
        print(json.dumps(record_traffic(args.record_traffic, args.workload)))
        return
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
        return
    if args.scenario == "adjoint":
        run_adjoint(args)
        return
    if args.scenario == "warmstart":
        run_warmstart(args)
        return
    if args.scenario == "congestion":
        run_congestion(args)
        return
    if args.scenario == "scaling":
        run_scaling(args)
        return
    if args.workload == "c4":
        run_batched(args)
        return
    run_ours(args, dist)


if __name__ == "__main__":
    main()
