"""bench.py host logic without a GPU: the reference arm's JSON line, rank behaviour, the
clock summary, the traffic record, and the replica timing reduction over gloo ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, env=e, timeout=600)


def test_reference_arm_line():
    r = _run(["--impl", "reference", "--scale", "0.0005", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "iterations/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_reference_arm_nonzero_rank_is_silent():
    r = _run(["--impl", "reference", "--scale", "0.0005", "--steps", "1", "--warmup", "0"],
             env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_parse_clocks():
    text = ("0, 1965, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Active\n"
            "0, 2032, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "0, 1900, 2032, 980.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.parse_clocks(text)
    assert c == {"sm_mhz": 1965.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    assert bench.parse_clocks("") is None


def test_record_traffic_parses_ncu_csv(tmp_path):
    """Two captured launches of each row kernel in ncu's CSV layout (header line, quoted
    fields, thousands separators, scaled units): per-launch means per kernel."""
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
           '"Metric Value"')
    rows = []
    for i, (kern, rd, wr, unit) in enumerate([
            ("k_stream_rows<float>", "400,000,000", "60,000,000", "byte"),
            ("k_link_rows<float>(pmp::View<float>)", "300", "20", "Mbyte"),
            ("k_stream_rows<float>", "410,000,000", "62,000,000", "byte"),
            ("k_link_rows<float>(pmp::View<float>)", "302", "18", "Mbyte")]):
        for metric, v in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr)):
            rows.append(f'"{i}","1","python","h","{kern}","1","7","(256, 1, 1)","(1184, 1, 1)",'
                        f'"0","10.3","Command line profiler metrics","{metric}","{unit}","{v}"')
    csv_path = tmp_path / "traffic.csv"
    csv_path.write_text("==PROF== Connected to process 1\n" + hdr + "\n" + "\n".join(rows) + "\n")
    out = tmp_path / "traffic.json"
    rec = bench.record_traffic(str(csv_path), "c2", out_path=str(out))
    s = rec["c2:k_stream_rows"]
    assert s["launches"] == 2 and s["read"] == 405_000_000 and s["write"] == 61_000_000
    assert s["dram_bytes_per_launch"] == 466_000_000
    l = rec["c2:k_link_rows"]
    assert l["read"] == 301_000_000 and l["write"] == 19_000_000
    assert s["source_sha"] == bench.row_sources_sha()
    assert json.loads(out.read_text()) == rec


def test_traffic_record_requires_matching_source():
    rec = bench.traffic_record("c2:k_link_rows")
    if rec is not None:
        assert rec["dram_bytes_per_launch"] > 0
    assert bench.traffic_record("c2:no_such_kernel") is None


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    # per-rank timed milliseconds and iterations: value = sum(iters) / max(time)
    ms = 100.0 + 50.0 * rank
    its = 1000 + rank
    q.put((rank, d.max(ms), d.sum(its)))
    d.close()


def test_replica_timing_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, sm in res:
        assert mx == 150.0 and sm == 2001.0
