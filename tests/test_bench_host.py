"""Host-side logic of bench.py, on CPU: multi-rank aggregation over gloo
(world size 2), the algorithmic-byte count, and the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import bench
from paper_2004_02290_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 1000.0 * (rank + 1)       # each rank's own replica of the workload
    seconds = 0.5 + 0.25 * rank       # the slower rank decides the time
    value, t = bench.aggregate(units, seconds, world)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"value": value, "t": t}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            res = json.load(f)
        assert res["t"] == pytest.approx(0.75)
        assert res["value"] == pytest.approx(3000.0 / 0.75)


def test_aggregate_single():
    v, t = bench.aggregate(500.0, 0.25, 1)
    assert v == pytest.approx(2000.0) and t == 0.25


def test_defaults_meet_the_timing_rules():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.config == "large_cls"


def test_method_bytes_counts_each_term():
    w = wl.Workload(name="x", points=np.zeros((10, 4), np.float32),
                    labels=np.zeros(10, np.int32), queries=np.zeros((2, 4), np.float32), k=3,
                    mode=wl.VOTE, w=1.0, table=wl.TABLE_HASH, seed=0)
    stats = np.array([[2, 5, 40], [3, 7, 60]], np.int64)
    # per query: 4*4 (query) + 8*3 (ids, dist2) + 4 (pred) + 4*3 (winner outputs) = 56
    # cells: 12 hash slots of 16 B; points: 100 rows of 4 floats
    assert bench.method_bytes(w, stats, 4, 2) == 2 * 56 + 12 * 16 + 100 * 16
    assert bench.method_bytes(w, stats, 4, 1) == 2 * 56 + 12 * 8 + 100 * 16


def test_profiled_traffic_ignores_stale_summaries(tmp_path, monkeypatch):
    p = tmp_path / "q_large_cls.md"
    p.write_text("workload: large_cls\nkernel_source_sha256_16: 0000\n"
                 "dram_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "q_{}.md"))
    assert bench.profiled_traffic("large_cls") is None
    p.write_text(f"workload: large_cls\nkernel_source_sha256_16: {bench.query_kernel_sha()}\n"
                 "dram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic("large_cls") == 123.0
    assert bench.profiled_traffic("skewed_reg") is None  # no summary for it
    # a summary filed under one workload's name but taken on another
    (tmp_path / "q_tiny.md").write_text(
        f"workload: large_cls\nkernel_source_sha256_16: {bench.query_kernel_sha()}\n"
        "dram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic("tiny") is None


def test_committed_summaries_match_their_names():
    import glob
    import re
    for path in glob.glob(os.path.join(ROOT, "profiles", "query_kernel_*_ncu.md")):
        text = open(path).read()
        wk = re.search(r"workload:\s*(\S+)", text)
        assert wk, path
        name = os.path.basename(path)[len("query_kernel_"):-len("_ncu.md")]
        if name in ("large_cls", "skewed_reg", "tiny"):
            assert wk.group(1) == name, path


def test_query_order_per_workload():
    class K:
        KNN_QUERY_SORTED = 2
    assert bench.query_order("skewed_reg") == "cell"
    assert bench.query_order("large_cls") == "input"
    assert bench.query_flags(K, "skewed_reg") == 2 and bench.query_flags(K, "large_cls") == 0
    assert bench.query_flags(K, "skewed_reg", "input") == 0
    assert bench.query_flags(K, "large_cls", "cell") == 2


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "tiny",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "queries/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == "tiny"


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "tiny",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
