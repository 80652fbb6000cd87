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
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.config == "batched"


def test_method_bytes_counts_each_term():
    w = wl.Workload(name="x", points=np.zeros((10, 4), np.float32),
                    labels=np.zeros(10, np.int32), queries=np.zeros((2, 4), np.float32), k=3,
                    mode=wl.VOTE, w=1.0, table=wl.TABLE_HASH, seed=0)
    stats = np.array([[2, 5, 40], [3, 7, 60]], np.int64)
    # per query: 4*4 (query) + 8*3 (ids, dist2) + 4 (pred) + 4*3 (winner outputs) = 56
    # cells: 12 hash slots of 16 B; points: 100 rows of 4 floats
    assert bench.method_bytes(w, stats, 4, 2) == 2 * 56 + 12 * 16 + 100 * 16
    assert bench.method_bytes(w, stats, 4, 1) == 2 * 56 + 12 * 8 + 100 * 16


def _summary(workload, phase, sha, dram=123, extra=""):
    return (f"workload: {workload}\nphase: {phase}\nkernel_source_sha256_16: {sha}\n"
            f"dram_bytes_per_launch: {dram}\n{extra}")


def test_profiled_ignores_stale_summaries(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    p = tmp_path / "q_large_cls_ncu.md"
    p.write_text(_summary("large_cls", "query.search", "0000"))
    assert bench.profiled("large_cls", "query.search") is None
    p.write_text(_summary("large_cls", "query.search", bench.query_kernel_sha(),
                          extra="issue_active_pct: 80.5\nwarp_inst_per_query: 5010\n"))
    got = bench.profiled("large_cls", "query.search")
    assert got["dram_bytes_per_launch"] == 123.0 and got["warp_inst_per_query"] == 5010.0
    assert bench.profiled_traffic("large_cls") == 123.0
    assert bench.profiled("skewed_reg", "query.search") is None  # no summary for it
    assert bench.profiled("large_cls", "query.coop") is None     # another kernel


def test_profiled_build_kernel_summary_keys_on_its_own_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    p = tmp_path / "s_tiny_ncu.md"
    p.write_text(_summary("tiny", "build.small", bench.query_kernel_sha(),
                          extra="kernel_sources: build_kernels.cu\n"))
    assert bench.profiled("tiny", "build.small") is None  # the query source's hash
    p.write_text(_summary("tiny", "build.small", bench.kernel_sha(("build_kernels.cu",)),
                          dram=5e5, extra="kernel_sources: build_kernels.cu\n"))
    assert bench.profiled("tiny", "build.small")["dram_bytes_per_launch"] == 5e5
    p.write_text(_summary("tiny", "build.small", "0000", extra="kernel_sources: nofile.cu\n"))
    assert bench.profiled("tiny", "build.small") is None


def test_roofline_uses_measured_traffic_and_issue_rate(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    (tmp_path / "b_ncu.md").write_text(_summary(
        "batched", "query.d6.k32.hash", bench.query_kernel_sha(), dram=2.0e8,
        extra="bound: issue\nissue_active_pct: 88.8\nwarp_inst_per_query: 20000\n"))
    peaks = {"hbm_gbs": 6800.0}
    r = bench.roofline("batched", "query.d6.k32.hash", 40.0, 1_000_000, 1.0e11, peaks,
                       "measured", {"sm_mhz": 2000.0}, 50.0)
    assert r["kernel"] == "qk::batch_query_kernel<6, 1, 0, 0>"
    assert r["bound"] == "issue"
    assert r["achieved"] == pytest.approx(2.0e8 / 0.040 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["method_bytes_per_s"] == pytest.approx(1.0e11 / 0.040 / 1e9)
    assert r["cross_check"]["below_peak"]
    ipk = 152 * 4 * 2000.0e6
    assert r["issue"]["frac"] == pytest.approx(20000 * 1_000_000 / 0.040 / ipk)
    # no profile on the current source: no DRAM figure, no fraction
    r = bench.roofline("batched", "query.d2.k32.dense", 4.0, 10, 1.0e9, peaks, "measured",
                       None, 50.0)
    assert r["traffic"] is None and r["frac"] is None and r["bound"] is None


def test_kernel_names_of_phases():
    assert bench.kernel_of_phase("query.d3.k64.dense.coop") == "qk::batch_heavy_kernel<3, 2, 1, 0>"
    assert bench.kernel_of_phase("query.d4.k32.hash.exact") == "qk::batch_query_kernel<4, 1, 0, 1>"
    assert bench.kernel_of_phase("build.sort").startswith("radix_hist_kernel")


def test_committed_summaries_name_their_workload():
    import glob
    for path in glob.glob(os.path.join(ROOT, "profiles", "*_ncu.md")):
        text = open(path).read()
        assert bench._field(text, "workload"), path


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


def test_reference_arm_batched_times_a_fixed_sample():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--batch-count", "6",
                        "--ref-step-seconds", "0.2", "--steps", "2", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads([l for l in r.stdout.splitlines() if l.strip()][-1])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC_BATCHED
    assert d["config"]["workload"] == "batched" and d["config"]["sample_problems"] >= 1
    # the line's value is the sample's queries over the time the steps took
    q = d["config"]["sample_queries"]
    assert d["value"] == pytest.approx(q / (d["ms_per_step"] * 1e-3), rel=1e-6)
