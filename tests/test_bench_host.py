"""Host side of the benchmark contract, without a GPU: the reference arm (the
oracle timed on the host cores) prints one JSON line with the GPU arm's
metric, unit and direction; the roofline's traffic figure is used only while
the kernel's sources hash to the captured version; the workload config names
the 128^2 workload."""
import json
import subprocess
import sys

import bench


def test_reference_arm_prints_the_gpu_arms_metric():
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
         "--ref-sample-steps", "2"],
        capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "forward solves/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"] == bench.workload_config(4096)


def test_traffic_follows_the_kernel_sources(monkeypatch):
    k = "k_solve2d_tc128<2>"
    sha = bench.sources_sha256(k)
    assert sha == bench.sources_sha256(k) and len(sha) == 64
    monkeypatch.setitem(bench.TRAFFIC, k, {"sha256": sha, "bytes": 123})
    assert bench.traffic_of(k) == 123
    monkeypatch.setitem(bench.TRAFFIC, k, {"sha256": "0" * 64, "bytes": 123})
    assert bench.traffic_of(k) is None  # sources changed since the capture
    assert bench.traffic_of("no_such_kernel") is None


def test_committed_traffic_matches_the_committed_kernel():
    """The traffic figure committed with the bench belongs to the kernel as it
    stands (a change to the kernel must come with a new capture)."""
    assert bench.traffic_of("k_solve2d_tc128<2>") is not None


def test_workload_config_names_the_workload():
    c = bench.workload_config(4096)
    assert c["grid"] == 128 and c["imex_steps"] == 8000 and c["chains"] == 4096
    assert "128^2" in c["workload"] and "L2" in c["l2"]
    assert not any(k in c for k in ("model", "seq_len", "global_batch"))
