"""The bench's reference arm (the FP64 CPU oracle timed on host cores): one JSON line on rank 0 with
the own arm's metric, unit and direction, nothing on the other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3"]


def _run(rank):
    env = dict(os.environ, RANK=str(rank))
    r = subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_line_on_rank_zero():
    lines = _run(0)
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    assert _run(1) == []


def test_roofline_of_the_pair_classes():
    """The roofline object: the dominant class by summed time, the method's flops over its time against
    the measured FP32 rate, and DRAM traffic only where the capture is of the current kernel."""
    import bench
    import inputs
    cfg = inputs.config3(seed=3)
    peaks = {"ffma": {"value": 80.0}}
    ms = {"pairs_fp32": 100.0, "pairs_fp64class": 300.0, "self_weights": 50.0}
    n = {"pairs_fp32": 20, "pairs_fp64class": 10, "self_weights": 4}
    work = {"pairs_fp32": 4.0e12, "pairs_fp64class": 6.0e12}
    r = bench.roofline(ms, n, work, cfg, peaks)
    assert r["kernel_class"] == "pairs_fp64class" and r["launches"] == 10
    assert abs(r["achieved"] - 20.0) < 1e-9 and abs(r["frac"] - 0.25) < 1e-12   # 6e12 flops in 0.3 s
    assert r["traffic"] is None and r["traffic_last_capture"]["bytes_per_launch"] > 0
    r32 = bench.roofline(ms, n, work, cfg, peaks, dom="pairs_fp32")
    assert abs(r32["frac"] - 0.5) < 1e-12 and r32["traffic"] == bench.TRAFFIC["pairs_fp32"]
    assert "traffic_last_capture" not in r32
