"""bench.py's output: one JSON line with the fields its consumers read, run
as a user would (a subprocess, a 512^3 volume, a few steps), and the
per-frame JSON lines of --frame-log."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_prints_one_complete_json_line(tmp_path):
    log = tmp_path / "frames.jsonl"
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "6", "--warmup", "3", "--volume", "512",
           "--no-extra", "--no-cpu-baseline", "--frame-log", str(log)]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "gpu_launches"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 6 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["gpu_launches"] == 2 * 6
    assert abs(d["value"] - 6 / (d["ms_per_step"] * 6 / 1e3)) / d["value"] < 1e-3
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0 < r["frac"] < 1.5
    assert r["achieved"] == pytest.approx(r["frac"] * r["peak"], rel=1e-3)
    assert r["algorithmic_bytes_per_launch"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["d2h_bytes_per_step"] == 2 * 1440 * 1600 * 16 and e["h2d_bytes_per_step"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["config"]["workload"] and d["config"]["volume"] == [512, 512, 512]
    frames = [json.loads(ln) for ln in open(log)]
    assert len(frames) == 6 and all(f["leg"] == "render" for f in frames)
    for f in frames:
        assert f["samples"] > 0 and f["bricks_touched"] <= f["bricks_selected"] and f["frame_ms"] > 0
