"""Host-side pieces of bench.py that run without a GPU: the FP64 oracle leg (the CPU
baseline and the reference arm) on a small scene, and the JSON line's shape."""
import json
import subprocess
import sys
import os

import bench
from paper_2507_20239_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_view_seconds_small_scene():
    sc = synth.orbit_scene(1, n=3000, width=160, height=106, f=160.0)
    total, spent, sample, cores = bench.oracle_view_seconds(sc, 4)
    assert total > 0 and spent > 0 and cores >= 1
    assert "tiles" in sample


def test_reference_arm_json_line():
    env = dict(os.environ)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", "4000", "--cpu-sample-tiles", "4"],
                         capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "views/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
