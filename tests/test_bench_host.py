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
    total, spent, sample, threads, used = bench.oracle_view_seconds(sc, 4)
    assert total > 0 and spent > 0 and threads >= 1 and used > 0
    assert "tiles" in sample


def test_cpu_baseline_reports_measured_cores_and_single_thread():
    import torch
    sc = synth.orbit_scene(1, n=3000, width=160, height=106, f=160.0)
    n0 = torch.get_num_threads()
    cb = bench.cpu_baseline(sc, 4)
    assert torch.get_num_threads() == n0
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] > 0
    assert cb["single_thread"]["value"] > 0 and cb["host_cores"] >= 1


def test_fp32_peak_from_device_properties_and_clock(monkeypatch):
    import torch

    class Props:
        multi_processor_count = 152
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: Props())
    peak, inp = bench.fp32_peak_tflops(0, {"sm_max_mhz": 2070.0}, {})
    assert abs(peak - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9 and inp["sms"] == 152
    peak, inp = bench.fp32_peak_tflops(0, {"sm_max_mhz": None}, {"sm_max_mhz": 1000.0})
    assert abs(peak - 152 * 128 * 2 * 1e9 / 1e12) < 1e-9 and "MEASURED_PEAKS" in inp["mhz_source"]


def test_reference_arm_json_line():
    env = dict(os.environ)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--n", "4000", "--cpu-sample-tiles", "4"],
                         capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "views/s" and line["value"] > 0
    # the run the arguments ask for: K timed steps after W warm-ups
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    # a step is one bounded sample: its wall time, and the fraction of a view it covers
    assert 0 < line["view_fraction_per_step"] <= 1
    assert abs(line["value"] * line["ms_per_step"] / 1000 - line["view_fraction_per_step"]) < 0.05
