"""The benchmark's JSON line on a GPU: `python bench.py --quick` runs the
256x256x4 film step, prints one line, and that line carries every key the
measurement contract asks for, with values in their physical ranges."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_bench_quick_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "5", "--warmup", "3", "--quick"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks",
              "demag_evals_per_s", "timing_context"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["dtype"] == "f32" and d["scaling"] == "weak"
    assert d["config"]["grid"] == [256, 256, 4] and "flushed" in d["config"]["l2"]
    # 262144 cells per step; a step takes between 1 us and 1 ms
    assert 262144 / 1e-3 < d["value"] < 262144 / 1e-6
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - 262144) < 1e-6 * 262144
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert 0 < rf["frac"] < 1.5 and abs(rf["achieved"] / rf["peak"] - rf["frac"]) < 1e-9
    assert rf["traffic"] is None or rf["traffic"] > 0
    e2e = d["e2e"]
    assert e2e["unit"] == d["unit"] and 0 < e2e["value"] <= d["value"] * 1.05
    assert e2e["h2d_bytes_per_step"] == 12 * 262144 and e2e["d2h_bytes_per_step"] == 12 * 262144
    assert d["gpu_launches"] == 2 * 5
    assert d["demag_evals_per_s"] > 0
    bd = d["e2e_breakdown"]
    assert 0 < bd["event_span_us_median"] <= bd["wall_us_median"] and bd["device_buffers_call_us_median"] > 0
    tc = d["timing_context"]
    assert tc["event_pair_around_tiny_kernel_after_flush_us"] > 0
    assert tc["flushed_16_step_calls"]["ms_per_step"] > 0
