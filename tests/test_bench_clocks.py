"""The bench line's `clocks` object from nvidia-smi samples: a fake
nvidia-smi on PATH prints rows in the queried CSV form and the sampler
reports the median SM clock under load (samples above half the maximum),
the maximum clock and every throttle reason seen Active."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ROWS = """0, 2070, 2070, 910.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2055, 2070, 1212.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1980, 2070, 1300.2, 0x0000000000000020, Not Active, Active, Not Active, Not Active
0, 345, 2070, 98.0, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active
"""


def test_clock_sampler_summarises_the_samples(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\ncat <<'EOF'\n" + ROWS + "EOF\nexec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.delenv("MM_CLOCKS_CSV", raising=False)
    import bench
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    c = s.stop()
    assert c["samples"] == 4
    assert c["sm_max_mhz"] == 2070.0
    assert c["sm_mhz"] == 2055.0                 # median of 2070, 2055, 1980; the idle 345 left out
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(s.path)            # the raw samples are removed unless kept


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    import bench
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() is None
    assert not os.path.exists(s.path)            # no sampler: no file left behind
