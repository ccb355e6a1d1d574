"""bench.py's clock sampler on CPU, with a stand-in for nvidia-smi on PATH that prints one CSV line
every 20 ms: a loaded clock of 2070 MHz, then, from its 20th line on, a throttled 1500 MHz with
sw_power_cap active. The sampler keeps only the lines that arrive within the timed window, so a
window before the change reports 2070 MHz and no reason, and one after it reports 1500 MHz and
sw_power_cap."""

import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/sh
i=0
while [ $i -lt 400 ]; do
  if [ $i -lt 20 ]; then
    echo "0, 2070, 2070, 900.0, 100, 0x0, Not Active, Not Active, Not Active, Not Active"
  else
    echo "0, 1500, 2070, 1400.0, 100, 0x4, Not Active, Not Active, Not Active, Active"
  fi
  i=$((i+1))
  sleep 0.02
done
"""


def test_clock_samples_are_taken_from_the_timed_window(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])

    c = bench.ClockSampler(0)
    c.start()
    assert c.lines, "start() returns once the first sample has arrived"
    t0 = time.perf_counter()
    time.sleep(0.1)
    t1 = time.perf_counter()
    time.sleep(0.8)                      # well past the change of clock
    t2 = time.perf_counter()
    time.sleep(0.2)
    t3 = time.perf_counter()
    lines = list(c.lines)
    early = c.stop((t0, t1))
    c.lines = lines
    late = c.stop((t2, t3))
    assert early["sm_mhz"] == 2070.0 and early["reasons"] == [] and early["samples"] >= 2
    assert late["sm_mhz"] == 1500.0 and late["reasons"] == ["sw_power_cap"] and late["samples"] >= 2
    assert early["sm_max_mhz"] == late["sm_max_mhz"] == 2070.0
