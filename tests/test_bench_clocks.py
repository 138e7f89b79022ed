"""bench.py's clock sampler on the CPU, against a stand-in nvidia-smi on PATH
that prints the queried CSV fields every 20 ms: the median SM clock, the
maximum clock and the active throttle reasons of the samples taken inside
the timed region; without nvidia-smi the summary is empty, not an error."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/sh
i=0
while true; do
  if [ $i -lt 3 ]; then echo "1200, 2070, 300.0, Not Active, Not Active, Not Active, Not Active";
  else echo "1965, 2070, 1350.5, Not Active, Not Active, Not Active, Active"; fi
  i=$((i+1)); sleep 0.02
done
"""


def test_summary_of_samples_in_region(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import bench
    with bench.ClockSampler(0) as c:
        time.sleep(0.4)
    s = c.summary()
    assert s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == 1965.0          # the median under load
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] >= 3


def test_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench
    with bench.ClockSampler(0) as c:
        pass
    s = c.summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["reasons"] == []
