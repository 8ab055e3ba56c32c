"""Clock sampling of bench.py against a fake nvidia-smi on the host: the lines
of this process's GPU are picked by UUID among several GPUs, only samples
inside the marked timed region count, and throttle reasons are collected."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = r"""#!/bin/bash
# fake nvidia-smi: two GPUs, one line each every 20 ms; GPU 1 (ours) reports
# 1980 MHz before the marker file exists and 2070 MHz with sw_power_cap after
while true; do
  ts=$(date +"%Y/%m/%d %H:%M:%S.%3N")
  echo "$ts, 0, GPU-00000000-0000-0000-0000-000000000000, 1500, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active"
  if [ -e "$MARK" ]; then
    echo "$ts, 1, GPU-11111111-2222-3333-4444-555555555555, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"
  else
    echo "$ts, 1, GPU-11111111-2222-3333-4444-555555555555, 1980, 2070, 200.0, 0x0, Not Active, Not Active, Not Active, Not Active"
  fi
  sleep 0.02
done
"""


def _fake_smi(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    mark = tmp_path / "mark"
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    monkeypatch.setenv("MARK", str(mark))
    return mark


def test_samples_inside_the_region_of_our_gpu(tmp_path, monkeypatch):
    mark = _fake_smi(tmp_path, monkeypatch)
    s = bench.ClockSampler(0, uuid="11111111-2222-3333-4444-555555555555", interval_ms=20)
    s.start()
    assert s.lines, "first sample not awaited"
    time.sleep(0.2)                  # samples before the region (1980 MHz) are dropped
    mark.touch()
    time.sleep(0.1)
    s.mark_start()
    time.sleep(0.5)
    s.mark_stop()
    time.sleep(0.2)
    c = s.stop()
    assert c["window"] == "timed region"
    assert c["samples"] >= 5
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_index_fallback_and_missing_tool(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    s = bench.ClockSampler(0, uuid=None, interval_ms=20)   # no UUID: index 0 of two GPUs
    s.start()
    s.mark_start()
    time.sleep(0.3)
    s.mark_stop()
    c = s.stop()
    assert c["sm_mhz"] == 1500.0 and c["reasons"] == []
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["sm_mhz"] is None and c["samples"] == 0
