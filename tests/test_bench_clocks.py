"""bench.py's clock record: nvidia-smi rows taken inside the timed region only, their median SM
clock and the throttle reasons seen.  A fake nvidia-smi on PATH writes rows on the CPU."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/sh
# rows every 50 ms: SM clock falls 2070 -> 1900 after the fourth row; power cap from the sixth
i=0
while [ $i -lt 400 ]; do
  if [ $i -lt 4 ]; then c=2070; else c=1900; fi
  if [ $i -ge 6 ]; then cap=Active; else cap="Not Active"; fi
  echo "0, $c, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, $cap"
  i=$((i+1))
  sleep 0.05
done
"""


def _fake_smi(tmp_path, monkeypatch, body=FAKE):
    p = tmp_path / "nvidia-smi"
    p.write_text(body)
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")


def test_rows_before_the_mark_are_dropped(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    time.sleep(0.45)        # rows 0..8 or so before the timed region
    c.mark()
    time.sleep(0.5)
    out = c.stop()
    assert out["samples"] >= 3
    assert out["sm_mhz"] == 1900.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert "note" not in out


def test_a_region_shorter_than_one_interval_keeps_the_last_row(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch, FAKE.replace("sleep 0.05", "sleep 5"))
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)     # returns once the first row is there
    c.mark()
    out = c.stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    assert "shorter than one interval" in out["note"]


def test_no_nvidia_smi_gives_no_record(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.mark()
    assert c.stop() is None
