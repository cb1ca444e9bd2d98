"""CPU: bench.py's clock sampler, with a fake nvidia-smi on PATH. The sampler
is started before the warm-up (its start-up stays out of the timed region),
start() returns once the first sample is written, and stop() summarises only
the samples taken after mark(), the start of the timed region."""
from __future__ import annotations

import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

# Writes one CSV sample every 50 ms: SM clock 1000 MHz for the first ten
# samples (the "warm-up"), 2070 MHz after; nine fields as the query asks,
# sw_power_cap Active throughout. It waits 0.3 s before its first line and
# exits by itself after 200 samples, so a failed test leaves nothing running.
FAKE = r'''#!/usr/bin/env python3
import sys, time
time.sleep(0.3)
i = 0
while i < 200:
    mhz = 1000 if i < 10 else 2070
    sys.stdout.write(f"0, {mhz}, 2070, 500.0, 0x4, Not Active, Not Active, Not Active, Active\n")
    sys.stdout.flush()
    i += 1
    time.sleep(0.05)
'''


def _fake_smi(tmp_path, monkeypatch):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(FAKE)
    f.chmod(f.stat().st_mode | stat.S_IEXEC | stat.S_IXGRP | stat.S_IXOTH)
    monkeypatch.setenv("PATH", f"{d}{os.pathsep}{os.environ.get('PATH', '')}")
    monkeypatch.setenv("KDT_CLOCKS_DIR", str(tmp_path / "clocks"))


def test_start_waits_for_the_first_sample_and_stop_reads_after_the_mark(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    c = bench.Clocks(0)
    t0 = time.perf_counter()
    c.start()
    assert time.perf_counter() - t0 >= 0.25          # waited through the sampler's start-up
    assert os.path.getsize(c.path) > 0
    time.sleep(0.7)                                   # past the ten 1000 MHz samples
    c.mark()
    time.sleep(0.5)
    r = c.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert 3 <= r["samples"] <= 15                    # the timed region's samples only
    assert r["reasons"] == ["sw_power_cap"]


def test_a_region_shorter_than_a_sample_falls_back_to_every_sample(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.2)
    c.mark()
    r = c.stop()                                      # no sample after the mark
    assert r["samples"] >= 1 and r["sm_mhz"] is not None


def test_no_nvidia_smi_is_reported_not_raised(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))         # nothing to run
    monkeypatch.setenv("KDT_CLOCKS_DIR", str(tmp_path / "clocks"))
    c = bench.Clocks(0)
    c.start()
    c.mark()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
