"""Host logic of bench.py that needs no GPU: the clock sampler's parsing,
its restriction to the timed region and its throttle-reason report, driven
by a stand-in nvidia-smi script that prints rows in the query's CSV format;
and the JSON line of the reference arm, which times the oracle on the host."""
import os
import stat
import time

import pytest

import bench

ROW = "echo \"$(date +'%Y/%m/%d %H:%M:%S.%3N'), 0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, {swt}, Not Active\""


def _fake_smi(tmp_path, body):
    p = tmp_path / "nvidia-smi"
    p.write_text("#!/bin/bash\n" + body + "\n")
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def _sample(monkeypatch, path, before=0.3, inside=0.7, after=0.3):
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ.get("PATH", ""))
    c = bench.Clocks(0)
    time.sleep(before)
    c.mark_start()
    time.sleep(inside)
    c.mark_end()
    time.sleep(after)
    tmp = c.path
    out = c.stop()
    assert not os.path.exists(tmp)
    return out


def test_clocks_keep_only_the_timed_region(tmp_path, monkeypatch):
    # 1000 MHz outside the timed region, 2070 about inside it: most samples
    # are taken outside, so without the restriction the median would be 1000
    body = ("t0=$(date +%s.%N); while true; do now=$(date +%s.%N); "
            "if awk -v a=$now -v b=$t0 'BEGIN{exit !(a-b>0.55 && a-b<1.15)}'; then "
            + ROW.format(sm=2070, swt="Not Active") + "; else "
            + ROW.format(sm=1000, swt="Not Active") + "; fi; sleep 0.1; done")
    out = _sample(monkeypatch, _fake_smi(tmp_path, body), before=0.6, inside=0.5, after=0.8)
    assert out["samples_in_timed_region"] is True
    assert out["samples"] <= 7
    assert out["sm_mhz"] == 2070.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_clocks_report_throttle_reasons(tmp_path, monkeypatch):
    body = "while true; do " + ROW.format(sm=1800, swt="Active") + "; sleep 0.1; done"
    out = _sample(monkeypatch, _fake_smi(tmp_path, body))
    assert out["reasons"] == ["sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1800.0


def test_clocks_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.Clocks(0)
    tmp = c.path
    assert c.stop() is None
    assert not os.path.exists(tmp)


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle on the host cores, bounded
    samples) prints one JSON line with the keys of the bench contract, on
    the same metric and unit as the GPU arm, and an e2e entry that moves no
    bytes across the host link."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "3", "--warmup", "3", "--ref-sample", "4096"],
                         capture_output=True, text=True, timeout=300, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
