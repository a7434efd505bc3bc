"""Host logic of bench.py that needs no GPU: the reference arm (the CPU oracle
timed on the host) and its JSON line, the ranks that must stay silent, and the
clock sampler's reading of nvidia-smi (through a stand-in nvidia-smi)."""
import json
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          cwd=ROOT, env=e, timeout=300)


def test_reference_arm_prints_one_line_with_the_contract_keys():
    import bench
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == bench.WORKLOADS["c3"][6]  # the gb300 arm's default workload
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_output():
    r = _bench("--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
               env={"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_names_the_workloads_it_does_not_cover():
    r = _bench("--impl", "reference", "--workload", "c4")
    assert r.returncode == 0
    d = json.loads(r.stdout.strip())
    assert d["impl"] == "reference" and "unavailable" in d


FAKE_SMI = """#!/bin/sh
# stand-in for nvidia-smi --query-gpu=...: three samples, then wait to be stopped
echo "1965, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "2070, 2070, 1310.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "2055, 2070, 1290.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
sleep 30
"""


def test_clock_sampler_reads_clocks_and_throttle_reasons(tmp_path, monkeypatch):
    import bench
    smi = tmp_path / "nvidia-smi"
    smi.write_text(FAKE_SMI)
    smi.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler("0")
    s.start()
    for _ in range(50):
        if len(s.rows) >= 3:
            break
        time.sleep(0.05)
    c = s.stop()
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler("0")
    s.start()
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
