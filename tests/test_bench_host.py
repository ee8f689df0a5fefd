"""Host side of bench.py, without a GPU: the clock-sample summary that decides
whether a run saw throttling, the percentile used for p50/p99, and the
reference arm's JSON line (the oracle timed on the host cores)."""

import importlib.util
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


bench = _bench()


def line(sm, smax, reasons=("Not Active",) * 4, power="900.00"):
    return ", ".join(["0", str(sm), str(smax), power, "0x0000000000000000", *reasons]) + "\n"


def test_clock_summary_under_load():
    lines = [line(345, 2070)] * 3 + [line(2070, 2070)] * 10 + [line(2055, 2070)] * 5
    got = bench.ClockSampler.summarize(lines)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 18}


def test_clock_summary_reports_throttle_reasons():
    pc = ("Not Active", "Not Active", "Not Active", "Active")
    th = ("Active", "Active", "Not Active", "Not Active")
    got = bench.ClockSampler.summarize([line(1900, 2070, pc)] * 4 + [line(1500, 2070, th)])
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert got["sm_mhz"] == 1900.0 and got["samples"] == 5


def test_clock_summary_tolerates_missing_values():
    assert bench.ClockSampler.summarize([]) is None
    assert bench.ClockSampler.summarize(["garbage\n", "\n"]) is None
    got = bench.ClockSampler.summarize([line("[N/A]", "[N/A]")] * 2 + [line(1000, 2070)])
    assert got["sm_mhz"] == 1000.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3


def test_percentile():
    v = list(range(101))
    assert bench.percentile(v, 50) == 50 and bench.percentile(v, 99) == 99 and bench.percentile(v, 0) == 0
    assert bench.percentile([], 50) is None
    assert bench.percentile([7], 99) == 7


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--cpu-seconds", "2"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == "terms/s"
    assert j["value"] > 0 and j["higher_is_better"] is True and j["steps"] == 1 and j["warmup"] == 3
    assert j["n_gpus"] == 1 and j["data"] == "synthetic" and j["config"]["workload"] == bench.WORKLOAD
    assert j["e2e"] == {"value": j["value"], "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1 and "k-ranges" in cb["sample"]


@pytest.mark.parametrize("rank", ["1"])
def test_reference_arm_is_silent_on_other_ranks(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_sampler_start_stop_with_a_fake_nvidia_smi(tmp_path, monkeypatch):
    """The sampler's whole start/stop path against a stand-in nvidia-smi that
    prints samples every 50 ms until it is terminated."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "while true; do\n"
                    "  echo '0, 2070, 2070, 1100.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.05\n"
                    "done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    import time

    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.4)
    got = s.stop()
    assert got is not None and got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] >= 2
    assert not os.path.exists(s.path)


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() is None
    assert not os.path.exists(s.path)               # its sample file is gone too
