"""Host logic of the autotuner (paper_1008_3171_gb300/autotune.py) with a stand-in
for the library: each setting reaches the plan through a tune-table file, the
fastest setting wins, and a setting that changes the result stops the sweep."""

import importlib.util
import json
import os
import time

import pytest

from conftest import ROOT


def _autotune():
    spec = importlib.util.spec_from_file_location("autotune_host", os.path.join(ROOT, "paper_1008_3171_gb300",
                                                                                 "autotune.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


at = _autotune()


class FakeLib:
    """Plan objects that read the tune table they are given, like bbp_plan_create."""

    def __init__(self):
        self.seen = []

    def Plan(self, device, guard_bits, tune_table):
        with open(tune_table) as fh:
            setting = json.load(fh)
        self.seen.append(setting)
        lib = self

        class P:
            def __init__(self):
                self.setting = setting
                self.closed = False

            def close(self):
                self.closed = True
                lib.closed = getattr(lib, "closed", 0) + 1

        return P()


def test_sweep_picks_the_fastest_and_records_every_value():
    lib = FakeLib()
    delay = {64: 0.02, 128: 0.005, 256: 0.012}

    def work(p):
        time.sleep(delay[p.setting["cta"]])
        return "same sum", 1000

    measured = {}
    best = at._sweep(lib, "cta", (64, 128, 256), {"run": 32, "streams": 1}, work, measured, reps=2)
    assert best == 128
    assert set(measured["cta"]) == {"64", "128", "256"}
    assert measured["cta"]["128"] > measured["cta"]["64"]          # terms per second
    assert all(s["run"] == 32 and s["streams"] == 1 for s in lib.seen)
    assert [s["cta"] for s in lib.seen] == [64, 128, 256]
    assert lib.closed == 3                                          # every plan is released


def test_sweep_stops_when_a_setting_changes_the_result():
    lib = FakeLib()

    def work(p):
        return ("other" if p.setting["limb_bump"] == 1 else "sum"), 10

    with pytest.raises(RuntimeError, match="limb_bump=1 changed the result"):
        at._sweep(lib, "limb_bump", (0, 1), {}, work, {}, reps=1)
    assert lib.closed == 2


def test_tune_table_file_is_removed_after_the_plan_reads_it():
    lib = FakeLib()
    paths = []
    orig = lib.Plan

    def plan(device, guard_bits, tune_table):
        paths.append(tune_table)
        return orig(device, guard_bits, tune_table)

    lib.Plan = plan
    at._plan(lib, run=64, grab=4)
    assert paths and not os.path.exists(paths[0])
    assert lib.seen == [{"run": 64, "grab": 4}]
