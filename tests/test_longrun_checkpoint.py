"""Host side of checkpointed long runs (paper_1008_3171_gb300/longrun.py): the
checkpoint records exactly the finished shards and their accumulators, survives
a save/load round trip, refuses a checkpoint of another query, and resumes with
the shards still missing.  The checkpoint module is loaded by file path, so no
GPU and no compiled library are needed."""

import importlib.util
import json
import os
import sys

import pytest

from conftest import ROOT


def _module():
    path = os.path.join(ROOT, "paper_1008_3171_gb300", "longrun.py")
    spec = importlib.util.spec_from_file_location("longrun_host_only", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod          # dataclasses look the module up by name
    spec.loader.exec_module(mod)
    return mod


lr = _module()


def test_fresh_checkpoint_has_every_shard_left():
    ck = lr.Checkpoint.fresh(0, 10**14 + 1, 256, 64, 8, 10)
    assert ck.remaining() == list(range(8))
    assert ck.slots == [0] * 10 and ck.done == []


def test_add_records_shards_in_any_order():
    ck = lr.Checkpoint.fresh(0, 1001, 64, 64, 5, 4)
    ck.add(3, [1, -1, 2, 3], 0.5)           # device values come back as signed int64
    ck.add(0, [5, 6, 7, 8], 0.25)
    assert ck.done == [0, 3] and ck.remaining() == [1, 2, 4]
    assert ck.slots == [5, 6, 7, 8] and ck.seconds == pytest.approx(0.75)
    ck2 = lr.Checkpoint.fresh(0, 1001, 64, 64, 5, 4)
    ck2.add(1, [1, -1, 2, 3], 0.0)
    assert ck2.slots[1] == (1 << 64) - 1     # stored unsigned, modulo 2^64
    with pytest.raises(ValueError):
        ck.add(3, [0, 0, 0, 0], 0.0)        # twice
    with pytest.raises(ValueError):
        ck.add(5, [0, 0, 0, 0], 0.0)        # out of range
    with pytest.raises(ValueError):
        ck.add(1, [0, 0, 0], 0.0)           # wrong accumulator count


def test_save_load_round_trip_and_resume(tmp_path):
    path = str(tmp_path / "run.json")
    fresh = lr.Checkpoint.fresh(0, 10**13 + 1, 256, 64, 6, 10)
    assert lr.Checkpoint.load_or_fresh(path, fresh) is fresh      # no file yet
    big = [(1 << 64) - 1 - i for i in range(10)]
    fresh.add(2, big, 12.5)
    fresh.save(path)
    assert os.listdir(tmp_path) == ["run.json"]                    # temporary file replaced
    back = lr.Checkpoint.load_or_fresh(path, lr.Checkpoint.fresh(0, 10**13 + 1, 256, 64, 6, 10))
    assert back.slots == big and back.done == [2] and back.remaining() == [0, 1, 3, 4, 5]
    assert back.seconds == pytest.approx(12.5)
    raw = json.load(open(path))
    assert raw["n"] == str(10**13 + 1) and all(isinstance(v, str) for v in raw["slots"])


@pytest.mark.parametrize("other", [
    (1, 10**13 + 1, 256, 64, 6, 10),     # other formula
    (0, 10**13 + 3, 256, 64, 6, 10),     # other position
    (0, 10**13 + 1, 128, 64, 6, 6),      # other width
    (0, 10**13 + 1, 256, 96, 6, 11),     # other guard
    (0, 10**13 + 1, 256, 64, 7, 10),     # other shard count
])
def test_checkpoint_of_another_query_is_refused(tmp_path, other):
    path = str(tmp_path / "run.json")
    lr.Checkpoint.fresh(0, 10**13 + 1, 256, 64, 6, 10).save(path)
    with pytest.raises(ValueError):
        lr.Checkpoint.load_or_fresh(path, lr.Checkpoint.fresh(*other))


def test_corrupt_checkpoints_are_refused(tmp_path):
    good = lr.Checkpoint.fresh(0, 99, 64, 64, 4, 4).to_json()
    for bad in ({**good, "format": "x"}, {**good, "done": [1, 1]}, {**good, "done": [4]}):
        with pytest.raises(ValueError):
            lr.Checkpoint.from_json(bad)
    with pytest.raises(ValueError):
        lr.Checkpoint.fresh(0, 99, 64, 64, 0, 4)
