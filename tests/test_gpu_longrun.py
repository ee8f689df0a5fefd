"""Checkpointed long run on the GPU: a run stopped after some shards and resumed
from its checkpoint file (by a new plan, as a new process would) gives the same
bits and certified count as one uninterrupted bbp_bits call, and a resumed run
that finds every shard done only finalizes."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,P,shards,first", [(10**9 + 1, 256, 5, 2), (10**6, 64, 3, 1), (654_321, 1000, 4, 3)])
def test_stop_and_resume_equals_uninterrupted(tmp_path, n, P, shards, first):
    import paper_1008_3171_gb300 as bbp
    from paper_1008_3171_gb300 import longrun

    path = str(tmp_path / "ck.json")
    r1 = longrun.run(n, P, shards, path, max_shards=first)
    assert r1["done"] == first and "bits_hex" not in r1
    r2 = longrun.run(n, P, shards, path)
    assert r2["done"] == shards and r2["added"] == shards - first
    with bbp.Plan(device=0, guard_bits=64) as plan:
        bits, valid = plan.bits(n, P)
    assert (int(r2["bits_hex"], 16), r2["valid_bits"]) == (bits, valid)
    r3 = longrun.run(n, P, shards, path)
    assert r3["added"] == 0 and r3["bits_hex"] == r2["bits_hex"]


def test_resumed_run_matches_the_suppressed_m9_row(tmp_path, pins):
    from paper_1008_3171_gb300 import longrun

    pin = pins["suppressed_m9"]
    path = str(tmp_path / "m9.json")
    longrun.run(pin["n"], 256, 4, path, max_shards=1)
    r = longrun.run(pin["n"], 256, 4, path)
    paper = int(pin["hex"], 16) >> (4 * len(pin["hex"]) - 256)
    v = r["valid_bits"]
    assert v >= 200 and int(r["bits_hex"], 16) >> (256 - v) == paper >> (256 - v)
