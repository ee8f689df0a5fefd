"""Every launch configuration the autotuner can pick computes the same exact sums:
terms per run, pairs per thread (1 or 2 streams), CTA size, accumulator limb
class, the Montgomery width crossover (small moduli on the two-limb path) and
queue hand-out size change only the schedule or the arithmetic route, never a
bit of the result."""

import json
import os
import tempfile

import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

SETTINGS = [
    {"run": 2, "streams": 1, "grab": 1},
    {"run": 16, "streams": 2, "grab": 3},
    {"run": 64, "streams": 1, "grab": 32},
    {"run": 128, "streams": 2, "grab": 8},
    {"run": 64, "cta": 64, "limb_bump": 1, "wide_min_bits": 5},
    {"run": 32, "streams": 2, "cta": 128, "wide_min_bits": 17, "grab": 2},
    {"run": 64, "cta": 32, "limb_bump": 2, "wide_min_bits": 29},
    {"run": 64, "streams": 1, "wide_min_bits": 31},
    {"run": 128, "streams": 2, "wide_min_bits": 32, "cta": 192},
    {"run": 8, "wide_min_bits": 30, "grab": 5},
]


def plan_with(bbp, setting, guard=64):
    fd, path = tempfile.mkstemp(suffix=".json")
    with os.fdopen(fd, "w") as fh:
        json.dump(setting, fh)
    try:
        return bbp.Plan(device=0, guard_bits=guard, tune_table=path)
    finally:
        os.unlink(path)


@pytest.mark.parametrize("setting", SETTINGS, ids=[json.dumps(s) for s in SETTINGS])
def test_settings_give_identical_sums(setting):
    import paper_1008_3171_gb300 as bbp

    p = plan_with(bbp, setting)
    try:
        for n, P, j, kb, ke in [(10**12, 256, 0, 5 * 10**10, 5 * 10**10 + 70_001),
                                (10**12, 256, 5, 3, 200_003), (10**9 + 1, 128, 3, 0, None),
                                (99_991, 64, 6, 0, None), (10**6, 100, 1, 1, 12_345),
                                (3 * 10**9 + 7, 64, 2, 2 * 10**8 - 40_000, 2 * 10**8 + 40_000),
                                (10**15 + 1, 256, 4, 7_036_874_417_765 - 20_000, 7_036_874_417_765 + 20_000)]:
            assert p.partial_sum(0, j, kb, ke, n, P) == oracle.c_partial_sum(0, j, kb, ke, n, P, 64)
        ns, Ps = workloads.batched_queries(count=48, seed=17, lo=2.0, hi=6.5)
        vals, valid, _ = bbp.bbp_bits_batch(p.handle, 0, ns, Ps)
        for q, (n, P) in enumerate(zip(ns, Ps)):
            assert (vals[q], valid[q]) == oracle.c_bits(n, P, 64)
    finally:
        p.close()


def test_montgomery_width_setting_is_applied():
    """Moduli from 2^4 to 2^20 move to the two-limb path when wide_min_bits = 5: the
    result is unchanged and the modelled multiply count rises (13 instead of 4
    halves per squaring)."""
    import paper_1008_3171_gb300 as bbp

    default = plan_with(bbp, {})
    wide = plan_with(bbp, {"wide_min_bits": 5})
    try:
        assert default.bits(10**6, 64) == wide.bits(10**6, 64) == oracle.c_bits(10**6, 64, 64)
        d, w = default.stats(), wide.stats()
        assert d["terms"] == w["terms"]
        assert w["imad_model"] > 1.5 * d["imad_model"]
    finally:
        default.close()
        wide.close()
