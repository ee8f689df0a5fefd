"""The batched persistent pass (bbp_bits_batch) against the oracle (and, for
queries too large to run through the oracle here, the paper's printed rows and
the single-query path), bit for bit, on seeded mixed-size batches."""

import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbp():
    import paper_1008_3171_gb300 as m

    return m


@pytest.fixture(scope="module")
def plan(bbp):
    p = bbp.Plan(device=0, guard_bits=64)
    yield p
    p.close()


def test_small_batch_matches_oracle(bbp, plan):
    ns, Ps = workloads.batched_queries(count=160, seed=5, lo=0.0, hi=6.0, precisions=(1, 8, 64, 100, 128, 256))
    ns += [1, 2, 9, 10, 11, 100]
    Ps += [8, 64, 8, 1, 256, 1000]
    vals, valid, lat = bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)
    for q, (n, P) in enumerate(zip(ns, Ps)):
        assert (vals[q], valid[q]) == oracle.c_bits(n, P, 64), (q, n, P)
    assert all(v >= 0 for v in lat)


def test_batch_matches_single_query_path(bbp, plan):
    ns, Ps = workloads.batched_queries(count=96, seed=7, lo=4.0, hi=9.3)
    vals, valid, _ = bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)
    for q, (n, P) in enumerate(zip(ns, Ps)):
        assert (vals[q], valid[q]) == plan.bits(n, P), (q, n, P)
        if n < 2 * 10**6:
            assert (vals[q], valid[q]) == oracle.c_bits(n, P, 64), (q, n, P)


def test_large_queries_in_a_batch_match_oracle(bbp, plan):
    """Queries of n = 1e7 .. 6e7 (moduli up to 2^29.2: both one-limb paths) among
    small ones, each checked against the oracle in full."""
    ns, Ps = workloads.batched_queries(count=24, seed=19, lo=3.0, hi=6.0)
    big = [10**7 + 1, 23_456_789, 41_234_567, 59_999_999]
    ns += big
    Ps += [256, 64, 128, 256]
    vals, valid, _ = bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)
    for q, (n, P) in enumerate(zip(ns, Ps)):
        assert (vals[q], valid[q]) == oracle.c_bits(n, P, 64), (q, n, P)


def test_batch_against_paper_rows(bbp, plan, pins):
    names = ["suppressed_m9", "suppressed_m10", "worked_example"]
    ns = [pins[nm]["n"] for nm in names]
    Ps = [pins[nm]["bits"] for nm in names]
    vals, valid, _ = bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)
    for nm, v, ok in zip(names, vals, valid):
        pin = pins[nm]
        ref = int(pin["hex"], 16) >> (4 * len(pin["hex"]) - pin["bits"])
        assert ok >= pin["bits"] - 32
        assert v >> (pin["bits"] - ok) == ref >> (pin["bits"] - ok)


def test_repeated_batches_replay_the_graph(bbp, plan):
    ns, Ps = workloads.batched_queries(count=64, seed=11, lo=3.0, hi=7.0)
    first = bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)[:2]
    for _ in range(3):
        assert bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)[:2] == first
    # a different batch of the same shape, then the first again
    ns2, Ps2 = workloads.batched_queries(count=64, seed=12, lo=3.0, hi=7.0)
    second = bbp.bbp_bits_batch(plan.handle, 0, ns2, Ps2)[:2]
    for q, (n, P) in enumerate(zip(ns2, Ps2)):
        assert (second[0][q], second[1][q]) == oracle.c_bits(n, P, 64)
    assert bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)[:2] == first


def test_bbp_formula_batch(bbp, plan):
    ns, Ps = workloads.batched_queries(count=40, seed=13, lo=1.0, hi=5.0)
    vals, valid, _ = bbp.bbp_bits_batch(plan.handle, 1, ns, Ps)
    for q, (n, P) in enumerate(zip(ns, Ps)):
        assert (vals[q], valid[q]) == oracle.c_bits(n, P, 64, "bbp")


def test_batch_errors(bbp, plan):
    with pytest.raises(bbp.BBPError):
        bbp.bbp_bits_batch(plan.handle, 0, [0], [64])
    with pytest.raises(bbp.BBPError):
        bbp.bbp_bits_batch(plan.handle, 0, [10], [5000])
    assert bbp.bbp_bits_batch(plan.handle, 0, [], []) == ([], [], [])
