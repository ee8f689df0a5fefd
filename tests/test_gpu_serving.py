"""Serving (bbp_submit / bbp_poll): continuous batching returns, for every query,
exactly the bits the query gets alone -- while other queries (a long one and many
short ones arriving over time) share the GPU with it -- and, for every query the
oracle can run here (n < 4e7, including two of n > 1e7), exactly the oracle's bits."""

import random
import time

import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbp():
    import paper_1008_3171_gb300 as m

    return m


def wait_all(bbp, plan, tickets, timeout_s=180.0):
    done = {}
    t_end = time.time() + timeout_s
    while len(done) < len(tickets) and time.time() < t_end:
        for t, (n, P) in tickets.items():
            if t in done:
                continue
            r = bbp.bbp_poll(plan.handle, t, P)
            if r is not None:
                done[t] = r
        time.sleep(0.002)
    assert len(done) == len(tickets), "serving did not finish in time"
    return done


def test_results_in_the_mix_equal_results_alone(bbp):
    plan = bbp.Plan(device=0, guard_bits=64, max_slots=64)
    try:
        tickets = {}
        long_n, long_P = 10**10 + 1, 256
        tickets[bbp.bbp_submit(plan.handle, long_n, long_P)] = (long_n, long_P)
        for n_big, P_big in ((12_345_679, 256), (33_333_331, 64)):   # checked against the oracle in full
            tickets[bbp.bbp_submit(plan.handle, n_big, P_big)] = (n_big, P_big)
        rng = random.Random(21)
        arrivals = workloads.serving_arrivals(40, rate_per_s=200.0, seed=21, lo=2.0, hi=8.0)
        t0 = time.time()
        for t_arr, n, P in arrivals:
            delay = t0 + t_arr - time.time()
            if delay > 0:
                time.sleep(delay)
            t = bbp.bbp_submit(plan.handle, n, P)
            assert t is not None
            tickets[t] = (n, P)
        done = wait_all(bbp, plan, tickets)
        info = bbp.bbp_serve_stats(plan.handle)
        assert info["iterations"] > 1 and info["pending"] == 0 and info["active"] == 0
        alone = bbp.Plan(device=0, guard_bits=64)
        try:
            for t, (n, P) in tickets.items():
                assert done[t] == alone.bits(n, P), (n, P)
                if n < 4 * 10**7:
                    assert done[t] == oracle.c_bits(n, P, 64), (n, P)
        finally:
            alone.close()
        assert rng is not None
    finally:
        plan.close()


def test_admission_is_bounded_by_the_slot_pool(bbp):
    plan = bbp.Plan(device=0, guard_bits=64, max_slots=1)
    try:
        first = bbp.bbp_submit(plan.handle, 10**11 + 1, 64)
        t_end = time.time() + 10
        while bbp.bbp_serve_stats(plan.handle)["active"] != 1 and time.time() < t_end:
            time.sleep(0.001)
        second = bbp.bbp_submit(plan.handle, 1000, 64)   # waits for the one slot
        assert second is not None
        assert bbp.bbp_submit(plan.handle, 1001, 64) is None  # the queue is as long as the pool
        done = wait_all(bbp, plan, {first: (10**11 + 1, 64), second: (1000, 64)})
        assert done[second] == oracle.c_bits(1000, 64, 64)
    finally:
        plan.close()


def test_tickets(bbp):
    plan = bbp.Plan(device=0, guard_bits=32)
    try:
        with pytest.raises(bbp.BBPError) as e:
            bbp.bbp_poll(plan.handle, 12345, 8)
        assert e.value.status == bbp.BBP_ENOTFOUND
        t = bbp.bbp_submit(plan.handle, 9, 8)
        done = wait_all(bbp, plan, {t: (9, 8)})
        assert done[t] == (0x3F, 8)
        with pytest.raises(bbp.BBPError) as e:
            bbp.bbp_poll(plan.handle, t, 8)
        assert e.value.status == bbp.BBP_ENOTFOUND
        with pytest.raises(bbp.BBPError):
            bbp.bbp_submit(plan.handle, 0, 8)
    finally:
        plan.close()


def test_query_too_large_for_the_queue_limbs_is_refused(bbp, tmp_path):
    """A query needing 2^32 - 2^24 or more warp tiles could overflow its 64-bit
    carry-save limbs in the queue kernels: bbp_submit and bbp_bits_batch refuse it
    with BBP_ERANGE while planning, before any launch.  With run = 2 and one term
    pair per thread a tile is 64 terms, so n = 5e11 (3.5e11 head terms, 5.5e9 tiles)
    is past the limit and n = 1e11 (1.1e9 tiles) is not."""
    import json

    table = tmp_path / "tune.json"
    table.write_text(json.dumps({"run": 2, "streams": 1}))
    plan = bbp.Plan(device=0, guard_bits=64, tune_table=str(table))
    try:
        with pytest.raises(bbp.BBPError) as e:
            bbp.bbp_submit(plan.handle, 5 * 10**11, 64)
        assert e.value.status == bbp.BBP_ERANGE
        with pytest.raises(bbp.BBPError) as e:
            bbp.bbp_bits_batch(plan.handle, 0, [1000, 5 * 10**11], [64, 64])
        assert e.value.status == bbp.BBP_ERANGE
        t = bbp.bbp_submit(plan.handle, 10**6, 64)      # a small query is still served
        assert t is not None
        assert wait_all(bbp, plan, {t: (10**6, 64)})[t] == oracle.c_bits(10**6, 64, 64)
    finally:
        plan.close()
