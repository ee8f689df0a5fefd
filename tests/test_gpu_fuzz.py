"""Random partial sums over the whole supported range of positions (moduli below
2^60) on both formulas against the oracle, and the range limit itself."""

import random

import pytest

import oracle
from oracle import bbp_oracle as o1

pytestmark = pytest.mark.gpu


def test_random_ranges_up_to_1e18():
    import paper_1008_3171_gb300 as bbp

    rng = random.Random(29)
    plans = {G: bbp.Plan(device=0, guard_bits=G) for G in (32, 64)}
    try:
        for trial in range(60):
            formula = rng.choice([0, 1])
            f = o1.FORMULAS[formula]
            n = int(10 ** rng.uniform(0, 18.06)) + 1
            P = rng.choice([1, 7, 32, 64, 96, 200, 256, 500])
            G = rng.choice([32, 64])
            W = o1.working_bits(P, G)
            j = rng.randrange(len(f.series))
            s = f.series[j]
            he = o1.head_end(f, s, n - 1)
            ne = o1.natural_end(f, s, n - 1, W)
            if s.a * (ne - 1) + s.b >= 1 << 60:
                continue
            kb = rng.randrange(0, ne + 1)
            ke = kb + rng.randrange(0, 4000) if rng.random() < 0.8 or ne - kb > 4000 else None
            got = plans[G].partial_sum(formula, j, kb, ke, n, P)
            want = oracle.c_partial_sum(formula, j, kb, ke, n, P, G)
            assert got == want, (formula, n, P, G, j, kb, ke, he)
    finally:
        for p in plans.values():
            p.close()


def test_range_limit():
    import paper_1008_3171_gb300 as bbp

    plan = bbp.Plan(device=0, guard_bits=64)
    try:
        # the largest series modulus is about n; 2^60 is the limit of the 64-bit path
        n_ok = (1 << 60) - (1 << 20)
        for j, kb in ((0, 10**17), (4, 1), (5, 2 * 10**17)):      # sampled ranges near the top
            got = plan.partial_sum(0, j, kb, kb + 300, n_ok, 64)
            assert got == oracle.c_partial_sum(0, j, kb, kb + 300, n_ok, 64, 64)
        with pytest.raises(bbp.BBPError) as e:
            plan.bits(1 << 60, 64)
        assert e.value.status == bbp.BBP_ERANGE
    finally:
        plan.close()
