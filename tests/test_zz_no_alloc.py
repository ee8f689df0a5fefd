"""The no-allocation partial sum (bbp_partial_sum_noalloc) against the oracle and
against the plan-based entry point (bbp_partial_sum_async), through the C ABI.

The no-allocation entry point serves callers that may not allocate device memory
once running; it keeps its accumulators in a fixed array inside the library that
every call reuses.  So it is called twice in a row per case: the second call must
not see anything left over from the first, and must leave the device's free memory
unchanged.  The cases cross every modulus-path boundary the entry point splits its
launches at (moduli of 2^29, 2^31 and 2^46).  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""

import pytest

import oracle

pytestmark = pytest.mark.gpu

CASES = [
    # (formula, series, k_begin, k_end, n, P, guard bits)
    (0, 0, 0, None, 10**6, 64, 32),
    (0, 3, 12_345, 400_000, 10**9 + 1, 256, 64),
    (1, 2, 0, None, 99_991, 96, 64),
    (0, 5, 10**9, 10**9 + 30_000, 10**12, 256, 64),
    (0, 6, 0, None, 1, 1000, 64),
    # moduli crossing 2^29 (series 10k + 1) and 2^31 (series 4k + 3)
    (0, 0, 53_687_091 - 20_000, 53_687_091 + 20_000, 10**12, 256, 64),
    (0, 6, 536_870_911 - 20_000, 536_870_911 + 20_000, 10**12, 128, 64),
    # moduli crossing 2^46 (series 10k + 9): the three- and four-word two-limb paths
    (0, 4, 7_036_874_417_765 - 15_000, 7_036_874_417_765 + 15_000, 10**16, 256, 64),
]


def test_noalloc_matches_oracle_and_plan_entry_point_twice_in_a_row():
    import torch

    import paper_1008_3171_gb300 as bbp

    stream = torch.cuda.current_stream().cuda_stream
    plans = {G: bbp.Plan(device=0, guard_bits=G) for G in (32, 64)}
    try:
        for formula, j, kb, ke, n, P, G in CASES:
            W = plans[G].working_bits(P)
            want = oracle.c_partial_sum(formula, j, kb, ke, n, P, G)
            ref = torch.zeros(W // 32, dtype=torch.int32, device="cuda")
            bbp.bbp_partial_sum_async(plans[G].handle, formula, j, kb, ke, n, P, ref.data_ptr(), stream)
            outs = [torch.full((W // 32,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
            torch.cuda.synchronize()
            for i, got in enumerate(outs):
                free_before = torch.cuda.mem_get_info()[0]
                bbp.bbp_partial_sum_noalloc(formula, j, kb, ke, n, P, G, got.data_ptr(), stream)
                torch.cuda.synchronize()
                if i == 1:   # after the first call on the device has looked up the scratch address
                    assert torch.cuda.mem_get_info()[0] == free_before, "the entry point allocated"
                assert torch.equal(got, ref), (formula, j, kb, ke, n, P, G)
                limbs = [int(v) & 0xFFFFFFFF for v in got.tolist()]
                assert sum(v << (32 * i) for i, v in enumerate(limbs)) == want, (formula, j, kb, ke, n, P, G)
    finally:
        for p in plans.values():
            p.close()


def test_noalloc_rejects_precision_beyond_its_scratch():
    import torch

    import paper_1008_3171_gb300 as bbp

    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(bbp.BBPError) as e:
        bbp.bbp_partial_sum_noalloc(0, 0, 0, None, 1000, 1280, 64, out.data_ptr(), None)
    assert e.value.status == bbp.BBP_ESCRATCH
