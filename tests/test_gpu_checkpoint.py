"""Checkpoint / resume of a long query (the paper persists partial sums so a run
can be killed and resumed, Sec. 4): the carry-save accumulators after some
shards are the checkpoint; a new plan restores them, adds the remaining shards
and finalizes, and the bits equal the oracle's (n = 1e9 + 1: the paper's Table 2
row for that position, whose first 256 bits the oracle is pinned to)."""

import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,P,shards,stop", [(10**9 + 1, 256, 8, 3), (10**6, 64, 5, 0), (123_457, 1000, 3, 2)])
def test_resume_from_host_checkpoint(pins, n, P, shards, stop):
    import torch

    import paper_1008_3171_gb300 as bbp

    stream = torch.cuda.current_stream().cuda_stream
    first = bbp.Plan(device=0, guard_bits=64)
    W = first.working_bits(P)
    L = W // 32
    slots = torch.zeros(L, dtype=torch.int64, device="cuda")
    for s in range(stop):
        bbp.bbp_accumulate_async(first.handle, 0, n, P, s, shards, slots.data_ptr(), stream)
    torch.cuda.synchronize()
    checkpoint = slots.cpu().tolist()            # persisted partial sums
    first.close()
    del slots

    second = bbp.Plan(device=0, guard_bits=64)
    try:
        slots = torch.tensor(checkpoint, dtype=torch.int64, device="cuda")
        for s in range(stop, shards):
            bbp.bbp_accumulate_async(second.handle, 0, n, P, s, shards, slots.data_ptr(), stream)
        out = torch.zeros((P + 7) // 8, dtype=torch.uint8, device="cuda")
        valid = torch.zeros(1, dtype=torch.int32, device="cuda")
        bbp.bbp_finalize_async(second.handle, 0, n, P, slots.data_ptr(), out.data_ptr(), valid.data_ptr(), 0, stream)
        torch.cuda.synchronize()
        raw = bytes(out.tolist())
        got = int.from_bytes(raw, "big") >> (8 * len(raw) - P)
        ok = int(valid.item())
        if n == 10**9 + 1:
            pin = pins["suppressed_m9"]
            ref = int(pin["hex"], 16) >> (4 * len(pin["hex"]) - pin["bits"])
            assert ok == P and got == ref >> (pin["bits"] - P)
        else:
            assert (got, ok) == oracle.c_bits(n, P, 64)
        assert (got, ok) == second.bits(n, P)
    finally:
        second.close()
