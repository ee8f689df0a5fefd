"""The device finalize (carry propagation, guard-bit certification, MSB-first
bytes) on constructed sums placed exactly on the certification boundaries, against
the oracle's rule: the top b bits of S are certified iff
B <= S mod 2^(W-b) <= 2^(W-b) - B, with B = N + J + 1 (Eq. 8 read for truncation)."""

import random

import pytest

from oracle import bbp_oracle as o1

pytestmark = pytest.mark.gpu


def finalize(bbp, plan, n, P, S, W, carry_save=False):
    import torch

    L = W // 32
    limbs = [(S >> (32 * i)) & 0xFFFFFFFF for i in range(L)]
    if carry_save:  # spread the value over the 64-bit slots: slot i += 2^32, slot i+1 -= 1
        for i in range(L - 1):
            if limbs[i + 1] > 0:
                limbs[i] += 1 << 32
                limbs[i + 1] -= 1
    slots = torch.tensor(limbs, dtype=torch.int64, device="cuda")
    out = torch.zeros((P + 7) // 8, dtype=torch.uint8, device="cuda")
    valid = torch.zeros(1, dtype=torch.int32, device="cuda")
    raw = torch.zeros(L, dtype=torch.int32, device="cuda")
    bbp.bbp_finalize_async(plan.handle, 0, n, P, slots.data_ptr(), out.data_ptr(), valid.data_ptr(),
                           raw.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got_S = sum((int(v) & 0xFFFFFFFF) << (32 * i) for i, v in enumerate(raw.tolist()))
    return bytes(out.tolist()), int(valid.item()), got_S


def test_certification_boundaries():
    import paper_1008_3171_gb300 as bbp

    rng = random.Random(23)
    for G in (32, 64):
        plan = bbp.Plan(device=0, guard_bits=G)
        try:
            for n, P in ((1000, 64), (10**6 + 3, 100), (54321, 1), (10**9, 256), (77, 33)):
                W = o1.working_bits(P, G)
                N = sum(o1.natural_end(o1.BELLARD, s, n - 1, W) for s in o1.BELLARD.series)
                B = o1.error_bound(o1.BELLARD, N)
                cases = []
                for b in (P, P - 1, max(P // 2, 0), 0):
                    low = W - b
                    top = rng.getrandbits(W) >> low << low
                    for g in (B - 1, B, B + 1, (1 << low) - B - 1, (1 << low) - B, (1 << low) - B + 1, 0,
                              (1 << low) - 1, rng.getrandbits(low)):
                        if 0 <= g < (1 << low):
                            cases.append(top | g)
                for S in cases:
                    for cs in (False, True):
                        raw, valid, got_S = finalize(bbp, plan, n, P, S, W, cs)
                        assert got_S == S
                        assert valid == o1.certified_bits(S, W, P, B), (n, P, G, hex(S))
                        assert raw == o1.to_bytes_msb_first(S >> (W - P), P)
        finally:
            plan.close()
