"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit for bit.

The accumulator is exact integer arithmetic modulo 2^W, so the tolerance is zero:
every partial sum, raw accumulator and output bit must equal the oracle's.  Cases
cover several tiles and ragged tails, the four modulus paths and every boundary
between them, k = 0 (m = 1), the head/tail boundary, the tail end, both formulas,
and sampled ranges at the full configuration sizes (n = 1e9, 1e12, 1e13).
"""

import json
import os
import random

import pytest

import oracle
from oracle import bbp_oracle as o1

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bbp():
    import paper_1008_3171_gb300 as m

    return m


@pytest.fixture(scope="module")
def plan64(bbp):
    p = bbp.Plan(device=0, guard_bits=64)
    yield p
    p.close()


@pytest.fixture(scope="module")
def plan32(bbp):
    p = bbp.Plan(device=0, guard_bits=32)
    yield p
    p.close()


def plans(plan32, plan64):
    return ((32, plan32), (64, plan64))


def hexpin(pin):
    return int(pin["hex"], 16) >> (4 * len(pin["hex"]) - pin["bits"])


# ---------------------------------------------------------------- pins

@pytest.mark.parametrize("formula", [0, 1])
def test_worked_example(plan32, plan64, pins, formula):
    for G, p in plans(plan32, plan64):
        assert p.bits(9, 8, formula) == (0x3F, 8)
        assert p.bits(1, 16, formula) == (0x243F, 16)


def test_config1_against_machin(plan32):
    """n = 1e6, P = 64 + 32 guard bits: checked against Machin-series pi bits."""
    with open(os.path.join(HERE, "golden", "machin_bits.json")) as fh:
        windows = {w["n"]: int(w["hex"], 16) for w in json.load(fh)["windows"]}
    v, valid = plan32.bits(10**6, 64)
    assert valid == 64
    assert v == windows[10**6] >> (256 - 64)


@pytest.mark.parametrize("name", ["suppressed_m9", "suppressed_m10", "suppressed_m11"])
def test_suppressed_table_rows(plan64, pins, name):
    pin = pins[name]
    v, valid = plan64.bits(pin["n"], pin["bits"])
    assert valid >= pin["bits"] - 32
    assert v >> (pin["bits"] - valid) == hexpin(pin) >> (pin["bits"] - valid)


def test_config3_headline_against_paper_row(plan64, pins):
    """n = 1e12, P = 256, G = 64.  Table 2's suppressed m = 12 row starts one bit later."""
    v, valid = plan64.bits(10**12, 256)
    assert valid == 256
    row = pins["suppressed_m12"]
    assert v & ((1 << 255) - 1) == hexpin(row) >> (row["bits"] - 255)


def test_config2_against_paper_row(plan64, pins):
    v, valid = plan64.bits(10**9, 128)
    assert valid == 128
    row = pins["suppressed_m9"]
    assert v & ((1 << 127) - 1) == hexpin(row) >> (row["bits"] - 127)


# ---------------------------------------------------------------- raw partial sums

def _ranges(rng, he, ne):
    rs = [(0, None), (0, 1), (0, 2), (1, 4), (max(0, he - 3), he + 3), (he, None), (he, ne),
          (ne - 1, ne + 10), (ne + 5, None), (3, 3)]
    for _ in range(4):
        a = rng.randrange(0, ne + 1)
        rs.append((a, a + rng.randrange(0, 3000)))
    return rs


@pytest.mark.parametrize("formula", [0, 1])
def test_partial_sums_small_n(plan32, plan64, formula):
    rng = random.Random(7 + formula)
    f = o1.FORMULAS[formula]
    for n in (1, 2, 3, 5, 9, 17, 100, 1001, 12345, 99991):
        for P in (1, 8, 64, 96, 256):
            for G, p in plans(plan32, plan64):
                W = o1.working_bits(P, G)
                for j, s in enumerate(f.series):
                    he = o1.head_end(f, s, n - 1)
                    ne = o1.natural_end(f, s, n - 1, W)
                    for kb, ke in _ranges(rng, he, ne):
                        got = p.partial_sum(formula, j, kb, ke, n, P)
                        want = oracle.c_partial_sum(formula, j, kb, ke, n, P, G, threads=4)
                        assert got == want, (formula, n, P, G, j, kb, ke)


def test_partial_sums_many_tiles(plan64):
    """Ranges spanning many warp tiles and CTAs with ragged ends, on the one-limb paths
    (n = 1e9 + 1: moduli below 2^30)."""
    rng = random.Random(11)
    n, P, G = 10**9 + 1, 128, 64
    for j in range(7):
        for kb, cnt in ((1, 200_000), (53_687_000, 150_001), (rng.randrange(1, 9 * 10**7), 123_457)):
            got = plan64.partial_sum(0, j, kb, kb + cnt, n, P)
            want = oracle.c_partial_sum(0, j, kb, kb + cnt, n, P, G)
            assert got == want, (j, kb, cnt)


@pytest.mark.parametrize("n", [10**12, 10**13, 2 * 10**15 - 3])
def test_partial_sums_full_size_sampled(plan64, n):
    """Sampled k-ranges of the full-size queries, in the launch configuration the bench uses."""
    rng = random.Random(n % 1000003)
    P, G = 256, 64
    f = o1.BELLARD
    W = o1.working_bits(P, G)
    for j, s in enumerate(f.series):
        he = o1.head_end(f, s, n - 1)
        ne = o1.natural_end(f, s, n - 1, W)
        starts = [1, he - 4000, rng.randrange(1, he - 5000), rng.randrange(1, he - 5000)]
        # the one-limb path boundaries (m crosses 2^29 and 2^31)
        starts.append(max(1, ((1 << 29) - s.b) // s.a - 1500))
        starts.append(max(1, ((1 << 31) - s.b) // s.a - 1500))
        for kb in starts:
            ke = kb + 3001
            got = plan64.partial_sum(0, j, kb, ke, n, P)
            want = oracle.c_partial_sum(0, j, kb, ke, n, P, G)
            assert got == want, (n, j, kb)
        got = plan64.partial_sum(0, j, he - 10, None, n, P)
        assert got == oracle.c_partial_sum(0, j, he - 10, None, n, P, G)
        assert ne > he


@pytest.mark.parametrize("formula", [0, 1])
@pytest.mark.parametrize("bits", [29, 30, 31, 32, 46, 47])
def test_modulus_path_boundaries(plan64, bits, formula):
    """k-ranges whose moduli cross 2^bits, on every series: the one-limb lazy and
    reduced paths meet at 2^29 (bitlen 30), the reduced one-limb path and the
    three-word two-limb path at 2^31 (bitlen 32), the three- and four-word two-limb
    paths at 2^46 (bitlen 47); 2^30 and 2^32 cross inside a path.  n = 2e15 - 3
    reaches all of them in the head, for Eq. 2 and Eq. 1."""
    n, P, G = 2 * 10**15 - 3, 256, 64
    f = o1.FORMULAS[formula]
    for j, s in enumerate(f.series):
        k_cross = ((1 << (bits - 1)) - s.b) // s.a
        for kb, cnt in ((max(1, k_cross - 1500), 3001), (max(1, k_cross - 70_000), 140_001)):
            got = plan64.partial_sum(formula, j, kb, kb + cnt, n, P)
            want = oracle.c_partial_sum(formula, j, kb, kb + cnt, n, P, G)
            assert got == want, (formula, bits, j, kb, cnt)


def test_raw_accumulator_matches_oracle(bbp, plan32, plan64):
    import torch

    rng = random.Random(3)
    for n in [1, 2, 9, 1000, 54321, 10**6] + [rng.randrange(1, 10**6) for _ in range(6)]:
        for P in (1, 31, 64, 100, 256):
            for G, p in plans(plan32, plan64):
                for formula in (0, 1):
                    W = o1.working_bits(P, G)
                    d_out = torch.zeros((P + 7) // 8, dtype=torch.uint8, device="cuda")
                    d_valid = torch.zeros(1, dtype=torch.int32, device="cuda")
                    d_limbs = torch.zeros(W // 32, dtype=torch.int32, device="cuda")
                    bbp.bbp_bits_async(p.handle, formula, n, P, d_out.data_ptr(), d_valid.data_ptr(),
                                       d_limbs.data_ptr(), torch.cuda.current_stream().cuda_stream)
                    torch.cuda.synchronize()
                    S, N = oracle.c_accumulate(formula, n, P, G)
                    got = sum((int(v) & 0xFFFFFFFF) << (32 * i) for i, v in enumerate(d_limbs.tolist()))
                    assert got == S, (n, P, G, formula)
                    f = o1.FORMULAS[formula]
                    valid = o1.certified_bits(S, W, P, o1.error_bound(f, N))
                    assert int(d_valid.item()) == valid
                    raw = bytes(d_out.tolist())
                    assert raw == o1.to_bytes_msb_first(S >> (W - P), P)


def test_bits_match_oracle(plan32, plan64):
    rng = random.Random(5)
    for n in [3, 77, 4096, 65537] + [rng.randrange(1, 2 * 10**6) for _ in range(5)]:
        for P in (8, 64, 100):
            for G, p in plans(plan32, plan64):
                assert p.bits(n, P) == oracle.c_bits(n, P, G), (n, P, G)


def test_bbp_formula_agrees_with_bellard_on_gpu(plan64):
    for n in (10**6 + 3, 10**8, 10**9 + 1):
        a, va = plan64.bits(n, 128, 0)
        b, vb = plan64.bits(n, 128, 1)
        v = min(va, vb)
        assert v >= 120
        assert a >> (128 - v) == b >> (128 - v)


def test_overlapping_windows_gpu(plan64):
    for n in (10**10 + 1, 10**11 + 1):
        hi, vh = plan64.bits(n, 256)
        lo, vl = plan64.bits(n - 4, 256)
        overlap = min(vh, vl - 4)
        assert overlap >= 240
        assert (lo >> (256 - 4 - overlap)) & ((1 << overlap) - 1) == hi >> (256 - overlap)


def test_repeatable(plan64):
    a = plan64.partial_sum(0, 3, 5, 2_000_005, 10**11, 256)
    b = plan64.partial_sum(0, 3, 5, 2_000_005, 10**11, 256)
    assert a == b


# ---------------------------------------------------------------- errors

def test_error_codes(bbp, plan64):
    h = plan64.handle
    bad = [
        lambda: bbp.bbp_partial_sum(h, 0, 7, 0, None, 100, 64),     # denominator out of range
        lambda: bbp.bbp_partial_sum(h, 1, 4, 0, None, 100, 64),
        lambda: bbp.bbp_partial_sum(h, 0, 0, 10, 5, 100, 64),       # k_begin > k_end
        lambda: bbp.bbp_partial_sum(h, 0, 0, 0, None, 0, 64),       # n = 0
        lambda: bbp.bbp_bits(h, 0, 64),
        lambda: bbp.bbp_bits(h, 10, 0),
        lambda: bbp.bbp_bits(h, 10, 5000),                          # W beyond 1280 bits
        lambda: bbp.bbp_bits_formula(h, 2, 10, 64),
    ]
    for fn in bad:
        with pytest.raises(bbp.BBPError) as e:
            fn()
        assert e.value.status == bbp.BBP_EINVAL
    with pytest.raises(bbp.BBPError) as e:
        bbp.bbp_bits(h, 1 << 61, 64)
    assert e.value.status == bbp.BBP_ERANGE


def test_strict_mode(bbp):
    p = bbp.Plan(device=0, guard_bits=32, strict=True)
    try:
        assert p.bits(9, 8) == (0x3F, 8)
    finally:
        p.close()


@pytest.mark.parametrize("P", [64, 96, 160, 288, 448, 512, 736, 1000, 1216])
def test_every_limb_class_matches_oracle(plan64, P):
    """W = roundup(P, 32) + 64 from 4 to 40 limbs: every compiled accumulator class
    (3, 4, 6, 10, 16, 24, 40 limbs), its lower and upper fill, on both modulus
    paths (a 64-bit-modulus slice of n = 1e12) and in whole queries."""
    assert plan64.bits(123_457, P) == oracle.c_bits(123_457, P, 64)
    assert plan64.bits(10**7 + 1, P) == oracle.c_bits(10**7 + 1, P, 64)
    for j in (0, 6):
        kb = 31 * 10**9 + 17
        got = plan64.partial_sum(0, j, kb, kb + 40_001, 10**12, P)
        assert got == oracle.c_partial_sum(0, j, kb, kb + 40_001, 10**12, P, 64), (P, j)


def test_imad_probe_kinds(bbp, plan64):
    """Every probe kind reports a positive issue rate, a full 32-bit product at most
    as fast as its low half; an unknown kind is refused."""
    rates = [plan64.imad_probe(k) for k in range(7)]
    assert all(r > 0 for r in rates)
    assert rates[5] <= rates[0] * 1.05 and rates[2] <= rates[0] * 1.05
    with pytest.raises(bbp.BBPError) as e:
        plan64.imad_probe(7)
    assert e.value.status == bbp.BBP_EINVAL


@pytest.mark.parametrize("P", [64, 1000])
@pytest.mark.parametrize("bits", [30, 32, 47])
def test_modulus_path_boundaries_small_and_large_accumulators(plan64, bits, P):
    """The path crossings (one-limb lazy/reduced, one-/two-limb, three-/four-word) with
    the smallest and the largest accumulator classes (4 and 40 limbs)."""
    n, G = 2 * 10**15 - 3, 64
    f = o1.BELLARD
    for j in (0, 5):
        s = f.series[j]
        kb = max(1, ((1 << (bits - 1)) - s.b) // s.a - 20_000)
        got = plan64.partial_sum(0, j, kb, kb + 40_001, n, P)
        want = oracle.c_partial_sum(0, j, kb, kb + 40_001, n, P, G)
        assert got == want, (bits, P, j)
