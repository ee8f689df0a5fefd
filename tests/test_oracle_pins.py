"""Pins for the oracle (CPU only).

The oracle is checked against things other than itself: bits the paper prints,
pi bits from Machin's formula (an unrelated method), the other BBP-type formula
(Eq. 1 against Eq. 2), the paper's n / n-4 overlap practice (Sec. 2, Sec. 3.1),
and the error bound (Eq. 8 read for truncation).  A last group plants mistakes in
copies of the oracle and checks that one of these pins catches each of them.
"""

import dataclasses
import json
import os
import random

import pytest

import oracle
from oracle import bbp_oracle as o1
from oracle import machin


def hex_value(pin):
    """The pin's P bits as an integer (the hex may carry padding bits below P)."""
    h = pin["hex"]
    return int(h, 16) >> (4 * len(h) - pin["bits"])


# ---------------------------------------------------------------- paper values

@pytest.mark.parametrize("formula", ["bellard", "bbp"])
@pytest.mark.parametrize("name", ["worked_example", "footnote_prefix"])
def test_worked_example(pins, name, formula):
    pin = pins[name]
    for G in (32, 64):
        v, valid = o1.bits(pin["n"], pin["bits"], G, formula)
        assert valid == pin["bits"]
        assert v == hex_value(pin)
        assert oracle.c_bits(pin["n"], pin["bits"], G, formula) == (v, valid)


def test_paper_rows_consistent_with_each_other(pins):
    # Table 2's m = 15 row, read from bit 10^15 + 53, is the true-bit listing of Sec. 3.1.
    row = pins["table2_m15"]
    fp = pins["fp64_example_true_bits"]
    offset = fp["n"] - row["n"]
    assert offset == 52
    assert (hex_value(row) >> (row["bits"] - offset - fp["bits"])) & ((1 << fp["bits"]) - 1) == hex_value(fp)
    # the abstract's statement: the bit at position 2e15 (fourth bit of Table 1) is 0
    t1 = pins["table1_2e15"]
    assert (hex_value(t1) >> (t1["bits"] - 4)) & 1 == 0


# ---------------------------------------------------------------- Machin pins

MACHIN_F = 10**5 + 512          # one Machin evaluation serves every window below 1e5


def machin_sample(seed, count, n_max):
    rng = random.Random(seed)
    ns = [1, 2, 3, 4, 5, 8, 9, 31, 32, 33, 100, n_max]
    ns += [rng.randrange(1, n_max + 1) for _ in range(count)]
    return ns


@pytest.mark.parametrize("formula", ["bellard", "bbp"])
def test_o1_matches_machin_up_to_1e5(formula):
    for n in machin_sample(11, 25, 10**5):
        for P, G in ((8, 32), (64, 32), (200, 64)):
            v, valid = o1.bits(n, P, G, formula)
            assert valid >= P - 8, (n, P, G, valid)
            want = machin.pi_bits(n, P, F=MACHIN_F)
            assert v >> (P - valid) == want >> (P - valid), (n, P, G)


def test_o2_matches_machin_at_1e6():
    """Machin windows near n = 1e6, stored by tests/golden/make_machin_golden.py."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "machin_bits.json")) as fh:
        windows = json.load(fh)["windows"]
    for w in windows:
        ref = int(w["hex"], 16)
        for P, G in ((64, 32), (128, 64), (256, 64)):
            v, valid = oracle.c_bits(w["n"], P, G, "bellard")
            assert valid == P
            assert v == ref >> (w["bits"] - P), (w["n"], P, G)


def _fractional_fixed(n, W):
    """floor({2^(n-1) pi} 2^W) from Machin, and Machin's error in those units (< 1)."""
    extra = 64
    F = MACHIN_F
    assert F >= n - 1 + W + extra
    Y, E = machin.pi_fixed(F)
    Y >>= F - (n - 1 + W + extra)
    assert E < (1 << (extra - 2))
    return (Y >> extra) & ((1 << W) - 1)


@pytest.mark.parametrize("formula", ["bellard", "bbp"])
def test_accumulator_within_error_bound(formula):
    """The whole W-bit accumulator, not only its top bits, is within B units of
    {2^d pi} 2^W: this catches a dropped or mis-signed term anywhere in the sum."""
    f = o1.FORMULAS[formula]
    for n in (1, 2, 7, 64, 1000, 4097, 54321):
        for P, G in ((32, 32), (96, 64)):
            W = o1.working_bits(P, G)
            S, N = o1.accumulate(f, n, P, G)
            X = _fractional_fixed(n, W)
            diff = (S - X) % (1 << W)
            dist = min(diff, (1 << W) - diff)
            assert dist <= o1.error_bound(f, N), (n, P, G, dist, N)


# ---------------------------------------------------------------- other formula / overlap

def test_bbp_formula_agrees_with_bellard_small():
    for n in machin_sample(5, 20, 20000):
        a, va = o1.bits(n, 64, 32, "bellard")
        b, vb = o1.bits(n, 64, 32, "bbp")
        v = min(va, vb)
        assert a >> (64 - v) == b >> (64 - v)


@pytest.mark.parametrize("n", [10**6 + 7, 10**7, 10**8])
def test_bbp_formula_agrees_with_bellard_large(n):
    a, va = oracle.c_bits(n, 64, 32, "bellard")
    b, vb = oracle.c_bits(n, 64, 32, "bbp")
    assert va >= 56 and vb >= 56
    v = min(va, vb)
    assert a >> (64 - v) == b >> (64 - v)


@pytest.mark.parametrize("n", [5, 1001, 123457, 10**7 + 1])
def test_overlapping_windows(n):
    """Sec. 2 / Sec. 3.1: runs at n and n - 4 must agree where they overlap."""
    P = 96
    hi, vh = oracle.c_bits(n, P, 64)
    lo, vl = oracle.c_bits(n - 4, P, 64)
    overlap = min(vh, vl - 4)
    assert overlap >= P - 12
    assert (lo >> (P - 4 - overlap)) & ((1 << overlap) - 1) == hi >> (P - overlap)


# ---------------------------------------------------------------- O1 == O2

def test_o1_o2_partial_sums_bit_exact():
    rng = random.Random(3)
    cases = [(1, 8, 32), (2, 64, 32), (9, 8, 64), (12345, 70, 32), (99991, 256, 64)]
    for n, P, G in cases:
        for fname, f in (("bellard", o1.BELLARD), ("bbp", o1.BBP)):
            W = o1.working_bits(P, G)
            for j in range(len(f.series)):
                end = o1.natural_end(f, f.series[j], n - 1, W)
                assert oracle.c_natural_end(fname, j, n, P, G) == end
                ranges = [(0, None), (0, 1), (end - 1, end + 5), (end, None), (3, 3)]
                for _ in range(4):
                    a = rng.randrange(0, end + 2)
                    ranges.append((a, a + rng.randrange(0, 50)))
                for kb, ke in ranges:
                    want = o1.partial_sum(f, j, kb, ke, n, P, G)
                    got = oracle.c_partial_sum(fname, j, kb, ke, n, P, G, threads=3)
                    assert got == want, (fname, n, P, G, j, kb, ke)


def test_certified_bits_rule():
    W, P, B = 96, 64, 10
    base = 0xABCDEF << (W - 24)
    # low 32 bits well inside [B, 2^32 - B]: all P bits certified
    assert o1.certified_bits(base | 1000, W, P, B) == P
    # low bits just below B: the last certified prefix ends where a 1 bit absorbs it
    assert o1.certified_bits(base | (B - 1), W, P, B) < P
    assert o1.certified_bits(base | B, W, P, B) == P
    top = (1 << (W - P)) - B
    assert o1.certified_bits(base | top, W, P, B) == P
    assert o1.certified_bits(base | (top + 1), W, P, B) < P


# ---------------------------------------------------------------- planted mistakes

def _mutants():
    f = o1.BELLARD
    out = []
    for j, s in enumerate(f.series):
        flipped = list(f.series)
        flipped[j] = dataclasses.replace(s, sign=-s.sign)
        out.append((f"sign{j}", dataclasses.replace(f, series=tuple(flipped))))
        shifted = list(f.series)
        shifted[j] = dataclasses.replace(s, c=s.c + 1)
        out.append((f"c{j}", dataclasses.replace(f, series=tuple(shifted))))
        dropped = tuple(x for i, x in enumerate(f.series) if i != j)
        out.append((f"drop{j}", dataclasses.replace(f, series=dropped)))
    swapped = list(f.series)
    swapped[1] = dataclasses.replace(swapped[1], a=swapped[1].b, b=swapped[1].a)
    out.append(("transposed_a_b", dataclasses.replace(f, series=tuple(swapped))))
    out.append(("no_alternation", dataclasses.replace(f, alternating=False)))
    out.append(("step", dataclasses.replace(f, step=9)))
    return out


@pytest.mark.parametrize("label,mutant", _mutants(), ids=[m[0] for m in _mutants()])
def test_machin_pin_catches_formula_mistakes(label, mutant):
    caught = False
    for n in (1, 17, 333, 5000):
        v, valid = o1.bits(n, 64, 32, mutant)
        if v != machin.pi_bits(n, 64, F=MACHIN_F):
            caught = True
            break
    assert caught, label


def test_bound_pin_catches_code_mistakes(monkeypatch):
    """Plant mistakes in the term routine itself: each must break the error-bound pin."""
    real = o1.term

    def dropped_last_head(f, s, d, k, W):
        return 0 if k == o1.head_end(f, s, d) - 1 else real(f, s, d, k, W)

    def off_by_one_exponent(f, s, d, k, W):
        return real(f, s, d + 1, k, W) if k == 3 else real(f, s, d, k, W)

    def rounded_up(f, s, d, k, W):
        return real(f, s, d, k, W) + (1 << 40)

    for planted in (dropped_last_head, off_by_one_exponent, rounded_up):
        monkeypatch.setattr(o1, "term", planted)
        with pytest.raises(AssertionError):
            test_accumulator_within_error_bound("bellard")
        monkeypatch.setattr(o1, "term", real)
