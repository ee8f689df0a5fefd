"""Host-side launch planning (bbp_explain, no GPU): for many positions, widths and
Montgomery crossovers, the ranges a query launches cover exactly the terms of
the definition, and every head range satisfies the bounds its kernel's
arithmetic needs.

Coverage is checked against the oracle's own series extents (Eq. 4 split, tail
end by truncation).  The bounds come from the Montgomery ladder the kernels run
(R = 2^64 on two limbs, 2^32 on one; REDC of T returns a value below 2m when
T < m R):
  * path 0 (one limb, lazy x < 2m): a squaring with the window's value s shifted
    in reduces x^2 2^s < 4 m^2 2^s, so 4 m 2^s < R for every s <= 2^window - 1;
  * path 3 (one limb, x < m after a conditional subtraction): m 2^s < R and
    m^2 2^s < 2^64;
  * path 1 (two limbs, three-word square): x < 2m with x^2 + 2^32 m < 2^96 keeps
    the first reduction step in two words, and that value shifted by s in three;
    the result (T 2^s + (u 2^s + u' 2^32) m) / 2^64 stays below 2m while
    4 m 2^s + 2^(32+s) < R;
  * path 2 (two limbs, four-word square): 4 m 2^s < R;
  * the first window starts from x = (R mod m) << w0 < m 2^w0 with w0 < 2^first,
    and the squaring after it (the general routine on the two-limb paths)
    carries a shift of at most one bit, so m 2^(2 w0 + 1) < R;
  * path 0 needs m < 2^29, path 3 2^29 <= m < 2^31, path 1 2^31 <= m < 2^46 at the
    default crossover, path 2 m < 2^60;
  * carrying R mod m along a run forms floor(R / m) * a in 64 bits.
"""

import importlib.util
import math
import os
import random

import pytest

from conftest import ROOT
from oracle import bbp_oracle as o1


@pytest.fixture(scope="module")
def bbp():
    spec = importlib.util.spec_from_file_location("_bbp_build", os.path.join(ROOT, "paper_1008_3171_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1008_3171_gb300 as m

    return m


def _positions():
    rng = random.Random(2024)
    ns = [1, 2, 3, 5, 9, 10, 11, 17, 100, 1001, 4096, 65537, 10**6, 10**9 + 1, 10**12, 10**13 + 1,
          10**14 + 1, 2 * 10**15 - 3, 10**16 + 7]
    ns += [int(10 ** rng.uniform(0, 16.5)) or 1 for _ in range(24)]
    return ns


CASES = [(f, n, P, G, wide)
         for f in (0, 1)
         for n in _positions()
         for P, G in ((1, 32), (64, 32), (256, 64), (1000, 64))
         for wide in (5, 17, 30, 32)]


def _check_plan(bbp, f, n, P, G, wide):
    ranges, terms = bbp.bbp_explain(f, n, P, G, wide)
    F = o1.FORMULAS[f]
    W = o1.working_bits(P, G)
    d = n - 1
    total = 0
    for j, s in enumerate(F.series):
        mine = [r for r in ranges if r["denominator"] == j]
        he = o1.head_end(F, s, d)
        ne = o1.natural_end(F, s, d, W)
        # heads first, then at most one tail range; contiguous, in k order
        k = 1 if (s.b == 1 and he > 0) else 0          # the m = 1 head term is 0 and is skipped
        seen_tail = False
        for r in mine:
            assert r["count"] > 0
            assert r["k_begin"] == k, (f, n, P, G, wide, j, r)
            k = r["k_begin"] + r["count"]
            if r["tail"]:
                assert not seen_tail and r["k_begin"] == he
                seen_tail = True
            else:
                assert not seen_tail and k <= he
                _check_head_bounds(s, r, wide, W, d, F)
        assert k == ne, (f, n, j, k, he, ne)            # ne >= he: the tail, if any, ends the series
        assert seen_tail == (ne > he)
        expected = ne - (1 if (s.b == 1 and he > 0) else 0)
        assert sum(r["count"] for r in mine) == expected
        total += expected
    assert terms == total


def _check_head_bounds(s, r, wide, W, d, F):
    k_last = r["k_begin"] + r["count"] - 1
    m_max = s.a * k_last + s.b
    m_min = s.a * r["k_begin"] + s.b
    assert m_min >= 3 and m_min % 2 == 1
    path, window, first = r["path"], r["window"], r["first"]
    two_limbs = path in (1, 2)
    R = 1 << (64 if two_limbs else 32)
    sh = (1 << window) - 1                                               # largest window shift
    if path == 0:
        assert m_max < 1 << 29 and m_max.bit_length() < wide
        assert 4 * m_max * (1 << sh) < R
    elif path == 3:
        assert m_min >= 1 << 29 and m_max < 1 << 31 and m_max.bit_length() < wide
        assert m_max * (1 << sh) < R and m_max * m_max * (1 << sh) < 1 << 64
    elif path == 1:
        assert m_max < 1 << 46 and m_min.bit_length() >= min(wide, 32)
        assert (2 * m_max) ** 2 + (1 << 32) * m_max < 1 << 96           # first step in two words
        assert ((2 * m_max) ** 2 // (1 << 32) + m_max) << sh < 1 << 96   # shifted: three words
        assert 4 * m_max * (1 << sh) + (1 << (32 + sh)) < R
    else:
        assert m_max < 1 << 60 and m_min.bit_length() >= 47
        assert 4 * m_max * (1 << sh) < R
    assert 1 <= window
    # R mod m is carried from k to k + 1 with q = floor(R / m): q * a must fit 64 bits
    assert (R // m_min) * s.a < 1 << 64
    fm = r["first_max"]
    assert fm >= (1 << first) - 1 and fm < (1 << (first + 1)) - 1 or first == 4
    for w0 in ((1 << first) - 1, fm):                                   # every first window; the largest
        assert m_max * (1 << (2 * w0 + 1)) < R                          # first squaring after the first window
        if two_limbs:
            assert m_max * (1 << w0) < 1 << 61                          # 2 x1 fits one word
    # every head term's exponent is >= 0, so the ladder exponent e + W >= W >= R's width
    e_last = d + s.c - F.step * k_last
    assert e_last >= 0 and e_last + W >= (64 if two_limbs else 32)
    assert r["imad"] > 0


@pytest.mark.parametrize("n", _positions())
def test_plan_covers_every_term_within_kernel_bounds(bbp, n):
    for f, n_, P, G, wide in CASES:
        if n_ == n:
            _check_plan(bbp, f, n, P, G, wide)


def test_default_headline_plan(bbp):
    """n = 1e12, P = 256, G = 64: 42 head launches (moduli from 3 to 2^40) and 7
    tail launches, 7e11 terms; the 64-bit ranges carry almost all of them."""
    ranges, terms = bbp.bbp_explain(0, 10**12, 256, 64, 32)
    heads = [r for r in ranges if not r["tail"]]
    assert len(ranges) - len(heads) == 7
    assert terms == 700_000_000_195
    wide = sum(r["count"] for r in heads if r["path"] > 0)
    assert wide / terms > 0.999


def test_first_window_bound_is_the_largest_the_first_squaring_allows(bbp):
    """Every head range's first-window bound is the largest w0 with
    bitlen(m_max) + 2 w0 + 1 <= R's width (so the extra first-window bit is not
    given away), and its first-window width is the most bits whose every value fits
    (at most 4): on the headline query the two-limb range of moduli up to 2^40 has
    bound 11 over a 3-bit window, so exponents whose top four bits read 8 to 11
    take a 4-bit first window."""
    for f, n, P, wide in ((0, 10**12, 256, 32), (0, 10**14 + 1, 256, 32), (1, 10**9, 128, 32),
                          (0, 10**7 + 1, 64, 5)):
        ranges, _ = bbp.bbp_explain(f, n, P, 64, wide)
        F = o1.FORMULAS["bellard" if f == 0 else "bbp"]
        for r in ranges:
            if r["tail"]:
                continue
            s = F.series[r["denominator"]]
            rb = 64 if r["path"] in (1, 2) else 32
            lmax = (s.a * (r["k_begin"] + r["count"] - 1) + s.b).bit_length()
            assert r["first_max"] == max(0, (rb - 1 - lmax) // 2), (f, n, r)
            h = max(i for i in range(5) if (1 << i) - 1 <= r["first_max"])
            assert r["first"] == h, (f, n, r)
    ranges, _ = bbp.bbp_explain(0, 10**12, 256, 64, 32)
    top = [r for r in ranges if not r["tail"] and r["denominator"] == 2][-1]
    assert (top["path"], top["window"], top["first"], top["first_max"]) == (1, 4, 3, 11)


def test_crossover_moves_small_moduli_to_two_limbs(bbp):
    for wide in (5, 10, 20, 30, 32):
        ranges, _ = bbp.bbp_explain(0, 10**7 + 1, 64, 64, wide)
        for r in ranges:
            if not r["tail"]:
                s = o1.BELLARD.series[r["denominator"]]
                m_max = s.a * (r["k_begin"] + r["count"] - 1) + s.b
                assert (r["path"] in (0, 3)) == (m_max.bit_length() < wide)


def test_one_limb_path_reaches_2_to_31(bbp):
    """At the default crossover every head term with a modulus below 2^31 runs on one
    limb: the n = 1e9 query (moduli below 2^30) has no two-limb head terms, and at
    n = 3e9 the moduli of 30 and 31 bits take path 3 and only those of 32 bits and
    more take the two-limb paths."""
    ranges, _ = bbp.bbp_explain(0, 10**9, 128, 64)
    assert all(r["path"] in (0, 3) for r in ranges if not r["tail"])
    assert any(r["path"] == 3 for r in ranges if not r["tail"])
    ranges, _ = bbp.bbp_explain(0, 3 * 10**9, 64, 64)
    for r in ranges:
        if r["tail"]:
            continue
        s = o1.BELLARD.series[r["denominator"]]
        lo = (s.a * r["k_begin"] + s.b).bit_length()
        hi = (s.a * (r["k_begin"] + r["count"] - 1) + s.b).bit_length()
        if r["path"] == 3:
            assert 30 <= lo and hi <= 31
        elif r["path"] in (1, 2):
            assert lo >= 32


def test_errors(bbp):
    with pytest.raises(bbp.BBPError) as e:
        bbp.bbp_explain(0, 0, 64)
    assert e.value.status == bbp.BBP_EINVAL
    for args in ((0, 100, 0, 64, 30), (0, 100, 64, 0, 30), (0, 100, 64, 48, 30), (0, 100, 1250, 64, 30),
                 (0, 100, 64, 64, 4), (0, 100, 64, 64, 33), (2, 100, 64, 64, 30)):
        with pytest.raises(bbp.BBPError) as e:
            bbp.bbp_explain(*args)
        assert e.value.status == bbp.BBP_EINVAL, args
    # a modulus reaching 2^60: n about 2^62 for Bellard's 4k + 1 series
    with pytest.raises(bbp.BBPError) as e:
        bbp.bbp_explain(0, 1 << 62, 64)
    assert e.value.status == bbp.BBP_ERANGE
    assert math.isfinite(bbp.bbp_explain(0, 1 << 40, 64)[0][0]["imad"])
