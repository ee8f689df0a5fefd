"""A word-level model of the head kernel's arithmetic, run on the CPU at the
extremes of the launch ranges the planner produces.

The kernels keep every value in 32-bit words and drop carries they have shown
cannot occur; the GPU parity tests sample terms, this model checks the claims
themselves.  It restates, word by word, what the device code does for one term
(in `csrc/bbp_device.cuh` and `process_tile` in `csrc/bbp_tile.cuh`):
  * -m^-1 mod 2^32 by Newton-Hensel lifting from the start (3 m) XOR 2 (three steps);
  * R mod m by bit-serial division, carried to k + 1 with R = q (m + a) + (r - a q);
  * the left-to-right ladder: a first window taken as (R mod m) << w0, then
    groups of `window` bits, each len - 1 plain Montgomery squarings and one
    squaring with the group's bits shifted in (aligned from the top, except on
    path 1 with 4-bit windows, where they are aligned from the bottom);
  * path 2 (and the first squaring of path 1): the square on four words, the
    shift by funnel shifts, two word-by-word REDC steps with the vanishing low
    word's carry taken as (word != 0) and u m1 accumulated by the multiply;
  * path 1: the square on three words (x1^2 low word only), the first REDC step
    summed in 32-bit carry chains into two words, the window shift applied to
    that two-word value, then the second REDC step;
  * one-word squaring and REDC, with lazy residues (path 0) or one conditional
    subtraction per squaring (path 3, moduli of 30 and 31 bits);
  * W/32 exact-division digits (Hensel), least significant first; a lane past
    the range enters them with x = 0.
Every dropped carry, truncated shift and narrowed product is asserted to be
zero or in range, the ladder result must be 2^E mod m, and the digits must
equal the oracle's term floor((2^e mod m) 2^W / m) mod 2^W (Eq. 5).  The launch
parameters (path, window, first window) come from the library's own planner
(bbp_explain); the exponents include the warp-maximum padding the kernel uses
and all-ones exponents that take the largest shift in every group.
"""

import importlib.util
import os
import random

import pytest

from conftest import ROOT
from oracle import bbp_oracle as o1

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def bbp():
    spec = importlib.util.spec_from_file_location("_bbp_build", os.path.join(ROOT, "paper_1008_3171_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1008_3171_gb300 as m

    return m


def neg_inverse32(m0):
    x = ((3 * m0) ^ 2) & M32
    assert (x * m0) & 31 == 1                # five correct bits to start
    for _ in range(3):                       # 5 -> 10 -> 20 -> 40 bits
        x = (x * ((2 - m0 * x) & M32)) & M32
    assert (x * m0) & M32 == 1
    return (-x) & M32


def r_mod_m_bitserial(m, rbits):
    l = m.bit_length()
    r, q = 1 << (l - 1), 0
    for _ in range(l - 1, rbits):
        r <<= 1
        q <<= 1
        assert r <= M64                      # r < m < 2^60 before doubling
        if r >= m:
            r -= m
            q |= 1
    assert q == (1 << rbits) // m and r == (1 << rbits) % m
    return q, r


def r_mod_m_advance(q, r, m_next, a, rbits):
    aq = q * a
    assert aq <= M64                         # formed in 64 bits
    if aq > r + 4 * m_next:
        return r_mod_m_bitserial(m_next, rbits)
    r2 = r - aq
    while r2 < 0:
        r2 += m_next
        q -= 1
    assert q == (1 << rbits) // m_next and r2 == (1 << rbits) % m_next
    return q, r2


def sqr_shift_redc64(x, s, m, mp, do_shift):
    """General squaring (path 2 and the first squaring of path 1): four-word square."""
    x0, x1 = x & M32, x >> 32
    assert x1 < 1 << 31                      # d1 = x1 << 1 in one word
    d1 = x1 << 1
    p00, p01, p11 = x0 * x0, x0 * d1, x1 * x1
    s1 = (p00 >> 32) + (p01 & M32)
    c = s1 >> 32
    s1 &= M32
    s2 = (p11 & M32) + (p01 >> 32) + c
    c = s2 >> 32
    s2 &= M32
    s3 = (p11 >> 32) + c
    assert s3 <= M32
    s0 = p00 & M32
    T = s0 | s1 << 32 | s2 << 64 | s3 << 96
    assert T == x * x
    if do_shift:
        assert 0 <= s < 32
        assert (T << s) >> 128 == 0          # funnel shifts keep four words
        T <<= s
    t0, t1, t2, t3 = T & M32, (T >> 32) & M32, (T >> 64) & M32, T >> 96
    m0, m1 = m & M32, m >> 32
    # step 1: word 0 vanishes
    u = (t0 * mp) & M32
    assert (t0 + u * m0) & M32 == 0
    h = ((u * m0) >> 32) + (1 if t0 else 0)
    assert h <= M32
    a = (t1 | t2 << 32) + u * m1
    t3 += a >> 64
    a &= M64
    a += h
    t3 += a >> 64
    a &= M64
    assert t3 <= M32
    t1, t2 = a & M32, a >> 32
    assert (T + u * m) >> 32 == t1 | t2 << 32 | t3 << 64
    # step 2: word 1 vanishes; the 64-bit multiply-add must not carry out
    u = (t1 * mp) & M32
    h = ((u * m0) >> 32) + (1 if t1 else 0)
    assert h <= M32
    a = (t2 | t3 << 32) + u * m1
    assert a <= M64
    a += h
    assert a <= M64
    assert a < 2 * m
    return a


def add32(a, b, cin=0):
    """One 32-bit add of a carry chain: (sum mod 2^32, carry out)."""
    v = a + b + cin
    return v & M32, v >> 32


def sqr_redc64_p1(x, s, m, mp, do_shift):
    """Path 1 (bitlen(m) <= 46, x < 2m): three-word square, first REDC step into two
    words by 32-bit carry chains, the window shift on that two-word value, then the
    second step.  Mirrors the two asm blocks of sqr_redc64_p1."""
    assert x < 2 * m
    x0, x1 = x & M32, x >> 32
    d1 = (x1 << 1) & M32                     # funnel shift of (x1 : 0) by one
    assert d1 == 2 * x1
    p00, p01 = x0 * x0, x0 * d1
    q0 = (x1 * x1) & M32
    assert x1 * x1 <= M32                    # only the low word of x1^2 is formed
    s0, h0 = p00 & M32, p00 >> 32
    b0, b1 = p01 & M32, p01 >> 32
    m0, m1 = m & M32, m >> 32
    u = (s0 * mp) & M32
    assert (s0 + u * m0) & M32 == 0
    h = (u * m0) >> 32
    z = u * m1
    z0, z1 = z & M32, z >> 32
    _, c = add32(s0, M32)                    # carry out = (s0 != 0)
    h0, c = add32(h0, b0, c)
    b1, c2 = add32(b1, q0, c)
    assert c2 == 0
    h0, c = add32(h0, z0)
    b1, c2 = add32(b1, z1, c)
    assert c2 == 0
    y0, c = add32(h0, h)
    y1, c2 = add32(b1, 0, c)
    assert c2 == 0                           # T' fits two words
    T = x * x
    assert y0 | y1 << 32 == (T + u * m) >> 32
    y2 = 0
    if do_shift:
        assert 0 <= s < 32
        y = (y0 | y1 << 32) << s
        assert y >> 96 == 0                  # three words after the shift
        y0, y1, y2 = y & M32, (y >> 32) & M32, y >> 64
    Y = y0 | y1 << 32 | y2 << 64
    u2 = (y0 * mp) & M32
    assert (y0 + u2 * m0) & M32 == 0
    h2 = (u2 * m0) >> 32
    z = u2 * m1
    z0, z1 = z & M32, z >> 32
    _, c = add32(y0, M32)
    b1, c = add32(y1, z0, c)
    b2, c2 = add32(y2, z1, c)
    assert c2 == 0
    r0, c = add32(b1, h2)
    r1, c2 = add32(b2, 0, c)
    assert c2 == 0
    r = r0 | r1 << 32
    assert r == (Y + u2 * m) >> 32
    assert r % m == (x * x << (s if do_shift else 0)) * pow(2, -64, m) % m
    assert r < 2 * m
    return r


def hensel_step64(x, m, mp):
    x0, x1 = x & M32, x >> 32
    q = (x0 * mp) & M32
    h = ((q * (m & M32)) >> 32) + (1 if x0 else 0)
    assert h <= M32
    r = q * (m >> 32) + h + x1
    assert r <= M64 and r == (x + q * m) >> 32 and (x + q * m) & M32 == 0
    return q, r


def sqr_shift_redc32(x, s, m, mp, do_shift, reduced):
    if reduced:
        assert x < m
    T = x * x
    if do_shift:
        T <<= s
    assert T <= M64
    t0, t1 = T & M32, T >> 32
    u = (t0 * mp) & M32
    r = t1 + ((u * m) >> 32) + (1 if t0 else 0)
    assert r <= M32 and r < 2 * m
    if reduced:                               # min(r, r - m) on 32-bit words
        r = min(r, (r - m) & M32)
        assert r < m
    return r


def ladder_term(path, window, first, m, E, W, extra, r_mod_m, valid=True, first_max=0, take_extra=False):
    """2^E mod m by the kernel's ladder, then the W-bit quotient digits.  take_extra:
    the warp's top first + 1 exponent bits fit first_max, so the first window takes
    one more bit (taken here whenever this term's own bits allow it)."""
    wide = path in (1, 2)
    rb = 64 if wide else 32
    mp = neg_inverse32(m & M32)
    v = E - rb
    assert v >= 0
    nb = v.bit_length() + extra              # the warp's longest exponent
    h = min(first, nb - 1) if nb > 0 else 0
    if take_extra and h + 1 <= nb - 1 and (v >> (nb - h - 1)) <= first_max:
        h += 1
    low = nb - h
    w0 = (v >> low) if h > 0 else 0
    x = r_mod_m << w0
    assert x < 1 << rb
    rem = v & ((1 << low) - 1) if low > 0 else 0

    def square(x, sh, shifted, general=False):
        if path == 2 or general:
            return sqr_shift_redc64(x, sh, m, mp, shifted)
        if path == 1:
            return sqr_redc64_p1(x, sh, m, mp, shifted)
        return sqr_shift_redc32(x, sh, m, mp, shifted, path == 3)

    p = low
    w4 = path == 1 and window == 4           # path 1: groups aligned from the bottom, the first one short
    if path == 1 and p > 0:                  # first group: its first squaring on the general routine
        ln = (p - 1) % 4 + 1 if w4 else min(window, p)
        p -= ln
        sh = (rem >> p) & ((1 << ln) - 1)
        if ln == 1:
            x = square(x, sh, True, general=True)
        else:
            x = square(x, 0, False, general=True)
            for i in range(ln - 1):
                last = i == ln - 2
                x = square(x, sh if last else 0, last)
    while p > 0:
        ln = min(window, p)
        p -= ln
        for i in range(ln):
            last = i == ln - 1
            sh = ((rem >> p) & ((1 << ln) - 1)) if last else 0
            x = square(x, sh, last)
    assert x % m == pow(2, E, m)
    if x >= m:
        x -= m
    if not valid:                            # a lane past the range: x = 0, all digits 0
        x = 0
    digits = []
    for _ in range(W // 32):
        if wide:
            q, x = hensel_step64(x, m, mp)
        else:
            q = (x * mp) & M32
            x = ((q * m) >> 32) + (1 if x else 0)
        digits.append(q)
    return sum(q << (32 * i) for i, q in enumerate(digits))


CONFIGS = [
    (0, 10**12, 256, 64, 32),
    (0, 10**14 + 1, 256, 64, 32),
    (0, 2 * 10**15 - 3, 256, 64, 32),
    (0, 10**17 + 1, 64, 32, 32),
    (1, 10**16 + 7, 1000, 64, 32),
    (0, 10**7 + 1, 64, 64, 5),
    (0, 10**9 + 1, 128, 64, 17),
    (0, 10**9 + 1, 128, 64, 32),
    (0, 3 * 10**9 + 7, 64, 64, 32),
    (1, 2 * 10**9 + 3, 256, 64, 31),
    (0, 10**10 + 1, 256, 64, 30),
]


def test_every_path_is_modelled(bbp):
    """The configurations reach every modulus path: one word lazy (0) and reduced (3),
    two words with the three-word square (1) and the four-word square (2)."""
    seen = set()
    for cfg in CONFIGS:
        seen |= _check_config(bbp, *cfg)
    assert seen == {0, 1, 2, 3}


def test_inverse_start_value_is_five_bits():
    """(3 m) XOR 2 is an inverse of every odd m modulo 2^5 (here: every odd residue mod
    2^16), and three lifting steps from it reach 32 bits for random odd words."""
    for m in range(1, 1 << 16, 2):
        assert (m * ((3 * m) ^ 2)) % 32 == 1
    rng = random.Random(3)
    for _ in range(2000):
        m = rng.randrange(1, 1 << 32) | 1
        assert (m * neg_inverse32(m)) & M32 == M32      # m (-m^-1) = -1


@pytest.mark.parametrize("f,n,P,G,wide", CONFIGS)
def test_word_model_matches_oracle_at_range_extremes(bbp, f, n, P, G, wide):
    _check_config(bbp, f, n, P, G, wide)


def _check_config(bbp, f, n, P, G, wide):
    rng = random.Random(n ^ (P << 8) ^ wide)
    F = o1.FORMULAS[f]
    W = o1.working_bits(P, G)
    d = n - 1
    ranges, _ = bbp.bbp_explain(f, n, P, G, wide)
    checked = 0
    paths = set()
    for r in ranges:
        if r["tail"]:
            continue
        s = F.series[r["denominator"]]
        path, window, first, fm = r["path"], r["window"], r["first"], r["first_max"]
        assert fm >= (1 << first) - 1
        rb = 64 if path in (1, 2) else 32
        k_last = r["k_begin"] + r["count"] - 1
        ks = sorted({r["k_begin"], min(r["k_begin"] + 1, k_last), k_last}
                    | {rng.randrange(r["k_begin"], k_last + 1) for _ in range(3)})
        q = rr = None
        prev = None
        for k in ks:
            m = s.a * k + s.b
            if prev is not None and k == prev + 1:
                q, rr = r_mod_m_advance(q, rr, m, s.a, rb)
            else:
                q, rr = r_mod_m_bitserial(m, rb)
            prev = k
            E = d + s.c - F.step * k + W
            want = o1.term(F, s, d, k, W)
            for extra in (0, 1, 9):               # a warp tile can span E from ~64 to ~20000
                for take in (False, True):
                    got = ladder_term(path, window, first, m, E, W, extra, rr, first_max=fm, take_extra=take)
                    assert got % (1 << W) == want, (f, n, k, extra, take)
            assert ladder_term(path, window, first, m, E, W, 0, rr, valid=False) == 0
            # the largest shifts: an all-ones exponent of the same length, at the range's largest modulus
            m_max = s.a * k_last + s.b
            L1 = max(1, (E - rb).bit_length())
            E1 = rb + (1 << L1) - 1
            x = ladder_term(path, window, first, m_max, E1, 64, 0, (1 << rb) % m_max)
            assert x == (-pow(2, E1, m_max) * pow(m_max, -1, 1 << 64)) % (1 << 64)
            # the largest first window: top bits equal to first_max, then all ones
            if fm >= 1 << first and L1 >= first + 3:
                v2 = (fm << (L1 - first - 1)) | ((1 << (L1 - first - 1)) - 1)
                E2 = rb + v2
                x = ladder_term(path, window, first, m_max, E2, 64, 0, (1 << rb) % m_max, first_max=fm,
                                take_extra=True)
                assert x == (-pow(2, E2, m_max) * pow(m_max, -1, 1 << 64)) % (1 << 64)
            checked += 1
            paths.add(path)
    assert checked > 0
    return paths


def test_quotient_digits_are_the_exact_division():
    """Fed s = x 2^W mod m, the digits q_i with s + (sum q_i 2^(32 i)) m = 0
    mod 2^W are floor(x 2^W / m): the W-bit fraction of x / m without a
    reciprocal (the ladder delivers s = 2^(e + W) mod m, i.e. x = 2^e mod m).
    Checked against the definition for random odd moduli of every width."""
    rng = random.Random(5)
    for _ in range(300):
        bits = rng.choice((5, 20, 29, 31, 40, 47, 52, 59))
        m = rng.randrange(1 << (bits - 1), 1 << bits) | 1
        x = rng.randrange(0, m)
        W = 32 * rng.randrange(2, 12)
        mp = neg_inverse32(m & M32)
        y, digits = (x << W) % m, []
        for _ in range(W // 32):
            q, y = hensel_step64(y, m, mp)
            digits.append(q)
        t = sum(q << (32 * i) for i, q in enumerate(digits))
        assert t == (x << W) // m


def tail_term_model(s, F, d, k, W):
    """Tail term (e < 0) as the tail kernel forms it: q = floor(2^W / m) from the
    exact-division digits of 2^W mod m (doubling, then Hensel steps), shifted
    right by b = -e (Sec. 4.3: shift, then divide to W - b bits)."""
    e = d + s.c - F.step * k
    b = -e
    m = s.a * k + s.b
    assert 1 <= b
    if b > W:
        return 0
    if m == 1:
        return 1 << (W - b)
    x = 1
    for _ in range(W):                        # 2^W mod m by doubling; m < 2^62 keeps 2x in 64 bits
        x <<= 1
        assert x <= M64
        if x >= m:
            x -= m
    mp = neg_inverse32(m & M32)
    digits = []
    for _ in range(W // 32):
        q, x = hensel_step64(x, m, mp)
        digits.append(q)
    q = sum(v << (32 * i) for i, v in enumerate(digits))
    assert q == (1 << W) // m % (1 << W)
    return q >> b


@pytest.mark.parametrize("f,n,P,G,wide", CONFIGS + [(0, 1, 64, 32, 30), (1, 2, 8, 32, 30), (0, 9, 8, 64, 30)])
def test_tail_model_matches_oracle(bbp, f, n, P, G, wide):
    F = o1.FORMULAS[f]
    W = o1.working_bits(P, G)
    d = n - 1
    ranges, _ = bbp.bbp_explain(f, n, P, G, wide)
    tails = [r for r in ranges if r["tail"]]
    assert tails
    for r in tails:
        s = F.series[r["denominator"]]
        for k in range(r["k_begin"], r["k_begin"] + r["count"]):
            assert tail_term_model(s, F, d, k, W) == o1.term(F, s, d, k, W), (f, n, k)
