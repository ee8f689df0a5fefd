"""Oracle O1: BBP digit extraction of pi written out with plain Python integers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library never
calls it and shares no code, table or helper with it.

What it computes (Sze, "The Two Quadrillionth Bit of pi is 0!", Sec. 3):

* To read the bits of pi that start at bit position ``n`` (counted from 1 after
  the radix point, Sec. 2 footnote: pi = 11.0010 0100 0011 1111..., so the eight
  bits starting at position 9 are 0x3F), compute the fractional part
  ``{2^d pi}`` with ``d = n - 1`` (Sec. 3: the (n+1)th bit comes from
  ``{2^n pi}``).
* A BBP-type formula (Eq. 1, or Bellard's Eq. 2) turns ``{2^d pi}`` into a signed
  combination of fractional parts of series (Eq. 3).  Each series
  ``sum_k 2^(d + c - step*k) / (a*k + b)`` is split (Eq. 4) into head terms
  ``A_k = (2^e mod m) / m`` for exponents ``e >= 0`` and tail terms
  ``B_k = 1 / (2^-e * m)`` for ``e < 0`` (Eq. 5).
* Every term is evaluated as an exact W-bit fixed-point fraction (Sec. 4.3:
  modular exponentiation, then a division carried to the working precision;
  a tail term is a shift followed by a division to ``W - b`` bits), and the
  signed terms are summed modulo 1, i.e. modulo ``2^W`` in fixed point (Eq. 3).

Readings taken where the paper is silent or leaves a choice open:

1. Each non-negative term is truncated (floor) to W fraction bits; its sign is
   applied afterwards, in two's complement modulo ``2^W``.
2. ``W = roundup(P, 32) + G`` with G guard bits; the output is the top P bits.
3. A term is a head term iff its exponent ``e >= 0``; at ``e = 0`` Eq. 5's two
   forms agree.
4. The tail stops at the first term whose truncated value is 0 (or whose
   ``W + e`` is negative): all later terms are smaller still.
5. A tail term is ``floor(2^(W+e) / m)`` -- shifting first and dividing to
   ``W - b`` bits gives the same integer as dividing then shifting.
6. Error bound (Eq. 8 restated for truncation): each evaluated term is off by
   less than one unit in the last place and the omitted tail of each series is
   below ``1/(1 - 2^-step)`` units, so ``|S - {2^d pi} 2^W| < N + J + 1`` units
   for N evaluated terms and J series.  The leading b bits are certified iff the
   low ``W - b`` bits ``g`` of S satisfy ``B <= g <= 2^(W-b) - B`` with
   ``B = N + J + 1``.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Iterable, Sequence


@dataclass(frozen=True)
class Series:
    """One series of a BBP-type formula: sum_k sign * (-1)^(alt*k) * 2^(d+c-step*k) / (a*k+b)."""

    a: int      # modulus slope: m_k = a*k + b
    b: int      # modulus offset
    sign: int   # +1 or -1, the sign in front of the series
    c: int      # exponent offset: the series' power-of-two coefficient is 2^c


@dataclass(frozen=True)
class Formula:
    name: str
    step: int            # exponent decrease per k (10 for Eq. 2, 4 for Eq. 1)
    alternating: bool    # (-1)^k factor present (Eq. 2) or not (Eq. 1)
    series: tuple[Series, ...]


# Eq. 2 (Bellard), read off term by term: 2^2/(10k+1) - 1/(10k+3) - 2^-4/(10k+5)
# - 2^-4/(10k+7) + 2^-6/(10k+9) - 2^-1/(4k+1) - 2^-6/(4k+3), all times (-1)^k 2^-10k.
BELLARD = Formula(
    name="bellard",
    step=10,
    alternating=True,
    series=(
        Series(10, 1, +1, 2),
        Series(10, 3, -1, 0),
        Series(10, 5, -1, -4),
        Series(10, 7, -1, -4),
        Series(10, 9, +1, -6),
        Series(4, 1, -1, -1),
        Series(4, 3, -1, -6),
    ),
)

# Eq. 1 (BBP) in the form of Eq. 3: 2^(d+2-4k)/(8k+1) - 2^(d-1-4k)/(2k+1)
# - 2^(d-4k)/(8k+5) - 2^(d-1-4k)/(4k+3), no alternation.
BBP = Formula(
    name="bbp",
    step=4,
    alternating=False,
    series=(
        Series(8, 1, +1, 2),
        Series(2, 1, -1, -1),
        Series(8, 5, -1, 0),
        Series(4, 3, -1, -1),
    ),
)

FORMULAS = {"bellard": BELLARD, "bbp": BBP, 0: BELLARD, 1: BBP}


def working_bits(P: int, G: int) -> int:
    """W = roundup(P, 32) + G (reading 2); G must be a positive multiple of 32."""
    if P <= 0:
        raise ValueError("P must be positive")
    if G <= 0 or G % 32:
        raise ValueError("G must be a positive multiple of 32")
    return -(-P // 32) * 32 + G


def exponent(f: Formula, s: Series, d: int, k: int) -> int:
    """e = d + c - step*k: the power of two in front of term k (Eq. 3 / Eq. 4)."""
    return d + s.c - f.step * k


def term(f: Formula, s: Series, d: int, k: int, W: int) -> int:
    """The unsigned W-bit fixed-point value of term k of one series (Eq. 5).

    Head term (e >= 0): A_k = (2^e mod m)/m, i.e. a modular exponentiation followed
    by a division carried to W fraction bits.  Tail term (e < 0): B_k = 2^e/m, i.e.
    a shift by b = -e bits then a division to W - b bits.  Both truncate (reading 1).
    """
    e = exponent(f, s, d, k)
    m = s.a * k + s.b
    if e >= 0:
        r = pow(2, e, m)                  # modular exponentiation (Sec. 4.3)
        return (r << W) // m              # division to W bits
    if W + e < 0:
        return 0
    return (1 << (W + e)) // m            # shift by -e, divide to W + e bits


def head_end(f: Formula, s: Series, d: int) -> int:
    """First k whose exponent is negative: head terms are k < head_end (Eq. 4)."""
    top = d + s.c
    return 0 if top < 0 else top // f.step + 1


def natural_end(f: Formula, s: Series, d: int, W: int) -> int:
    """First k after the head whose truncated tail term is 0 (reading 4).

    Terms k >= natural_end are all 0 once truncated, because 2^e shrinks and m grows.
    """
    k = head_end(f, s, d)
    while True:
        e = exponent(f, s, d, k)
        m = s.a * k + s.b
        if W + e < 0 or (1 << (W + e)) // m == 0:
            return k
        k += 1


def partial_sum(f: Formula, j: int, k_begin: int, k_end: int | None, n: int, P: int, G: int) -> int:
    """sum over k in [k_begin, k_end) of sign_j (-1)^k t_{j,k}, modulo 2^W.

    ``k_end=None`` means the natural end of series j.  Terms past the natural end
    are zero by definition and contribute nothing.
    """
    if n < 1:
        raise ValueError("n counts from 1")
    W = working_bits(P, G)
    d = n - 1
    s = f.series[j]
    end = natural_end(f, s, d, W)
    hi = end if k_end is None else min(k_end, end)
    acc = 0
    for k in range(k_begin, hi):
        t = term(f, s, d, k, W)
        if f.alternating and (k & 1):
            acc -= t
        else:
            acc += t
    return (s.sign * acc) % (1 << W)


def accumulate(f: Formula, n: int, P: int, G: int) -> tuple[int, int]:
    """(S, N): the full fixed-point sum S = {2^d pi} 2^W (mod 2^W) and the number
    N of evaluated terms, taken series by series as in Eq. 3."""
    W = working_bits(P, G)
    d = n - 1
    S = 0
    N = 0
    for j, s in enumerate(f.series):
        end = natural_end(f, s, d, W)
        N += end
        S += partial_sum(f, j, 0, None, n, P, G)
    return S % (1 << W), N


def error_bound(f: Formula, N: int) -> int:
    """Integer B with |S - {2^d pi} 2^W| < B units (reading 6)."""
    # each omitted tail is below 1/(1 - 2^-step) <= 1.07 units; J of them < J + 1
    return N + len(f.series) + 1


def certified_bits(S: int, W: int, P: int, B: int) -> int:
    """Largest b <= P such that the top b bits of S are those of the exact value."""
    for b in range(P, -1, -1):
        low = W - b
        g = S & ((1 << low) - 1)
        if B <= g <= (1 << low) - B:
            return b
    return 0


def bits(n: int, P: int, G: int = 64, formula: str | Formula = "bellard") -> tuple[int, int]:
    """(value, valid): the P bits of pi starting at position n as an integer
    (MSB = bit n), and how many leading bits the error bound certifies."""
    f = formula if isinstance(formula, Formula) else FORMULAS[formula]
    W = working_bits(P, G)
    S, N = accumulate(f, n, P, G)
    return S >> (W - P), certified_bits(S, W, P, error_bound(f, N))


def to_bytes_msb_first(value: int, P: int) -> bytes:
    """Pack P bits (MSB = first bit) into ceil(P/8) bytes; unused low bits are 0."""
    nbytes = (P + 7) // 8
    return (value << (nbytes * 8 - P)).to_bytes(nbytes, "big")


def to_limbs(x: int, W: int) -> list[int]:
    """Little-endian 32-bit limbs of x mod 2^W."""
    x %= 1 << W
    return [(x >> (32 * i)) & 0xFFFFFFFF for i in range(W // 32)]


def from_limbs(limbs: Sequence[int] | Iterable[int]) -> int:
    return sum(int(v) << (32 * i) for i, v in enumerate(limbs))
