"""Oracle O3: bits of pi from Machin's arctangent formula, in plain Python integers.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

This is an independent route to the bits of pi, used to pin the BBP oracle: it
shares nothing with the BBP digit-extraction method (Sec. 3 of Sze's paper) --
no modular exponentiation, no series in 2^-k.  It evaluates

    pi = 16 atan(1/5) - 4 atan(1/239),   atan(1/x) = sum_i (-1)^i / ((2i+1) x^(2i+1))

in F-bit fixed point.  Every term is floored, so each term is off by less than
one unit; the error of the result is bounded by 16 (T5 + 1) + 4 (T239 + 1)
units for T5 and T239 evaluated terms, and a bit window is only returned when
that bound cannot change it.
"""

from __future__ import annotations

from functools import lru_cache


def _atan_inv(x: int, F: int) -> tuple[int, int]:
    """(floor-sum approximation of atan(1/x) * 2^F, number of terms)."""
    power = (1 << F) // x           # floor(2^F / x^(2i+1)), updated by floor division
    x2 = x * x
    total = 0
    i = 0
    while power:
        t = power // (2 * i + 1)
        total = total - t if i & 1 else total + t
        power //= x2
        i += 1
    return total, i


@lru_cache(maxsize=4)
def pi_fixed(F: int) -> tuple[int, int]:
    """(Y, E): Y approximates pi * 2^F with |Y - pi 2^F| < E."""
    a5, n5 = _atan_inv(5, F)
    a239, n239 = _atan_inv(239, F)
    return 16 * a5 - 4 * a239, 16 * (n5 + 1) + 4 * (n239 + 1)


def pi_bits(n: int, P: int, guard: int = 64, F: int | None = None) -> int:
    """The P bits of pi starting at bit position n (1 = first bit after the
    radix point) as an integer, MSB first.  Raises if rounding could reach them."""
    if n < 1 or P < 1:
        raise ValueError("n and P count from 1")
    need = n - 1 + P + guard
    if F is None or F < need:
        F = need
    Y, E = pi_fixed(F)
    shift = F - (n - 1 + P)                 # bits below the window
    low = Y & ((1 << shift) - 1)
    if not (E <= low <= (1 << shift) - E):
        raise ArithmeticError("Machin window is within the rounding bound; raise guard")
    return (Y >> shift) & ((1 << P) - 1)
