"""Closed forms of the expected overlap upper bound (Section 3.4, Eq. 4-6).

TEST INFRASTRUCTURE (part of the oracle).  For two sets of n tokens each,
hashed uniformly into b bits, the paper gives the expected value of the
Theorem 1 bound (without the floor) for each generation method:

  Eq. 4 (Set):  E = n + (b-1)^(2n) / b^(2n-1) - (b-1)^n / b^(n-1)
  Eq. 5 (Xor):  E = n - (b/2) * sum over odd k in [1, 2n] of
                     C(2n, k) (1/b)^k ((b-1)/b)^(2n-k)
  Eq. 6 (Next): E = min(n^2 / b, n)            (an approximation)

Eq. 4 and Eq. 5 are evaluated exactly with rationals and returned as float.

The cutoff point (Section 3.5) is the set size at which the normalised
expected bound E(b, n)/n reaches the normalised overlap threshold u: the
largest n with E(b, n)/n <= u.  Its search runs to n in the thousands, so it
uses Eq. 4 and Eq. 5 in closed form (fp64):
  Eq. 4 = n + b q^(2n) - b q^n                    with q = (b-1)/b
  Eq. 5 = n - (b/4) (1 - (1 - 2/b)^(2n))
(the odd-k half of the binomial expansion of (q + 1/b)^(2n) is
((q + 1/b)^(2n) - (q - 1/b)^(2n)) / 2).
The Monte Carlo test in tests/test_oracle_pins.py draws random token sets,
builds their bitmaps with the oracle's Alg. 3a/3b and compares the mean of
(|r| + |s| - popcount(br xor bs)) / 2 with these values.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb


def e_set(b: int, n: int) -> float:
    """Eq. 4, exact rational arithmetic."""
    v = Fraction(n) + Fraction((b - 1) ** (2 * n), b ** (2 * n - 1)) \
        - Fraction((b - 1) ** n, b ** (n - 1))
    return float(v)


def e_xor(b: int, n: int) -> float:
    """Eq. 5, the odd-k binomial sum written out term by term."""
    s = Fraction(0)
    for k in range(1, 2 * n + 1, 2):
        s += comb(2 * n, k) * Fraction(1, b) ** k * Fraction(b - 1, b) ** (2 * n - k)
    return float(Fraction(n) - Fraction(b, 2) * s)


def e_next(b: int, n: int) -> float:
    """Eq. 6 (the paper's approximation)."""
    return min(n * n / b, float(n))


def e_set_closed(b: int, n: int) -> float:
    """Eq. 4 rearranged (fp64)."""
    q = (b - 1) / b
    return n + b * q ** (2 * n) - b * q ** n


def e_xor_closed(b: int, n: int) -> float:
    """Eq. 5 with its odd-k binomial sum in closed form (fp64)."""
    return n - (b / 4) * (1 - (1 - 2 / b) ** (2 * n))


def cutoff(b: int, u: float, method: str) -> int:
    """Section 3.5: the largest n with E(b, n)/n <= u, for method "set", "xor" or
    "next" (Eq. 4, 5, 6); u is the normalised overlap threshold."""
    e = {"set": e_set_closed, "xor": e_xor_closed, "next": e_next}[method]
    n = 1
    while e(b, n + 1) / (n + 1) <= u:
        n += 1
    return n
