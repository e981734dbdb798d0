"""Closed forms of the expected overlap upper bound (Section 3.4, Eq. 4-6).

TEST INFRASTRUCTURE (part of the oracle).  For two sets of n tokens each,
hashed uniformly into b bits, the paper gives the expected value of the
Theorem 1 bound (without the floor) for each generation method:

  Eq. 4 (Set):  E = n + (b-1)^(2n) / b^(2n-1) - (b-1)^n / b^(n-1)
  Eq. 5 (Xor):  E = n - (b/2) * sum over odd k in [1, 2n] of
                     C(2n, k) (1/b)^k ((b-1)/b)^(2n-k)
  Eq. 6 (Next): E = min(n^2 / b, n)            (an approximation)

Eq. 4 and Eq. 5 are evaluated exactly with rationals and returned as float.
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
