"""Path offsets of the movement-order pass (reading R6 of the straight path,
Sec. 2): step s of a path to (dx, dy) with L = max(|dx|, |dy|) sits at
round(s*d/L), halves away from zero.  The kernel forms each offset without an
integer division, as trunc(fl32(|s*d| * fl32(1/L) + 1/2)) with one fused
multiply-add, and that form is only valid because for |d| <= L <= 5 the
quotient is either exact in binary (L = 1, 2, 4) or at least 1/10 away from
a half.  This checks the single-precision form against the exact rational
rounding for every case the kernel meets, emulating the fused operation
exactly: the product and sum have at most 30 significant bits, so double
precision holds them exactly, and numpy rounds the double once to single."""
from fractions import Fraction
import math

import numpy as np


def exact_offset(num: int, L: int) -> int:
    r = math.floor(Fraction(abs(num), L) + Fraction(1, 2))
    return -r if num < 0 else r


def kernel_offset(num: int, L: int) -> int:
    inv = np.float32(1.0) / np.float32(L)  # correctly rounded reciprocal
    fused = float(abs(num)) * float(inv) + 0.5  # exact in double
    r = int(np.float32(fused))  # one rounding to nearest, then truncation
    return -r if num < 0 else r


def test_fused_form_rounds_like_the_exact_quotient():
    cases = 0
    for L in range(1, 6):
        for d in range(-L, L + 1):
            for s in range(1, L + 1):
                assert kernel_offset(s * d, L) == exact_offset(s * d, L), (L, d, s)
                cases += 1
    assert cases == 125


def test_check_tells_the_rounding_rules_apart():
    """The exact rule rounds halves away from zero; a form that rounded them
    to even (or truncated) would fail the check above at L = 2 and L = 4."""
    halves = [(num, L) for L in (2, 4) for num in range(-L * L, L * L + 1)
              if Fraction(num, L).denominator == 2]
    assert halves
    to_even = [round(Fraction(num, L)) for num, L in halves]
    away = [exact_offset(num, L) for num, L in halves]
    assert to_even != away
    assert any(int(Fraction(num, L)) != exact_offset(num, L) for num, L in halves)


def test_exact_rounding_is_odd_and_monotone():
    for L in range(1, 6):
        prev = None
        for num in range(-L * L, L * L + 1):
            r = exact_offset(num, L)
            assert r == -exact_offset(-num, L)
            assert prev is None or r >= prev
            prev = r
