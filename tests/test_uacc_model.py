"""A bit-level model of the pair loop's exact sum of m_j / r (UAcc in csrc/device.cuh).

Each term is P 2^e with P < 2^64. The accumulator is a 128-bit integer A times 2^L whose
window slides up so that the largest term sits at bits 56..119; the sum is rounded to a
double once, from its top 64 bits. This module restates those integer steps with Python
integers and checks them against exact rational sums. CPU only; the GPU tests check the
device code against the oracle.
"""
import math
import random
from fractions import Fraction

import pytest

M64 = (1 << 64) - 1


class UAccModel:
    def __init__(self):
        self.a0 = 0
        self.a1 = 0
        self.L = -(1 << 29)

    def add(self, P, e):
        s = e - self.L
        if s > 56:
            d = s - 56
            if d >= 128:
                self.a0 = self.a1 = 0
            elif d >= 64:
                self.a0 = self.a1 >> (d - 64)
                self.a1 = 0
            else:
                self.a0 = ((self.a0 >> d) | (self.a1 << (64 - d))) & M64
                self.a1 >>= d
            self.L += d
            s = 56
        if s >= 0:
            lo = (P << s) & M64
            hi = (P >> (64 - s)) if s else 0
        else:
            lo = P >> (-s) if s > -64 else 0
            hi = 0
        a0 = self.a0 + lo
        carry = 1 if a0 > M64 else 0
        self.a0 = a0 & M64
        a1 = self.a1 + hi + carry
        assert a1 <= M64, "128-bit overflow"
        self.a1 = a1

    def value(self):
        def to_double(Sn, e2):
            mant = (Sn >> 11) + ((Sn >> 10) & 1)
            ex = e2 + 11
            if mant >> 53:
                mant >>= 1
                ex += 1
            return math.ldexp(mant, ex)

        if self.a1:
            z = 64 - self.a1.bit_length()
            top = ((self.a1 << z) | (self.a0 >> (64 - z))) & M64 if z else self.a1
            return to_double(top, self.L + 64 - z)
        if self.a0:
            z = 64 - self.a0.bit_length()
            return to_double((self.a0 << z) & M64, self.L - z)
        return 0.0


def _relerr(got, exact):
    return abs(Fraction(got) - exact) / exact


@pytest.mark.parametrize("spread", [0, 8, 64, 300])
def test_sum_is_exact_to_one_rounding(spread):
    """Terms whose exponents spread over 2^spread: the rounded sum is within 2^-53 (one
    rounding of the exact sum) plus the truncation of terms far below the largest."""
    rng = random.Random(spread)
    for _ in range(300):
        n = rng.randint(1, 256)
        terms = [(rng.getrandbits(64) | (1 << 63), rng.randint(-spread, spread) - 1000) for _ in range(n)]
        acc = UAccModel()
        for P, e in terms:
            acc.add(P, e)
        exact = sum(Fraction(P) * Fraction(2) ** e for P, e in terms)
        assert _relerr(acc.value(), exact) <= Fraction(1, 2 ** 53) * Fraction(1001, 1000)


def test_256_largest_terms_do_not_overflow():
    acc = UAccModel()
    for _ in range(256):
        acc.add(M64, 40)
    exact = Fraction(M64 * 256) * 2 ** 40
    assert _relerr(acc.value(), exact) <= Fraction(1, 2 ** 53)


def test_masked_adds_leave_the_sum_unchanged():
    """A masked pair adds P = 0 at the window's own exponent: a no-op, before or after the
    first real term."""
    acc = UAccModel()
    acc.add(0, acc.L)
    assert acc.value() == 0.0
    acc.add(12345 << 40, -7)
    state = (acc.a0, acc.a1, acc.L)
    acc.add(0, acc.L)
    assert (acc.a0, acc.a1, acc.L) == state


def test_a_growing_sequence_slides_the_window():
    """Each term twice the last: the window slides up at every add and the sum stays exact
    to one rounding (2^k - 1 times the first term)."""
    acc = UAccModel()
    P = 1 << 63
    for k in range(200):
        acc.add(P, k - 100)
    exact = Fraction(P) * (Fraction(2) ** 200 - 1) * Fraction(2) ** -100
    assert _relerr(acc.value(), exact) <= Fraction(1, 2 ** 53)
