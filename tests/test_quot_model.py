"""A model of the batched kernels' quotient by the total mass (quot in csrc/batched.cu):
q = S rM with rM = RN(1/M), then one correction fma(fma(-q, M, S), rM, q). The comment there
claims the correctly rounded S / M except in rare cases next to a rounding boundary, where
the result is one unit in the last place away. CPU only."""
import math
import random
from fractions import Fraction


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def quot(S, M, rM):
    q = S * rM
    return _fma(_fma(-q, M, S), rM, q)


def test_quotient_is_correctly_rounded_but_rarely_one_ulp_off():
    rng = random.Random(3)
    off = 0
    trials = 20000
    for _ in range(trials):
        M = rng.uniform(0.5, 2.0) * 10.0 ** rng.randint(-3, 3)
        S = rng.uniform(-1, 1) * 10.0 ** rng.randint(-20, 20)
        got, exact = quot(S, M, 1.0 / M), S / M          # Python's division is correctly rounded
        if got != exact:
            off += 1
            assert abs(got - exact) <= math.ulp(exact), (S, M, got, exact)
    assert off <= trials // 1000, off                    # rare: none seen in these 20000
