"""A bit-level model of the four-instruction FP64 reciprocal square root (rsqrt_fp64 in
csrc/device.cuh), used by the near pairs and the adjoint, checked against 60-digit
arithmetic.

The steps: a float seed of 1/sqrt built from x's exponent and top mantissa bits, made an
exact double y; e = fma(-x, y^2, 1); the binomial series y (1 + e/2 + 3e^2/8), with the e^2
term in float. The hardware seed is replaced by a float32 of 1/sqrt perturbed by up to
2^-21. CPU only; the GPU tests check the device code against the oracle.
"""
import math
import random
import struct
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _double(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _fbits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _float(b):
    return struct.unpack("<f", struct.pack("<I", b))[0]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _approx_float_of(x):
    """float from the leading bits of a normal double (truncated), 0 below the float range."""
    hi = _bits(x) >> 32
    e = ((hi >> 20) & 0x7FF) - 1023 + 127
    m = (hi & 0xFFFFF) << 3
    if not 0 < e < 255:
        return np.float32(0.0)
    return np.float32(_float((hi & 0x80000000) | (e << 23) | m))


def _double_of_nonneg_float(f):
    b = _fbits(float(f))
    e = (b >> 23) & 0xFF
    m = b & 0x7FFFFF
    if e == 0:
        return 0.0
    return _double((((e - 127 + 1023) << 20) | (m >> 3)) << 32 | ((m << 29) & 0xFFFFFFFF))


def rsqrt_model(x, seed_rel):
    b = _bits(x)
    hi, lo = b >> 32, b & 0xFFFFFFFF
    E = ((hi >> 20) & 0x7FF) - 1023
    k = E >> 1
    fe = E - 2 * k
    mant = ((hi & 0xFFFFF) << 3) | (lo >> 29)
    mx = _float(((127 + fe) << 23) | mant)
    yf = np.float32(1.0 / math.sqrt(mx) * (1.0 + seed_rel))
    yb = _fbits(float(yf))
    ye = ((yb >> 23) & 0xFF) - 127 + 1023 - k
    ym = yb & 0x7FFFFF
    y = _double(((ye << 20) | (ym >> 3)) << 32 | ((ym << 29) & 0xFFFFFFFF))
    y2 = y * y                                   # exact: y has 24 significant bits
    assert Fraction(y2) == Fraction(y) ** 2
    e = _fma(-x, y2, 1.0)
    ef = _approx_float_of(e)
    c2 = _double_of_nonneg_float(np.float32(np.float32(0.375) * ef) * ef)
    c = _fma(0.5, e, c2)
    return _fma(y, c, y)


@pytest.mark.parametrize("seed_rel", [-2.0 ** -21, 0.0, 2.0 ** -21])
def test_rsqrt_within_one_ulp(seed_rel):
    getcontext().prec = 60
    rng = random.Random(5)
    worst = 0.0
    for _ in range(3000):
        x = 10.0 ** rng.uniform(-300, 300) * rng.uniform(1, 10)
        got = rsqrt_model(x, seed_rel)
        ref = 1 / Decimal(x).sqrt()
        worst = max(worst, float(abs((Decimal(got) - ref) / ref)) / 2.0 ** -53)
    assert worst < 1.0, worst          # observed 0.98 units of 2^-53
