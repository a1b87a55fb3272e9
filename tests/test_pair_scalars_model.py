"""A bit-level model of the integer-pipe pair scalars, checked against 60-digit arithmetic.

The pair kernels compute r^2, 1/r and m/r^3 from the binary64 significands in 64-bit
integer arithmetic (pair_scalars_core and u64_to_double in csrc/device.cuh), seeded by a
float reciprocal square root. This module restates those integer steps with Python
integers, replaces the hardware seed by a float32 of 1/sqrt perturbed by up to 2^-21
(the algorithm needs only |1 - r^2 y^2| < 2^-20), and bounds the error of each result
over separations from 1e-60 to 1e12 with any ratio of the components. It checks the
algorithm; the GPU tests check the device code against the oracle. CPU only.
"""
import math
import random
import struct
from decimal import Decimal, getcontext

import numpy as np
import pytest

M64 = (1 << 64) - 1


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _fbits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _float(b):
    return struct.unpack("<f", struct.pack("<I", b))[0]


def _sig(x):
    """(biased exponent, significand with the hidden bit) of |x|; (0, 0) for zero."""
    b = _bits(x) & ~(1 << 63)
    e = b >> 52
    return (e, (b & ((1 << 52) - 1)) | (1 << 52)) if e else (0, 0)


def _umulhi(a, b):
    return (a * b) >> 64


def _to_double(Sn, e2):
    """Sn 2^e2, Sn in [2^63, 2^64), to the nearest double (ties up), as u64_to_double."""
    mant = (Sn >> 11) + ((Sn >> 10) & 1)
    ex = e2 + 11
    if mant >> 53:
        mant >>= 1
        ex += 1
    return math.ldexp(mant, ex)


def _mass(x):
    e, m = _sig(x)
    return m << 11, e - 1075 - 11


def pair_scalars_model(dx, dy, dz, mi, mj, seed_rel):
    """(1/r, m_j/r^3, m_i/r^3) by the integer steps of pair_scalars_core."""
    comps = [_sig(d) for d in (dx, dy, dz)]
    E = max(e for e, _ in comps)
    F = 0
    for e, m in comps:
        sh = 2 + 2 * (E - e)
        T = (m * m) >> 42                           # (m^2 >> 42), m < 2^53
        F += (T >> sh) if (e and sh < 64) else 0
    assert 0 < F < (1 << 64)
    z = 64 - F.bit_length()
    M = F << z                                      # r^2 = (M / 2^63) 2^Er
    Er = 2 * E - 2043 - z
    k, p = Er >> 1, Er & 1
    mx = _float(((127 + p) << 23) | ((M >> 40) & 0x7FFFFF))
    yf = float(np.float32(1.0 / math.sqrt(mx) * (1.0 + seed_rel)))
    yb = _fbits(yf)
    eyf = (yb >> 23) & 0xFF
    myf = (yb & 0x7FFFFF) | 0x800000
    Y2 = myf * myf
    sh = 301 - p - 2 * eyf
    Pfix = ((M * Y2) >> sh) & M64
    efix = (1 << 62) - Pfix                         # e 2^62 (signed)
    et = efix >> 20
    cfix = (efix >> 1) + ((3 * et * et) >> 25)
    Rm = (1 << 62) + cfix
    R = myf * Rm                                    # < 2^87
    Rh = R >> 64
    zR = 64 - Rh.bit_length()
    Rn = (R >> (64 - zR)) & M64                     # top 64 bits of R
    eR = 64 - zR + eyf - 212 - k                    # 1/r = Rn 2^eR
    R2 = _umulhi(Rn, Rn)
    R3 = _umulhi(R2, Rn)
    out = [_to_double(Rn, eR)]
    for mass in (mj, mi):
        mm, me = _mass(mass)
        S = _umulhi(mm, R3)
        zs = 64 - S.bit_length()
        out.append(_to_double((S << zs) & M64, me + 3 * eR + 192 - zs))
    return out


def _exact(dx, dy, dz, mi, mj):
    getcontext().prec = 60
    r2 = Decimal(dx) ** 2 + Decimal(dy) ** 2 + Decimal(dz) ** 2
    rinv = 1 / r2.sqrt()
    return rinv, Decimal(mj) * rinv ** 3, Decimal(mi) * rinv ** 3


@pytest.mark.parametrize("seed_rel", [-2.0 ** -21, 0.0, 2.0 ** -21])
def test_integer_pair_scalars_within_one_ulp(seed_rel):
    rng = random.Random(7)
    worst = [0.0, 0.0, 0.0]
    for _ in range(1500):
        sc = 10.0 ** rng.uniform(-60, 12)
        comps = [rng.uniform(-1, 1) * sc * (10.0 ** rng.uniform(-8, 0) if rng.random() < 0.3 else 1.0)
                 for _ in range(3)]
        if rng.random() < 0.1:
            comps[rng.randrange(3)] = 0.0
        if all(c == 0.0 for c in comps):
            continue
        mi, mj = 10.0 ** rng.uniform(-6, 1), 10.0 ** rng.uniform(-6, 1)
        got = pair_scalars_model(*comps, mi, mj, seed_rel)
        ref = _exact(*comps, mi, mj)
        for q in range(3):
            rel = abs((Decimal(got[q]) - ref[q]) / ref[q])
            worst[q] = max(worst[q], float(rel) / 2.0 ** -53)
    # each result is rounded once from ~60 correct bits: within one unit of 2^-53
    assert max(worst) < 1.0, worst


def test_model_rejects_a_dropped_correction_term():
    """The model is sensitive to its own steps: without the 3e^2/8 term the error grows to
    ~2^-40 for the largest seed error."""
    dx, dy, dz, mi, mj = 0.37, -1.25, 0.5, 1.0, 2.0

    def without_e2(seed_rel):
        # the same steps with cfix = e/2 only
        comps = [_sig(d) for d in (dx, dy, dz)]
        E = max(e for e, _ in comps)
        F = sum(((m * m) >> 42) >> (2 + 2 * (E - e)) for e, m in comps)
        z = 64 - F.bit_length()
        M = F << z
        Er = 2 * E - 2043 - z
        k, p = Er >> 1, Er & 1
        yf = float(np.float32(1.0 / math.sqrt(_float(((127 + p) << 23) | ((M >> 40) & 0x7FFFFF))) * (1 + seed_rel)))
        yb = _fbits(yf)
        eyf, myf = (yb >> 23) & 0xFF, (yb & 0x7FFFFF) | 0x800000
        Pfix = ((M * myf * myf) >> (301 - p - 2 * eyf)) & M64
        efix = (1 << 62) - Pfix
        R = myf * ((1 << 62) + (efix >> 1))
        return R * 2.0 ** (eyf - 150 - 62 - k)

    exact = float(_exact(dx, dy, dz, mi, mj)[0])
    assert abs(without_e2(2.0 ** -21) / exact - 1) > 2.0 ** -45
    assert abs(pair_scalars_model(dx, dy, dz, mi, mj, 2.0 ** -21)[0] / exact - 1) < 2.0 ** -52
