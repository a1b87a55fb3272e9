"""A model of the float filters of the MST builders (the Boruvka nearest-neighbour search
k_nfn, the Prim kernel's key intervals and the divide-and-conquer relaxations), checked
against the exact FP64 squared distance.

The search skips the exact distance of a candidate whose float lower bound exceeds a float
upper bound of the best distance so far. That is safe only if the lower bound never exceeds
the FP64 squared distance ((dx*dx + dy*dy) + dz*dz, each operation rounded) and the upper
bound never falls below it. This module restates the float steps with numpy float32 (and
exact rationals where a fused multiply-add may be contracted) and checks both bounds on
adversarial coordinates: large offsets with small separations, separations at float
rounding boundaries, tiny and subnormal values. CPU only.
"""
from fractions import Fraction

import numpy as np

F = np.float32


def _f32_of(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _err_bound(x, y, z):
    """Per-body error term: max |coordinate| 2^-23 + 1e-37 (as the float copies carry)."""
    m = np.maximum(np.abs(x), np.maximum(np.abs(y), np.abs(z)))
    return (m * F(2.0 ** -23) + F(1e-37)).astype(np.float32)


def _shrink(d, e):
    """max(fmaf(d, -2^-22, d) - e, 0): the fmaf is exact in float64, then rounded once."""
    t = (d.astype(np.float64) * (1.0 - 2.0 ** -22)).astype(np.float32)
    return np.maximum(t - e, F(0.0))


MARGIN = F(2.0 ** -144)   # absolute allowance for roundings below 2^-126 (<= 2^-150 each)


def _lower_plain(lx, ly, lz, margin=MARGIN):
    return np.maximum(((lx * lx + ly * ly) + lz * lz) * F(1.0 - 2.0 ** -20) - margin, F(0.0))


def _fma32(a, b, c):
    """fmaf: a*b + c rounded once (exact rationals, then float32)."""
    return F(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def _lower_fused(lx, ly, lz, margin=MARGIN):
    """The same with the additions contracted, as the compiler may do and as the
    divide-and-conquer builder writes it: s = fma(lz, lz, fma(ly, ly, lx*lx)), then
    fma(s, -2^-20, s) - margin."""
    out = np.empty(len(lx), np.float32)
    for k in range(len(lx)):
        s = _fma32(lz[k], lz[k], _fma32(ly[k], ly[k], lx[k] * lx[k]))
        out[k] = max(_fma32(s, F(-2.0 ** -20), s) - margin, F(0.0))
    return out


def _d2_exact(xi, yi, zi, xj, yj, zj):
    dx, dy, dz = xi - xj, yi - yj, zi - zj
    return (dx * dx + dy * dy) + dz * dz


def _cases(rng, n):
    """Body pairs (float64) of many kinds."""
    kinds = []
    base = rng.uniform(-1, 1, (n, 3)) * 10.0 ** rng.uniform(-30, 15, (n, 1))
    sep = rng.uniform(-1, 1, (n, 3)) * 10.0 ** rng.uniform(-40, 2, (n, 1)) * np.abs(base).max(axis=1, keepdims=True)
    kinds.append((base, base + sep))
    # separations of a few float ulps of large offsets
    off = rng.uniform(1e3, 1e14, (n, 3)) * rng.choice([-1, 1], (n, 3))
    ulp = np.spacing(off.astype(np.float32)).astype(np.float64)
    kinds.append((off, off + ulp * rng.integers(-3, 4, (n, 3)) + rng.uniform(-0.5, 0.5, (n, 3)) * ulp))
    # tiny and subnormal-in-float coordinates
    tiny = rng.uniform(-1, 1, (n, 3)) * 10.0 ** rng.uniform(-48, -30, (n, 1))
    kinds.append((tiny, tiny * rng.uniform(0.5, 1.5, (n, 3))))
    # equal floats but different doubles
    v = rng.uniform(-1, 1, (n, 3)) * 1e6
    kinds.append((v, v + np.spacing(v) * rng.integers(1, 50, (n, 3))))
    return kinds


def test_float_lower_bound_never_exceeds_the_fp64_distance():
    rng = np.random.default_rng(11)
    for ri, rj in _cases(rng, 20000):
        fi, fj = _f32_of(ri), _f32_of(rj)
        ei = _err_bound(fi[:, 0], fi[:, 1], fi[:, 2])
        ej = _err_bound(fj[:, 0], fj[:, 1], fj[:, 2])
        e = ei + ej
        lx, ly, lz = (_shrink(np.abs(fi[:, c] - fj[:, c]), e) for c in range(3))
        d = _d2_exact(ri[:, 0], ri[:, 1], ri[:, 2], rj[:, 0], rj[:, 1], rj[:, 2])
        lo = _lower_plain(lx, ly, lz).astype(np.float64)
        assert np.all(lo <= d), (lo[lo > d][:4], d[lo > d][:4])
        sub = np.flatnonzero(d < 1e-36)[:300]          # the subnormal-square regime
        sub = np.concatenate([sub, np.arange(200)])
        lo_f = _lower_fused(lx[sub], ly[sub], lz[sub]).astype(np.float64)
        assert np.all(lo_f <= d[sub])


def test_the_absolute_margin_is_needed():
    """Without the 2^-144 the bound exceeds the distance in the subnormal-square regime (and
    even the distance rounded up to a float, which the search compares with): squares and
    sums below 2^-126 round by up to 2^-150 in absolute terms, which no relative factor
    covers. Separations below ~1e-19 with coordinates below ~1e-4 reach that regime."""
    rng = np.random.default_rng(11)
    ri, rj = _cases(rng, 20000)[0]
    fi, fj = _f32_of(ri), _f32_of(rj)
    e = _err_bound(fi[:, 0], fi[:, 1], fi[:, 2]) + _err_bound(fj[:, 0], fj[:, 1], fj[:, 2])
    lx, ly, lz = (_shrink(np.abs(fi[:, c] - fj[:, c]), e) for c in range(3))
    d = _d2_exact(ri[:, 0], ri[:, 1], ri[:, 2], rj[:, 0], rj[:, 1], rj[:, 2])
    f = d.astype(np.float32)
    d_up = np.where(f.astype(np.float64) < d, np.nextafter(f, np.float32(np.inf)), f)
    lo0 = _lower_plain(lx, ly, lz, margin=F(0.0))
    bad = lo0 > d_up
    assert bad.any() and np.all(d[bad] < 1e-36)


def test_float_upper_bound_of_the_best_distance():
    """bhi = float(d) rounded up, times (1 + 2^-20), is never below d; with the lower bound
    this makes a skipped candidate strictly farther than the best one."""
    rng = np.random.default_rng(12)
    d = 10.0 ** rng.uniform(-60, 30, 100000)
    f = d.astype(np.float32)
    up = np.where(f.astype(np.float64) < d, np.nextafter(f, np.float32(np.inf)), f)
    bhi = (up * F(1.0 + 2.0 ** -20)).astype(np.float64)
    assert np.all(bhi >= d)


def test_the_filter_is_not_vacuous():
    """Well separated pairs get a positive lower bound within 1e-5 of the distance."""
    rng = np.random.default_rng(13)
    ri = rng.uniform(-1, 1, (1000, 3))
    rj = rng.uniform(-1, 1, (1000, 3))
    fi, fj = _f32_of(ri), _f32_of(rj)
    e = _err_bound(fi[:, 0], fi[:, 1], fi[:, 2]) + _err_bound(fj[:, 0], fj[:, 1], fj[:, 2])
    lx, ly, lz = (_shrink(np.abs(fi[:, c] - fj[:, c]), e) for c in range(3))
    d = _d2_exact(ri[:, 0], ri[:, 1], ri[:, 2], rj[:, 0], rj[:, 1], rj[:, 2])
    lo = _lower_plain(lx, ly, lz).astype(np.float64)
    ok = d > 1e-2
    assert np.all(lo[ok] > d[ok] * (1 - 1e-5))


def _prim_terms(fi, fj):
    """The Prim kernel's per-pair float terms: |differences|, their error radii
    (|x_u| + |x_w| + |dx|) 2^-23 + 1e-37, and the bodies' own radii max|x| 2^-23 + 1e-37."""
    ad = np.abs(fi - fj)
    ex = ((np.abs(fi) + np.abs(fj)) + ad) * F(2.0 ** -23) + F(1e-37)
    eu = _err_bound(fi[:, 0], fi[:, 1], fi[:, 2])
    ew = _err_bound(fj[:, 0], fj[:, 1], fj[:, 2])
    return ad, ex.astype(np.float32), eu, ew


def test_prim_key_interval_and_quick_test():
    """The Prim kernel's interval [lo, hi] of a squared distance holds the FP64 value (hi is
    used only above 1e-30), and its quick test on the largest coordinate difference,
    fmaf(a, -2^-22, a) - (e_u + e_w), never exceeds the FP64 distance itself."""
    rng = np.random.default_rng(21)
    for ri, rj in _cases(rng, 20000):
        fi, fj = _f32_of(ri), _f32_of(rj)
        ad, ex, eu, ew = _prim_terms(fi, fj)
        l = np.maximum(ad - ex, F(0.0))
        h = ad + ex
        lo = np.maximum(((l[:, 0] * l[:, 0] + l[:, 1] * l[:, 1]) + l[:, 2] * l[:, 2]) * F(1.0 - 2.0 ** -20)
                        - MARGIN, F(0.0)).astype(np.float64)
        hi = (((h[:, 0] * h[:, 0] + h[:, 1] * h[:, 1]) + h[:, 2] * h[:, 2]) * F(1.0 + 2.0 ** -20)).astype(np.float64)
        d = _d2_exact(ri[:, 0], ri[:, 1], ri[:, 2], rj[:, 0], rj[:, 1], rj[:, 2])
        assert np.all(lo <= d)
        used = hi >= 1e-30
        assert np.all(hi[used] >= d[used])
        a = ad.max(axis=1)
        quick = ((a.astype(np.float64) * (1.0 - 2.0 ** -22)).astype(np.float32) - (eu + ew)).astype(np.float64)
        assert np.all(quick <= np.sqrt(d) * (1 + 2.0 ** -50))


def _grow(d, e):
    """fmaf(d, 2^-22, d) + e: the fmaf is exact in float64, then rounded once; then the sum."""
    t = (d.astype(np.float64) * (1.0 + 2.0 ** -22)).astype(np.float32)
    return (t + e).astype(np.float32)


def _upper_plain(hx, hy, hz):
    return (((hx * hx + hy * hy) + hz * hz) * F(1.0 + 2.0 ** -20) + MARGIN).astype(np.float32)


def _upper_fused(hx, hy, hz):
    """The upper bound with the additions contracted (fma(hz, hz, fma(hy, hy, hx*hx)), then
    fma(s, 2^-20, s) + margin), as the compiler may emit it."""
    out = np.empty(len(hx), np.float32)
    for k in range(len(hx)):
        s = _fma32(hz[k], hz[k], _fma32(hy[k], hy[k], hx[k] * hx[k]))
        out[k] = _fma32(s, F(2.0 ** -20), s) + MARGIN
    return out


def test_nearest_neighbour_upper_bound_never_falls_below_the_fp64_distance():
    """k_nfn's first step takes the least float upper bound over a vertex's candidates and
    lists only the candidates whose lower bound does not exceed it: safe only if the upper
    bound is never below the FP64 squared distance (overflow gives inf, which is safe)."""
    rng = np.random.default_rng(31)
    with np.errstate(over="ignore"):
        for ri, rj in _cases(rng, 20000):
            fi, fj = _f32_of(ri), _f32_of(rj)
            e = _err_bound(fi[:, 0], fi[:, 1], fi[:, 2]) + _err_bound(fj[:, 0], fj[:, 1], fj[:, 2])
            hx, hy, hz = (_grow(np.abs(fi[:, c] - fj[:, c]), e) for c in range(3))
            d = _d2_exact(ri[:, 0], ri[:, 1], ri[:, 2], rj[:, 0], rj[:, 1], rj[:, 2])
            hi = _upper_plain(hx, hy, hz).astype(np.float64)
            assert np.all(hi >= d), (hi[hi < d][:4], d[hi < d][:4])
            sub = np.concatenate([np.flatnonzero(d < 1e-36)[:300], np.arange(300)])
            hf = _upper_fused(hx[sub], hy[sub], hz[sub]).astype(np.float64)
            assert np.all(hf >= d[sub])


def test_nearest_neighbour_bounds_are_tight():
    """For well separated pairs the upper bound is within 1e-5 of the distance, so the listed
    candidates are those within about 1e-5 of the nearest."""
    rng = np.random.default_rng(32)
    ri = rng.uniform(-1, 1, (1000, 3))
    rj = rng.uniform(-1, 1, (1000, 3))
    fi, fj = _f32_of(ri), _f32_of(rj)
    e = _err_bound(fi[:, 0], fi[:, 1], fi[:, 2]) + _err_bound(fj[:, 0], fj[:, 1], fj[:, 2])
    hx, hy, hz = (_grow(np.abs(fi[:, c] - fj[:, c]), e) for c in range(3))
    d = _d2_exact(ri[:, 0], ri[:, 1], ri[:, 2], rj[:, 0], rj[:, 1], rj[:, 2])
    hi = _upper_plain(hx, hy, hz).astype(np.float64)
    ok = d > 1e-2
    assert np.all(hi[ok] < d[ok] * (1 + 1e-5))
