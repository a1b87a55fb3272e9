"""Pins of the GBS error norm (Eq. gbs-criterion, readings R6-R8) on hand-worked cases.

The criterion compares the change between the last two extrapolants, dS = T_kk - T_{k-1,k-1},
with the state advanced by one substep delta = H/n_kfix along its derivative at the step
start, S(s0) + delta S'(s0), per 3-vector in the Euclidean norm. In the LogH equations
(Sec. 2.1) S' is V/(T+B) for an edge vector X, A/U for an edge velocity V and 1/(T+B) for t.

Every case below uses the same step-start state of a three-body tree 0 <- 1 <- 2 (root 0),
with k_fix = 8 (n_kfix = 16), H = 8, so delta = 1/2, and T0 = 1/2, B = 3/2 (T0 + B = 2),
U0 = 4, t0 = 1:

  edge 1: X0 = (1, 2, 4),  V0 = (4, 4, 8),  A0 = (-16, 16, 8)
          X0 + delta V0/(T0+B) = (1, 2, 4) + (1, 1, 2)  = (2, 3, 6), norm 7
          V0 + delta A0/U0     = (4, 4, 8) + (-2, 2, 1) = (2, 6, 9), norm 11
  edge 2: X0 = (0, 4, 8),  V0 = (4, 0, 0),  A0 = (0, 32, 56)
          X0 + delta V0/(T0+B) = (1, 4, 8), norm 9
          V0 + delta A0/U0     = (4, 4, 7), norm 9
  time:   t0 + delta/(T0+B)    = 1 + 1/4 = 5/4

The differences dS are planted as integer vectors with integer norms ((1,2,2): 3, (2,3,6): 7,
(3,4,12): 13, (2,10,11): 15) times s = 2^-30, on top of extrapolants near 100 (not near the
start state, so that a derivative taken from the extrapolants instead of the step start shows),
and the root's entries carry large differences that must be skipped. Each case makes a
different ratio the largest, so that each of these slips changes eps: a dropped delta S' term,
S' taken at the end of the step, A0 not divided by U0, the drift rate without B, the substep of
the first division (H/2) in place of the last (H/16), a 1-norm in place of the 2-norm, a sum
of the ratios in place of their maximum, the root included, a wrong sign of delta S'.
"""
import math

import numpy as np
import pytest

import oracle as O

S_UNIT = 2.0 ** -30
PARENT = [-1, 0, 1]
X0 = np.array([[0, 0, 0], [1, 2, 4], [0, 4, 8]], float)
V0 = np.array([[0, 0, 0], [4, 4, 8], [4, 0, 0]], float)
A0 = np.array([[0, 0, 0], [-16, 16, 8], [0, 32, 56]], float)
T0, B, U0, t0, H, KFIX = 0.5, 1.5, 4.0, 1.0, 8.0, 8


def extrapolants(dX, dV, dt, root=(1000.0, 1000.0, 1000.0)):
    """Tprev near 100 and Tkk = Tprev + the planted differences (exact in binary64)."""
    n = 3
    Tprev = 100.0 + 3.0 * np.arange(6 * n + 1)
    d = np.zeros(6 * n + 1)
    d[0:3] = root
    d[9:12] = root
    for v, x in dX.items():
        d[3 * v:3 * v + 3] = np.asarray(x, float) * S_UNIT
    for v, x in dV.items():
        d[9 + 3 * v:9 + 3 * v + 3] = np.asarray(x, float) * S_UNIT
    d[18] = dt * S_UNIT
    Tkk = Tprev + d
    assert np.array_equal(Tkk - Tprev, d, equal_nan=True)
    return Tkk, Tprev


def eps_of(Tkk, Tprev, x0=X0, v0=V0, a0=A0):
    return O.gbs_error(PARENT, Tkk, Tprev, x0, v0, a0, t0, T0, B, U0, H, KFIX)


BASE_X = {1: (1, 2, 2), 2: (1, 2, 2)}     # 3s/7 and 3s/9
BASE_V = {1: (1, 2, 2), 2: (1, 2, 2)}     # 3s/11 and 3s/9
BASE_T = 1.0                              # s/(5/4)


def test_denominators_by_hand():
    """The step-start denominators of the docstring, from the stated S' of Sec. 2.1."""
    delta = H / (2 * KFIX)
    assert delta == 0.5
    assert np.linalg.norm(X0[1] + delta * V0[1] / (T0 + B)) == 7.0
    assert np.linalg.norm(V0[1] + delta * A0[1] / U0) == 11.0
    assert np.linalg.norm(X0[2] + delta * V0[2] / (T0 + B)) == 9.0
    assert np.linalg.norm(V0[2] + delta * A0[2] / U0) == 9.0
    assert t0 + delta / (T0 + B) == 1.25


@pytest.mark.parametrize("case,dX,dV,dt,expected", [
    # edge 1 position: |(2,3,6)| s / 7 = s
    ("X1", {1: (2, 3, 6)}, {}, BASE_T, 1.0),
    # edge 1 velocity: |(3,4,12)| s / 11 = 13 s / 11
    ("V1", {}, {1: (3, 4, 12)}, BASE_T, 13.0 / 11.0),
    # edge 2 position: |(2,10,11)| s / 9 = 15 s / 9
    ("X2", {2: (2, 10, 11)}, {}, BASE_T, 15.0 / 9.0),
    # edge 2 velocity: |(3,4,12)| s / 9 = 13 s / 9
    ("V2", {}, {2: (3, 4, 12)}, BASE_T, 13.0 / 9.0),
    # time: 3 s / (5/4) = 12 s / 5
    ("t", {}, {}, 3.0, 12.0 / 5.0),
])
def test_each_term_by_hand(case, dX, dV, dt, expected):
    Tkk, Tprev = extrapolants({**BASE_X, **dX}, {**BASE_V, **dV}, dt)
    eps = eps_of(Tkk, Tprev)
    assert eps == pytest.approx(expected * S_UNIT, rel=4e-16), (case, eps / S_UNIT, expected)


def test_largest_ratio_not_largest_numerator():
    """The maximum is over the ratios, not the numerators. With dX2 = (2,3,6) s and
    dV1 = (3,4,12) s the ratios are 7/9 and 13/11, so eps = 13 s/11. With dV1 = (2,3,6) s
    instead, V1 and X2 have equal numerators (7 s) but V1's ratio is 7/11 and X2's 7/9 wins."""
    Tkk, Tprev = extrapolants({1: (1, 2, 2), 2: (2, 3, 6)}, {1: (3, 4, 12), 2: (1, 2, 2)}, 1.0)
    assert eps_of(Tkk, Tprev) == pytest.approx(13.0 / 11.0 * S_UNIT, rel=4e-16)
    Tkk, Tprev = extrapolants({1: (1, 2, 2), 2: (2, 3, 6)}, {1: (2, 3, 6), 2: (1, 2, 2)}, 0.0)
    assert eps_of(Tkk, Tprev) == pytest.approx(7.0 / 9.0 * S_UNIT, rel=4e-16)


def test_root_is_skipped_even_when_not_a_number():
    """The root has no edge: its entries (here 1000 and then NaN) never enter eps."""
    Tkk, Tprev = extrapolants({1: (2, 3, 6)}, {}, 1.0, root=(math.nan, 1000.0, 1000.0))
    assert eps_of(Tkk, Tprev) == pytest.approx(S_UNIT, rel=4e-16)


def test_zero_denominator_is_floored_not_nan():
    """An edge whose advanced start state is exactly zero: X0 = (-1, 0, 0), V0 = (4, 0, 0) give
    X0 + delta V0/(T0+B) = 0. With no change there the ratio is 0/1e-300 = 0 (not 0/0); with a
    change s it is s/1e-300, finite and dominant."""
    x0 = X0.copy()
    x0[2] = (-1.0, 0.0, 0.0)
    Tkk, Tprev = extrapolants({1: (1, 2, 2), 2: (0, 0, 0)}, BASE_V, 1.0)
    assert eps_of(Tkk, Tprev, x0=x0) == pytest.approx(S_UNIT / 1.25, rel=4e-16)
    Tkk, Tprev = extrapolants({1: (1, 2, 2), 2: (1, 0, 0)}, BASE_V, 1.0)
    eps = eps_of(Tkk, Tprev, x0=x0)
    assert math.isfinite(eps) and eps == pytest.approx(S_UNIT / 1e-300, rel=4e-16)


def test_nan_ratio_makes_eps_nan():
    """A non-finite division result (R8): eps is NaN, so the step is rejected."""
    Tkk, Tprev = extrapolants(BASE_X, BASE_V, 1.0)
    Tkk[9 + 3 * 1 + 1] = math.nan
    assert math.isnan(eps_of(Tkk, Tprev))
    Tkk, Tprev = extrapolants(BASE_X, BASE_V, 1.0)
    Tkk[18] = math.inf
    Tprev[18] = math.inf
    assert math.isnan(eps_of(Tkk, Tprev))


def test_scaling_laws():
    """eps is linear in the planted differences and, for dt alone, scales as 1/(t0 + delta/(T0+B)):
    doubling H moves the time denominator from 5/4 to 3/2."""
    Tkk, Tprev = extrapolants({1: (0, 0, 0), 2: (0, 0, 0)}, {1: (0, 0, 0), 2: (0, 0, 0)}, 3.0)
    e1 = eps_of(Tkk, Tprev)
    e2 = O.gbs_error(PARENT, Tkk, Tprev, X0, V0, A0, t0, T0, B, U0, 2 * H, KFIX)
    assert e1 == pytest.approx(3 * S_UNIT / 1.25, rel=4e-16)
    assert e2 == pytest.approx(3 * S_UNIT / 1.5, rel=4e-16)
    e3 = O.gbs_error(PARENT, Tkk, Tprev, X0, V0, A0, t0, T0, B, U0, H, 4)  # delta = 1: 1 + 1/2
    assert e3 == pytest.approx(3 * S_UNIT / 1.5, rel=4e-16)
