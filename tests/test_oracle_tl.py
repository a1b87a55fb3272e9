"""Pins of the oracle's fixed-step run and its tangent-linear (forward-mode derivative).

The tangent-linear is written from the Cartesian LogH equations (Sec. 2.1-2.2) with
Aitken-Neville extrapolation (Sec. 4.2); it is pinned here against facts that do not come
from itself:
- central finite differences (h = 1e-6) of the oracle's MST-coordinate fixed-step run;
- translation invariance: shifting every initial position (or velocity) by one vector
  changes nothing after the centre-of-mass shift, so the tangent of the final state is 0;
- rotation equivariance: the dynamics and the MST commute with rotations, so an
  infinitesimal rotation of the initial state rotates the final state, d r_f = W x r_f,
  d v_f = W x v_f, and leaves the energy unchanged;
- its primal equals the MST-coordinate run (the two forms agree in real arithmetic).
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_03180_gb300 import workloads as W

N, STEPS = 16, 5


@pytest.fixture(scope="module")
def case():
    m, r, v = W.plummer(N, 7)
    # off the centre-of-mass frame, so that the initial shift (and its mass tangent) acts
    r = r + np.array([0.4, -0.3, 0.2])
    v = v + np.array([0.1, 0.05, -0.2])
    U = O.potential(m, O.com_shift(m, r))
    H = 0.02 * U
    st = W.Stream(99, 1)
    w = dict(r=(st.uniform(3 * N) - 0.5).reshape(N, 3), v=(st.uniform(3 * N) - 0.5).reshape(N, 3), E=0.7)
    return m, r, v, H, w, st


def loss_of(m, r, v, H, w):
    s = O.System(m, r, v)
    s.fixed_run(H, STEPS)
    S = s.state()
    return float((w["r"] * S["r"]).sum() + (w["v"] * S["v"]).sum() + w["E"] * s.energy()["E"])


@pytest.mark.parametrize("which", ["r", "v", "m", "all"])
def test_tl_matches_central_differences(case, which):
    m, r, v, H, w, st = case
    dm = (st.uniform(N) - 0.5) * 0.1 * m if which in ("m", "all") else np.zeros(N)
    dr = (st.uniform(3 * N) - 0.5).reshape(N, 3) if which in ("r", "all") else np.zeros((N, 3))
    dv = (st.uniform(3 * N) - 0.5).reshape(N, 3) if which in ("v", "all") else np.zeros((N, 3))
    tl = O.fixed_run_tl(m, r, v, dm, dr, dv, H, STEPS)
    dL = float((w["r"] * tl["dr"]).sum() + (w["v"] * tl["dv"]).sum() + w["E"] * tl["dE"])
    h = 1e-6
    fd = (loss_of(m + h * dm, r + h * dr, v + h * dv, H, w) - loss_of(m - h * dm, r - h * dr, v - h * dv, H, w)) / (2 * h)
    assert abs(dL - fd) <= 1e-5 * abs(fd), (dL, fd)


def test_tl_translation_invariance(case):
    m, r, v, H, w, st = case
    c = np.array([0.3, -0.2, 0.5])
    for dr, dv in [(np.tile(c, (N, 1)), np.zeros((N, 3))), (np.zeros((N, 3)), np.tile(c, (N, 1)))]:
        tl = O.fixed_run_tl(m, r, v, np.zeros(N), dr, dv, H, STEPS)
        assert np.abs(tl["dr"]).max() < 1e-13 and np.abs(tl["dv"]).max() < 1e-13
        assert abs(tl["dE"]) < 1e-13


def test_tl_rotation_equivariance(case):
    m, r, v, H, w, st = case
    Om = np.array([0.2, 0.7, -0.4])
    tl = O.fixed_run_tl(m, r, v, np.zeros(N), np.cross(Om, r), np.cross(Om, v), H, STEPS)
    er = np.abs(tl["dr"] - np.cross(Om, tl["r"])).max() / np.abs(tl["dr"]).max()
    ev = np.abs(tl["dv"] - np.cross(Om, tl["v"])).max() / np.abs(tl["dv"]).max()
    assert er < 1e-11 and ev < 1e-11
    assert abs(tl["dE"]) < 1e-12


def test_tl_primal_equals_mst_run(case):
    m, r, v, H, w, st = case
    tl = O.fixed_run_tl(m, r, v, np.zeros(N), np.zeros((N, 3)), np.zeros((N, 3)), H, STEPS)
    s = O.System(m, r, v)
    s.fixed_run(H, STEPS)
    S = s.state()
    assert np.abs(tl["r"] - S["r"]).max() <= 1e-12 * np.abs(S["r"]).max()
    assert np.abs(tl["v"] - S["v"]).max() <= 1e-12 * np.abs(S["v"]).max()
    assert abs(tl["E"] - s.energy()["E"]) <= 1e-12 * abs(tl["E"])
    assert np.abs(tl["dr"]).max() == 0.0 and tl["dE"] == 0.0
