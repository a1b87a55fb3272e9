"""Pins of the CPU oracle to facts the paper and the mathematics fix (no GPU).

Each test names the passage it follows. A plausible slip in the oracle (a dropped term,
a wrong sign, index or operand order) should fail at least one of these.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2001_03180_gb300 import workloads as W
from tests import helpers as Hh
from tests.helpers import golden


def rand_points(n, seed):
    st = W.Stream(seed, 99)
    return (st.uniform(3 * n).reshape(n, 3) - 0.5) * 2.0


# ----------------------------------------------------------------- MST (Sec. 3.1-3.4)

@pytest.mark.parametrize("n,seed", [(3, 1), (4, 2), (5, 3), (6, 4), (7, 5), (7, 6)])
def test_prim_equals_bruteforce_mst(n, seed):
    """Sec. 3.1: distinct weights give a unique MST; Prim must find the lightest of all
    N^(N-2) spanning trees."""
    r = rand_points(n, seed)
    r = r - r.mean(0)
    root, parent, level, order = O.prim(r)
    assert Hh.edge_set(parent) == Hh.mst_bruteforce(r)


@pytest.mark.parametrize("n,seed", [(50, 1), (200, 2), (500, 3)])
def test_prim_equals_kruskal(n, seed):
    r = rand_points(n, seed)
    root, parent, level, order = O.prim(r - r.mean(0))
    assert Hh.edge_set(parent) == Hh.mst_kruskal(r - r.mean(0))


def test_prim_cut_and_cycle_properties():
    """Sec. 3.1: every tree edge is the lightest edge across the cut it defines; every
    non-tree edge is the heaviest on the cycle it closes."""
    n = 80
    r = rand_points(n, 11)
    r = r - r.mean(0)
    root, parent, level, order = O.prim(r)
    d2 = ((r[:, None, :] - r[None, :, :]) ** 2).sum(-1)
    for v in range(n):
        p = parent[v]
        if p < 0:
            continue
        # component of v after removing edge (v, p): v's subtree
        sub = {v}
        changed = True
        while changed:
            changed = False
            for u in range(n):
                if u not in sub and parent[u] in sub:
                    sub.add(u)
                    changed = True
        inside = np.array(sorted(sub))
        outside = np.array([u for u in range(n) if u not in sub])
        assert d2[np.ix_(inside, outside)].min() == d2[v, p]
    for i in range(0, n, 7):
        for j in range(i + 1, n, 5):
            if parent[i] == j or parent[j] == i:
                continue
            path = Hh.tree_path(parent, i, j)
            wmax = max(d2[path[k], path[k + 1]] for k in range(len(path) - 1))
            assert d2[i, j] >= wmax


def test_prim_indexing_rules():
    """Sec. 3.4: root at level 0, closest to the COM; vertices indexed in insertion order;
    each parent inserted before its child; level = parent's level + 1."""
    m, r, v = W.plummer(300, 7)
    root, parent, level, order = O.prim(r)
    assert root == int(np.argmin((r * r).sum(1)))
    assert parent[root] == -1 and level[root] == 0 and order[0] == root
    assert sorted(order) == list(range(300))
    pos = {int(u): k for k, u in enumerate(order)}
    for u in range(300):
        if u != root:
            assert pos[int(parent[u])] < pos[u]
            assert level[u] == level[parent[u]] + 1


def test_prim_ties_hand_computed():
    """Square with equal edges: root = lowest index among equidistant; argmin ties go to the
    lowest index; a key is only replaced by a strictly smaller weight."""
    r = np.array([[1.0, 1.0, 0.0], [-1.0, 1.0, 0.0], [-1.0, -1.0, 0.0], [1.0, -1.0, 0.0]])
    root, parent, level, order = O.prim(r)
    assert root == 0
    assert list(parent) == [-1, 0, 1, 0]
    assert list(order) == [0, 1, 2, 3]
    assert list(level) == [0, 1, 2, 1]


def test_mst_shallower_than_chain():
    """Sec. 3.5 / Fig. mean_L: with a root near the COM, <L_MST> is below the chain's
    (N-1)/2 by a factor of a few for N = 10..1000."""
    for n, seed in [(30, 1), (300, 2), (1000, 3)]:
        m, r, v = W.plummer(n, seed)
        _, parent, level, _ = O.prim(r)
        ratio = ((n - 1) / 2) / level.mean()
        assert 1.5 < ratio < 50, ratio


# ----------------------------------------------------------------- near rule (Eq. LCA)

@pytest.mark.parametrize("n_d", [1, 2, 3])
def test_near_rule_equals_tree_distance(n_d):
    m, r, v = W.plummer(120, 3)
    _, parent, level, _ = O.prim(r)
    for i in range(120):
        dist = Hh.tree_distance_bfs(parent, i)
        for j in range(120):
            if j != i:
                assert O.is_near(parent, level, i, j, n_d) == (dist[j] <= n_d)


def test_near_rule_nd2_is_parent_grandparent_sibling():
    """For N_d = 2 the LCA rule reduces to: parent, grandparent, child, grandchild, sibling."""
    m, r, v = W.plummer(150, 4)
    _, parent, level, _ = O.prim(r)
    gp = [parent[p] if p >= 0 else -1 for p in parent]
    for i in range(150):
        for j in range(150):
            if i == j:
                continue
            rule = (parent[i] == j or gp[i] == j or parent[j] == i or gp[j] == i
                    or (parent[i] == parent[j] and parent[i] >= 0))
            assert O.is_near(parent, level, i, j, 2) == rule


def test_near_separation_exact_on_integer_lattice():
    """Walking the tree over edge vectors reproduces r_j - r_i exactly when all
    coordinates are small integers (every sum is exact)."""
    st = W.Stream(5, 1)
    r = np.floor(st.uniform(3 * 60).reshape(60, 3) * 1000.0) - 500.0
    _, parent, level, _ = O.prim(r - r.mean(0))
    X = O.to_mst(parent, r)
    for i in range(60):
        for j in range(60):
            if i != j and O.is_near(parent, level, i, j, 3):
                assert np.array_equal(O.near_sep(parent, level, X, i, j), r[j] - r[i])


# ----------------------------------------------------------------- transforms (Sec. 3.5)

def test_round_trip_mst_coordinates():
    """Build then deconstruct: r -> X -> r within <L>-scaled rounding (Sec. 3.5)."""
    m, r, v = W.plummer(1000, 9)
    _, parent, level, _ = O.prim(r)
    X = O.to_mst(parent, r)
    back = O.from_mst(m, parent, X)
    ref = O.com_shift(m, r)
    tol = 4 * level.max() * np.finfo(float).eps * np.abs(r).max()
    assert np.abs(back - ref).max() <= tol


def test_round_trip_exact_on_dyadic_grid():
    st = W.Stream(6, 2)
    n = 64
    r = (np.floor(st.uniform(3 * n).reshape(n, 3) * 64.0) - 32.0) / 8.0
    m = np.full(n, 1.0 / 64)
    r = r - r.mean(0)  # mean of multiples of 1/8 over 64 points is exact
    _, parent, level, _ = O.prim(r)
    back = O.from_mst(m, parent, O.to_mst(parent, r))
    assert np.array_equal(back, r)


# ----------------------------------------------------------------- forces (Eq. 1-2)

def test_forces_are_gradient_of_force_function():
    """m_i a_i = dU/dr_i (U is the negative potential energy, Eq. 1-2); checked by central
    differences of the Cartesian U."""
    m, r, v = W.plummer(40, 12)
    _, parent, level, _ = O.prim(r)
    X = O.to_mst(parent, r)
    a, U = O.forces(m, r, parent, level, X, n_d=2)
    h = 1e-6
    for i in [0, 7, 19, 33]:
        for k in range(3):
            rp = r.copy(); rp[i, k] += h
            rm = r.copy(); rm[i, k] -= h
            g = (O.potential(m, rp) - O.potential(m, rm)) / (2 * h)
            assert abs(m[i] * a[i, k] - g) <= 1e-7 * max(1.0, abs(g))
    assert abs(U - O.potential(m, r)) <= 1e-13 * U


def test_two_body_force_closed_form():
    m = np.array([2.0, 3.0])
    r = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    _, parent, level, _ = O.prim(r - (m[:, None] * r).sum(0) / 5.0)
    X = O.to_mst(parent, r)
    a, U = O.forces(m, r, parent, level, X, n_d=2, G=2.0)
    # |d| = 5: a_0 = G m_1 d/125, a_1 = -G m_0 d/125, U = G m0 m1 / 5
    d = np.array([3.0, 4.0, 0.0])
    assert np.allclose(a[0], 2.0 * 3.0 * d / 125.0, rtol=0, atol=1e-16)
    assert np.allclose(a[1], -2.0 * 2.0 * d / 125.0, rtol=0, atol=1e-16)
    assert U == pytest.approx(2.0 * 6.0 / 5.0, rel=1e-16)


def test_kinetic_and_potential_closed_forms():
    """Sec. 2.1: T = sum m v^2 / 2 and U = sum_{i<j} G m_i m_j / r_ij, on configurations
    with exact values: three bodies on a 3-4-5 triangle (U = G (m0 m1/5 + m0 m2/3 + m1 m2/4))
    and velocities of integer components; the system's E = T - U and zero P, L at rest."""
    m = np.array([2.0, 3.0, 4.0])
    r = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [3.0, 0.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, -2.0, 0.0], [0.0, 0.0, 3.0]])
    assert O.kinetic(m, v) == 0.5 * (2.0 * 1.0 + 3.0 * 4.0 + 4.0 * 9.0)
    assert O.potential(m, r, G=1.5) == pytest.approx(1.5 * (6.0 / 5.0 + 8.0 / 3.0 + 12.0 / 4.0), rel=1e-15)
    e = O.System(m, r, np.zeros_like(v)).energy()
    assert e["E"] == pytest.approx(-(6.0 / 5.0 + 8.0 / 3.0 + 12.0 / 4.0), rel=1e-15)
    assert np.abs(e["P"]).max() == 0.0 and np.abs(e["L"]).max() == 0.0


def test_forces_newton_third_law_and_near_rule_consistency():
    m, r, v = W.plummer_smbh_binary(300, 2)
    _, parent, level, _ = O.prim(r)
    X = O.to_mst(parent, r)
    a2, U2 = O.forces(m, r, parent, level, X, n_d=2)
    a0, U0 = O.forces(m, r, parent, level, X, n_d=0)
    scale = np.abs(m[:, None] * a2).max()
    assert np.abs((m[:, None] * a2).sum(0)).max() <= 1e-12 * scale
    # the near-pair formula changes only rounding for a generic configuration
    assert np.abs(a2 - a0).max() <= 1e-10 * np.abs(a0).max()
    assert abs(U2 - U0) <= 1e-12 * U0


# ----------------------------------------------------------------- GBS pieces (Sec. 2.3, 4.2)

@pytest.mark.parametrize("kf", [2, 4, 8])
def test_neville_exact_on_polynomials(kf):
    """Aitken-Neville extrapolation to x = h^2 -> 0 reproduces any polynomial of degree
    < k_fix in x exactly, and for x^k_fix gives (-1)^(k_fix+1) prod x_k (Lagrange remainder)."""
    nseq = np.array([2 * (k + 1) for k in range(kf)], np.int32)
    x = 1.0 / nseq.astype(float) ** 2
    st = W.Stream(kf, 3)
    coef = st.uniform(kf) - 0.5
    S = np.polyval(coef, x)  # degree kf-1, constant term coef[-1]
    Tkk, _ = O.neville(nseq, S[:, None])
    assert Tkk[0] == pytest.approx(coef[-1], abs=1e-13)
    Tkk, _ = O.neville(nseq, (x ** kf)[:, None])
    assert Tkk[0] == pytest.approx((-1) ** (kf + 1) * np.prod(x), rel=1e-10)


@pytest.mark.parametrize("kf", [2, 4, 8])
def test_neville_second_output_is_the_previous_diagonal(kf):
    """The convergence test compares successive extrapolants (Sec. 4.2, reading R7): the second
    output is T_{kf-1,kf-1}, the extrapolation from the first kf-1 divisions alone. For
    f = x^(kf-1), monic of degree kf-1 with kf-1 nodes x_1..x_{kf-1}, the interpolant's value at 0
    is f(0) - prod(0 - x_i) = (-1)^kf prod_{i<kf} x_i, while T_kk is exact (0). The other
    reading, T_{kf,kf-1} (nodes x_2..x_kf), would give (-1)^kf prod_{i>1} x_i instead."""
    nseq = np.array([2 * (k + 1) for k in range(kf)], np.int32)
    x = 1.0 / nseq.astype(float) ** 2
    Tkk, Tprev = O.neville(nseq, (x ** (kf - 1))[:, None])
    assert Tkk[0] == pytest.approx(0.0, abs=1e-15)
    want = (-1) ** kf * np.prod(x[:-1])
    other = (-1) ** kf * np.prod(x[1:])
    assert Tprev[0] == pytest.approx(want, rel=1e-10)
    assert abs(Tprev[0] - other) > 0.5 * abs(want - other)
    # a polynomial of degree < kf-1 is reproduced exactly by both diagonals
    st = W.Stream(kf, 4)
    coef = st.uniform(kf - 1) - 0.5
    Tkk, Tprev = O.neville(nseq, np.polyval(coef, x)[:, None])
    assert Tprev[0] == pytest.approx(coef[-1], abs=1e-13)


@pytest.mark.parametrize("kf", [2, 3])
def test_gbs_order_on_harmonic_oscillator(kf):
    """Even-power error expansion (Sec. 2.3): with k_fix divisions the extrapolated step has
    local error O(H^(2 k_fix + 1)); halving H divides the error by about 2^(2 k_fix + 1)."""
    errs = []
    for H in [0.4, 0.2]:
        out, _ = O.gbs_harmonic(1.0, 1.0, 0.0, H, kf)
        errs.append(math.hypot(out[0] - math.cos(H), out[1] + math.sin(H)))
    order = math.log2(errs[0] / errs[1])
    assert abs(order - (2 * kf + 1)) < 0.35, (errs, order)


def test_division_scheduler_speedups():
    """Eq. speedup-div: S_div = sum n_k / max C_i; N_div = k_fix gives (k_fix+1)/2 and
    N_div <= k_fix/2 gives N_div (Sec. 4.2, tests/golden/scheduler.txt)."""
    gd = golden("scheduler")
    for kf in [4, 6, 8, 10]:
        tot = kf * (kf + 1)
        mx, g = O.div_assign(kf, kf)
        assert tot / mx == (kf + gd["s_div_max_num"]) / 2
        for nd in range(1, kf // 2 + 1):
            mx, g = O.div_assign(kf, nd)
            assert tot / mx == pytest.approx(gd["s_div_slope"] * nd, rel=0.15)
        mx, g = O.div_assign(kf, kf // 2)
        assert tot / mx == kf / 2
        mx, g = O.div_assign(kf, 1)
        assert mx == tot and set(g) == {0}
    mx, g = O.div_assign(8, 4)
    assert list(g) == [0, 1, 2, 3, 3, 2, 1, 0]


# ----------------------------------------------------------------- Kepler (Sec. 2.1, 5.1)

def test_logh_leapfrog_kepler_orbit_exact():
    """Sec. 2.1: the LogH leapfrog gives the exact Keplerian orbit; only the time has an
    error. E, L and the Laplace-Runge-Lenz vector stay at rounding level over many large
    steps, without extrapolation."""
    m, r, v = W.kepler_binary(seed=3, e=0.9)
    E0, L0, A0 = Hh.two_body_invariants(m[0], m[1], r, v)
    s = O.System(m, r, v)
    B = s.state()["B"]
    t = 0.0
    for _ in range(400):
        out = s.leapfrog(4, 0.3 * B)  # large fictitious step, 4 substeps
        t = out["t"]
        s.set_state(t, out["r"], out["v"])
    S = s.state()
    E1, L1, A1 = Hh.two_body_invariants(m[0], m[1], S["r"], S["v"])
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.abs(L1 - L0).max() <= 1e-12 * np.linalg.norm(L0)
    assert np.abs(A1 - A0).max() <= 1e-11 * np.linalg.norm(A0)
    assert t > 10.0  # the orbit has gone round several times


@pytest.mark.parametrize("case", ["plummer64", "kepler", "plummer257"])
def test_gbs_step_reverses_within_its_error(case):
    """Sec. 2.1 / 2.3: the LogH leapfrog is time-symmetric, and extrapolating it in even powers
    of the substep keeps the symmetry up to the extrapolated step's own truncation error (a
    linear combination of symmetric maps is not exactly symmetric). So a step of H followed
    by one of -H from its result returns to the start within that error: the round trip
    misses by less than the step's error estimate eps, and by far less than the step moved.
    A first-order (non-symmetric) drift/kick split misses by O(H)."""
    if case == "plummer64":
        (m, r, v), H = W.workload("plummer64"), 0.05
    elif case == "kepler":
        (m, r, v), H = W.kepler_binary(seed=2, e=0.7), 0.3
    else:
        (m, r, v), H = W.plummer(257, 8), 0.015
    s = O.System(m, r, v)
    st0 = s.state()
    a = s.attempt(H)
    back = O.System(m, r, v)
    back.set_state(a["t"], a["r"], a["v"])
    b = back.attempt(-H)
    rel = lambda x, y: float(np.abs(x - y).max() / np.abs(y).max())  # noqa: E731
    moved = rel(a["r"], st0["r"])
    assert moved > 1e-4
    miss_r, miss_v = rel(b["r"], st0["r"]), rel(b["v"], st0["v"])
    assert miss_r < max(a["eps"], 1e-13) and miss_v < max(a["eps"], 1e-13), (miss_r, miss_v, a["eps"])
    assert miss_r < 1e-6 * moved
    assert abs(b["t"] - st0["t"]) <= max(a["eps"], 1e-13) * abs(a["t"])


@pytest.mark.parametrize("k_fix,H0", [(4, 0.25), (6, 0.5), (8, 1.0)])
def test_error_estimate_has_order_2kfix_minus_1(k_fix, H0):
    """Sec. 2.3 and Eq. hnext: with k_fix divisions the error estimate (the difference of the last
    two diagonal extrapolants) shrinks as H^(2 k_fix - 1), the order that Eq. hnext's exponent
    1/(2k - 1) assumes. On a circular Kepler orbit the local slope of log eps against log H,
    over H0 * 2^(-3/4 .. -1/4), is 2 k_fix - 1 to 0.25. A dropped or unsquared ratio in the
    tableau, a wrong division sequence or a first-order leapfrog changes the slope."""
    m, r, v = W.kepler_binary(seed=2, e=0.0)
    s = O.System(m, r, v, k_fix=k_fix)
    Hs = H0 * 2.0 ** (np.arange(-3, 0) / 4)
    eps = np.array([s.attempt(H)["eps"] for H in Hs])
    assert eps.max() < 1e-5 and eps.min() > 1e-12, eps
    slopes = np.diff(np.log(eps)) / np.diff(np.log(Hs))
    assert np.all(np.abs(slopes - (2 * k_fix - 1)) < 0.25), slopes


@pytest.mark.parametrize("k_fix,a_gbs,eta", [(8, 0.9, 1e-10), (8, 0.7, 1e-8), (6, 0.9, 1e-10), (4, 0.8, 1e-9)])
def test_step_control_settles_at_a_gbs_power(k_fix, a_gbs, eta):
    """Eq. hnext on an error estimate of order 2k - 1 (previous test): H_next = a (eta/eps)^(1/(2k-1)) H
    makes the next estimate a^(2k-1) eta whatever eps was, so after a few accepted steps (the first,
    from the q U dt guess of Sec. 2.4, is halved a few times) on a
    circular orbit (constant error constant) every eps is a_GBS^(2 k_fix - 1) eta. Observed to
    0.1 % from the fourth step; the test allows 1 %. An exponent of 1/(2k) would settle at
    a^(2k) eta (10 % lower at a = 0.9), a missing safety factor at eta itself."""
    m, r, v = W.kepler_binary(seed=2, e=0.0)
    s = O.System(m, r, v, eta=eta, k_fix=k_fix, a_gbs=a_gbs)
    ratios = []
    for i in range(8):
        rc, st = s.integrate(1e3, max_steps=1)
        assert rc == 0 and st["accepted"] == 1 and (i == 0 or st["rejected"] == 0)
        ratios.append(st["eps_last"] / eta)
    target = a_gbs ** (2 * k_fix - 1)
    assert np.all(np.abs(np.array(ratios[3:]) / target - 1) < 1e-2), (ratios, target)


def test_gbs_kepler_matches_analytic_solution():
    """A full run with GBS (eta = 1e-12) lands on the Kepler solution at the end time."""
    m, r, v = W.kepler_binary(seed=4, e=0.9)
    s = O.System(m, r, v, eta=1e-12)
    rc, st = s.integrate(5.0)
    assert rc == 0 and abs(st["t"] - 5.0) <= 1e-9
    S = s.state()
    dr, dv = Hh.kepler_propagate(r[1] - r[0], v[1] - v[0], m.sum(), S["t"])
    assert np.abs((S["r"][1] - S["r"][0]) - dr).max() <= 1e-9
    assert np.abs((S["v"][1] - S["v"][0]) - dv).max() <= 1e-8 * np.linalg.norm(dv)


# ----------------------------------------------------------------- conservation, driver

def test_plummer64_conservation_and_end_time():
    """Plummer N=64 to t=1 (eta=1e-12): |dE/E| in the 1e-14 regime (abstract), angular
    momentum conserved, the end time met to t_tol (Sec. 2.4)."""
    m, r, v = W.workload("plummer64")
    s = O.System(m, r, v)
    e0 = s.energy()
    rc, st = s.integrate(1.0)
    e1 = s.energy()
    assert rc == 0
    assert abs(st["t"] - 1.0) <= 1e-10
    assert abs((e1["E"] - e0["E"]) / e0["E"]) < 1e-13
    # the extrapolated state conserves the quadratic invariant L to about eta per step
    Lscale = float((m * np.linalg.norm(r, axis=1) * np.linalg.norm(v, axis=1)).sum())
    assert np.abs(e1["L"] - e0["L"]).max() < 1e-11 * Lscale
    assert np.abs(e1["P"]).max() < 1e-15
    assert st["accepted"] > 10


def test_pythagorean_three_body():
    """Sec. 5.2: the lightest body escapes; the remaining binary has a_23 ~ 5.5 pc for sides of
    30/40/50 pc (0.55 for sides 3/4/5) and e_23 ~ 0.99; escape angle ~ 71.4 deg."""
    m, r, v = W.pythagorean()
    s = O.System(m, r, v)
    rc, st = s.integrate(100.0)
    assert rc == 0
    S = s.state()
    dr = S["r"][2] - S["r"][1]
    dv = S["v"][2] - S["v"][1]
    M = m[1] + m[2]
    E = 0.5 * dv @ dv - M / np.linalg.norm(dr)
    a = -M / (2 * E)
    Lv = np.cross(dr, dv)
    e = math.sqrt(1 + 2 * E * (Lv @ Lv) / M ** 2)
    beta = math.degrees(math.atan2(S["r"][0][1], S["r"][0][0]))
    gd = golden("pythagorean")
    assert a == pytest.approx(gd["a23"] / gd["side_scale"], abs=0.01)
    assert e == pytest.approx(gd["e23"], abs=0.005)
    assert beta == pytest.approx(gd["beta1"], abs=0.5)


def test_lidov_kozai_oscillations():
    """Sec. 5.3 (tests/golden/lidov_kozai.txt): the hierarchical triple with i0 = 80 deg
    shows Lidov-Kozai cycles. Checked over the first two cycles against the paper and two
    closed forms of the quadrupole test-particle theory:
    - the set-up reading: the paper's test-particle e_max is sqrt(1 - 5/3 cos^2 i0), and
      the minimum inclination is i_crit = arccos sqrt(3/5);
    - the run: the first cycle's peak eccentricity is within 0.006 of the paper's 0.983
      (the peaks depend a little on the orbital phases, which the paper does not give) and
      above the test-particle value; the inclination bottoms out within 0.5 deg of i_crit;
    - the cycle period gives roughly ten cycles in 100 Myr (G = 1, 1e9 Msun, pc units: one
      time unit is sqrt(pc^3 / (G 1e9 Msun)) = 471.5 yr with G = 4.3009e-3 pc (km/s)^2/Msun)."""
    gd = golden("lidov_kozai")
    i0 = math.radians(80.0)
    assert math.sqrt(1 - 5 / 3 * math.cos(i0) ** 2) == pytest.approx(gd["e_max_test_particle"], abs=1e-3)
    i_crit = math.degrees(math.acos(math.sqrt(0.6)))
    assert i_crit == pytest.approx(gd["i_crit"], abs=0.05)
    m, r, v = W.lidov_kozai()
    s = O.System(m, r, v)
    M = m[0] + m[1]
    peaks, cur, cur_t, i_min = [], 0.0, 0.0, 90.0
    t_stop = 40000.0
    while True:
        rc, st = s.integrate(t_stop, max_steps=1)
        assert rc == 0
        S = s.state()
        dr, dv = S["r"][1] - S["r"][0], S["v"][1] - S["v"][0]
        E = 0.5 * dv @ dv - M / np.linalg.norm(dr)
        L = np.cross(dr, dv)
        e = math.sqrt(max(0.0, 1 + 2 * E * (L @ L) / M ** 2))
        i_min = min(i_min, math.degrees(math.acos(L[2] / np.linalg.norm(L))))
        if e > cur:
            cur, cur_t = e, S["t"]
        if e < 0.5 and cur > 0.9:
            peaks.append((cur, cur_t))
            cur = 0.0
        if abs(S["t"] - t_stop) <= 1e-10 * t_stop:
            break
    assert len(peaks) == 2, peaks
    e1 = peaks[0][0]
    assert gd["e_max_test_particle"] < e1 and abs(e1 - gd["e_max"]) < 0.006, peaks
    assert abs(i_min - i_crit) < 0.5, i_min
    v_unit_kms = math.sqrt(4.3009e-3 * 1e9)  # sqrt(G M / 1 pc)
    t_unit_yr = 3.0857e13 / v_unit_kms / 3.15576e7  # 1 pc in km over v_unit, in years
    period_myr = (peaks[1][1] - peaks[0][1]) * t_unit_yr / 1e6
    cycles = gd["duration"] / period_myr
    assert 0.8 * gd["oscillations"] <= cycles <= 1.2 * gd["oscillations"], (cycles, period_myr)
