"""Pins of the chained coordinates (Sec. 2.2), the Hernquist initial conditions (Sec. 6.1) and
the oracle's rebuild test (Sec. 3.5).

Chain: a Hamiltonian path whose first link is the globally shortest pair, never shorter
than the MST, a hand-computed case, and <L_chain> = (N-1)/2 against <L_MST> in the paper's
range (Fig. mean_L: a factor 2-10 for N = 10..1000).
Hernquist: the distribution function integrates back to the density (Eddington's
inversion, checked by quadrature), and a large sample follows the enclosed-mass law and the
velocity-dispersion profile of the distribution function.
Rebuild run: exact on a dyadic state (every transform is then exact), topology unchanged
over the run, and the paper's claim that MST coordinates accumulate less error than the
chain when the deconstruction adds the root's kept position.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from paper_2001_03180_gb300 import workloads as W

from tests.helpers import edge_set, golden, mst_kruskal, sqdist


def tree_length(r, parent):
    return sum(math.sqrt(sqdist(r, v, int(p))) for v, p in enumerate(parent) if p >= 0)


@pytest.mark.parametrize("n, seed", [(7, 1), (60, 2), (379, 3)])
def test_chain_structure(n, seed):
    m, r, v = W.plummer(n, seed)
    tail, par, lev, order = O.chain(r)
    assert order[0] == tail and sorted(order.tolist()) == list(range(n))
    assert par[tail] == -1 and all(par[order[k]] == order[k - 1] for k in range(1, n))
    assert lev.tolist() == np.argsort(order).tolist()
    # the first link is the globally shortest inter-particle vector
    d2 = ((r[:, None, :] - r[None, :, :]) ** 2).sum(axis=2)
    np.fill_diagonal(d2, np.inf)
    i, j = np.unravel_index(np.argmin(d2), d2.shape)
    links = {tuple(sorted((int(order[k]), int(order[k + 1])))) for k in range(n - 1)}
    assert tuple(sorted((int(i), int(j)))) in links
    # a spanning tree, so never shorter than the MST
    assert edge_set(par) == links
    mst = mst_kruskal(r)
    mst_len = sum(math.sqrt(sqdist(r, a, b)) for a, b in mst)
    assert tree_length(r, par) >= mst_len * (1 - 1e-12)


def test_chain_hand_computed():
    """Points on a line at 0, 1, 3, 7 and 1.5 (indices 0..4): the shortest pair is (1, 4)
    (0.5 apart; tail 1, head 4). Then 0 joins the tail (1 from body 1; body 2 is 1.5 from
    body 4), then 2 joins the head (1.5 from body 4; body 3 is 5.5), then 3 joins the head
    (4 from body 2). Chain from the tail: 0, 1, 4, 2, 3."""
    x = np.array([0.0, 1.0, 3.0, 7.0, 1.5])
    r = np.stack([x, np.zeros(5), np.zeros(5)], axis=1)
    tail, par, lev, order = O.chain(r)
    assert order.tolist() == [0, 1, 4, 2, 3] and tail == 0
    assert par.tolist() == [-1, 0, 4, 2, 1]


def test_chain_levels_against_mst_levels():
    """Fig. mean_L: <L_chain> = (N-1)/2, and <L_MST> is always lower, by a factor that starts
    near 2 at N = 10 and grows with N (the paper reads ~2-10 up to N = 1000 for rho ~ 1/r;
    these Hernquist samples give ~2.3 at N = 10 and ~18 at N = 1000)."""
    ratios = []
    for n in (10, 100, 1000):
        rs = []
        for seed in (1, 2, 3):
            m, r, v, _ = W.hernquist(n, seed)
            _, _, lev_c, _ = O.chain(r)
            _, _, lev_m, _ = O.prim(r)
            assert lev_c.mean() == (n - 1) / 2
            rs.append(lev_c.mean() / lev_m.mean())
        ratios.append(float(np.mean(rs)))
    gd = golden("mst_claims")
    assert 0.75 * gd["chain_over_mst_mean_level_low"] < ratios[0] < 1.75 * gd["chain_over_mst_mean_level_low"], ratios
    assert ratios[0] < ratios[1] < ratios[2], ratios


def test_hernquist_df_reproduces_the_density():
    a = 1.0 / (1.0 + math.sqrt(2.0))
    for rr in (0.02, 0.2, 1.0, 5.0):
        psi = 1.0 / (rr + a)
        val, _ = quad(lambda v: 4 * math.pi * v * v * float(W.hernquist_df(psi - 0.5 * v * v, a=a)), 0,
                      math.sqrt(2 * psi), limit=200)
        rho = a / (2 * math.pi * rr * (rr + a) ** 3)
        assert abs(val / rho - 1) < 1e-7, (rr, val / rho - 1)


def test_hernquist_sample_statistics():
    n = 4000
    m, r, v, draws = W.hernquist(n, 7, reject_hard_binaries=False)
    a = 1.0 / (1.0 + math.sqrt(2.0))
    rad = np.linalg.norm(r, axis=1)
    # enclosed-mass law (truncated at 20 half-mass radii): M(<r)/M(<r_cut) = (r/(r+a))^2 / (r_c/(r_c+a))^2
    rc = 20.0
    norm = (rc / (rc + a)) ** 2
    for x in (0.3, 1.0, 3.0):
        frac = float((rad < x).mean())
        expect = (x / (x + a)) ** 2 / norm
        assert abs(frac - expect) < 4 * math.sqrt(expect * (1 - expect) / n) + 0.01, (x, frac, expect)
    # velocity dispersion in shells against <v^2>(r) = 4 pi int v^4 f dv / rho
    speed2 = (v * v).sum(axis=1)
    for lo, hi in ((0.2, 0.4), (0.8, 1.2), (2.0, 3.0)):
        sel = (rad >= lo) & (rad < hi)
        rmid = float(np.median(rad[sel]))
        psi = 1.0 / (rmid + a)
        num, _ = quad(lambda u: 4 * math.pi * u ** 4 * float(W.hernquist_df(psi - 0.5 * u * u, a=a)), 0,
                      math.sqrt(2 * psi), limit=200)
        rho = a / (2 * math.pi * rmid * (rmid + a) ** 3)
        expect = num / rho
        got = float(speed2[sel].mean())
        assert abs(got / expect - 1) < 0.1, (lo, hi, got, expect)


def test_hernquist_has_no_hard_binary():
    for seed in (1, 9):
        m, r, v, draws = W.hernquist(379, seed)
        assert not W.has_hard_binary(m, r, v)
        assert draws >= 1


@pytest.mark.parametrize("coords", [0, 1])
@pytest.mark.parametrize("deconstruct", [0, 1, 2, 3])
def test_rebuild_exact_on_dyadic_state(coords, deconstruct):
    """Small integers times powers of two with equal power-of-two masses: every difference,
    path sum and centre-of-mass shift is exact, so the state never changes."""
    st = W.Stream(5, 1)
    h = 12  # mirrored pairs p, -p: the centre of mass is exactly the origin
    r = np.floor(st.uniform(3 * h) * 64).reshape(h, 3) * 0.25 + 0.125
    v = np.floor(st.uniform(3 * h) * 16).reshape(h, 3) * 0.125 + 0.0625
    r = np.concatenate([r, -r])
    v = np.concatenate([v, -v])
    m = np.full(2 * h, 0.25)
    out = O.rebuild_run(m, r, v, coords, 200, 50, [0, 200], deconstruct)
    assert np.array_equal(out["r"], r) and np.array_equal(out["v"], v)
    assert out["E"][0] == out["E"][1] and out["topo_changes"] == 0


def test_rebuild_mst_accumulates_less_error_than_chain_with_root_kept():
    """Sec. 3.5: with the root's position kept, MST coordinates accumulate several times less
    energy error than the chain (mean over seeds, N = 379 Hernquist, 1000 rebuilds)."""
    mst, chn = [], []
    for seed in (1, 2, 3):
        m, r, v, _ = W.hernquist(379, seed)
        for coords, acc in ((0, mst), (1, chn)):
            out = O.rebuild_run(m, r, v, coords, 1000, 500, [0, 1000], 1)
            acc.append(abs(out["E"][1] / out["E"][0] - 1))
            assert out["topo_changes"] == 0
    # the paper reads an order of magnitude at 1e5 rebuilds; at 1e3 a factor 3 is asked
    assert np.mean(chn) > 0.3 * golden("mst_claims")["rebuild_chain_over_mst_error"] * np.mean(mst), \
        (np.mean(chn), np.mean(mst))


@pytest.mark.parametrize("coords", [0, 1])
def test_rebuild_from_the_root_outwards_does_not_accumulate(coords):
    """Deconstruction from the root outwards (w_v = w_parent(v) + X_v, parents first, the root
    kept) undoes the build up to one rounding per edge, and once a body's parent is unchanged
    fl(w_p + fl(w_v - w_p)) returns w_v (the subtraction and the addition are then exact in all
    but rare cases): after the first cycle the state stays where it is. The energy error after
    1000 cycles therefore equals the one after 10, while the per-vertex path sums (rule 1) grow
    by about the cycle ratio."""
    m, r, v, _ = W.hernquist(379, 4)
    out = O.rebuild_run(m, r, v, coords, 1000, 500, [0, 10, 1000], 2)
    E = out["E"]
    assert abs(E[2] / E[0] - 1) <= max(abs(E[1] / E[0] - 1), 1e-16) * 1.5
    assert abs(E[2] / E[0] - 1) < 2e-15
    walk = O.rebuild_run(m, r, v, coords, 1000, 500, [0, 10, 1000], 1)["E"]
    assert abs(walk[2] / walk[0] - 1) > 10 * abs(walk[1] / walk[0] - 1)
    # the root keeps its position exactly
    root = O.prim(r)[0] if coords == 0 else O.chain(r)[0]
    assert np.array_equal(out["r"][root], r[root]) and np.array_equal(out["v"][root], v[root])


def test_chain_end_tie_joins_the_tail():
    """Tail (0,0) and head (1,0) start the chain (squared distance 1, the shortest); body 2 at
    (0.5, 2) is 4.25 from both ends (exact) and joins the tail (the reading for a tie);
    body 3 at (10, 0) then joins the head. Chain from the tail: 2, 0, 1, 3."""
    r = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, 2.0, 0.0], [10.0, 0.0, 0.0]])
    tail, par, lev, order = O.chain(r)
    assert order.tolist() == [2, 0, 1, 3] and tail == 2


def test_compensated_energy_is_the_rounded_exact_sum():
    """orc_energy_comp sums the FP64 terms m v^2 / 2 and G m_i m_j / r_ij with compensation:
    each sum equals math.fsum of the same terms (the correctly rounded exact sum) to about
    one rounding, where a plain running sum of ~5e5 terms is off by much more."""
    m, r, v = W.plummer(1000, 11)
    n = len(m)
    T = [0.5 * (m[i] * ((v[i, 0] * v[i, 0] + v[i, 1] * v[i, 1]) + v[i, 2] * v[i, 2])) for i in range(n)]
    U = []
    for i in range(n):
        d = r[i] - r[i + 1:]
        w2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        U.extend(((m[i] * m[i + 1:]) / np.sqrt(w2)).tolist())
    ref = math.fsum(T) - math.fsum(U)
    got = O.energy_comp(m, r, v)
    assert abs(got - ref) <= 4e-16 * abs(ref), (got, ref)
