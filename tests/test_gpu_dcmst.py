"""Divide-and-conquer spanning tree (Sec. 3.3, mst_method = 1) on the GPU against the oracle.

Root, parent and level must be bit-identical to the oracle's tree for the same
centre-of-mass positions (the tree is a discrete result); the order is the breadth-first
walk, checked for validity (a tree has several). One GBS attempt on the tree must match
the oracle's attempt on the same tree to 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_03180_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA GPU", allow_module_level=True)

from paper_2001_03180_gb300 import build as B  # noqa: E402

B.build()
from paper_2001_03180_gb300 import mstar as M  # noqa: E402

O.set_threads(16)


def gpu_tree(m, r, v, nsub):
    g = M.Integrator(m, r, v, mst_method=1, mst_nsub=nsub)
    root, parent, level, order = g.mst(with_order=True)
    g.close()
    return root, parent, level, order


def check(m, r, v, nsub=0):
    rc = O.com_shift(m, np.asarray(r, np.float64))
    root_o, par_o, lev_o, _, _, _ = O.dc_mst(rc, nsub)
    root, par, lev, order = gpu_tree(m, r, v, nsub)
    assert root == root_o
    assert np.array_equal(par, par_o)
    assert np.array_equal(lev, lev_o)
    n = len(m)
    assert order[0] == root and sorted(order.tolist()) == list(range(n))
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    assert np.all(np.diff(lev[order]) >= 0)
    nonroot = par >= 0
    assert np.all(pos[par[nonroot]] < pos[np.flatnonzero(nonroot)])


@pytest.mark.parametrize("n, seed", [(2, 1), (3, 2), (100, 3), (1000, 4), (4097, 5)])
def test_dc_tree_matches_oracle_plummer(n, seed):
    check(*W.plummer(n, seed))


@pytest.mark.parametrize("nsub", [1, 2, 7, 64, 200])
def test_dc_tree_matches_oracle_subgraph_counts(nsub):
    check(*W.plummer(200, 6), nsub=nsub)


def test_dc_tree_matches_oracle_workloads():
    check(*W.workload("plummer2048_smbh_binary"))
    check(*W.workload("plummer10k_two_smbh"))
    check(*W.workload("plummer10k_two_smbh"), nsub=1024)


def test_dc_tree_ties():
    # the hand-computed tie cases of the oracle's pins, then a cubic lattice (many equal distances)
    sq = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1.0, 1.0, 0.0]])
    check(np.ones(4), sq, np.zeros((4, 3)), nsub=1)
    tri = np.array([[-3.0, 0.0, 0.0], [1.0, 1.0, 0.5], [1.0, 0.5, 1.0]])
    m3 = np.array([1.0, 1.0, 1.0])
    check(m3, tri, np.zeros((3, 3)), nsub=2)
    g = np.arange(6.0)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    for nsub in (0, 8, 27):
        check(np.ones(len(lat)), lat, np.zeros_like(lat), nsub=nsub)


def test_attempt_on_dc_tree_matches_oracle():
    m, r, v = W.workload("plummer2048_smbh_binary")
    H = 2e-4 * O.potential(m, O.com_shift(m, r))
    g = M.Integrator(m, r, v, mst_method=1)
    a = g.attempt(H)
    g.close()
    o = O.System(m, r, v, mst_method=1)
    b = o.attempt(H)
    rel = lambda x, y: float(np.abs(x - y).max() / np.abs(y).max())  # noqa: E731
    assert rel(a["r"], b["r"]) < 1e-12 and rel(a["v"], b["v"]) < 1e-12
    assert abs(a["t"] - b["t"]) <= 1e-12 * abs(b["t"])


def test_invalid_subgraph_count_rejected():
    m, r, v = W.plummer(50, 1)
    with pytest.raises(M.MstarError) as e:
        M.Integrator(m, r, v, mst_method=1, mst_nsub=1025)
    assert e.value.code == M.MSTAR_ERR_INVALID_ARG
    with pytest.raises(M.MstarError):
        M.Integrator(m, r, v, mst_method=2)


def test_run_to_t1_on_dc_tree_matches_oracle():
    """Plummer 64 (8 subgraphs) to t = 1 with the divide-and-conquer tree in every step: the
    end state agrees with the oracle's run on the same trees, and over 7 realisations (the start
    and six starts perturbed at the 1e-15 level) the GPU's energy errors are within 10x of the
    oracle's, median and maximum."""
    m, r, v = W.workload("plummer64")
    dg, do = [], []
    for k in range(7):
        mk, rk, vk = W.perturbed(m, r, v, k)
        g = M.Integrator(mk, rk, vk, mst_method=1)
        o = O.System(mk, rk, vk, mst_method=1)
        e0g, e0o = g.energy()["E"], o.energy()["E"]
        rc, st = g.step(1.0)
        rco, sto = o.integrate(1.0)
        assert rc == 0 and rco == 0
        if k == 0:
            S, So = g.state(), o.state()
            rel = lambda x, y: float(np.abs(x - y).max() / np.abs(y).max())  # noqa: E731
            assert rel(S["r"], So["r"]) < 1e-9 and rel(S["v"], So["v"]) < 1e-9
        dg.append(abs((g.energy()["E"] - e0g) / e0g))
        do.append(abs((o.energy()["E"] - e0o) / e0o))
        g.close()
    dg, do = np.asarray(dg), np.asarray(do)
    assert np.median(dg) <= 10 * np.median(do), (dg.tolist(), do.tolist())
    assert dg.max() <= 10 * do.max(), (dg.tolist(), do.tolist())
