"""The rebuild test of Sec. 3.5 on the GPU (mstar_rebuild_test) against the oracle.

The transforms are pure additions, subtractions and one division per component, done in
the CPU definition's order, and the energies are compensated sums in index order: the GPU's
energies, final states, topology-change counts and mean levels must equal the oracle's bit
for bit, for both coordinate systems and all four deconstruction rules (per-vertex path sums
with the centre-of-mass shift or the root kept; from the root outwards with the root kept,
or followed by the shift).
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


def run_both(systems, jobs, cycles, topo_every, samples):
    sy = [systems[s] for s, _, _ in jobs]
    g = M.mstar_rebuild_test(sy, [c for _, c, _ in jobs], [d for _, _, d in jobs], cycles, topo_every, samples)
    for k, (s, c, d) in enumerate(jobs):
        m, r, v = systems[s]
        o = O.rebuild_run(m, r, v, c, cycles, topo_every, samples, d)
        assert np.array_equal(g["E"][k], o["E"]), (k, g["E"][k], o["E"])
        assert np.array_equal(g["r"][k], o["r"]) and np.array_equal(g["v"][k], o["v"]), k
        assert g["topo_changes"][k] == o["topo_changes"] and g["mean_level"][k] == o["mean_level"], k
    return g


def test_rebuild_test_bit_identical_to_oracle_hernquist379():
    systems = [W.hernquist(379, s)[:3] for s in (1, 2)]
    jobs = [(s, c, d) for s in (0, 1) for c in (0, 1) for d in (0, 1, 2, 3)]
    run_both(systems, jobs, 300, 100, [0, 1, 10, 100, 300])


@pytest.mark.parametrize("n", [2, 3, 33, 600])
def test_rebuild_test_other_sizes(n):
    systems = [W.plummer(n, n)]
    jobs = [(0, c, d) for c in (0, 1) for d in (0, 1, 2, 3)]
    run_both(systems, jobs, 40, 7, [0, 3, 40])


def test_rebuild_test_rejects_bad_arguments():
    m, r, v = W.plummer(M.MSTAR_REBUILD_MAX_N + 1, 1)
    with pytest.raises(M.MstarError) as e:
        M.mstar_rebuild_test([(m, r, v)], [0], [0], 1, 1, [0])
    assert e.value.code == M.MSTAR_ERR_INVALID_ARG
    m, r, v = W.plummer(10, 1)
    with pytest.raises(M.MstarError):
        M.mstar_rebuild_test([(m, r, v)], [2], [0], 1, 1, [0])
    with pytest.raises(M.MstarError):
        M.mstar_rebuild_test([(m, r, v)], [0], [4], 1, 1, [0])
    with pytest.raises(M.MstarError):
        M.mstar_rebuild_test([(m, r, v)], [0], [0], 5, 1, [3, 2])
