"""The allocation-free pair loop (mstar_accelerations_noalloc) against the context path and
against the oracle's Cartesian (n_d = 0) pair loop.

mstar_accelerations_noalloc serves callers that may not allocate device memory (a
sub-integrator inside a code whose memory manager owns the device heap, or a loop that
cannot afford cudaMalloc's synchronisation): its scratch is a static device array shared
by all calls. This file is collected last so that a failure here cannot hide the other
tests; it also passes on its own in a fresh process.
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


def context_reference(m, r, v):
    """Accelerations and U from the existing entry point (a context with n_d = 0, every
    pair Cartesian), and the centre-of-mass positions that context works on."""
    g = M.Integrator(m, r, v, n_d=0)
    a, U = g.accelerations()
    rc = g.state()["r"]
    g.close()
    return a, U, rc


def noalloc(m, rc, G=1.0):
    dev = torch.device("cuda")
    mt = torch.tensor(m, dtype=torch.float64, device=dev)
    rt = torch.tensor(rc, dtype=torch.float64, device=dev)
    at = torch.empty_like(rt)
    Ut = torch.empty(1, dtype=torch.float64, device=dev)
    rc_ = M.mstar_accelerations_noalloc(len(m), mt, rt, G, at, Ut, torch.cuda.current_stream().cuda_stream)
    assert rc_ == M.MSTAR_OK, M.mstar_strerror(rc_)
    torch.cuda.synchronize()
    return at.cpu().numpy(), float(Ut.item())


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    # first call at the maximum size, second call smaller and ragged: the second must not
    # see anything the first left in the shared scratch
    for m, r, v in [W.plummer(M.MSTAR_NOALLOC_MAX_N, 2), W.plummer(333, 8)]:
        a_ref, U_ref, rc = context_reference(m, r, v)
        a, U = noalloc(m, rc)
        assert np.abs(a - a_ref).max() <= 1e-13 * np.abs(a_ref).max()
        assert abs(U - U_ref) <= 1e-13 * U_ref


@pytest.mark.parametrize("n", [2, 129, 333, 2047, M.MSTAR_NOALLOC_MAX_N])
def test_noalloc_matches_oracle_cartesian_forces(n):
    """Element by element against the oracle's pair loop with every pair Cartesian (n_d = 0),
    on the same centre-of-mass positions: sizes with a ragged last 128-body tile (129, 333,
    2047), the smallest system and the maximum."""
    m, r, v = W.plummer(n, 40 + n) if n > 2 else W.kepler_binary(seed=3)
    rc = O.com_shift(m, r)
    root, par, lev, order = O.prim(rc)
    X = O.to_mst(par, rc)
    ao, Uo = O.forces(m, rc, par, lev, X, n_d=0)
    a, U = noalloc(m, rc)
    assert np.abs(a - ao).max() <= 1e-13 * np.abs(ao).max()
    assert abs(U - Uo) <= 1e-13 * Uo


def test_noalloc_rejects_oversize_and_host_pointers():
    m, r, v = W.plummer(64, 1)
    dev = torch.device("cuda")
    n = M.MSTAR_NOALLOC_MAX_N + 1
    big_m = torch.ones(n, dtype=torch.float64, device=dev)
    big_r = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    a = torch.empty((n, 3), dtype=torch.float64, device=dev)
    U = torch.empty(1, dtype=torch.float64, device=dev)
    assert M.mstar_accelerations_noalloc(n, big_m, big_r, 1.0, a, U) == M.MSTAR_ERR_UNSUPPORTED
    a_h = np.empty((64, 3))
    U_h = np.empty(1)
    assert M.mstar_accelerations_noalloc(64, m, r, 1.0, a_h, U_h) == M.MSTAR_ERR_INVALID_ARG
