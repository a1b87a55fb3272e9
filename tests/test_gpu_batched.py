"""Batched independent systems (mstar_step_batched) against the oracle, system by system.

One launch advances every system by one GBS step attempt (one CTA per system with
divisions spread over four groups of 1, 2 or 4 warps by the greedy recipe of Sec. 4.2, or
groups of 8 or 16 lanes with one body per lane for systems of at most 16 bodies). With eta = 1
every attempt is accepted, so one launch at a fixed H must reproduce the oracle's single
attempt for each system (1e-12 relative per system) under every schedule; with eta = 1e-12
repeated launches must land every system on t_end with the oracle's end state.
"""
import math

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


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def mixed_systems():
    st = W.Stream(17, 3)
    out = [W.kepler_binary(seed=2, e=0.7), W.pythagorean(),
           W.hierarchical_triple(1.0, 1.0, 0.1, 1.0, 0.3, 20.0, 0.0, math.radians(60.0), st)]
    for n, seed in [(5, 1), (12, 7), (16, 8), (33, 2), (64, 3), (100, 4), (257, 5), (512, 6)]:
        out.append(W.plummer(n, seed))
    return out


def step_sizes(systems):
    """A fictitious step of about 2e-3 time units for each system (H ~ U dt)."""
    H = []
    for m, r, v in systems:
        U = O.potential(m, O.com_shift(m, r))
        H.append(2e-3 * U)
    return np.array(H)


SCHEDULES = {"default": None, "g1": [1] * 7, "g2": [2] * 7, "g4": [4] * 7, "mixed": [4, 2, 1, 4, 2, 1, 2],
             "segments": [0, 0, 2, 1, 1, 1, 2], "split1": [-1] * 7, "split2": [-2] * 7, "split4": [-4] * 7,
             "split_mixed": [0, -4, 1, -1, -2, 2, -4]}


@pytest.mark.parametrize("name", list(SCHEDULES))
def test_one_launch_matches_oracle_attempt(name):
    systems = mixed_systems()
    H = step_sizes(systems)
    b = M.Batch(systems, eta_gbs=1.0)
    if SCHEDULES[name] is not None:
        b.set_schedule(SCHEDULES[name])
        assert list(b.schedule()) == SCHEDULES[name]
    b.set_H(H)
    st = b.step(1e9, launches=1)
    assert st["accepted"] == len(systems) and st["failed"] == 0
    S = b.state()
    for s, (m, r, v) in enumerate(systems):
        o = O.System(m, r, v)
        a = o.attempt(H[s])
        assert relerr(S["r"][s], a["r"]) < 1e-12, s
        assert relerr(S["v"][s], a["v"]) < 1e-12, s
        assert abs(S["t"][s] - a["t"]) <= 1e-12 * abs(a["t"]), s
        if a["eps"] > 1e-11:
            assert abs(S["eps"][s] - a["eps"]) <= 1e-2 * a["eps"], (s, S["eps"][s], a["eps"])
    b.close()


def test_full_size_batch_sampled_against_oracle():
    """The benchmark's 4096-system workload (2..199 bodies, every size class up to 256) in the
    benchmark's launch configuration: the autotuned schedule, every node in one graph launch.
    With eta = 1 every attempt is accepted. In each size class the largest system and eight
    spread over the class match the oracle's attempt at the same H."""
    systems = W.batched_systems(4096, 3)
    trip = [(s.m, s.r, s.v) for s in systems]
    H = step_sizes(trip)
    b = M.Batch(trip, eta_gbs=1.0)
    sched, _ = b.autotune(1e9, repeats=1)
    assert list(b.schedule()) == list(sched)
    b.set_H(H)
    st = b.step(1e9, launches=1)
    assert st["accepted"] == len(systems) and st["failed"] == 0
    S = b.state()
    b.close()
    sizes = np.array([len(s.m) for s in systems])
    pick = set()
    for lo, hi in [(2, 8), (9, 16), (17, 32), (33, 64), (65, 128), (129, 256)]:
        idx = np.flatnonzero((sizes >= lo) & (sizes <= hi))
        assert len(idx) > 0, (lo, hi)
        pick.add(int(idx[np.argmax(sizes[idx])]))
        pick.update(int(i) for i in idx[np.linspace(0, len(idx) - 1, 8).astype(int)])
    for s in sorted(pick):
        a = O.System(*trip[s]).attempt(H[s])
        assert relerr(S["r"][s], a["r"]) < 1e-12, (s, sizes[s])
        assert relerr(S["v"][s], a["v"]) < 1e-12, (s, sizes[s])
        assert abs(S["t"][s] - a["t"]) <= 1e-12 * abs(a["t"]), (s, sizes[s])


@pytest.mark.parametrize("G", [1, 2, 4])
def test_split_attempt_is_bit_identical_to_one_cta(G):
    """The split schedule -G runs the same arithmetic as the one-CTA schedule G: start, the
    four groups' divisions and the finish, with the same partial sums in the same order."""
    systems = mixed_systems()
    H = step_sizes(systems)
    out = []
    for sched in ([G] * 7, [-G] * 7):
        b = M.Batch(systems)
        b.set_schedule(sched)
        b.set_H(H)
        b.step(1e9, launches=3)
        out.append(b.state())
        b.close()
    for key in ("t", "eps", "status"):
        assert np.array_equal(out[0][key], out[1][key]), key
    for s in range(len(systems)):
        assert np.array_equal(out[0]["r"][s], out[1]["r"][s]) and np.array_equal(out[0]["v"][s], out[1]["v"][s]), s


@pytest.mark.parametrize("n_d", [0, 1])
def test_one_launch_other_near_rules(n_d):
    """The batched kernels with N_d = 0 and 1 (Sec. 3.4) against the oracle's attempt with the
    same rule, every system (segment kernels and CTAs)."""
    systems = mixed_systems()
    H = step_sizes(systems)
    b = M.Batch(systems, eta_gbs=1.0, n_d=n_d)
    b.set_H(H)
    st = b.step(1e9, launches=1)
    assert st["accepted"] == len(systems) and st["failed"] == 0
    S = b.state()
    for s, (m, r, v) in enumerate(systems):
        a = O.System(m, r, v, n_d=n_d).attempt(H[s])
        assert relerr(S["r"][s], a["r"]) < 1e-12, s
        assert relerr(S["v"][s], a["v"]) < 1e-12, s
    b.close()


def test_batch_integrates_to_end_time_like_the_oracle():
    systems = mixed_systems()
    t_end = 0.05
    b = M.Batch(systems)
    for _ in range(400):
        st = b.step(t_end, launches=5)
        if st["finished"] == len(systems):
            break
    assert st["finished"] == len(systems) and st["failed"] == 0
    S = b.state()
    assert np.all(S["status"] == 1)
    for s, (m, r, v) in enumerate(systems):
        o = O.System(m, r, v)
        rc, sto = o.integrate(t_end)
        assert rc == 0
        So = o.state()
        assert abs(S["t"][s] - t_end) <= 1e-10 * t_end
        assert relerr(S["r"][s], So["r"]) < 1e-9, s
        assert relerr(S["v"][s], So["v"]) < 1e-9, s
    b.close()


def test_batch_rejects_oversize_and_bad_input():
    m, r, v = W.plummer(M.MSTAR_BATCH_MAX_N + 1, 1)
    with pytest.raises(M.MstarError) as e:
        M.Batch([W.plummer(10, 1), (m, r, v)])
    assert e.value.code == M.MSTAR_ERR_UNSUPPORTED
    m, r, v = W.plummer(10, 2)
    r = r.copy()
    r[2, 0] = np.inf
    with pytest.raises(M.MstarError) as e:
        M.Batch([(m, r, v)])
    assert e.value.code == M.MSTAR_ERR_NONFINITE
    m1, r1, v1 = W.plummer(10, 3)
    with pytest.raises(M.MstarError) as e:                     # a one-body system has no pairs
        M.Batch([W.plummer(10, 1), (m1[:1], r1[:1], v1[:1])])
    assert e.value.code == M.MSTAR_ERR_INVALID_ARG


def test_autotune_keeps_the_state_and_picks_a_valid_schedule():
    systems = mixed_systems()
    H = step_sizes(systems)
    b = M.Batch(systems, eta_gbs=1.0)
    b.set_H(H)
    before = b.state()
    sched, ms = b.autotune(1e9, repeats=1)
    assert ms > 0 and set(sched.tolist()) <= {0, 1, 2, 4, -1, -2, -4}
    assert list(b.schedule()) == sched.tolist()
    after = b.state()
    for key in ("t", "eps", "status"):
        assert np.array_equal(before[key], after[key])
    for s in range(len(systems)):
        assert np.array_equal(before["r"][s], after["r"][s]) and np.array_equal(before["v"][s], after["v"][s])
    st = b.step(1e9, launches=1)  # the H set above survived the trials
    assert st["accepted"] == len(systems)
    S = b.state()
    for s, (m, r, v) in enumerate(systems):
        a = O.System(m, r, v).attempt(H[s])
        assert relerr(S["r"][s], a["r"]) < 1e-12, s
        assert relerr(S["v"][s], a["v"]) < 1e-12, s
    b.close()


def test_batch_rejects_bad_schedule():
    b = M.Batch([W.plummer(10, 1)])
    assert list(b.schedule()) == [0, 0, 1, 1, 1, 2, 4]
    # width 3; segments above 16 bodies; split width 3
    for bad in ([1, 2, 3, 4, 1, 1, 1], [0, 0, 0, 1, 1, 1, 1], [1, 1, 1, -3, 1, 1, 1]):
        with pytest.raises(M.MstarError) as e:
            b.set_schedule(bad)
        assert e.value.code == M.MSTAR_ERR_INVALID_ARG
    assert list(b.schedule()) == [0, 0, 1, 1, 1, 2, 4]
    b.close()
