"""A model of the work split of k_division_cta<C> (csrc/step.cu): the tile-pair tasks of a
division's pair sums, how a cluster of C CTAs deals them out, the per-CTA and cross-CTA sums, and
the share of near partners each task takes. CPU only.

The kernel's rules, restated:
- nb = npad / 32 body tiles give ntp = nb (nb + 1) / 2 tile pairs (I <= J) in row-major order;
- each tile pair's partner steps (k = 0..31, or k = 1..16 on the diagonal, where step 16 counts
  only lanes < 16) are split into S = clamp(16 C / ntp, 1, 8) chunks; task w = tp S + s;
- CTA r of the cluster takes the tasks w = r + C lw (lw = 0, 1, ...), at most 16 of them;
- the partials of body b (tile t) are the tasks with I == t (i-side) or J == t (j-side); each CTA
  adds those of its own tasks, and the cluster adds the CTAs' sums;
- near partner number k of a body in tile I goes to the task with rank k mod (nb - I) S among the
  tasks whose i-side is tile I, ordered (J - I) S + s.
"""
import itertools

import numpy as np
import pytest

TASKS_PER_CTA = 16


def split(nb, C):
    ntp = nb * (nb + 1) // 2
    S = max(1, min(8, (TASKS_PER_CTA * C) // ntp))
    return ntp, S, ntp * S


def tile_pairs(nb):
    return [(I, J) for I in range(nb) for J in range(I, nb)]


def steps(diag, s, S):
    if diag:
        return range(1 + (16 * s) // S, 1 + (16 * (s + 1)) // S)
    return range((32 * s) // S, (32 * (s + 1)) // S)


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("C", [1, 2, 4, 8])
def test_every_unordered_pair_once_and_every_cta_within_its_warps(nb, C):
    ntp, S, ntask = split(nb, C)
    assert ntask <= TASKS_PER_CTA * C
    per_cta = [0] * C
    seen = np.zeros((32 * nb, 32 * nb), np.int32)
    tps = tile_pairs(nb)
    for w in range(ntask):
        per_cta[w % C] += 1
        I, J = tps[w // S]
        s = w % S
        diag = I == J
        for k in steps(diag, s, S):
            for lane in range(32):
                if diag and k == 16 and lane >= 16:
                    continue
                i, j = 32 * I + lane, 32 * J + (lane + k) % 32
                seen[min(i, j), max(i, j)] += 1
    assert max(per_cta) <= TASKS_PER_CTA
    assert np.array_equal(seen, np.triu(np.ones_like(seen), 1))


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("C", [1, 2, 4, 8])
def test_each_task_partial_is_added_once_per_body(nb, C):
    """The two-level sum: every task touching a body's tile contributes to exactly one CTA's sum
    for that body, on the side that holds the body (the diagonal's single plane on the i-side)."""
    ntp, S, ntask = split(nb, C)
    tps = tile_pairs(nb)
    for t in range(nb):
        counted = {}
        for r in range(C):
            wt = 0
            for (I, J) in tps:
                for q in range(S):
                    if wt % C == r and (I == t or J == t):
                        counted[wt] = counted.get(wt, 0) + 1
                        assert (I == t) or (J == t and I != J)
                    wt += 1
        touching = [w for w in range(ntask) if t in tps[w // S]]
        assert sorted(counted) == touching and all(v == 1 for v in counted.values())


def near_list(parent, i, n_d):
    """The kernel's enumeration order: parent, children, grandparent, grandchildren, siblings."""
    kids = [[] for _ in parent]
    for v, p in enumerate(parent):
        if p >= 0:
            kids[p].append(v)
    out = []
    p = parent[i]
    if n_d >= 1:
        if p >= 0:
            out.append(p)
        out += kids[i]
    if n_d >= 2:
        if p >= 0 and parent[p] >= 0:
            out.append(parent[p])
        for c in kids[i]:
            out += kids[c]
        if p >= 0:
            out += [s for s in kids[p] if s != i]
    return out


@pytest.mark.parametrize("n,C", [(31, 1), (64, 4), (100, 8), (160, 8), (160, 2)])
def test_each_near_partner_is_taken_by_one_task(n, C):
    rng = np.random.default_rng(n + C)
    parent = [-1] + [int(rng.integers(0, v)) for v in range(1, n)]  # a random rooted tree
    npad = -(-n // 32) * 32
    nb = npad // 32
    ntp, S, ntask = split(nb, C)
    tps = tile_pairs(nb)
    for i in range(n):
        I = i // 32
        partners = near_list(parent, i, 2)
        taken = [0] * len(partners)
        for w in range(ntask):
            TI, TJ = tps[w // S]
            if TI != I:
                continue
            count, share = (nb - I) * S, (TJ - I) * S + w % S
            for k in range(len(partners)):
                if k % count == share:
                    taken[k] += 1
        assert all(x == 1 for x in taken), (i, partners, taken)
        # the near list holds each partner once (the tree distance rule of N_d = 2)
        assert len(set(partners)) == len(partners)
