"""A model of the breadth-first orientation loop of k_orient (csrc/boruvka.cu), which turns the
undirected spanning tree of the step into parent and level (tree depth) arrays. CPU only.

Each warp is a coroutine over the shared queue, the shared tail counter and the visited marks;
a scheduler picks which warp runs next, so warps can be interleaved in any order the hardware
allows between barriers. Lanes of a warp share its reads of the tail; each lane expands its
queue entry in lane order and appends by an atomic increment of the tail.

The loop as first written read the level's end (the tail) right after the barrier that ends a
level. A warp that ran ahead could then expand its part of the level and append the next level
before a slower warp read the tail: the slow warp took a later end, expanded next-level vertices
a level early (their depth one short) and left the loop out of step with the others. The fixed
loop puts a barrier between every warp's read of the tail and any append.

The kernel now runs the walk in one warp (`run_warp_ballot` below): a level is taken 32 vertices
at a time, one per lane; in every round the lanes that found an unvisited neighbour append it at
their rank among them (a ballot), so there is no shared tail counter, no block barrier, and the
queue order is fixed given the adjacency lists.
"""
import numpy as np
import pytest

from tests import helpers as Hh


def random_tree(n, seed):
    rng = np.random.default_rng(seed)
    par = [-1] + [int(rng.integers(0, i)) for i in range(1, n)]
    perm = rng.permutation(n)
    edges = [(int(perm[v]), int(perm[par[v]])) for v in range(1, n)]
    root = int(perm[int(rng.integers(0, n))])
    return edges, root


def star_of_paths(arms, length):
    """A root with `arms` paths of `length` vertices: every level is wider than one warp's share."""
    edges, nxt = [], 1
    for _ in range(arms):
        prev = 0
        for _ in range(length):
            edges.append((prev, nxt))
            prev, nxt = nxt, nxt + 1
    return edges, 0


def run_model(n, edges, root, nwarps, lanes, policy, fixed, seed=0):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    S = {"qtail": 1}
    s_q = [0] * n
    s_a = [-2] * n
    level = [-9] * n
    s_a[root] = -1
    s_q[0] = root
    nt = nwarps * lanes

    def warp(w):
        h, depth = 0, 0
        while True:
            t = min(S["qtail"], n)  # every lane of the warp reads the same value
            yield "step"
            if fixed:
                yield "barrier"
            if h >= t:
                return
            it = 0
            while True:
                qs = [h + w * lanes + ln + it * nt for ln in range(lanes)]
                qs = [q for q in qs if q < t]
                if not qs:
                    break
                for q in qs:
                    u = s_q[q]
                    level[u] = depth
                    for x in adj[u]:
                        if s_a[x] == -2:
                            s_a[x] = u
                            slot = S["qtail"]
                            S["qtail"] += 1
                            if slot < n:
                                s_q[slot] = x
                    yield "step"
                it += 1
            h = t
            depth += 1
            yield "barrier"

    rng = np.random.default_rng(seed)
    gens = [warp(w) for w in range(nwarps)]
    state = ["run"] * nwarps
    diverged = False
    while True:
        runnable = [w for w in range(nwarps) if state[w] == "run"]
        if not runnable:
            waiting = [w for w in range(nwarps) if state[w] == "bar"]
            if not waiting:
                break
            # warps that left the loop count as arrived (as exited warps do on the GPU); a
            # barrier that others pass after some warps left is recorded as divergence
            diverged |= len(waiting) != nwarps
            state = ["run" if x == "bar" else x for x in state]
            continue
        w = runnable[0] if policy == "lowest_first" else int(rng.choice(runnable))
        try:
            ev = next(gens[w])
            if ev == "barrier":
                state[w] = "bar"
        except StopIteration:
            state[w] = "done"
    return s_a, level, s_q, diverged


def check(n, edges, root, s_a, level, s_q, diverged):
    parent_ref = [-1] * n
    dist = [-1] * n
    dist[root] = 0
    frontier = [root]
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    for u in frontier:
        for x in adj[u]:
            if dist[x] < 0:
                dist[x] = dist[u] + 1
                parent_ref[x] = u
                frontier.append(x)
    return not diverged and level == dist and s_a == parent_ref and sorted(s_q) == list(range(n))


def test_old_loop_mislevels_under_a_warp_that_runs_ahead():
    """Warp 0 runs until it blocks, so the other warps read the tail only after its appends:
    they expand vertices of the next level with this level's depth."""
    edges, root = star_of_paths(arms=12, length=4)
    n = len(edges) + 1
    s_a, level, s_q, diverged = run_model(n, edges, root, nwarps=3, lanes=2, policy="lowest_first", fixed=False)
    assert diverged
    depth = Hh.tree_distance_bfs(_parents(n, edges, root), root)
    assert any(0 <= level[v] < depth[v] for v in range(n))


def _parents(n, edges, root):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    par = [-1] * n
    seen = [False] * n
    seen[root] = True
    q = [root]
    for u in q:
        for x in adj[u]:
            if not seen[x]:
                seen[x] = True
                par[x] = u
                q.append(x)
    return par


@pytest.mark.parametrize("tree", ["star", "random40", "random200", "path"])
def test_fixed_loop_is_exact_under_every_schedule_tried(tree):
    if tree == "star":
        edges, root = star_of_paths(arms=12, length=4)
    elif tree == "path":
        edges, root = star_of_paths(arms=1, length=30)
    else:
        edges, root = random_tree(int(tree[6:]), seed=int(tree[6:]))
    n = len(edges) + 1
    for nwarps, lanes in ((1, 4), (3, 2), (4, 8)):
        assert check(n, edges, root, *run_model(n, edges, root, nwarps, lanes, "lowest_first", fixed=True))
        for seed in range(60):
            out = run_model(n, edges, root, nwarps, lanes, "random", fixed=True, seed=seed)
            assert check(n, edges, root, *out), (nwarps, lanes, seed)


def test_old_loop_fails_under_random_schedules_too():
    """Not only the hand-picked order: plain random interleavings break the old loop."""
    edges, root = random_tree(200, seed=200)
    n = len(edges) + 1
    bad = 0
    for seed in range(60):
        bad += not check(n, edges, root, *run_model(n, edges, root, 4, 8, "random", fixed=False, seed=seed))
    assert bad > 0


def run_warp_ballot(n, edges, root, lanes=32):
    """The one-warp loop of k_orient, lane by lane: the same reads, ballots and appends."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    s_q = [0] * n
    s_a = [-2] * n
    level = [-9] * n
    s_a[root] = -1
    s_q[0] = root
    h, t, depth = 0, 1, 0
    while h < t:
        tail = t
        for base in range(h, t, lanes):
            us = [s_q[base + ln] if base + ln < t else -1 for ln in range(lanes)]
            pos = [0] * lanes
            for ln, u in enumerate(us):
                if u >= 0:
                    level[u] = depth
            while any(u >= 0 and pos[ln] < len(adj[u]) for ln, u in enumerate(us)):
                found = []
                for ln, u in enumerate(us):   # every lane reads before any lane writes (one round)
                    w = -1
                    if u >= 0 and pos[ln] < len(adj[u]):
                        w = adj[u][pos[ln]]
                        pos[ln] += 1
                        if s_a[w] != -2:
                            w = -1
                    found.append(w)
                rank = 0
                for ln, w in enumerate(found):
                    if w >= 0:
                        s_a[w] = us[ln]
                        if tail + rank < n:
                            s_q[tail + rank] = w
                        rank += 1
                tail += rank
        h, t, depth = t, min(tail, n), depth + 1
    return s_a, level, s_q


@pytest.mark.parametrize("tree", ["star", "random40", "random200", "random2050", "path"])
@pytest.mark.parametrize("lanes", [4, 32])
def test_one_warp_ballot_loop_is_exact_and_level_ordered(tree, lanes):
    if tree == "star":
        edges, root = star_of_paths(arms=40, length=6)
    elif tree == "path":
        edges, root = star_of_paths(arms=1, length=70)
    else:
        edges, root = random_tree(int(tree[6:]), seed=int(tree[6:]))
    n = len(edges) + 1
    s_a, level, s_q = run_warp_ballot(n, edges, root, lanes)
    assert check(n, edges, root, s_a, level, s_q, False)
    # the queue lists the tree level by level, and the same order every time
    assert [level[u] for u in s_q] == sorted(level[u] for u in s_q)
    assert run_warp_ballot(n, edges, root, lanes)[2] == s_q
