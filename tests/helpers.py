"""Independent closed forms and brute-force references used by the tests.

Nothing here calls the oracle or the CUDA library: these are the textbook facts the
oracle (and through it the GPU path) is pinned to.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def golden(name):
    """Values the paper prints, from tests/golden/<name>.txt (each file cites its passage):
    one `key value [unit]` per line, '#' starts a comment."""
    out = {}
    with open(f"{GOLDEN}/{name}.txt") as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out[line[0]] = float(line[1])
    return out


def two_body_invariants(m1, m2, r, v, G=1.0):
    """Energy E, angular momentum L and Laplace-Runge-Lenz vector A of the relative orbit
    (Sec. 5.1: E = mu v^2/2 - G mu M/r, L = mu r x v). A is taken with the specific angular
    momentum, A = v x (r x v) - G M r_hat, so that |A| = e G M; the printed form mixes
    mu-scaled and unscaled terms and is only invariant for mu = 1."""
    M = m1 + m2
    mu = m1 * m2 / M
    dr = r[1] - r[0]
    dv = v[1] - v[0]
    E = 0.5 * mu * dv @ dv - G * mu * M / np.linalg.norm(dr)
    L = mu * np.cross(dr, dv)
    A = np.cross(dv, np.cross(dr, dv)) - G * M * dr / np.linalg.norm(dr)
    return E, L, A


def kepler_propagate(dr0, dv0, mu, t):
    """Analytic two-body propagation of the relative state (dr0, dv0) by time t (bound
    orbit), via Kepler's equation and the Lagrange f and g functions."""
    r0 = np.linalg.norm(dr0)
    v0sq = dv0 @ dv0
    a = 1.0 / (2.0 / r0 - v0sq / mu)
    n = math.sqrt(mu / a ** 3)
    ecosE0 = 1.0 - r0 / a
    esinE0 = (dr0 @ dv0) / math.sqrt(mu * a)
    e = math.hypot(ecosE0, esinE0)
    E0 = math.atan2(esinE0, ecosE0)
    M = E0 - esinE0 + n * t
    E = M
    for _ in range(100):
        dE = (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
        E -= dE
        if abs(dE) < 1e-16:
            break
    dE = E - E0
    f = 1.0 - a / r0 * (1.0 - math.cos(dE))
    g = t - (dE - math.sin(dE)) / n
    dr = f * dr0 + g * dv0
    rr = np.linalg.norm(dr)
    fdot = -math.sqrt(mu * a) / (rr * r0) * math.sin(dE)
    gdot = 1.0 - a / rr * (1.0 - math.cos(dE))
    dv = fdot * dr0 + gdot * dv0
    return dr, dv


def sqdist(r, i, j):
    d = r[i] - r[j]
    return float(d @ d)


def edge_set(parent):
    return {(min(v, int(p)), max(v, int(p))) for v, p in enumerate(parent) if p >= 0}


def mst_bruteforce(r):
    """Minimum spanning tree of the complete graph by enumerating every labelled tree
    (Pruefer sequences, N^(N-2) of them) and keeping the lightest (Euclidean weights)."""
    n = len(r)
    w = {(i, j): math.sqrt(sqdist(r, i, j)) for i in range(n) for j in range(i + 1, n)}
    best = None
    best_edges = None
    for seq in itertools.product(range(n), repeat=n - 2):
        degree = [1] * n
        for x in seq:
            degree[x] += 1
        edges = []
        for x in seq:
            leaf = min(i for i in range(n) if degree[i] == 1)
            edges.append((min(leaf, x), max(leaf, x)))
            degree[leaf] -= 1
            degree[x] -= 1
        u, v = [i for i in range(n) if degree[i] == 1]
        edges.append((min(u, v), max(u, v)))
        tot = sum(w[e] for e in edges)
        if best is None or tot < best:
            best, best_edges = tot, set(edges)
    return best_edges


def mst_kruskal(r):
    """Kruskal's algorithm with union-find on squared distances."""
    n = len(r)
    edges = sorted((sqdist(r, i, j), i, j) for i in range(n) for j in range(i + 1, n))
    par = list(range(n))

    def find(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x

    out = set()
    for _, i, j in edges:
        a, b = find(i), find(j)
        if a != b:
            par[a] = b
            out.add((i, j))
    return out


def tree_distance_bfs(parent, src):
    """Hop distance from src to every vertex of the tree given by parent pointers."""
    n = len(parent)
    adj = [[] for _ in range(n)]
    for v, p in enumerate(parent):
        if p >= 0:
            adj[v].append(int(p))
            adj[int(p)].append(v)
    dist = [-1] * n
    dist[src] = 0
    q = [src]
    for u in q:
        for w in adj[u]:
            if dist[w] < 0:
                dist[w] = dist[u] + 1
                q.append(w)
    return dist


def tree_path(parent, i, j):
    """Vertices on the tree path from i to j."""
    anc_i = [i]
    while parent[anc_i[-1]] >= 0:
        anc_i.append(int(parent[anc_i[-1]]))
    anc_j = [j]
    while parent[anc_j[-1]] >= 0:
        anc_j.append(int(parent[anc_j[-1]]))
    set_j = set(anc_j)
    lca = next(x for x in anc_i if x in set_j)
    up = anc_i[: anc_i.index(lca) + 1]
    down = anc_j[: anc_j.index(lca)]
    return up + down[::-1]
