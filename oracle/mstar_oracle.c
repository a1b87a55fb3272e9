/*
 * MSTAR oracle (see mstar_oracle.h). TEST INFRASTRUCTURE ONLY.
 *
 * Every function follows the paper's steps in its order and notation; nothing is
 * blocked, fused or reordered beyond what the definitions state. Section, equation
 * and algorithm names refer to Rantala et al., "MSTAR - a fast parallelised
 * algorithmically regularised integrator with minimum spanning tree coordinates".
 *
 * Readings taken where the paper is silent (the CUDA path implements the same):
 *  - (X, V, t) are the integrated variables; Cartesian r, v are rebuilt from them after
 *    every drift and kick (Sec. 2.2: chained velocities are transformed back).
 *  - Rebuild = per-vertex path sum of edge vectors, summed from the vertex up to the
 *    root, then a centre-of-mass shift (Sec. 3.5 counts L(V_i) additions per vertex).
 *  - Prim ties: argmin takes the lowest index; keys decrease only on strict '<'.
 *  - Error: eps = max over edge vectors X_v, V_v (3-vector norms) and the scalar t of
 *    |T_kk - T_{k-1,k-1}| / |S(s0) + (H/n_kfix) S'(s0)|, S' = V/(T+B), A/U, 1/(T+B).
 *  - Step growth factor a_GBS (eta/eps)^(1/(2 k_fix - 1)) clamped to [fac_min, fac_max].
 */
#include "mstar_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void orc_set_threads(int nthreads) { g_threads = nthreads < 1 ? 1 : nthreads; }
int orc_get_threads(void) { return g_threads; }

void orc_params_default(orc_params* p) {
  p->eta = 1e-12;
  p->a_gbs = 0.9;
  p->fac_min = 0.2;
  p->fac_max = 2.0;
  p->q_first = 0.1;
  p->t_tol = 1e-10;
  p->G = 1.0;
  p->k_fix = 8;
  p->n_d = 2;
  p->max_halvings = 30;
  p->max_time_iter = 8;
  p->mst_method = 0;
  p->mst_nsub = 0;
}

/* ---------------------------------------------------------------- energies (Eq. 1) */

static double norm2(const double* x) { return (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]; }

double orc_kinetic(int n, const double* m, const double* v) {
  double T = 0.0;
  for (int i = 0; i < n; ++i) T += m[i] * norm2(v + 3 * i);
  return 0.5 * T;
}

double orc_potential(int n, const double* m, const double* r, double G) {
  /* U = sum_i sum_{j>i} G m_i m_j / |r_j - r_i| */
  double U = 0.0;
  for (int i = 0; i < n; ++i) {
    double ui = 0.0;
    for (int j = i + 1; j < n; ++j) {
      double d[3] = {r[3 * j] - r[3 * i], r[3 * j + 1] - r[3 * i + 1], r[3 * j + 2] - r[3 * i + 2]};
      ui += m[j] / sqrt(norm2(d));
    }
    U += G * m[i] * ui;
  }
  return U;
}

void orc_com_shift(int n, const double* m, double* w) {
  double M = 0.0, c[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i) {
    M += m[i];
    for (int k = 0; k < 3; ++k) c[k] += m[i] * w[3 * i + k];
  }
  for (int k = 0; k < 3; ++k) c[k] = c[k] / M;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) w[3 * i + k] -= c[k];
}

/* ---------------------------------------------------------------- MST (Sec. 3.2, 3.4) */

/* Squared Euclidean edge weight. sqrt is monotone, so squared weights give the same MST
   as the Euclidean weights of Sec. 3.1. Two roundings per product/sum (no contraction). */
static double w2(const double* r, int u, int v) {
  double dx = r[3 * u] - r[3 * v], dy = r[3 * u + 1] - r[3 * v + 1], dz = r[3 * u + 2] - r[3 * v + 2];
  return (dx * dx + dy * dy) + dz * dz;
}

int orc_prim(int n, const double* r, int* parent, int* level, int* order) {
  /* Root: the particle spatially closest to the centre of mass (the origin of the COM
     frame); lowest index on ties. */
  int root = 0;
  double best = norm2(r);
  for (int i = 1; i < n; ++i) {
    double d = norm2(r + 3 * i);
    if (d < best) { best = d; root = i; }
  }
  double* key = (double*)malloc(sizeof(double) * (size_t)n);
  char* in_tree = (char*)calloc((size_t)n, 1);
  for (int v = 0; v < n; ++v) { key[v] = INFINITY; parent[v] = -1; level[v] = 0; }
  in_tree[root] = 1;
  order[0] = root;
  int u = root;
  for (int it = 1; it < n; ++it) {
    /* relax the keys of the non-tree vertices with the vertex just added */
    for (int v = 0; v < n; ++v) {
      if (in_tree[v]) continue;
      double d = w2(r, u, v);
      if (d < key[v]) { key[v] = d; parent[v] = u; }
    }
    /* add the non-tree vertex with the minimum-weight edge to the tree */
    int next = -1;
    double kmin = INFINITY;
    for (int v = 0; v < n; ++v) {
      if (in_tree[v]) continue;
      if (next < 0 || key[v] < kmin) { kmin = key[v]; next = v; }
    }
    u = next;
    in_tree[u] = 1;
    order[it] = u;
    if (parent[u] < 0) parent[u] = root; /* only reachable with non-finite positions */
    level[u] = level[parent[u]] + 1;
  }
  free(key);
  free(in_tree);
  return root;
}

/* ---------------------------------------------------------------- chained coordinates (Sec. 2.2) */

int orc_chain(int n, const double* r, int* parent, int* level, int* order) {
  /* the shortest inter-particle vector: its ends are the first tail and head (lowest pair
     (i, j), i < j, on ties; i is the tail) */
  int ti = 0, hj = 1;
  double best = w2(r, 0, 1);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double d = w2(r, i, j);
      if (d < best) { best = d; ti = i; hj = j; }
    }
  int* dq = (int*)malloc(sizeof(int) * (size_t)(2 * n)); /* the chain as a deque */
  char* in = (char*)calloc((size_t)n, 1);
  int lo = n, hi = n + 1;
  dq[lo] = ti; dq[hi] = hj;
  in[ti] = 1; in[hj] = 1;
  for (int added = 2; added < n; ++added) {
    /* the particle closest to either end; the tail wins a tie between the ends, then the
       lowest index */
    int tail = dq[lo], head = dq[hi], bp = -1, bend = 0;
    double bd = INFINITY;
    for (int p = 0; p < n; ++p) {
      if (in[p]) continue;
      double dt = w2(r, p, tail), dh = w2(r, p, head);
      int end = dh < dt ? 1 : 0;
      double d = end ? dh : dt;
      if (bp < 0 || d < bd) { bd = d; bp = p; bend = end; }
    }
    in[bp] = 1;
    if (bend) dq[++hi] = bp; else dq[--lo] = bp;
  }
  /* labels from the tail: edge vector X_k = r_{c_{k+1}} - r_{c_k}, stored at c_{k+1} */
  for (int k = 0; k < n; ++k) {
    int p = dq[lo + k];
    order[k] = p;
    parent[p] = k ? dq[lo + k - 1] : -1;
    level[p] = k;
  }
  int tail = dq[lo];
  free(dq);
  free(in);
  return tail;
}

/* Neumaier's compensated summation */
typedef struct { double s, c; } comp_sum;
static void comp_add(comp_sum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x; else a->c += (x - t) + a->s;
  a->s = t;
}

double orc_energy_comp(int n, const double* m, const double* r, const double* v, double G) {
  comp_sum T = {0.0, 0.0}, U = {0.0, 0.0};
  for (int i = 0; i < n; ++i) comp_add(&T, 0.5 * (m[i] * norm2(v + 3 * i)));
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) comp_add(&U, (G * (m[i] * m[j])) / sqrt(w2(r, i, j)));
  return (T.s + T.c) - (U.s + U.c);
}

/* Deconstruction with the root's position kept: w_v = (X_v + X_parent(v) + ...) + w_root. */
static void from_edges_keep_root(int n, const int* parent, int root, const double* W, double* w) {
  double r0[3] = {w[3 * root], w[3 * root + 1], w[3 * root + 2]};
  for (int v = 0; v < n; ++v) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int u = v; parent[u] >= 0; u = parent[u])
      for (int k = 0; k < 3; ++k) s[k] += W[3 * u + k];
    for (int k = 0; k < 3; ++k) w[3 * v + k] = s[k] + r0[k];
  }
}

/* Deconstruction from the root outwards: in insertion order (every parent before its
   children) w_v = w_parent(v) + X_v, starting from the root's kept position, so that a body
   and its parent differ by one rounding of their edge vector. */
static void from_edges_root_down(int n, const int* parent, const int* order, const double* W, double* w) {
  for (int k = 0; k < n; ++k) {
    int v = order[k], p = parent[v];
    if (p < 0) continue;
    for (int c = 0; c < 3; ++c) w[3 * v + c] = w[3 * p + c] + W[3 * v + c];
  }
}

int orc_rebuild_run(int n, const double* m, double* r, double* v, int coords, int deconstruct, int cycles,
                    int topo_every, int nsample, const int* sample_at, double* E_out, int* topo_changes,
                    double* mean_level) {
  if (n < 2 || cycles < 0 || topo_every < 1 || (coords != 0 && coords != 1) || deconstruct < 0 || deconstruct > 3)
    return ORC_ERR_ARG;
  size_t b3 = sizeof(double) * 3 * (size_t)n;
  int* parent = (int*)malloc(sizeof(int) * (size_t)n);
  int* prev = (int*)malloc(sizeof(int) * (size_t)n);
  int* level = (int*)malloc(sizeof(int) * (size_t)n);
  int* order = (int*)malloc(sizeof(int) * (size_t)n);
  double* X = (double*)malloc(b3);
  double* V = (double*)malloc(b3);
  int changes = 0, s = 0;
  double lsum = 0.0;
  int builds = 0;
  while (s < nsample && sample_at[s] == 0) E_out[s++] = orc_energy_comp(n, m, r, v, 1.0);
  for (int c = 1; c <= cycles; ++c) {
    if ((c - 1) % topo_every == 0) {
      if (coords == 0) orc_prim(n, r, parent, level, order);
      else orc_chain(n, r, parent, level, order);
      if (builds) for (int i = 0; i < n; ++i) if (parent[i] != prev[i]) { ++changes; break; }
      memcpy(prev, parent, sizeof(int) * (size_t)n);
      for (int i = 0; i < n; ++i) lsum += level[i];
      ++builds;
    }
    /* build the coordinates, deconstruct them (Sec. 3.5) */
    orc_to_mst(n, parent, r, X);
    orc_to_mst(n, parent, v, V);
    if (deconstruct == 0) {
      orc_from_mst(n, m, parent, X, r);
      orc_from_mst(n, m, parent, V, v);
    } else if (deconstruct == 1) {
      from_edges_keep_root(n, parent, order[0], X, r);
      from_edges_keep_root(n, parent, order[0], V, v);
    } else {
      from_edges_root_down(n, parent, order, X, r);
      from_edges_root_down(n, parent, order, V, v);
      if (deconstruct == 3) {
        orc_com_shift(n, m, r);
        orc_com_shift(n, m, v);
      }
    }
    while (s < nsample && sample_at[s] == c) E_out[s++] = orc_energy_comp(n, m, r, v, 1.0);
  }
  if (topo_changes) *topo_changes = changes;
  if (mean_level) *mean_level = builds ? lsum / ((double)builds * n) : 0.0;
  free(parent); free(prev); free(level); free(order); free(X); free(V);
  return ORC_OK;
}

/* ---------------------------------------------------------------- divide-and-conquer MST (Sec. 3.3) */

#define DC_DEPTH 16

typedef struct {
  double d2;
  int i, j; /* i in the lower-numbered subgraph */
} dc_edge;

/* lexicographic (d2, i, j) */
static int dc_less(dc_edge a, dc_edge b) {
  if (a.d2 != b.d2) return a.d2 < b.d2;
  if (a.i != b.i) return a.i < b.i;
  return a.j < b.j;
}

typedef struct {
  int nleaf;
  int* leaf_of;     /* subgraph of each body */
  int* leaf_start;  /* bodies of subgraph g: members[leaf_start[g] .. leaf_start[g+1]) */
  int* members;     /* ascending body index within each subgraph */
} dc_tree;

/* The octree partition into about `target` subgraphs: starting from the bounding cube,
   the cell holding the most bodies (the first in Morton order on ties) is replaced by its
   non-empty children, until there are at least `target` cells or the most populous cell
   cannot be split (one body, or depth DC_DEPTH). Children are ordered by their Morton
   digit (x, y, z bits from most to least significant), so the cells stay in Morton order.
   A cell is the range [lo, hi) of the bodies sorted by (key, index). */
typedef struct {
  int depth, lo, hi;
} dc_cell;

static int dc_partition(int n, const unsigned long long* skey, int target, dc_cell* cells) {
  int nc = 1;
  cells[0].depth = 0; cells[0].lo = 0; cells[0].hi = n;
  while (nc < target) {
    int best = 0;
    for (int c = 1; c < nc; ++c)
      if (cells[c].hi - cells[c].lo > cells[best].hi - cells[best].lo) best = c;
    dc_cell b = cells[best];
    if (b.hi - b.lo <= 1 || b.depth == DC_DEPTH) break;
    int shift = 3 * (DC_DEPTH - b.depth - 1);
    dc_cell kids[8];
    int nk = 0, p = b.lo;
    for (int dgt = 0; dgt < 8; ++dgt) {
      int q = p;
      while (q < b.hi && (int)((skey[q] >> shift) & 7u) == dgt) ++q;
      if (q > p) { kids[nk].depth = b.depth + 1; kids[nk].lo = p; kids[nk].hi = q; ++nk; }
      p = q;
    }
    for (int c = nc - 1; c > best; --c) cells[c + nk - 1] = cells[c];
    for (int k = 0; k < nk; ++k) cells[best + k] = kids[k];
    nc += nk - 1;
  }
  return nc;
}

int orc_dc_mst(int n, const double* r, int nsub, int* parent, int* level, int* order, int* leaf_of_out,
               int* nleaf_out) {
  /* root as for Prim: the body closest to the centre of mass, lowest index on ties */
  int root = 0;
  double best = norm2(r);
  for (int i = 1; i < n; ++i) {
    double d = norm2(r + 3 * i);
    if (d < best) { best = d; root = i; }
  }
  int target = nsub > 0 ? nsub : (int)ceil(sqrt((double)n));
  /* bounding cube: centre of the per-axis extent, half-size of the largest extent */
  double mn[3], mx[3], c0[3], hs = 0.0;
  for (int k = 0; k < 3; ++k) { mn[k] = r[k]; mx[k] = r[k]; }
  for (int i = 1; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      if (r[3 * i + k] < mn[k]) mn[k] = r[3 * i + k];
      if (r[3 * i + k] > mx[k]) mx[k] = r[3 * i + k];
    }
  for (int k = 0; k < 3; ++k) {
    c0[k] = (mn[k] + mx[k]) * 0.5;
    double e = (mx[k] - mn[k]) * 0.5;
    if (e > hs) hs = e;
  }
  /* Morton key of the cell path: at each depth the child is chosen by x >= centre */
  unsigned long long* key = (unsigned long long*)malloc(sizeof(unsigned long long) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    double c[3] = {c0[0], c0[1], c0[2]}, h = hs;
    unsigned long long kk = 0;
    for (int d = 0; d < DC_DEPTH; ++d) {
      h = h * 0.5;
      unsigned bits = 0;
      for (int k = 0; k < 3; ++k) {
        int b = r[3 * i + k] >= c[k];
        bits = (bits << 1) | (unsigned)b;
        c[k] = b ? c[k] + h : c[k] - h;
      }
      kk = (kk << 3) | bits;
    }
    key[i] = kk;
  }
  /* bodies sorted by (key, index): each cell of the partition is a contiguous range */
  int* sorted = (int*)malloc(sizeof(int) * (size_t)n);
  for (int i = 0; i < n; ++i) sorted[i] = i;
  for (int a = 1; a < n; ++a) { /* insertion sort by (key, index) */
    int x = sorted[a], b = a - 1;
    while (b >= 0 && (key[sorted[b]] > key[x] || (key[sorted[b]] == key[x] && sorted[b] > x))) {
      sorted[b + 1] = sorted[b];
      --b;
    }
    sorted[b + 1] = x;
  }
  unsigned long long* skey = (unsigned long long*)malloc(sizeof(unsigned long long) * (size_t)n);
  for (int q = 0; q < n; ++q) skey[q] = key[sorted[q]];
  dc_cell* cells = (dc_cell*)malloc(sizeof(dc_cell) * (size_t)(n + 8));
  int ncell = dc_partition(n, skey, target, cells);
  dc_tree t;
  t.leaf_of = (int*)malloc(sizeof(int) * (size_t)n);
  t.leaf_start = (int*)malloc(sizeof(int) * (size_t)(n + 1));
  t.members = (int*)malloc(sizeof(int) * (size_t)n);
  t.nleaf = ncell;
  for (int g = 0; g < ncell; ++g) {
    t.leaf_start[g] = cells[g].lo;
    /* members of the subgraph in ascending body index */
    int cnt = cells[g].hi - cells[g].lo;
    for (int q = 0; q < cnt; ++q) t.members[cells[g].lo + q] = sorted[cells[g].lo + q];
    for (int a = 1; a < cnt; ++a) {
      int* mm = t.members + cells[g].lo;
      int x = mm[a], b = a - 1;
      while (b >= 0 && mm[b] > x) { mm[b + 1] = mm[b]; --b; }
      mm[b + 1] = x;
    }
    for (int q = 0; q < cnt; ++q) t.leaf_of[t.members[cells[g].lo + q]] = g;
  }
  t.leaf_start[ncell] = n;
  free(sorted); free(skey); free(cells);
  int ng = t.nleaf;
  int* eu = (int*)malloc(sizeof(int) * (size_t)n);
  int* ev = (int*)malloc(sizeof(int) * (size_t)n);
  int ne = 0;
  /* Prim's algorithm inside every subgraph (complete graph on its bodies), from its lowest
     index; keys replaced only by strictly smaller distances; argmin lowest index */
  double* kd = (double*)malloc(sizeof(double) * (size_t)n);
  int* kp = (int*)malloc(sizeof(int) * (size_t)n);
  char* in = (char*)calloc((size_t)n, 1);
  for (int g = 0; g < ng; ++g) {
    const int* mem = t.members + t.leaf_start[g];
    int cnt = t.leaf_start[g + 1] - t.leaf_start[g];
    for (int q = 0; q < cnt; ++q) { kd[mem[q]] = INFINITY; kp[mem[q]] = -1; }
    int u = mem[0];
    in[u] = 1;
    for (int it = 1; it < cnt; ++it) {
      for (int q = 0; q < cnt; ++q) {
        int v = mem[q];
        if (in[v]) continue;
        double d = w2(r, u, v);
        if (d < kd[v]) { kd[v] = d; kp[v] = u; }
      }
      int nx = -1;
      for (int q = 0; q < cnt; ++q) {
        int v = mem[q];
        if (in[v]) continue;
        if (nx < 0 || kd[v] < kd[nx]) nx = v;
      }
      in[nx] = 1;
      eu[ne] = kp[nx]; ev[ne] = nx; ++ne;
      u = nx;
    }
  }
  free(kd); free(kp); free(in);
  /* meta-graph: subgraphs contracted to vertices; the weight of (a, b) is the cheapest
     edge between them (cut property), ties by the lowest (i in a, j in b) */
  dc_edge* W = (dc_edge*)malloc(sizeof(dc_edge) * (size_t)ng * (size_t)ng);
  for (int a = 0; a < ng; ++a)
    for (int b = a + 1; b < ng; ++b) {
      dc_edge e = {INFINITY, -1, -1};
      for (int p = t.leaf_start[a]; p < t.leaf_start[a + 1]; ++p)
        for (int q = t.leaf_start[b]; q < t.leaf_start[b + 1]; ++q) {
          dc_edge c = {w2(r, t.members[p], t.members[q]), t.members[p], t.members[q]};
          if (e.i < 0 || dc_less(c, e)) e = c;
        }
      W[(size_t)a * ng + b] = e;
      W[(size_t)b * ng + a] = e;
    }
  /* Prim's algorithm on the meta-graph from subgraph 0 */
  if (ng > 1) {
    dc_edge* key2 = (dc_edge*)malloc(sizeof(dc_edge) * (size_t)ng);
    char* in2 = (char*)calloc((size_t)ng, 1);
    for (int g = 0; g < ng; ++g) key2[g].i = -1;
    int u = 0;
    in2[0] = 1;
    for (int it = 1; it < ng; ++it) {
      for (int g = 0; g < ng; ++g) {
        if (in2[g]) continue;
        dc_edge c = W[(size_t)u * ng + g];
        if (key2[g].i < 0 || dc_less(c, key2[g])) key2[g] = c;
      }
      int nx = -1;
      for (int g = 0; g < ng; ++g) {
        if (in2[g]) continue;
        if (nx < 0 || dc_less(key2[g], key2[nx])) nx = g;
      }
      in2[nx] = 1;
      eu[ne] = key2[nx].i; ev[ne] = key2[nx].j; ++ne;
      u = nx;
    }
    free(key2); free(in2);
  }
  free(W);
  /* the union of the edges, ordered and labelled by a breadth-first walk from the root
     (neighbours in ascending index) */
  int* deg = (int*)calloc((size_t)n + 1, sizeof(int));
  for (int e = 0; e < ne; ++e) { deg[eu[e] + 1]++; deg[ev[e] + 1]++; }
  for (int i = 0; i < n; ++i) deg[i + 1] += deg[i];
  int* adj = (int*)malloc(sizeof(int) * (size_t)(2 * ne + 1));
  int* fill = (int*)calloc((size_t)n, sizeof(int));
  for (int e = 0; e < ne; ++e) {
    adj[deg[eu[e]] + fill[eu[e]]++] = ev[e];
    adj[deg[ev[e]] + fill[ev[e]]++] = eu[e];
  }
  for (int i = 0; i < n; ++i) { /* ascending neighbours: insertion sort of each list */
    for (int a = deg[i] + 1; a < deg[i + 1]; ++a) {
      int x = adj[a], b = a - 1;
      while (b >= deg[i] && adj[b] > x) { adj[b + 1] = adj[b]; --b; }
      adj[b + 1] = x;
    }
  }
  for (int i = 0; i < n; ++i) { parent[i] = -2; level[i] = 0; }
  parent[root] = -1;
  int head = 0, tail = 0;
  order[tail++] = root;
  while (head < tail) {
    int u = order[head++];
    for (int a = deg[u]; a < deg[u + 1]; ++a) {
      int w = adj[a];
      if (parent[w] == -2) { parent[w] = u; level[w] = level[u] + 1; order[tail++] = w; }
    }
  }
  if (leaf_of_out) memcpy(leaf_of_out, t.leaf_of, sizeof(int) * (size_t)n);
  if (nleaf_out) *nleaf_out = ng;
  free(deg); free(adj); free(fill);
  free(eu); free(ev);
  free(key); free(t.leaf_of); free(t.leaf_start); free(t.members);
  return root;
}

/* Eq. LCA with early exit: lift the deeper vertex, then both, counting traversed edges;
   the count at the lowest common ancestor is |L(V_i)-L(V_LCA)| + |L(V_j)-L(V_LCA)|. */
int orc_is_near(const int* parent, const int* level, int i, int j, int n_d) {
  if (i == j) return 0;
  int d = 0;
  while (level[i] > level[j]) { i = parent[i]; if (++d > n_d) return 0; }
  while (level[j] > level[i]) { j = parent[j]; if (++d > n_d) return 0; }
  while (i != j) {
    i = parent[i];
    j = parent[j];
    d += 2;
    if (d > n_d) return 0;
  }
  return 1;
}

/* r_j - r_i = (sum of X from j up to the LCA) - (sum of X from i up to the LCA), each
   sum accumulated upward starting at the vertex itself (Sec. 3.4). */
void orc_near_sep(const int* parent, const int* level, const double* X, int i, int j, double d[3]) {
  double si[3] = {0.0, 0.0, 0.0}, sj[3] = {0.0, 0.0, 0.0};
  int a = i, b = j;
  /* find the LCA first */
  while (level[a] > level[b]) a = parent[a];
  while (level[b] > level[a]) b = parent[b];
  while (a != b) { a = parent[a]; b = parent[b]; }
  int lca = a;
  for (int u = i; u != lca; u = parent[u])
    for (int k = 0; k < 3; ++k) si[k] += X[3 * u + k];
  for (int u = j; u != lca; u = parent[u])
    for (int k = 0; k < 3; ++k) sj[k] += X[3 * u + k];
  for (int k = 0; k < 3; ++k) d[k] = sj[k] - si[k];
}

void orc_to_mst(int n, const int* parent, const double* w, double* W) {
  for (int v = 0; v < n; ++v) {
    int p = parent[v];
    for (int k = 0; k < 3; ++k) W[3 * v + k] = (p < 0) ? 0.0 : w[3 * v + k] - w[3 * p + k];
  }
}

void orc_from_mst(int n, const double* m, const int* parent, const double* W, double* w) {
  for (int v = 0; v < n; ++v) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int u = v; parent[u] >= 0; u = parent[u])
      for (int k = 0; k < 3; ++k) s[k] += W[3 * u + k];
    for (int k = 0; k < 3; ++k) w[3 * v + k] = s[k];
  }
  orc_com_shift(n, m, w);
}

/* ---------------------------------------------------------------- forces (Eq. 2) */

void orc_forces(int n, const double* m, double G, const int* parent, const int* level, int n_d,
                const double* r, const double* X, double* a, double* U) {
  double* ui = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
  for (int i = 0; i < n; ++i) {
    double ai[3] = {0.0, 0.0, 0.0}, u = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      if (n_d > 0 && orc_is_near(parent, level, i, j, n_d)) {
        orc_near_sep(parent, level, X, i, j, d);
      } else {
        for (int k = 0; k < 3; ++k) d[k] = r[3 * j + k] - r[3 * i + k];
      }
      double rinv = 1.0 / sqrt(norm2(d));
      double s = G * m[j] * (rinv * rinv * rinv);
      for (int k = 0; k < 3; ++k) ai[k] += s * d[k];
      if (j > i) u += m[j] * rinv;
    }
    for (int k = 0; k < 3; ++k) a[3 * i + k] = ai[k];
    ui[i] = u;
  }
  double Us = 0.0;
  for (int i = 0; i < n; ++i) Us += G * m[i] * ui[i];
  *U = Us;
  free(ui);
}

/* ---------------------------------------------------------------- GBS (Sec. 2.3, 4.2) */

typedef void (*orc_op)(void* ctx, double h);

/* The leapfrog with n substeps over an interval h:
   D(h/2n) [K(h/n) D(h/n)]^(n-1) K(h/n) D(h/2n). */
static void orc_dkd(int n, double h, orc_op drift, orc_op kick, void* ctx) {
  double d = h / n;
  drift(ctx, 0.5 * d);
  for (int i = 0; i < n - 1; ++i) {
    kick(ctx, d);
    drift(ctx, d);
  }
  kick(ctx, d);
  drift(ctx, 0.5 * d);
}

void orc_neville(int kf, const int* nseq, int nvar, const double* S, double* Tkk, double* Tprev) {
  double* prev = (double*)malloc(sizeof(double) * (size_t)kf);
  double* cur = (double*)malloc(sizeof(double) * (size_t)kf);
  for (int q = 0; q < nvar; ++q) {
    for (int k = 0; k < kf; ++k) {
      cur[0] = S[(size_t)k * nvar + q];
      for (int j = 1; j <= k; ++j) {
        double ratio = (double)nseq[k] / (double)nseq[k - j];
        cur[j] = cur[j - 1] + (cur[j - 1] - prev[j - 1]) / (ratio * ratio - 1.0);
      }
      if (k == kf - 2) Tprev[q] = cur[k];
      double* t = prev; prev = cur; cur = t;
    }
    Tkk[q] = prev[kf - 1];
  }
  free(prev);
  free(cur);
}

int orc_div_assign(int kf, int ndiv, int* group) {
  int* load = (int*)calloc((size_t)ndiv, sizeof(int));
  for (int k = kf; k >= 1; --k) { /* n_k = 2k, largest first */
    int g = 0;
    for (int i = 1; i < ndiv; ++i)
      if (load[i] < load[g]) g = i;
    load[g] += 2 * k;
    group[k - 1] = g;
  }
  int mx = 0;
  for (int i = 0; i < ndiv; ++i) if (load[i] > mx) mx = load[i];
  free(load);
  return mx;
}

/* harmonic oscillator with the plain (0,0,1) leapfrog: drift x += h p, kick p -= h w^2 x */
typedef struct { double x, p, w; } harm_ctx;
static void harm_drift(void* c, double h) { harm_ctx* s = (harm_ctx*)c; s->x += h * s->p; }
static void harm_kick(void* c, double h) { harm_ctx* s = (harm_ctx*)c; s->p -= h * (s->w * s->w) * s->x; }

void orc_gbs_harmonic(double w, double x0, double p0, double H, int kf, double* out, double* out_prev) {
  int* nseq = (int*)malloc(sizeof(int) * (size_t)kf);
  double* S = (double*)malloc(sizeof(double) * 2 * (size_t)kf);
  for (int k = 0; k < kf; ++k) {
    nseq[k] = 2 * (k + 1);
    harm_ctx c = {x0, p0, w};
    orc_dkd(nseq[k], H, harm_drift, harm_kick, &c);
    S[2 * k] = c.x;
    S[2 * k + 1] = c.p;
  }
  orc_neville(kf, nseq, 2, S, out, out_prev);
  free(nseq);
  free(S);
}

/* ---------------------------------------------------------------- N-body system */

struct orc_system {
  int n;
  orc_params p;
  double *m, *r, *v;  /* Cartesian state, COM frame */
  double t, B, H;     /* physical time, binding energy B = -H_ham, next fictitious step */
  long long force_evals;
  /* per-step work */
  int *parent, *level, *order;
  int root;
  double *X0, *V0, *a0, *A0;
  double T0, U0;
  /* per-division work */
  double *S;          /* kf x (6n+1) division results */
  double *Tkk, *Tprev;
};

/* one leapfrog division's mutable state (the LogH equations of motion, Sec. 2.1-2.2) */
typedef struct {
  orc_system* s;
  double *X, *V, *r, *v, *a;
  double t, T, U;
} orc_div;

/* D(h): dX/ds = V/(T+B), dt/ds = 1/(T+B); then the Cartesian positions are rebuilt. */
static void nb_drift(void* c, double h) {
  orc_div* d = (orc_div*)c;
  orc_system* s = d->s;
  double f = h / (d->T + s->B);
  for (int v = 0; v < s->n; ++v)
    for (int k = 0; k < 3; ++k) d->X[3 * v + k] += f * d->V[3 * v + k];
  d->t += f;
  orc_from_mst(s->n, s->m, s->parent, d->X, d->r);
}

/* K(h): dV/ds = A/U with A_v = a_v - a_parent(v); then v is rebuilt and T updated. */
static void nb_kick(void* c, double h) {
  orc_div* d = (orc_div*)c;
  orc_system* s = d->s;
  orc_forces(s->n, s->m, s->p.G, s->parent, s->level, s->p.n_d, d->r, d->X, d->a, &d->U);
  s->force_evals++;
  double f = h / d->U;
  for (int v = 0; v < s->n; ++v) {
    int pv = s->parent[v];
    if (pv < 0) continue;
    for (int k = 0; k < 3; ++k) d->V[3 * v + k] += f * (d->a[3 * v + k] - d->a[3 * pv + k]);
  }
  orc_from_mst(s->n, s->m, s->parent, d->V, d->v);
  d->T = orc_kinetic(s->n, s->m, d->v);
}

static int all_finite(int n, const double* x) {
  for (int i = 0; i < n; ++i) if (!isfinite(x[i])) return 0;
  return 1;
}

orc_system* orc_create(int n, const double* m, const double* r, const double* v, const orc_params* p) {
  if (n < 2 || !p || p->k_fix < 2 || p->n_d < 0) return NULL;
  for (int i = 0; i < n; ++i) if (!(m[i] > 0.0) || !isfinite(m[i])) return NULL;
  if (!all_finite(3 * n, r) || !all_finite(3 * n, v)) return NULL;
  orc_system* s = (orc_system*)calloc(1, sizeof(orc_system));
  s->n = n;
  s->p = *p;
  size_t n3 = sizeof(double) * 3 * (size_t)n;
  s->m = (double*)malloc(sizeof(double) * (size_t)n);
  s->r = (double*)malloc(n3);
  s->v = (double*)malloc(n3);
  memcpy(s->m, m, sizeof(double) * (size_t)n);
  memcpy(s->r, r, n3);
  memcpy(s->v, v, n3);
  orc_com_shift(n, s->m, s->r);
  orc_com_shift(n, s->m, s->v);
  double T = orc_kinetic(n, s->m, s->v), U = orc_potential(n, s->m, s->r, p->G);
  s->B = U - T; /* B = -H with H = T - U (Eq. 1) */
  s->t = 0.0;
  s->H = 0.0;   /* unset: the first step uses ds = q U dt */
  s->parent = (int*)malloc(sizeof(int) * (size_t)n);
  s->level = (int*)malloc(sizeof(int) * (size_t)n);
  s->order = (int*)malloc(sizeof(int) * (size_t)n);
  s->X0 = (double*)malloc(n3);
  s->V0 = (double*)malloc(n3);
  s->a0 = (double*)malloc(n3);
  s->A0 = (double*)malloc(n3);
  size_t nv = 6 * (size_t)n + 1;
  s->S = (double*)malloc(sizeof(double) * nv * (size_t)p->k_fix);
  s->Tkk = (double*)malloc(sizeof(double) * nv);
  s->Tprev = (double*)malloc(sizeof(double) * nv);
  return s;
}

void orc_free(orc_system* s) {
  if (!s) return;
  free(s->m); free(s->r); free(s->v);
  free(s->parent); free(s->level); free(s->order);
  free(s->X0); free(s->V0); free(s->a0); free(s->A0);
  free(s->S); free(s->Tkk); free(s->Tprev);
  free(s);
}

void orc_get_state(const orc_system* s, double* t, double* r, double* v, double* H, double* B) {
  size_t n3 = sizeof(double) * 3 * (size_t)s->n;
  if (t) *t = s->t;
  if (r) memcpy(r, s->r, n3);
  if (v) memcpy(v, s->v, n3);
  if (H) *H = s->H;
  if (B) *B = s->B;
}

void orc_set_H(orc_system* s, double H) { s->H = H; }

/* Start of a GBS step: MST of the current positions, edge vectors, and the derivative
   information at s0 that the convergence criterion needs (one force evaluation). */
static void orc_prepare(orc_system* s) {
  int n = s->n;
  if (s->p.mst_method == 1)
    s->root = orc_dc_mst(n, s->r, s->p.mst_nsub, s->parent, s->level, s->order, NULL, NULL);
  else
    s->root = orc_prim(n, s->r, s->parent, s->level, s->order);
  orc_to_mst(n, s->parent, s->r, s->X0);
  orc_to_mst(n, s->parent, s->v, s->V0);
  s->T0 = orc_kinetic(n, s->m, s->v);
  orc_forces(n, s->m, s->p.G, s->parent, s->level, s->p.n_d, s->r, s->X0, s->a0, &s->U0);
  s->force_evals++;
  orc_to_mst(n, s->parent, s->a0, s->A0);
}

static double vnorm(double x, double y, double z) { return sqrt((x * x + y * y) + z * z); }

/* Eq. gbs-criterion in the reading R6-R8: the change between the last two extrapolants,
   relative to the state advanced by one substep delta = H/n_kfix (n_kfix = 2 k_fix, Eq.
   seq-deuflhard) along its derivative at the step start s0 (the LogH equations, Sec. 2.1:
   dX/ds = V/(T+B), dV/ds = A/U, dt/ds = 1/(T+B)), as a Euclidean norm per 3-vector. */
double orc_gbs_error(int n, const int* parent, const double* Tkk, const double* Tprev, const double* X0,
                     const double* V0, const double* A0, double t0, double T0, double B, double U0, double H,
                     int k_fix) {
  double delta = H / (2 * k_fix);
  double rate = 1.0 / (T0 + B);
  double eps = 0.0;
  int nan_seen = 0;
  for (int v = 0; v < n; ++v) {
    if (parent[v] < 0) continue;
    const double* dX = Tkk + 3 * v; const double* pX = Tprev + 3 * v;
    const double* dV = Tkk + 3 * (size_t)n + 3 * v; const double* pV = Tprev + 3 * (size_t)n + 3 * v;
    const double* x0 = X0 + 3 * v; const double* v0 = V0 + 3 * v; const double* a0 = A0 + 3 * v;
    double num = vnorm(dX[0] - pX[0], dX[1] - pX[1], dX[2] - pX[2]);
    double den = vnorm(x0[0] + delta * (v0[0] * rate), x0[1] + delta * (v0[1] * rate),
                       x0[2] + delta * (v0[2] * rate));
    double q = num / fmax(den, 1e-300);
    if (isnan(q)) nan_seen = 1; else if (q > eps) eps = q;
    num = vnorm(dV[0] - pV[0], dV[1] - pV[1], dV[2] - pV[2]);
    den = vnorm(v0[0] + delta * (a0[0] / U0), v0[1] + delta * (a0[1] / U0), v0[2] + delta * (a0[2] / U0));
    q = num / fmax(den, 1e-300);
    if (isnan(q)) nan_seen = 1; else if (q > eps) eps = q;
  }
  {
    double num = fabs(Tkk[6 * (size_t)n] - Tprev[6 * (size_t)n]);
    double den = fabs(t0 + delta * rate);
    double q = num / fmax(den, 1e-300);
    if (isnan(q)) nan_seen = 1; else if (q > eps) eps = q;
  }
  return nan_seen ? NAN : eps;
}

/* k_fix leapfrog divisions from the current state, Neville-Aitken extrapolation, and the
   error of Eq. gbs-criterion. Leaves T_{kf,kf} in s->Tkk. Returns eps (NaN if any ratio
   is not a number). */
static double orc_divisions(orc_system* s, double H) {
  int n = s->n, kf = s->p.k_fix;
  size_t nv = 6 * (size_t)n + 1, n3 = sizeof(double) * 3 * (size_t)n;
  int* nseq = (int*)malloc(sizeof(int) * (size_t)kf);
  orc_div d;
  d.s = s;
  d.X = (double*)malloc(n3); d.V = (double*)malloc(n3);
  d.r = (double*)malloc(n3); d.v = (double*)malloc(n3); d.a = (double*)malloc(n3);
  for (int k = 0; k < kf; ++k) {
    nseq[k] = 2 * (k + 1);
    memcpy(d.X, s->X0, n3); memcpy(d.V, s->V0, n3);
    memcpy(d.r, s->r, n3); memcpy(d.v, s->v, n3);
    d.t = s->t; d.T = s->T0; d.U = s->U0;
    orc_dkd(nseq[k], H, nb_drift, nb_kick, &d);
    double* Sk = s->S + (size_t)k * nv;
    memcpy(Sk, d.X, n3);
    memcpy(Sk + 3 * (size_t)n, d.V, n3);
    Sk[6 * (size_t)n] = d.t;
  }
  orc_neville(kf, nseq, (int)nv, s->S, s->Tkk, s->Tprev);
  double eps = orc_gbs_error(n, s->parent, s->Tkk, s->Tprev, s->X0, s->V0, s->A0, s->t, s->T0, s->B, s->U0, H, kf);
  free(nseq);
  free(d.X); free(d.V); free(d.r); free(d.v); free(d.a);
  return eps;
}

int orc_attempt(orc_system* s, double H, double* eps, double* r_out, double* v_out, double* t_out,
                double* U0_out) {
  int n = s->n;
  orc_prepare(s);
  double e = orc_divisions(s, H);
  if (eps) *eps = e;
  if (U0_out) *U0_out = s->U0;
  if (r_out) orc_from_mst(n, s->m, s->parent, s->Tkk, r_out);
  if (v_out) orc_from_mst(n, s->m, s->parent, s->Tkk + 3 * (size_t)n, v_out);
  if (t_out) *t_out = s->Tkk[6 * (size_t)n];
  return ORC_OK;
}

int orc_leapfrog(orc_system* s, int nsub, double H, double* r_out, double* v_out, double* t_out) {
  int n = s->n;
  size_t n3 = sizeof(double) * 3 * (size_t)n;
  orc_prepare(s);
  orc_div d;
  d.s = s;
  d.X = (double*)malloc(n3); d.V = (double*)malloc(n3);
  d.r = (double*)malloc(n3); d.v = (double*)malloc(n3); d.a = (double*)malloc(n3);
  memcpy(d.X, s->X0, n3); memcpy(d.V, s->V0, n3);
  memcpy(d.r, s->r, n3); memcpy(d.v, s->v, n3);
  d.t = s->t; d.T = s->T0; d.U = s->U0;
  orc_dkd(nsub, H, nb_drift, nb_kick, &d);
  if (r_out) orc_from_mst(n, s->m, s->parent, d.X, r_out);
  if (v_out) orc_from_mst(n, s->m, s->parent, d.V, v_out);
  if (t_out) *t_out = d.t;
  free(d.X); free(d.V); free(d.r); free(d.v); free(d.a);
  return ORC_OK;
}

void orc_set_state(orc_system* s, double t, const double* r, const double* v) {
  size_t n3 = sizeof(double) * 3 * (size_t)s->n;
  s->t = t;
  memcpy(s->r, r, n3);
  memcpy(s->v, v, n3);
}

int orc_integrate(orc_system* s, double t_end, int max_steps, orc_stats* st) {
  const orc_params* p = &s->p;
  int kf = p->k_fix;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  long long fe0 = s->force_evals;
  int rc = ORC_OK;
  double tol = p->t_tol * fabs(t_end);
  while (st->accepted < max_steps) {
    if (fabs(t_end - s->t) <= tol) break;
    orc_prepare(s);
    /* Sec. 2.4: the first step is ds = q U dt; afterwards the GBS controller's step,
       clamped so that the estimated end time t + ds/U does not pass t_end; past t_end
       (an overshoot) further steps of ds = U (t_end - t) head back to it. */
    double dt = t_end - s->t;
    double Hs = (s->H == 0.0) ? p->q_first * s->U0 * dt : fabs(s->H) * (dt < 0 ? -1.0 : 1.0);
    int clamped = 0;
    if (fabs(Hs / s->U0) >= fabs(dt)) { Hs = s->U0 * dt; clamped = 1; }
    if (clamped) {
      if (st->time_iters >= p->max_time_iter) break;
      st->time_iters++;
    }
    double eps = 0.0;
    int halvings = 0;
    for (;;) {
      eps = orc_divisions(s, Hs);
      if (eps <= p->eta) break;
      st->rejected++;
      if (++halvings > p->max_halvings) { rc = ORC_ERR_NO_CONVERGENCE; goto done; }
      Hs *= 0.5;
    }
    /* accept: deconstruct the extrapolated MST coordinates into the Cartesian state */
    orc_from_mst(s->n, s->m, s->parent, s->Tkk, s->r);
    orc_from_mst(s->n, s->m, s->parent, s->Tkk + 3 * (size_t)s->n, s->v);
    s->t = s->Tkk[6 * (size_t)s->n];
    /* Eq. hnext with k = k_fix */
    double fac = (eps > 0.0) ? p->a_gbs * pow(p->eta / eps, 1.0 / (2 * kf - 1)) : p->fac_max;
    if (fac < p->fac_min) fac = p->fac_min;
    if (fac > p->fac_max) fac = p->fac_max;
    s->H = fac * Hs;
    st->accepted++;
    st->eps_last = eps;
  }
done:
  st->force_evals = s->force_evals - fe0;
  st->H = s->H;
  st->t = s->t;
  return rc;
}

void orc_energy(const orc_system* s, double* E, double* T, double* U, double P[3], double L[3]) {
  int n = s->n;
  double t = orc_kinetic(n, s->m, s->v), u = orc_potential(n, s->m, s->r, s->p.G);
  if (T) *T = t;
  if (U) *U = u;
  if (E) *E = t - u;
  double p[3] = {0, 0, 0}, l[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const double* r = s->r + 3 * i; const double* v = s->v + 3 * i;
    for (int k = 0; k < 3; ++k) p[k] += s->m[i] * v[k];
    l[0] += s->m[i] * (r[1] * v[2] - r[2] * v[1]);
    l[1] += s->m[i] * (r[2] * v[0] - r[0] * v[2]);
    l[2] += s->m[i] * (r[0] * v[1] - r[1] * v[0]);
  }
  if (P) for (int k = 0; k < 3; ++k) P[k] = p[k];
  if (L) for (int k = 0; k < 3; ++k) L[k] = l[k];
}

/* ---------------------------------------------------------------- fixed-step runs */

int orc_fixed_run(orc_system* s, double H, int nsteps) {
  int n = s->n;
  size_t n3 = sizeof(double) * 3 * (size_t)n;
  double* r = (double*)malloc(n3);
  double* v = (double*)malloc(n3);
  for (int i = 0; i < nsteps; ++i) {
    double eps, t;
    orc_attempt(s, H, &eps, r, v, &t, NULL);
    orc_set_state(s, t, r, v);
  }
  free(r);
  free(v);
  return ORC_OK;
}

/* Tangent-linear (forward-mode derivative) of the fixed-step run, in Cartesian form.
   Exactly (in real arithmetic) the MST-coordinate step equals the Cartesian one: the
   edge vectors X = r_v - r_parent are a linear change of variables, the near-pair edge
   sums equal r_j - r_i, and the rebuild is its inverse plus a shift that is the identity
   on the centre-of-mass frame. So the derivative of the step is taken here from the
   Cartesian LogH equations of Sec. 2.1-2.2:
     D(h): f = h / (T + B), r += f v        with T = sum m |v|^2 / 2
     K(h): g = h / U,       v += g a        with a, U of Eq. 1-2
   B = U0 - T0 of the initial COM-frame state (Eq. 1), k_fix leapfrog divisions per step
   and Aitken-Neville extrapolation (linear in the division results, so the tangents are
   extrapolated with the same tableau). Every quantity carries its tangent (value, d). */

/* a_i = G sum_j m_j d_ij / |d_ij|^3, U = G sum_{i<j} m_i m_j / |d_ij|, d_ij = r_j - r_i,
   with tangents for a tangent (dr, dm). */
static void tl_forces(int n, const double* m, const double* dm, double G, const double* r, const double* dr,
                      double* a, double* da, double* U, double* dU) {
  double* ui = (double*)calloc((size_t)n, sizeof(double));
  double* dui = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 8) num_threads(g_threads)
  for (int i = 0; i < n; ++i) {
    double ax = 0, ay = 0, az = 0, dax = 0, day = 0, daz = 0, u = 0, du = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3], dd[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = r[3 * j + k] - r[3 * i + k];
        dd[k] = dr[3 * j + k] - dr[3 * i + k];
      }
      double r2 = norm2(d), rr = sqrt(r2), r3 = r2 * rr, r5 = r3 * r2;
      double dot = (d[0] * dd[0] + d[1] * dd[1]) + d[2] * dd[2];
      /* d/dx of m_j d / r^3 = dm_j d / r^3 + m_j (dd / r^3 - 3 d (d . dd) / r^5) */
      ax += m[j] * d[0] / r3;
      ay += m[j] * d[1] / r3;
      az += m[j] * d[2] / r3;
      dax += dm[j] * d[0] / r3 + m[j] * (dd[0] / r3 - 3.0 * d[0] * dot / r5);
      day += dm[j] * d[1] / r3 + m[j] * (dd[1] / r3 - 3.0 * d[1] * dot / r5);
      daz += dm[j] * d[2] / r3 + m[j] * (dd[2] / r3 - 3.0 * d[2] * dot / r5);
      if (j > i) {
        /* d/dx of m_i m_j / r = (dm_i m_j + m_i dm_j) / r - m_i m_j (d . dd) / r^3 */
        u += m[j] / rr;
        du += (dm[i] * m[j] + m[i] * dm[j]) / rr - m[i] * m[j] * dot / r3;
      }
    }
    a[3 * i] = G * ax; a[3 * i + 1] = G * ay; a[3 * i + 2] = G * az;
    da[3 * i] = G * dax; da[3 * i + 1] = G * day; da[3 * i + 2] = G * daz;
    ui[i] = m[i] * u;
    dui[i] = du;
  }
  double Us = 0.0, dUs = 0.0;
  for (int i = 0; i < n; ++i) {
    Us += G * ui[i];
    dUs += G * dui[i];
  }
  *U = Us;
  *dU = dUs;
  free(ui);
  free(dui);
}

/* T = sum m |v|^2 / 2 and its tangent sum (dm |v|^2 / 2 + m v . dv) */
static void tl_kinetic(int n, const double* m, const double* dm, const double* v, const double* dv, double* T,
                       double* dT) {
  double t = 0.0, dt = 0.0;
  for (int i = 0; i < n; ++i) {
    double v2 = norm2(v + 3 * i);
    double vdv = (v[3 * i] * dv[3 * i] + v[3 * i + 1] * dv[3 * i + 1]) + v[3 * i + 2] * dv[3 * i + 2];
    t += m[i] * v2;
    dt += dm[i] * v2 + 2.0 * m[i] * vdv;
  }
  *T = 0.5 * t;
  *dT = 0.5 * dt;
}

/* w -= sum m w / M with its tangent: d(sum m w / M) = (sum (dm w + m dw) - (sum m w / M) dM) / M */
static void tl_com_shift(int n, const double* m, const double* dm, double* w, double* dw) {
  double M = 0.0, dM = 0.0, c[3] = {0, 0, 0}, dc[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    M += m[i];
    dM += dm[i];
    for (int k = 0; k < 3; ++k) {
      c[k] += m[i] * w[3 * i + k];
      dc[k] += dm[i] * w[3 * i + k] + m[i] * dw[3 * i + k];
    }
  }
  for (int k = 0; k < 3; ++k) {
    c[k] /= M;
    dc[k] = (dc[k] - c[k] * dM) / M;
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      w[3 * i + k] -= c[k];
      dw[3 * i + k] -= dc[k];
    }
}

typedef struct {
  int n;
  const double *m, *dm;
  double G, B, dB;
  double *r, *v, *dr, *dv, *a, *da;
} tl_div;

static void tl_drift(void* c, double h) {
  tl_div* d = (tl_div*)c;
  double T, dT;
  tl_kinetic(d->n, d->m, d->dm, d->v, d->dv, &T, &dT);
  double f = h / (T + d->B);
  double df = -h * (dT + d->dB) / ((T + d->B) * (T + d->B));
  for (int i = 0; i < 3 * d->n; ++i) {
    d->dr[i] += df * d->v[i] + f * d->dv[i];
    d->r[i] += f * d->v[i];
  }
}

static void tl_kick(void* c, double h) {
  tl_div* d = (tl_div*)c;
  double U, dU;
  tl_forces(d->n, d->m, d->dm, d->G, d->r, d->dr, d->a, d->da, &U, &dU);
  double g = h / U, dg = -h * dU / (U * U);
  for (int i = 0; i < 3 * d->n; ++i) {
    d->dv[i] += dg * d->a[i] + g * d->da[i];
    d->v[i] += g * d->a[i];
  }
}

int orc_fixed_run_tl(int n, const double* m_in, const double* r_in, const double* v_in, const double* dm_in,
                     const double* dr_in, const double* dv_in, const orc_params* p, double H, int nsteps,
                     double* r_f, double* v_f, double* E_f, double* dr_f, double* dv_f, double* dE_f) {
  if (n < 2 || !p || p->k_fix < 2 || nsteps < 0) return ORC_ERR_ARG;
  int kf = p->k_fix;
  size_t n3 = 3 * (size_t)n, b3 = sizeof(double) * n3, nv = 6 * (size_t)n;
  double* m = (double*)malloc(sizeof(double) * (size_t)n);
  double* dm = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(m, m_in, sizeof(double) * (size_t)n);
  memcpy(dm, dm_in, sizeof(double) * (size_t)n);
  double *r = (double*)malloc(b3), *v = (double*)malloc(b3), *dr = (double*)malloc(b3), *dv = (double*)malloc(b3);
  memcpy(r, r_in, b3); memcpy(v, v_in, b3); memcpy(dr, dr_in, b3); memcpy(dv, dv_in, b3);
  tl_com_shift(n, m, dm, r, dr);
  tl_com_shift(n, m, dm, v, dv);
  tl_div d;
  d.n = n; d.m = m; d.dm = dm; d.G = p->G;
  d.a = (double*)malloc(b3); d.da = (double*)malloc(b3);
  d.r = (double*)malloc(b3); d.v = (double*)malloc(b3); d.dr = (double*)malloc(b3); d.dv = (double*)malloc(b3);
  {
    double U, dU, T, dT;
    tl_forces(n, m, dm, p->G, r, dr, d.a, d.da, &U, &dU);
    tl_kinetic(n, m, dm, v, dv, &T, &dT);
    d.B = U - T;  /* B = -H with H = T - U (Eq. 1) */
    d.dB = dU - dT;
  }
  int* nseq = (int*)malloc(sizeof(int) * (size_t)kf);
  double* S = (double*)malloc(sizeof(double) * nv * (size_t)kf);
  double* dS = (double*)malloc(sizeof(double) * nv * (size_t)kf);
  double* Tkk = (double*)malloc(sizeof(double) * nv);
  double* Tprev = (double*)malloc(sizeof(double) * nv);
  for (int step = 0; step < nsteps; ++step) {
    for (int k = 0; k < kf; ++k) {
      nseq[k] = 2 * (k + 1);
      memcpy(d.r, r, b3); memcpy(d.v, v, b3); memcpy(d.dr, dr, b3); memcpy(d.dv, dv, b3);
      orc_dkd(nseq[k], H, tl_drift, tl_kick, &d);
      memcpy(S + (size_t)k * nv, d.r, b3);
      memcpy(S + (size_t)k * nv + n3, d.v, b3);
      memcpy(dS + (size_t)k * nv, d.dr, b3);
      memcpy(dS + (size_t)k * nv + n3, d.dv, b3);
    }
    orc_neville(kf, nseq, (int)nv, S, Tkk, Tprev);
    memcpy(r, Tkk, b3); memcpy(v, Tkk + n3, b3);
    orc_neville(kf, nseq, (int)nv, dS, Tkk, Tprev);
    memcpy(dr, Tkk, b3); memcpy(dv, Tkk + n3, b3);
  }
  {
    double U, dU, T, dT;
    tl_forces(n, m, dm, p->G, r, dr, d.a, d.da, &U, &dU);
    tl_kinetic(n, m, dm, v, dv, &T, &dT);
    if (E_f) *E_f = T - U;
    if (dE_f) *dE_f = dT - dU;
  }
  if (r_f) memcpy(r_f, r, b3);
  if (v_f) memcpy(v_f, v, b3);
  if (dr_f) memcpy(dr_f, dr, b3);
  if (dv_f) memcpy(dv_f, dv, b3);
  free(m); free(dm); free(r); free(v); free(dr); free(dv);
  free(d.a); free(d.da); free(d.r); free(d.v); free(d.dr); free(d.dv);
  free(nseq); free(S); free(dS); free(Tkk); free(Tprev);
  return ORC_OK;
}
