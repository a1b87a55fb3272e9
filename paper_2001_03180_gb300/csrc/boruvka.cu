// Exact MST for the GBS step by Boruvka rounds over the whole GPU.
//
// Sec. 3.2 builds the MST with Prim's algorithm; its N sequential iterations keep a GPU on
// one SM. When all squared distances that decide the tree are distinct, the MST is unique
// (Sec. 3.1), so any exact MST algorithm yields Prim's tree. Boruvka's rounds are
// parallel: every vertex finds its nearest vertex outside its component (exact FP64
// comparisons, filtered by rigorous float lower bounds), every component takes its
// cheapest outgoing edge, and components merge along those edges. If two different
// candidates ever compare exactly equal in FP64, the tree could depend on tie-breaking
// rules, and the caller falls back to the Prim kernel, which applies the paper's rule.
// The tree is then oriented from Prim's root (the body closest to the centre of mass) by a
// breadth-first walk, which gives the same parent and level as Prim's indexing.
//
// Distances are computed exactly as the CPU definition does: ((dx*dx)+(dy*dy))+(dz*dz)
// with dx = x_u - x_v, each operation rounded separately.
#include <climits>
#include <cstring>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

constexpr int kBT = 128;  // vertices per CTA in the nearest-foreign-neighbour search

__device__ __forceinline__ double d2_exact(const double* X, const double* Y, const double* Z, int u, int v) {
  const double dx = __dsub_rn(X[u], X[v]), dy = __dsub_rn(Y[u], Y[v]), dz = __dsub_rn(Z[u], Z[v]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Float bounds of the FP64 squared distance ((dx*dx)+(dy*dy))+(dz*dz) of two vertices from
// their float copies: each coordinate difference errs by at most (|x_i| + |x_j|) 2^-24 + |dx|
// 2^-24, and e = e_i + e_j holds (max|coordinate_i| + max|coordinate_j|) 2^-23 + 2e-37.
// (1 -/+ 2^-20) covers the relative rounding of the float sums of squares and the FP64
// distance's own (< 2^-50); 2^-144 the absolute rounding (<= 2^-150 per operation) of squares
// and sums below 2^-126. Overflowing squares make hi infinite, which bounds nothing away.
__device__ __forceinline__ float d2_lower(float dx, float dy, float dz, float e) {
  const float lx = fmaxf(fmaf(dx, -0x1p-22f, dx) - e, 0.0f);
  const float ly = fmaxf(fmaf(dy, -0x1p-22f, dy) - e, 0.0f);
  const float lz = fmaxf(fmaf(dz, -0x1p-22f, dz) - e, 0.0f);
  return fmaxf(((lx * lx + ly * ly) + lz * lz) * (1.0f - 0x1p-20f) - 0x1p-144f, 0.0f);
}
__device__ __forceinline__ float d2_upper(float dx, float dy, float dz, float e) {
  const float hx = fmaf(dx, 0x1p-22f, dx) + e, hy = fmaf(dy, 0x1p-22f, dy) + e, hz = fmaf(dz, 0x1p-22f, dz) + e;
  return ((hx * hx + hy * hy) + hz * hz) * (1.0f + 0x1p-20f) + 0x1p-144f;
}

constexpr int kNfnList = 4;  // candidates a thread lists for exact evaluation

// Nearest foreign neighbour (smallest exact squared distance to a vertex of another
// component) of every vertex whose cached neighbour is missing or has become internal;
// CTA (tile, part) scans the part-th slice of the candidates. Writes per (vertex, part)
// the exact distance bits and the neighbour; exact equal distances to two different
// candidates at the minimum set *tie.
//
// Three steps, so that the FP64 distances (and their divergent, long-latency code) run only
// for the few candidates that can be the nearest: the least float upper bound over the
// foreign candidates; the candidates whose float lower bound does not exceed it, listed in
// index order (a candidate above it is strictly farther than the nearest); their exact
// distances. A vertex with more than kNfnList listed candidates scans the part again, taking
// the exact distance of every candidate whose lower bound does not exceed the bound.
__global__ void __launch_bounds__(kBT)
k_nfn(int n, int npad, int nparts, const double* __restrict__ X, const double* __restrict__ Y,
      const double* __restrict__ Z, const float* __restrict__ f4, const int* __restrict__ comp,
      const int* __restrict__ nbr, unsigned long long* __restrict__ partD, int* __restrict__ partJ,
      int* __restrict__ flags) {
  // The round's gate: flags[2] = 1 once the tree is complete (flags[1] = n - 1 edges, written
  // by the previous round's k_hook) or a tie has been seen (flags[0]); the round's kernels then
  // return at once, and flags[3] counts the rounds that ran. Rounds can thus be issued ahead of
  // the host's check: a round after the last one needed changes nothing (without the gate it
  // would find no foreign neighbour and report a tie). The search opens every round, so its
  // first CTA publishes the decision for the round's later kernels (none of which writes
  // flags[2]). A tie set by another CTA while the search runs can make CTAs decide differently;
  // the build then falls back to the Prim kernel, so nothing of that round is used.
  const bool stop = (flags[0] != 0) || (flags[1] >= n - 1);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    flags[2] = stop;
    if (!stop) flags[3] += 1;
  }
  if (stop) return;
  int* tie = flags;
  __shared__ float sx[kBT], sy[kBT], sz[kBT], se[kBT];
  __shared__ int sc[kBT];
  __shared__ int slist[kNfnList][kBT];
  __shared__ int any;
  const int i = blockIdx.x * kBT + threadIdx.x;
  const int part = blockIdx.y;
  bool need = false;
  int ci = -1;
  if (i < n) {
    ci = comp[i];
    const int b = nbr[i];
    need = (b < 0) || (comp[b] == ci);
  }
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  if (need) any = 1;
  __syncthreads();
  if (!any) return;
  const float xi = i < n ? f4[4 * i] : 0.0f, yi = i < n ? f4[4 * i + 1] : 0.0f, zi = i < n ? f4[4 * i + 2] : 0.0f;
  const float ei = i < n ? f4[4 * i + 3] : 0.0f;
  const int per = (n + nparts - 1) / nparts;
  const int j_lo = part * per, j_hi = min(n, j_lo + per);
  float bhi = __int_as_float(0x7f800000);
  int listed = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int t0 = j_lo; t0 < j_hi; t0 += kBT) {
      __syncthreads();
      const int j = t0 + threadIdx.x;
      if (j < j_hi) {
        sx[threadIdx.x] = f4[4 * j];
        sy[threadIdx.x] = f4[4 * j + 1];
        sz[threadIdx.x] = f4[4 * j + 2];
        se[threadIdx.x] = f4[4 * j + 3];
        sc[threadIdx.x] = comp[j];
      }
      __syncthreads();
      if (!need) continue;
      const int cnt = min(kBT, j_hi - t0);
      if (pass == 0) {
        for (int q = 0; q < cnt; ++q) {
          const float h = d2_upper(fabsf(xi - sx[q]), fabsf(yi - sy[q]), fabsf(zi - sz[q]), ei + se[q]);
          if (sc[q] != ci) bhi = fminf(bhi, h);
        }
      } else {
        for (int q = 0; q < cnt; ++q) {
          const float lo = d2_lower(fabsf(xi - sx[q]), fabsf(yi - sy[q]), fabsf(zi - sz[q]), ei + se[q]);
          if (lo <= bhi && sc[q] != ci) {
            if (listed < kNfnList) slist[listed][threadIdx.x] = t0 + q;
            ++listed;
          }
        }
      }
    }
  }
  if (!need) return;
  unsigned long long bD = ~0ull;
  int bj = -1;
  int mytie = 0;
  auto consider = [&](int jj) {
    const unsigned long long db = key_bits(d2_exact(X, Y, Z, i, jj));
    if (db < bD) {
      bD = db;
      bj = jj;
    } else if (db == bD && jj != bj) {
      mytie = 1;
    }
  };
  if (listed <= kNfnList) {
    for (int k = 0; k < listed; ++k) consider(slist[k][threadIdx.x]);
  } else {
    for (int jj = j_lo; jj < j_hi; ++jj) {
      if (comp[jj] == ci) continue;
      const float lo = d2_lower(fabsf(xi - f4[4 * jj]), fabsf(yi - f4[4 * jj + 1]), fabsf(zi - f4[4 * jj + 2]),
                                ei + f4[4 * jj + 3]);
      if (lo <= bhi) consider(jj);
    }
  }
  partD[(size_t)part * npad + i] = bD;
  partJ[(size_t)part * npad + i] = bj;
  if (mytie) atomicOr(tie, 1);
}

// Merge the parts: exact minimum, ties flagged; cache the neighbour.
__global__ void k_nfn_merge(int n, int npad, int nparts, const int* __restrict__ comp, int* __restrict__ nbr,
                            unsigned long long* __restrict__ nbrD, const unsigned long long* __restrict__ partD,
                            const int* __restrict__ partJ, int* __restrict__ tie, const int* __restrict__ stop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || *stop) return;
  const int b = nbr[i];
  if (b >= 0 && comp[b] != comp[i]) return;
  unsigned long long bD = ~0ull;
  int bj = -1;
  // the parts in ascending order, their values loaded four at a time ahead of the comparisons
  for (int p0 = 0; p0 < nparts; p0 += 4) {
    unsigned long long d[4];
    int j[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool in = p0 + k < nparts;
      d[k] = in ? partD[(size_t)(p0 + k) * npad + i] : ~0ull;
      j[k] = in ? partJ[(size_t)(p0 + k) * npad + i] : -1;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (j[k] < 0) continue;
      if (d[k] < bD) {
        bD = d[k];
        bj = j[k];
      } else if (d[k] == bD && j[k] != bj) {
        atomicOr(tie, 1);
      }
    }
  }
  nbr[i] = bj;
  nbrD[i] = bD;
}

__global__ void k_comp_min(int n, const int* __restrict__ comp, const unsigned long long* __restrict__ nbrD,
                           unsigned long long* __restrict__ cmin, const int* __restrict__ stop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !*stop) atomicMin(&cmin[comp[i]], nbrD[i]);
}

__global__ void k_comp_edge(int n, const int* __restrict__ comp, const unsigned long long* __restrict__ nbrD,
                            const unsigned long long* __restrict__ cmin, int* __restrict__ cidx,
                            int* __restrict__ ccnt, int* __restrict__ tie, const int* __restrict__ stop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || *stop) return;
  const int c = comp[i];
  if (nbrD[i] == cmin[c]) {
    if (atomicAdd(&ccnt[c], 1) > 0) atomicOr(tie, 1);  // two cheapest edges of equal weight
    cidx[c] = i;
  }
}

// Hook every component onto the component at the far end of its cheapest edge. Two
// components that chose each other chose the same edge (weights distinct); the smaller
// label becomes the root and records the edge once.
__global__ void k_hook(int n, const int* __restrict__ comp, const int* __restrict__ nbr, const int* __restrict__ cidx,
                       int* __restrict__ nxt, int* __restrict__ eu, int* __restrict__ ev, int* __restrict__ ecount,
                       const int* __restrict__ stop) {
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= n || *stop || comp[C] != C) return;
  const int i = cidx[C];
  const int j = nbr[i];
  const int T = comp[j];
  const int jT = nbr[cidx[T]];
  const bool mutual = comp[jT] == C;
  if (mutual && C < T) {
    nxt[C] = C;
  } else {
    nxt[C] = T;
  }
  if (!mutual || C < T) {
    const int e = atomicAdd(ecount, 1);
    if (e < n - 1) {
      eu[e] = i;
      ev[e] = j;
    }
  }
}

__global__ void k_relabel(int n, int* __restrict__ comp, const int* __restrict__ nxt,
                          unsigned long long* __restrict__ cmin, int* __restrict__ ccnt, const int* __restrict__ stop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || *stop) return;
  int c = comp[i];
  for (int guard = 0; guard < n && nxt[c] != c; ++guard) c = nxt[c];
  comp[i] = c;
  cmin[i] = ~0ull;
  ccnt[i] = 0;
}

__global__ void k_boruvka_init(int n, const double* __restrict__ X, const double* __restrict__ Y,
                               const double* __restrict__ Z, float* __restrict__ f4, int* __restrict__ comp,
                               int* __restrict__ nbr, unsigned long long* __restrict__ cmin, int* __restrict__ ccnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = __double2float_rn(X[i]), y = __double2float_rn(Y[i]), z = __double2float_rn(Z[i]);
  f4[4 * i] = x;
  f4[4 * i + 1] = y;
  f4[4 * i + 2] = z;
  f4[4 * i + 3] = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))) * 0x1p-23f + 1e-37f;
  comp[i] = i;
  nbr[i] = -1;
  cmin[i] = ~0ull;
  ccnt[i] = 0;
}

// Orient the tree from Prim's root: adjacency from the edge list, then a breadth-first
// walk in one CTA (levels are tree depths, independent of the visiting order). The
// adjacency, the visited marks and the queue live in shared memory (5n + 1 ints).
__global__ void __launch_bounds__(1024, 1)
k_orient(int n, const double* __restrict__ X, const double* __restrict__ Y, const double* __restrict__ Z,
         const int* __restrict__ eu, const int* __restrict__ ev, int* __restrict__ adj_off, int* __restrict__ adj,
         int* __restrict__ parent, int* __restrict__ level, int* __restrict__ root_out, int* __restrict__ queue) {
  extern __shared__ int smi[];
  int* s_off = smi;           // n + 1
  int* s_adj = s_off + n + 1; // 2 (n - 1)
  int* s_a = s_adj + 2 * n;   // n: degrees, then the parents
  int* s_q = s_a + n;         // n: fill counters, then the queue
  __shared__ unsigned long long rk[32];
  __shared__ int ri[32];
  __shared__ int part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int v = tid; v < n; v += nt) {
    s_a[v] = 0;
    s_q[v] = 0;
  }
  // root: closest to the origin (COM frame), lowest index on ties
  unsigned long long bk = ~0ull;
  int bi = INT_MAX;
  for (int w = tid; w < n; w += nt) {
    const double x = X[w], y = Y[w], z = Z[w];
    const unsigned long long k =
        key_bits(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    if (k < bk || (k == bk && w < bi)) {
      bk = k;
      bi = w;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_down_sync(0xffffffffu, bk, o);
    const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
    if (k2 < bk || (k2 == bk && i2 < bi)) {
      bk = k2;
      bi = i2;
    }
  }
  if ((tid & 31) == 0) {
    rk[tid >> 5] = bk;
    ri[tid >> 5] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (nt >> 5); ++w)
      if (rk[w] < rk[0] || (rk[w] == rk[0] && ri[w] < ri[0])) {
        rk[0] = rk[w];
        ri[0] = ri[w];
      }
  }
  // (endpoints outside [0, n) cannot come from the tree builders; they are skipped so that
  // no shared-memory index leaves its array)
  for (int e = tid; e < n - 1; e += nt) {
    const int a = eu[e], b = ev[e];
    if ((unsigned)a < (unsigned)n && (unsigned)b < (unsigned)n) {
      atomicAdd(&s_a[a], 1);
      atomicAdd(&s_a[b], 1);
    }
  }
  __syncthreads();
  const int root = ri[0];
  // exclusive scan of the degrees: contiguous chunks per thread, then the chunk sums
  const int chunk = (n + nt - 1) / nt;
  const int b0 = tid * chunk, b1 = min(n, b0 + chunk);
  int sum = 0;
  for (int v = b0; v < b1; ++v) sum += s_a[v];
  {
    int total;
    sum = block_exclusive_scan(sum, part, &total);
    if (tid == 0) s_off[n] = total;
  }
  for (int v = b0; v < b1; ++v) {
    s_off[v] = sum;
    sum += s_a[v];
  }
  __syncthreads();
  for (int e = tid; e < n - 1; e += nt) {
    const int a = eu[e], b = ev[e];
    if ((unsigned)a < (unsigned)n && (unsigned)b < (unsigned)n) {
      s_adj[s_off[a] + atomicAdd(&s_q[a], 1)] = b;
      s_adj[s_off[b] + atomicAdd(&s_q[b], 1)] = a;
    }
  }
  __syncthreads();
  for (int v = tid; v < n; v += nt) s_a[v] = -2;  // not yet reached
  __syncthreads();
  if (tid == 0) {
    s_a[root] = -1;
    s_q[0] = root;
    root_out[0] = root;
  }
  __syncthreads();
  // Level by level in warp 0: [h, t) is the current level, taken 32 vertices at a time, one per
  // lane. Each lane walks its vertex's neighbours; in every round the lanes that found an
  // unvisited neighbour append it at their rank among them (ballot), so the queue order is
  // fixed given the adjacency lists and no block barrier is needed between levels (a level holds ~35 vertices on average
  // at N = 2050, where 59 levels with block barriers cost about 1 us each). In a tree a vertex
  // is reached from its parent only, so no vertex is appended twice. (Parent and level do not
  // depend on the order of the adjacency lists, which the atomic fill above leaves open.)
  if (tid < 32) {
    const int lane = tid;
    const unsigned lt = (1u << lane) - 1u;
    int h = 0, t = 1, depth = 0;
    while (h < t) {
      int tail = t;
      for (int base = h; base < t; base += 32) {
        const int q = base + lane;
        const int u = q < t ? s_q[q] : -1;
        if (u >= 0) level[u] = depth;
        int a = u >= 0 ? s_off[u] : 0;
        const int aend = u >= 0 ? s_off[u + 1] : 0;
        while (__any_sync(0xffffffffu, a < aend)) {
          int w = -1;
          if (a < aend) {
            w = s_adj[a];
            ++a;
            if (s_a[w] != -2) w = -1;
          }
          const unsigned found = __ballot_sync(0xffffffffu, w >= 0);
          if (w >= 0) {
            s_a[w] = u;
            const int slot = tail + __popc(found & lt);
            if (slot < n) s_q[slot] = w;
          }
          tail += __popc(found);
          __syncwarp();  // this round's marks and appends are seen by every lane in the next
        }
        __syncwarp();
      }
      h = t;
      t = min(tail, n);
      ++depth;
    }
  }
  __syncthreads();
  for (int v = tid; v < n; v += nt) {
    parent[v] = s_a[v];
    queue[v] = s_q[v];
  }
  for (int v = tid; v <= n; v += nt) adj_off[v] = s_off[v];
  for (int a = tid; a < 2 * (n - 1); a += nt) adj[a] = s_adj[a];
}

}  // namespace

// Orientation of an undirected spanning tree (edges eu[e]-ev[e], e < n-1) from Prim's root
// into d.parent, d.level, d.root; `queue` receives the breadth-first order.
cudaError_t launch_orient(mstar_ctx* c, const int* eu, const int* ev, int* adj_off, int* adj, int* queue) {
  const int n = c->n;
  const double* X = c->d.r;
  const size_t smem = sizeof(int) * (5 * (size_t)n + 1);
  cudaError_t e = cudaFuncSetAttribute(k_orient, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_orient<<<1, 1024, smem, c->stream>>>(n, X, X + c->npad, X + 2 * (size_t)c->npad, eu, ev, adj_off, adj,
                                         c->d.parent, c->d.level, c->d.root, queue);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

// Boruvka MST of d.r into parent/level/root; returns cudaSuccess and sets *tied when a
// tie was seen (the caller then runs the Prim kernel). Scratch lives in the pair partial
// buffer, which is free while the tree is being built.
cudaError_t launch_mst_boruvka(mstar_ctx* c, bool* tied) {
  const int n = c->n, npad = c->npad;
  // the candidates are split into parts, one CTA row each, until the search has about four
  // CTAs per SM (a CTA scanning alone is bound by its latency) or a part would hold fewer than
  // kBT candidates; at most 16
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    sms = 1;
  }
  const int nbt = (n + kBT - 1) / kBT;
  int nparts = 1;
  while (nparts < 16 && nbt * nparts < 4 * sms && n / (2 * nparts) >= kBT) nparts *= 2;
  char* base = reinterpret_cast<char*>(c->d.P);
  auto take = [&](size_t bytes) {
    char* p = base;
    base += (bytes + 255) & ~size_t(255);
    return p;
  };
  float* f4 = reinterpret_cast<float*>(take(sizeof(float) * 4 * npad));
  int* comp = reinterpret_cast<int*>(take(sizeof(int) * npad));
  int* nbr = reinterpret_cast<int*>(take(sizeof(int) * npad));
  unsigned long long* nbrD = reinterpret_cast<unsigned long long*>(take(8 * (size_t)npad));
  unsigned long long* cmin = reinterpret_cast<unsigned long long*>(take(8 * (size_t)npad));
  int* cidx = reinterpret_cast<int*>(take(sizeof(int) * npad));
  int* ccnt = reinterpret_cast<int*>(take(sizeof(int) * npad));
  int* nxt = reinterpret_cast<int*>(take(sizeof(int) * npad));
  int* eu = reinterpret_cast<int*>(take(sizeof(int) * npad));
  int* ev = reinterpret_cast<int*>(take(sizeof(int) * npad));
  int* adj_off = reinterpret_cast<int*>(take(sizeof(int) * (npad + 1)));
  int* adj = reinterpret_cast<int*>(take(sizeof(int) * 2 * npad));
  int* queue = reinterpret_cast<int*>(take(sizeof(int) * npad));
  unsigned long long* partD = reinterpret_cast<unsigned long long*>(take(8 * (size_t)npad * nparts));
  int* partJ = reinterpret_cast<int*>(take(sizeof(int) * (size_t)npad * nparts));
  int* flags = reinterpret_cast<int*>(take(sizeof(int) * 4));  // [0] tie, [1] edge count, [2] gate, [3] rounds run
  const size_t p_bytes = (size_t)c->nslots * c->NT * 4 * npad * sizeof(double);
  if ((size_t)(base - reinterpret_cast<char*>(c->d.P)) > p_bytes) {  // scratch does not fit: use Prim
    *tied = true;
    return cudaSuccess;
  }
  const double* X = c->d.r;
  const double* Y = X + npad;
  const double* Z = Y + npad;
  const int nb = (n + 255) / 256;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int) * 4, c->stream);
  if (e != cudaSuccess) return e;
  k_boruvka_init<<<nb, 256, 0, c->stream>>>(n, X, Y, Z, f4, comp, nbr, cmin, ccnt);
  MSTAR_LAUNCHED(c);
  int edges = 0;
  *tied = false;
  // The first check comes after as many rounds as the context's last build ran (consecutive
  // steps build trees of nearly the same point set), then after every further round.
  int round = 0;
  while (round < 64 && edges < n - 1) {
    const int batch = round == 0 ? (c->mst_rounds > 0 ? c->mst_rounds : 1) : 1;
    for (int b = 0; b < batch && round < 64; ++b, ++round) {
      k_nfn<<<dim3((n + kBT - 1) / kBT, nparts), kBT, 0, c->stream>>>(n, npad, nparts, X, Y, Z, f4, comp, nbr,
                                                                       partD, partJ, flags);
      k_nfn_merge<<<(n + 63) / 64, 64, 0, c->stream>>>(n, npad, nparts, comp, nbr, nbrD, partD, partJ, flags,
                                                       flags + 2);
      k_comp_min<<<nb, 256, 0, c->stream>>>(n, comp, nbrD, cmin, flags + 2);
      k_comp_edge<<<nb, 256, 0, c->stream>>>(n, comp, nbrD, cmin, cidx, ccnt, flags, flags + 2);
      k_hook<<<nb, 256, 0, c->stream>>>(n, comp, nbr, cidx, nxt, eu, ev, flags + 1, flags + 2);
      k_relabel<<<nb, 256, 0, c->stream>>>(n, comp, nxt, cmin, ccnt, flags + 2);
      c->launches += 6;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(c->host_buf, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    int fl[4];
    std::memcpy(fl, c->host_buf, sizeof(fl));
    if (fl[0]) {
      *tied = true;
      return cudaSuccess;
    }
    edges = fl[1];
    c->mst_rounds = fl[3];
  }
  if (edges != n - 1) {  // cannot happen without ties; be safe
    *tied = true;
    return cudaSuccess;
  }
  return launch_orient(c, eu, ev, adj_off, adj, queue);
}

}  // namespace mstar
