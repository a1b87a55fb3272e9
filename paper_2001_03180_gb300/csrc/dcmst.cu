// Divide-and-conquer spanning tree of Sec. 3.3 on the GPU.
//
// The paper's large-N alternative to Prim's MST: split the bodies into about sqrt(N)
// subgraphs with an octree, build the MST of every subgraph and of the meta-graph whose
// vertices are the contracted subgraphs and whose edge weights are the cheapest edges
// between them (the cut property), and order the union of these edges by a walk from the
// root. The result is a spanning tree a few per cent longer than the MST that is locally
// the MST of every subgraph.
//
// Rules (each also the CPU definition's):
// - bounding cube: the centre of each coordinate's extent, half-size the largest half-extent;
//   at each of 16 depths a body goes to the child whose centre it is not below (x >= c);
//   the Morton key concatenates the x, y, z choices, most significant first;
// - partition: starting from the cube, the cell with the most bodies (the first in Morton
//   order on ties) is replaced by its non-empty children until there are at least
//   `nsub` cells or the most populous cell cannot split (one body or depth 16);
// - subgraph MSTs: Prim from the subgraph's lowest body index; a key is replaced only by a
//   strictly smaller squared distance; the next vertex is the lowest (key, index);
// - meta weights: for subgraphs a < b, the lexicographic minimum of (d^2, i, j) over
//   i in a, j in b; the meta-graph's Prim starts at subgraph 0 and compares these triples;
// - the walk: breadth first from the body closest to the centre of mass (lowest index on
//   ties); parent and level are unique for a tree whatever the visiting order.
// Squared distances are ((dx*dx)+(dy*dy))+(dz*dz) with dx = x_u - x_v, each operation rounded
// separately, as in the Prim kernel.
#include <climits>
#include <cmath>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

constexpr int kDepth = 16;
constexpr int kIdxBits = 14;
constexpr unsigned long long kIdxMask = (1ull << kIdxBits) - 1;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
static_assert(MSTAR_MAX_N <= (1 << kIdxBits), "a body index must fit below the Morton key");

struct DcEdge {
  unsigned long long d;  // bits of the non-negative squared distance (ordered like the value)
  int i, j;              // i in the lower-numbered subgraph
};

__device__ __forceinline__ bool dc_less(const DcEdge& a, const DcEdge& b) {
  if (a.d != b.d) return a.d < b.d;
  if (a.i != b.i) return a.i < b.i;
  return a.j < b.j;
}

struct Cell {
  int depth, lo, hi;
};

// Device scratch of the builder (carved from the context workspace).
struct DcLayout {
  int npow2, mc;                 // sort length (power of two >= n), cell capacity
  unsigned long long* sorted;    // (Morton key << 14 | body), sorted
  double* bounds;                // centre x, y, z, half-size
  float4* f4;                    // per body: float x, y, z and their conversion error bound
  Cell* cells;                   // mc cells
  int* ncell;                    // [1]
  int* leafid;                   // subgraph of each sorted position
  int* leaf_start;               // mc + 1
  unsigned long long* key;       // Prim keys by sorted position
  float* keyf;                   // the keys rounded up to float
  int* kp;                       // Prim parent candidates by sorted position
  DcEdge* W;                     // mc x mc meta weights (a < b entries)
  int *eu, *ev;                  // the n - 1 tree edges
  int *adj_off, *adj, *queue;    // orientation
  size_t bytes;
};

int target_of(int n, int nsub) { return nsub > 0 ? nsub : (int)ceil(sqrt((double)n)); }

DcLayout dc_layout(int n, int nsub, char* base) {
  DcLayout L{};
  L.npow2 = 2;
  while (L.npow2 < n) L.npow2 <<= 1;
  const int target = target_of(n, nsub);
  L.mc = target + 8 < n ? target + 8 : n;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  L.sorted = reinterpret_cast<unsigned long long*>(take(8 * (size_t)L.npow2));
  L.bounds = reinterpret_cast<double*>(take(4 * sizeof(double)));
  L.f4 = reinterpret_cast<float4*>(take(sizeof(float4) * (size_t)n));
  L.cells = reinterpret_cast<Cell*>(take(sizeof(Cell) * (size_t)L.mc));
  L.ncell = reinterpret_cast<int*>(take(sizeof(int)));
  L.leafid = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  L.leaf_start = reinterpret_cast<int*>(take(sizeof(int) * (size_t)(L.mc + 1)));
  L.key = reinterpret_cast<unsigned long long*>(take(8 * (size_t)n));
  L.keyf = reinterpret_cast<float*>(take(sizeof(float) * (size_t)n));
  L.kp = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  L.W = reinterpret_cast<DcEdge*>(take(sizeof(DcEdge) * (size_t)L.mc * L.mc));
  L.eu = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  L.ev = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  L.adj_off = reinterpret_cast<int*>(take(sizeof(int) * (size_t)(n + 1)));
  L.adj = reinterpret_cast<int*>(take(sizeof(int) * 2 * (size_t)n));
  L.queue = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
  L.bytes = (off + 255) & ~size_t(255);
  return L;
}

// Bounding cube (one CTA): centre of each coordinate's extent, largest half-extent.
__global__ void __launch_bounds__(1024, 1)
k_dc_bounds(int n, const double* __restrict__ X, const double* __restrict__ Y, const double* __restrict__ Z,
            double* __restrict__ bounds) {
  __shared__ double red[32][6];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int i = tid; i < n; i += blockDim.x) {
    const double c[3] = {X[i], Y[i], Z[i]};
    for (int k = 0; k < 3; ++k) {
      v[k] = fmin(v[k], c[k]);
      v[3 + k] = fmax(v[3 + k], c[k]);
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < 3; ++k) {
      v[k] = fmin(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
      v[3 + k] = fmax(v[3 + k], __shfl_xor_sync(0xffffffffu, v[3 + k], o));
    }
  if (lane == 0)
    for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (tid == 0) {
    double mn[3], mx[3], hs = 0.0;
    for (int k = 0; k < 3; ++k) {
      mn[k] = red[0][k];
      mx[k] = red[0][3 + k];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        mn[k] = fmin(mn[k], red[w][k]);
        mx[k] = fmax(mx[k], red[w][3 + k]);
      }
      bounds[k] = __dmul_rn(__dadd_rn(mn[k], mx[k]), 0.5);
      const double e = __dmul_rn(__dsub_rn(mx[k], mn[k]), 0.5);
      if (e > hs) hs = e;
    }
    bounds[3] = hs;
  }
}

// Packed Morton keys (padding: all ones, sorted last) and the float copies of the positions
// with a bound on their conversion error (for the meta-weight filter).
__global__ void __launch_bounds__(256)
k_dc_keys(int n, int npow2, const double* __restrict__ X, const double* __restrict__ Y, const double* __restrict__ Z,
          const double* __restrict__ bounds, unsigned long long* __restrict__ sorted, float4* __restrict__ f4) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npow2) return;
  if (i >= n) {
    sorted[i] = ~0ull;
    return;
  }
  const double p[3] = {X[i], Y[i], Z[i]};
  double c[3] = {bounds[0], bounds[1], bounds[2]}, h = bounds[3];
  unsigned long long kk = 0;
  for (int d = 0; d < kDepth; ++d) {
    h = __dmul_rn(h, 0.5);
    unsigned bits = 0;
    for (int k = 0; k < 3; ++k) {
      const int b = p[k] >= c[k];
      bits = (bits << 1) | (unsigned)b;
      c[k] = b ? __dadd_rn(c[k], h) : __dsub_rn(c[k], h);
    }
    kk = (kk << 3) | bits;
  }
  sorted[i] = (kk << kIdxBits) | (unsigned long long)i;
  const float fx = __double2float_rn(p[0]), fy = __double2float_rn(p[1]), fz = __double2float_rn(p[2]);
  f4[i] = make_float4(fx, fy, fz, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))) * 0x1p-22f + 1e-37f);
}

// Bitonic sort of npow2 keys in shared memory (one CTA).
__global__ void __launch_bounds__(1024, 1) k_dc_sort(int npow2, unsigned long long* __restrict__ a) {
  extern __shared__ unsigned long long s[];
  for (int i = threadIdx.x; i < npow2; i += blockDim.x) s[i] = a[i];
  __syncthreads();
  for (int k = 2; k <= npow2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const unsigned long long x = s[i], y = s[p];
          if ((x > y) == ((i & k) == 0)) {
            s[i] = y;
            s[p] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < npow2; i += blockDim.x) a[i] = s[i];
}

// First position in [lo, hi) whose Morton digit at `shift` exceeds `dgt` (digits are
// non-decreasing inside a cell).
__device__ int digit_end(const unsigned long long* __restrict__ sorted, int lo, int hi, int shift, unsigned dgt) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (((sorted[mid] >> shift) & 7u) <= dgt) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Greedy octree partition (thread 0), then the subgraph of every sorted position and the
// subgraph starts (cells partition [0, n); their starts are flagged and scanned).
__global__ void __launch_bounds__(1024, 1)
k_dc_partition(int n, int target, int mc, const unsigned long long* __restrict__ gsorted, Cell* __restrict__ cells,
               int* __restrict__ ncell, int* __restrict__ leafid, int* __restrict__ leaf_start) {
  extern __shared__ unsigned long long sorted[];  // n keys
  __shared__ int s_nc;
  __shared__ int wsum[32];
  const int tid = threadIdx.x;
  for (int p = tid; p < n; p += blockDim.x) sorted[p] = gsorted[p];
  __syncthreads();
  if (tid == 0) {
    int nc = 1;
    cells[0] = Cell{0, 0, n};
    while (nc < target) {
      int best = 0;
      for (int c = 1; c < nc; ++c) {
        const int cb = cells[best].hi - cells[best].lo, cc = cells[c].hi - cells[c].lo;
        if (cc > cb || (cc == cb && cells[c].lo < cells[best].lo)) best = c;
      }
      const Cell b = cells[best];
      if (b.hi - b.lo <= 1 || b.depth == kDepth) break;
      const int shift = 3 * (kDepth - b.depth - 1) + kIdxBits;
      int p = b.lo, first = 1;
      for (unsigned dgt = 0; dgt < 8; ++dgt) {
        const int q = digit_end(sorted, p, b.hi, shift, dgt);
        if (q > p) {
          const Cell kid{b.depth + 1, p, q};
          if (first) {
            cells[best] = kid;
            first = 0;
          } else if (nc < mc) {
            cells[nc++] = kid;
          }
        }
        p = q;
      }
    }
    s_nc = nc;
    *ncell = nc;
  }
  for (int p = tid; p < n; p += blockDim.x) leafid[p] = 0;
  __syncthreads();
  const int nc = s_nc;
  for (int c = tid; c < nc; c += blockDim.x) leafid[cells[c].lo] = 1;
  __syncthreads();
  // inclusive scan of the start flags over the sorted positions: chunk per thread
  const int ch = (n + blockDim.x - 1) / blockDim.x;
  const int b0 = tid * ch, b1 = min(n, b0 + ch);
  int local = 0;
  for (int p = b0; p < b1; ++p) local += leafid[p];
  int incl = local;
  const int lane = tid & 31, warp = tid >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  int run = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
  for (int p = b0; p < b1; ++p) {
    const int f = leafid[p];
    run += f;
    leafid[p] = run - 1;
    if (f) leaf_start[run - 1] = p;
  }
  if (tid == 0) leaf_start[nc] = n;
}

// Prim inside every subgraph: one CTA of kLpThreads per subgraph. A subgraph of up to
// kLeafSmem bodies is staged in shared memory (positions, their float copies, keys and the
// keys rounded up to float, candidate parents, body indices); larger ones work from global
// memory. The thread that owns a position (its offset from the subgraph start, mod the CTA
// size) keeps its key and candidate parent; kp = -2 marks tree vertices. A relaxation
// computes the exact FP64 distance only when the rigorous float lower bound does not exceed
// the key rounded up: otherwise the distance is certainly above the key and the strict
// update cannot happen.
constexpr int kLeafSmem = 1024;
constexpr int kLpThreads = 128;

__device__ __forceinline__ float dc_lower_bound(const float4& p, const float4& q) {
  const float dx = fabsf(p.x - q.x), dy = fabsf(p.y - q.y), dz = fabsf(p.z - q.z);
  const float e = p.w + q.w;
  const float lx = fmaxf(0.f, fmaf(dx, -0x1p-22f, dx) - e), ly = fmaxf(0.f, fmaf(dy, -0x1p-22f, dy) - e),
              lz = fmaxf(0.f, fmaf(dz, -0x1p-22f, dz) - e);
  const float s = fmaf(lz, lz, fmaf(ly, ly, lx * lx));
  // relative rounding of normal results, and 2^-144 for the absolute rounding (<= 2^-150 per
  // operation) of squares and sums below 2^-126
  return fmaxf(fmaf(s, -0x1p-20f, s) - 0x1p-144f, 0.0f);
}

struct LpCand {
  unsigned long long k;
  int v, q;
};

__device__ __forceinline__ bool lp_less(const LpCand& a, const LpCand& b) {
  return a.k < b.k || (a.k == b.k && a.v < b.v);
}

__global__ void __launch_bounds__(kLpThreads)
k_dc_local_prim(const int* __restrict__ ncell, const int* __restrict__ leaf_start,
                const unsigned long long* __restrict__ sorted, const double* __restrict__ X,
                const double* __restrict__ Y, const double* __restrict__ Z, const float4* __restrict__ f4,
                unsigned long long* __restrict__ gkey, float* __restrict__ gkeyf, int* __restrict__ gkp,
                int* __restrict__ eu, int* __restrict__ ev) {
  extern __shared__ double sm[];
  __shared__ LpCand red[2][kLpThreads / 32];
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (g >= *ncell) return;
  const int lo = leaf_start[g], hi = leaf_start[g + 1], cnt = hi - lo;
  const bool shared = cnt <= kLeafSmem;
  double* sx = sm;
  double* sy = sx + kLeafSmem;
  double* sz = sy + kLeafSmem;
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(sz + kLeafSmem);
  float4* sf = reinterpret_cast<float4*>(skey + kLeafSmem);
  float* skeyf = reinterpret_cast<float*>(sf + kLeafSmem);
  int* skp = reinterpret_cast<int*>(skeyf + kLeafSmem);
  int* bid = skp + kLeafSmem;
  unsigned long long* key = shared ? skey : gkey + lo;
  float* keyf = shared ? skeyf : gkeyf + lo;
  int* kp = shared ? skp : gkp + lo;
  LpCand st{~0ull, INT_MAX, -1};
  for (int q = tid; q < cnt; q += kLpThreads) {
    const int b = (int)(sorted[lo + q] & kIdxMask);
    if (shared) {
      sx[q] = X[b];
      sy[q] = Y[b];
      sz[q] = Z[b];
      sf[q] = f4[b];
      bid[q] = b;
    }
    key[q] = kInfBits;
    keyf[q] = INFINITY;
    kp[q] = -1;
    if (b < st.v) st = LpCand{0, b, q};
  }
  // the start vertex: the lowest body index of the subgraph
  for (int o = 16; o > 0; o >>= 1) {
    LpCand c;
    c.k = 0;
    c.v = __shfl_xor_sync(0xffffffffu, st.v, o);
    c.q = __shfl_xor_sync(0xffffffffu, st.q, o);
    if (c.v < st.v) st = c;
  }
  if (lane == 0) red[0][warp] = st;
  __syncthreads();
  for (int w = 0; w < kLpThreads / 32; ++w)
    if (red[0][w].v < st.v) st = red[0][w];
  if ((st.q % kLpThreads) == tid) kp[st.q] = -2;
  int u = st.v;
  double ux = X[u], uy = Y[u], uz = Z[u];
  float4 uf = f4[u];
  const int e0 = lo - g;  // local edges of the earlier subgraphs: sum (size - 1)
  for (int it = 1; it < cnt; ++it) {
    LpCand best{~0ull, INT_MAX, -1};
    for (int q = tid; q < cnt; q += kLpThreads) {
      if (kp[q] == -2) continue;
      const int v = shared ? bid[q] : (int)(sorted[lo + q] & kIdxMask);
      unsigned long long k = key[q];
      const float4 fv = shared ? sf[q] : f4[v];
      if (dc_lower_bound(uf, fv) <= keyf[q]) {
        const double vx = shared ? sx[q] : X[v], vy = shared ? sy[q] : Y[v], vz = shared ? sz[q] : Z[v];
        const double dx = __dsub_rn(ux, vx), dy = __dsub_rn(uy, vy), dz = __dsub_rn(uz, vz);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        const unsigned long long d = key_bits(d2);
        if (d < k) {
          k = d;
          key[q] = d;
          keyf[q] = __double2float_ru(d2);
          kp[q] = u;
        }
      }
      const LpCand c{k, v, q};
      if (lp_less(c, best)) best = c;
    }
    for (int o = 16; o > 0; o >>= 1) {
      LpCand c;
      c.k = __shfl_xor_sync(0xffffffffu, best.k, o);
      c.v = __shfl_xor_sync(0xffffffffu, best.v, o);
      c.q = __shfl_xor_sync(0xffffffffu, best.q, o);
      if (lp_less(c, best)) best = c;
    }
    if (lane == 0) red[it & 1][warp] = best;
    __syncthreads();
    for (int w = 0; w < kLpThreads / 32; ++w)
      if (lp_less(red[it & 1][w], best)) best = red[it & 1][w];
    if ((best.q % kLpThreads) == tid) {
      eu[e0 + it - 1] = kp[best.q];
      ev[e0 + it - 1] = best.v;
      kp[best.q] = -2;
    }
    u = best.v;
    if (shared) {
      ux = sx[best.q];
      uy = sy[best.q];
      uz = sz[best.q];
      uf = sf[best.q];
    } else {
      ux = X[u];
      uy = Y[u];
      uz = Z[u];
      uf = f4[u];
    }
  }
}

// Meta-graph weights: CTA (a, b), a < b, reduces (d^2, i, j) over i in a, j in b. A thread
// takes partners j of b and scans a in shared-memory chunks; the exact FP64 distance is
// computed only when a rigorous float lower bound does not exceed the best exact value so
// far (rounded up to float), so every pair that can win or tie is decided exactly.
constexpr int kMetaChunk = 512;

__global__ void __launch_bounds__(256)
k_dc_meta_w(const int* __restrict__ ncell, int mc, const int* __restrict__ leaf_start,
            const unsigned long long* __restrict__ sorted, const double* __restrict__ X,
            const double* __restrict__ Y, const double* __restrict__ Z, const float4* __restrict__ f4,
            DcEdge* __restrict__ W) {
  __shared__ float4 sf[kMetaChunk];
  __shared__ int si[kMetaChunk];
  __shared__ DcEdge red[8];
  const int a = blockIdx.x, b = blockIdx.y;
  const int nc = *ncell;
  if (a >= nc || b >= nc || b <= a) return;
  const int la = leaf_start[a], sa = leaf_start[a + 1] - la;
  const int lb = leaf_start[b], sb = leaf_start[b + 1] - lb;
  DcEdge best{~0ull, INT_MAX, INT_MAX};
  float bestf = INFINITY;
  for (int c0 = 0; c0 < sa; c0 += kMetaChunk) {
    const int cn = min(kMetaChunk, sa - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < cn; t += blockDim.x) {
      const int i = (int)(sorted[la + c0 + t] & kIdxMask);
      si[t] = i;
      sf[t] = f4[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < sb; q += blockDim.x) {
      const int j = (int)(sorted[lb + q] & kIdxMask);
      const float4 fj = f4[j];
      for (int t = 0; t < cn; ++t) {
        if (dc_lower_bound(sf[t], fj) > bestf) continue;
        const int i = si[t];
        const double dx = __dsub_rn(X[i], X[j]), dy = __dsub_rn(Y[i], Y[j]), dz = __dsub_rn(Z[i], Z[j]);
        const DcEdge c{key_bits(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz))), i,
                       j};
        if (dc_less(c, best)) {
          best = c;
          bestf = __double2float_ru(__longlong_as_double((long long)c.d));
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    DcEdge c;
    c.d = __shfl_xor_sync(0xffffffffu, best.d, o);
    c.i = __shfl_xor_sync(0xffffffffu, best.i, o);
    c.j = __shfl_xor_sync(0xffffffffu, best.j, o);
    if (dc_less(c, best)) best = c;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w)
      if (dc_less(red[w], best)) best = red[w];
    W[(size_t)a * mc + b] = best;
  }
}

// Prim on the meta-graph from subgraph 0 (one warp; keys in shared memory). Its edges go
// after the n - ncell local edges.
__global__ void __launch_bounds__(32)
k_dc_meta_prim(int n, const int* __restrict__ ncell, int mc, const DcEdge* __restrict__ W, int* __restrict__ eu,
               int* __restrict__ ev) {
  __shared__ DcEdge key[kDcMaxSub + 8];
  __shared__ unsigned char in[kDcMaxSub + 8];
  const int lane = threadIdx.x;
  const int nc = *ncell;
  for (int g = lane; g < nc; g += 32) {
    key[g] = DcEdge{~0ull, -1, -1};
    in[g] = g == 0;
  }
  __syncwarp();
  int u = 0;
  for (int it = 1; it < nc; ++it) {
    DcEdge bk{~0ull, INT_MAX, INT_MAX};
    int bg = INT_MAX;
    // four weights per lane are loaded together, then folded in ascending g
    for (int g0 = lane; g0 < nc; g0 += 128) {
      DcEdge cs[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int g = g0 + 32 * t;
        cs[t] = (g < nc && !in[g]) ? (u < g ? W[(size_t)u * mc + g] : W[(size_t)g * mc + u]) : DcEdge{~0ull, -1, -1};
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int g = g0 + 32 * t;
        if (g >= nc || in[g]) continue;
        if (key[g].i < 0 || dc_less(cs[t], key[g])) key[g] = cs[t];
        if (bg == INT_MAX || dc_less(key[g], bk)) {
          bk = key[g];
          bg = g;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      DcEdge c;
      c.d = __shfl_xor_sync(0xffffffffu, bk.d, o);
      c.i = __shfl_xor_sync(0xffffffffu, bk.i, o);
      c.j = __shfl_xor_sync(0xffffffffu, bk.j, o);
      const int g2 = __shfl_xor_sync(0xffffffffu, bg, o);
      if (g2 != INT_MAX && (bg == INT_MAX || dc_less(c, bk) || (!dc_less(bk, c) && g2 < bg))) {
        bk = c;
        bg = g2;
      }
    }
    if (lane == 0) {
      in[bg] = 1;
      eu[n - nc + it - 1] = bk.i;
      ev[n - nc + it - 1] = bk.j;
    }
    __syncwarp();
    u = bg;
  }
}

}  // namespace

size_t dc_scratch_bytes(int n, int nsub) { return dc_layout(n, nsub, nullptr).bytes; }

cudaError_t launch_mst_dc(mstar_ctx* c) {
  const int n = c->n;
  if (!c->d.dc) return cudaErrorInvalidValue;
  const DcLayout L = dc_layout(n, c->p.mst_nsub, c->d.dc);
  const int target = target_of(n, c->p.mst_nsub);
  const double* X = c->d.r;
  const double* Y = X + c->npad;
  const double* Z = Y + c->npad;
  cudaStream_t s = c->stream;
  k_dc_bounds<<<1, 1024, 0, s>>>(n, X, Y, Z, L.bounds);
  k_dc_keys<<<(L.npow2 + 255) / 256, 256, 0, s>>>(n, L.npow2, X, Y, Z, L.bounds, L.sorted, L.f4);
  const size_t smem = 8 * (size_t)L.npow2;
  cudaError_t e = cudaFuncSetAttribute(k_dc_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dc_sort<<<1, 1024, smem, s>>>(L.npow2, L.sorted);
  const size_t psmem = 8 * (size_t)n;
  if ((e = cudaFuncSetAttribute(k_dc_partition, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem)) !=
      cudaSuccess)
    return e;
  k_dc_partition<<<1, 1024, psmem, s>>>(n, target, L.mc, L.sorted, L.cells, L.ncell, L.leafid, L.leaf_start);
  const size_t lsmem = (size_t)kLeafSmem * (3 * sizeof(double) + 8 + sizeof(float4) + sizeof(float) + 2 * sizeof(int));
  if ((e = cudaFuncSetAttribute(k_dc_local_prim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem)) !=
      cudaSuccess)
    return e;
  k_dc_local_prim<<<L.mc, kLpThreads, lsmem, s>>>(L.ncell, L.leaf_start, L.sorted, X, Y, Z, L.f4, L.key, L.keyf,
                                                   L.kp, L.eu, L.ev);
  k_dc_meta_w<<<dim3(L.mc, L.mc), 256, 0, s>>>(L.ncell, L.mc, L.leaf_start, L.sorted, X, Y, Z, L.f4, L.W);
  k_dc_meta_prim<<<1, 32, 0, s>>>(n, L.ncell, L.mc, L.W, L.eu, L.ev);
  c->launches += 7;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_orient(c, L.eu, L.ev, L.adj_off, L.adj, L.queue)) != cudaSuccess) return e;
  return cudaMemcpyAsync(c->d.order, L.queue, sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
}

}  // namespace mstar
