// Prim's minimum spanning tree on the GPU (Sec. 3.2) with the indexing of Sec. 3.4.
//
// One CTA builds the whole tree: Prim's N iterations are sequential, and keeping the tree
// inside one SM turns every iteration's global argmin into a block reduction with two
// barriers. Each thread owns up to VPT vertices and keeps their keys (squared distance to
// the tree, as float intervals) in registers together with a summary of its smallest
// bounds, rebuilt only when one of its keys changed; parents, levels, FP32 copies of the
// positions and their rounding radii live in shared memory.
//
// Keys must decide exactly as the CPU definition does, where every distance is computed in
// FP64 as ((dx*dx)+(dy*dy))+(dz*dz) without contraction. One SM issues only ~1.6 FP64
// instructions per clock and Prim's ~50 key decreases per iteration would each cost a
// divergent FP64 sequence, so keys are carried as rigorous float intervals and FP64
// distances are evaluated only when an interval comparison cannot decide (derivation beside
// the code). The tree, order and levels are those of the plain algorithm.
#include <climits>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

__device__ __forceinline__ void argmin_combine(unsigned long long& k, int& i, unsigned long long k2, int i2) {
  if (k2 < k || (k2 == k && i2 < i)) {
    k = k2;
    i = i2;
  }
}

// Lexicographic (key, index) minimum over the block; every thread receives the winner.
__device__ __forceinline__ void block_argmin(unsigned long long& k, int& i, unsigned long long* rk, int* ri,
                                             unsigned long long* wk, int* wi) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long k2 = __shfl_down_sync(0xffffffffu, k, o);
    int i2 = __shfl_down_sync(0xffffffffu, i, o);
    argmin_combine(k, i, k2, i2);
  }
  if (blockDim.x == 32) {  // one warp: lane 0 holds the minimum
    k = __shfl_sync(0xffffffffu, k, 0);
    i = __shfl_sync(0xffffffffu, i, 0);
    return;
  }
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    rk[warp] = k;
    ri[warp] = i;
  }
  __syncthreads();
  if (warp == 0) {
    k = lane < nw ? rk[lane] : ~0ull;
    i = lane < nw ? ri[lane] : INT_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long k2 = __shfl_down_sync(0xffffffffu, k, o);
      int i2 = __shfl_down_sync(0xffffffffu, i, o);
      argmin_combine(k, i, k2, i2);
    }
    if (lane == 0) {
      *wk = k;
      *wi = i;
    }
  }
  __syncthreads();
  k = *wk;
  i = *wi;
}

// Per-thread summary for the argmin: the smallest upper bound (with its index) and the two
// smallest lower bounds (index of the smallest). Non-negative float bit patterns order like
// the values, and 0xffffffff sorts after every real key (+inf included).
struct Cand {
  unsigned hk;
  int hidx;
  unsigned l1;
  int l1idx;
  unsigned l2;
};

__device__ __forceinline__ Cand cand_identity() { return Cand{0xffffffffu, INT_MAX, 0xffffffffu, INT_MAX, 0xffffffffu}; }

__device__ __forceinline__ void cand_combine(Cand& a, const Cand& b) {
  if (b.hk < a.hk || (b.hk == a.hk && b.hidx < a.hidx)) {
    a.hk = b.hk;
    a.hidx = b.hidx;
  }
  if (b.l1 < a.l1 || (b.l1 == a.l1 && b.l1idx < a.l1idx)) {
    a.l2 = min(a.l1, b.l2);
    a.l1 = b.l1;
    a.l1idx = b.l1idx;
  } else {
    a.l2 = min(a.l2, b.l1);
  }
}

__device__ __forceinline__ Cand cand_shfl_down(const Cand& c, int o) {
  Cand r;
  r.hk = __shfl_down_sync(0xffffffffu, c.hk, o);
  r.hidx = __shfl_down_sync(0xffffffffu, c.hidx, o);
  r.l1 = __shfl_down_sync(0xffffffffu, c.l1, o);
  r.l1idx = __shfl_down_sync(0xffffffffu, c.l1idx, o);
  r.l2 = __shfl_down_sync(0xffffffffu, c.l2, o);
  return r;
}

__device__ __forceinline__ double exact_d2(double xa, double ya, double za, double xb, double yb, double zb) {
  const double dx = __dsub_rn(xa, xb), dy = __dsub_rn(ya, yb), dz = __dsub_rn(za, zb);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Keys are kept as float intervals [klo, khi] that provably contain the exact FP64 key
// (the squared distance to the tree, computed as the CPU definition does), plus
// skey >= sqrt(khi) with margin. For a new tree vertex u and a non-tree vertex w:
//  - if some coordinate's lower bound |dx| - err >= skey, then d(u,w)^2 > key: no update;
//  - else with the interval [lo, hi] of d(u,w)^2: hi < klo -> certain update; lo >= khi ->
//    certain no update; otherwise the FP64 distances are compared exactly.
// The argmin is certain when the vertex with the smallest upper bound also has the
// smallest lower bound and the second-smallest lower bound lies above that upper bound;
// otherwise the exact keys of all vertices whose interval reaches down to it decide.
// Every decision therefore equals the one the exact FP64 comparison makes.
template <int VPT>
__global__ void __launch_bounds__(1024, 1)
k_prim(int n, int npad, const double* __restrict__ r, int* __restrict__ parent_out,
       int* __restrict__ level_out, int* __restrict__ order_out, int* __restrict__ root_out) {
  extern __shared__ float sm_f[];
  float* xf = sm_f;
  float* yf = xf + n;
  float* zf = yf + n;
  float* ew = zf + n;  // per-vertex error radius: max|coordinate| * 2^-23 + 1e-37
  int* par = reinterpret_cast<int*>(ew + n);
  short* lvl = reinterpret_cast<short*>(par + n);
  __shared__ unsigned long long rk[32], wk;
  __shared__ int ri[32], wi;
  __shared__ Cand rc[32];
  __shared__ Cand wc;

  const double* X = r;
  const double* Y = r + npad;
  const double* Z = r + 2 * (size_t)npad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;

  for (int w = tid; w < n; w += nt) {
    const float x = __double2float_rn(X[w]), y = __double2float_rn(Y[w]), z = __double2float_rn(Z[w]);
    xf[w] = x;
    yf[w] = y;
    zf[w] = z;
    ew[w] = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))) * 0x1p-23f + 1e-37f;
    par[w] = -1;
    lvl[w] = 0;
  }

  // Root: the particle closest to the centre of mass (the origin), lowest index on ties.
  unsigned long long bk = ~0ull;
  int bi = INT_MAX;
  for (int w = tid; w < n; w += nt) {
    double x = X[w], y = Y[w], z = Z[w];
    double d = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    argmin_combine(bk, bi, key_bits(d), w);
  }
  __syncthreads();
  block_argmin(bk, bi, rk, ri, &wk, &wi);
  const int root = bi;

  const float kInf = __int_as_float(0x7f800000);
  float klo[VPT], khi[VPT], skey[VPT];
  unsigned intree = 0;
#pragma unroll
  for (int s = 0; s < VPT; ++s) {
    klo[s] = kInf;
    khi[s] = kInf;
    skey[s] = kInf;
    int w = tid + s * nt;
    if (w >= n || w == root) intree |= 1u << s;
  }
  if (tid == 0) {
    order_out[0] = root;
    root_out[0] = root;
  }

  Cand c = cand_identity();
  bool dirty = true;  // this thread's summary must be rebuilt from its slots
  int u = root;
  for (int it = 1; it < n; ++it) {
    const float xfu = xf[u], yfu = yf[u], zfu = zf[u], eu = ew[u];
    const float axu = fabsf(xfu), ayu = fabsf(yfu), azu = fabsf(zfu);
#pragma unroll
    for (int s = 0; s < VPT; ++s) {
      if (intree & (1u << s)) continue;
      const int w = tid + s * nt;
      const float xw = xf[w], yw = yf[w], zw = zf[w];
      const float dxf = xfu - xw, dyf = yfu - yw, dzf = zfu - zw;
      const float ax = fabsf(dxf), ay = fabsf(dyf), az = fabsf(dzf);
      // Quick test on the largest coordinate difference a: |d_true| >= a - (a + max|u| +
      // max|w|) 2^-24 (float copies round to nearest, the difference rounds once); the test
      // subtracts a 2^-22 + (max|u| + max|w|) 2^-23, which also covers its own two roundings.
      // skey >= sqrt(khi (1 + 2^-20)).
      const float a = fmaxf(ax, fmaxf(ay, az));
      if (fmaf(a, -0x1p-22f, a) - (eu + ew[w]) >= skey[s]) continue;
      // Full float interval of d(u,w)^2. |x - fl(x)| <= 2^-24 |fl(x)| and the float
      // difference errs by <= 2^-24 |dxf|; 2^-23 doubles that allowance, 1e-37 covers
      // subnormal coordinates.
      const float ex = (axu + fabsf(xw) + ax) * 0x1p-23f + 1e-37f;
      const float ey = (ayu + fabsf(yw) + ay) * 0x1p-23f + 1e-37f;
      const float ez = (azu + fabsf(zw) + az) * 0x1p-23f + 1e-37f;
      const float lx = fmaxf(ax - ex, 0.0f), ly = fmaxf(ay - ey, 0.0f), lz = fmaxf(az - ez, 0.0f);
      const float hx = ax + ex, hy = ay + ey, hz = az + ez;
      // (1 -/+ 2^-20) absorbs the float roundings of the sums of squares and the FP64
      // distance's own relative error (< 2^-50); hi is trusted only above 1e-30, where no
      // square that matters can underflow. Below 2^-126 the roundings are absolute (<= 2^-150
      // per operation), which the 2^-144 taken off lo covers; lo stays >= 0, as the
      // bit-pattern comparisons of the keys need.
      const float lo = fmaxf(((lx * lx + ly * ly) + lz * lz) * (1.0f - 0x1p-20f) - 0x1p-144f, 0.0f);
      const float hi = ((hx * hx + hy * hy) + hz * hz) * (1.0f + 0x1p-20f);
      if (hi < klo[s] && hi >= 1e-30f) {
        klo[s] = lo;
        khi[s] = hi;
        skey[s] = __fsqrt_ru(__fmul_ru(hi, 1.0f + 0x1p-20f));
        par[w] = u;
        dirty = true;
      } else if (!(lo >= khi[s])) {
        const double xw64 = X[w], yw64 = Y[w], zw64 = Z[w];
        const double d = exact_d2(X[u], Y[u], Z[u], xw64, yw64, zw64);
        const int p = par[w];
        const double key =
            p >= 0 ? exact_d2(X[p], Y[p], Z[p], xw64, yw64, zw64) : __longlong_as_double(0x7ff0000000000000LL);
        if (d < key) {
          klo[s] = __double2float_rd(d);
          khi[s] = __double2float_ru(d);
          skey[s] = __fsqrt_ru(__fmul_ru(khi[s], 1.0f + 0x1p-20f));
          par[w] = u;
          dirty = true;
        }
      }
    }
    if (dirty) {
      c = cand_identity();
#pragma unroll
      for (int s = 0; s < VPT; ++s)
        if (!(intree & (1u << s)))
          cand_combine(c, Cand{__float_as_uint(khi[s]), tid + s * nt, __float_as_uint(klo[s]), tid + s * nt,
                               0xffffffffu});
      dirty = false;
    }
    // block reduction of the candidate summaries
    // the warp's summary by warp-wide minima (redux): the least upper bound and its index, the
    // least lower bound and its index, and the least lower bound other than that one (the
    // winner's own second bound, or another vertex's least bound); the same values the
    // pairwise cand_combine tree gives, in every lane
    Cand cw;
    cw.hk = __reduce_min_sync(0xffffffffu, c.hk);
    cw.hidx = (int)__reduce_min_sync(0xffffffffu, c.hk == cw.hk ? (unsigned)c.hidx : 0xffffffffu);
    cw.l1 = __reduce_min_sync(0xffffffffu, c.l1);
    cw.l1idx = (int)__reduce_min_sync(0xffffffffu, c.l1 == cw.l1 ? (unsigned)c.l1idx : 0xffffffffu);
    cw.l2 = __reduce_min_sync(0xffffffffu, (c.l1 == cw.l1 && c.l1idx == cw.l1idx) ? c.l2 : c.l1);
    if (nw > 1) {
      if (lane == 0) rc[warp] = cw;
      __syncthreads();
      if (warp == 0) {
        cw = lane < nw ? rc[lane] : cand_identity();
        for (int o = 16; o > 0; o >>= 1) cand_combine(cw, cand_shfl_down(cw, o));
        if (lane == 0) wc = cw;
      }
      __syncthreads();
      cw = wc;
    }
    int nxt;
    if (cw.l1idx == cw.hidx && cw.l2 > cw.hk) {
      nxt = cw.hidx;
    } else {
      // exact argmin over every vertex whose lower bound does not exceed the best upper bound
      bk = ~0ull;
      bi = INT_MAX;
#pragma unroll
      for (int s = 0; s < VPT; ++s) {
        if (intree & (1u << s)) continue;
        const int w = tid + s * nt;
        if (__float_as_uint(klo[s]) <= cw.hk) {
          const int p = par[w];
          const double key = p >= 0 ? exact_d2(X[p], Y[p], Z[p], X[w], Y[w], Z[w])
                                    : __longlong_as_double(0x7ff0000000000000LL);
          argmin_combine(bk, bi, key_bits(key), w);
        }
      }
      block_argmin(bk, bi, rk, ri, &wk, &wi);
      nxt = bi;
    }
    if (tid == nxt % nt) {
      intree |= 1u << (nxt / nt);
      dirty = true;
      int p = par[nxt];
      if (p < 0) {  // only with non-finite positions
        p = root;
        par[nxt] = p;
      }
      lvl[nxt] = (short)(lvl[p] + 1);
      order_out[it] = nxt;
    }
    u = nxt;
    __syncthreads();
  }
  __syncthreads();
  for (int w = tid; w < n; w += nt) {
    parent_out[w] = par[w];
    level_out[w] = lvl[w];
  }
}

// Grandparents, the children lists (CSR, each list in ascending index) and the bodies in
// order of (level, index) of the tree. The last is a bitonic sort of the keys level * 2^14
// + index (n <= 2^14) in shared memory.
__global__ void __launch_bounds__(1024, 1)
k_tree(int n, int npad, const int* __restrict__ parent, const int* __restrict__ level, int* __restrict__ gp,
       int* __restrict__ child_off, int* __restrict__ child_idx, int* __restrict__ bylev) {
  extern __shared__ int sm_i[];
  int* cnt = sm_i;        // n
  int* pos = cnt + n;     // n
  __shared__ int part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int w = tid; w < n; w += nt) {
    cnt[w] = 0;
    pos[w] = 0;
  }
  __syncthreads();
  for (int v = tid; v < npad; v += nt) {
    if (v >= n) {
      gp[v] = -3;
      continue;
    }
    int p = parent[v];
    gp[v] = p >= 0 ? parent[p] : -1;
    if (p >= 0) atomicAdd(&cnt[p], 1);
  }
  __syncthreads();
  // exclusive scan of cnt: contiguous chunks per thread, then a scan of the chunk sums
  const int chunk = (n + nt - 1) / nt;
  const int b = tid * chunk, e = min(n, b + chunk);
  int s = 0;
  for (int w = b; w < e; ++w) s += cnt[w];
  {
    int total;
    s = block_exclusive_scan(s, part, &total);
    if (tid == 0) child_off[n] = total;
  }
  for (int w = b; w < e; ++w) {
    int x = cnt[w];
    cnt[w] = s;  // now the offset
    child_off[w] = s;
    s += x;
  }
  __syncthreads();
  for (int v = tid; v < n; v += nt) {
    int p = parent[v];
    if (p >= 0) child_idx[cnt[p] + atomicAdd(&pos[p], 1)] = v;
  }
  __syncthreads();
  __threadfence_block();
  for (int p = tid; p < n; p += nt) {  // insertion sort of each (short) list
    int lo = child_off[p], hi = child_off[p + 1];
    for (int a = lo + 1; a < hi; ++a) {
      int x = child_idx[a], c = a - 1;
      while (c >= lo && child_idx[c] > x) {
        child_idx[c + 1] = child_idx[c];
        --c;
      }
      child_idx[c + 1] = x;
    }
  }
  // (level, index) order; the keys reuse cnt and pos (P <= 2n entries)
  __syncthreads();
  int P = 1;
  while (P < n) P <<= 1;
  unsigned* key = reinterpret_cast<unsigned*>(sm_i);
  for (int i = tid; i < P; i += nt) key[i] = i < n ? ((unsigned)level[i] << 14) | (unsigned)i : 0xffffffffu;
  __syncthreads();
  // each thread takes compare-exchange pairs p = tid, tid + nt, ...: i = the p-th index with
  // bit j clear, partner i + j; four pairs at a time so that their loads overlap
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int p0 = tid; p0 < P / 2; p0 += 4 * nt) {
        unsigned a[4], b[4];
        int ii[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int p = p0 + t * nt;
          ii[t] = 2 * p - (p & (j - 1));
          if (p < P / 2) {
            a[t] = key[ii[t]];
            b[t] = key[ii[t] + j];
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (p0 + t * nt < P / 2 && (a[t] > b[t]) == ((ii[t] & k) == 0)) {
            key[ii[t]] = b[t];
            key[ii[t] + j] = a[t];
          }
      }
      __syncthreads();
    }
  for (int i = tid; i < npad; i += nt) bylev[i] = i < n ? (int)(key[i] & 0x3fffu) : i;
}

template <int VPT>
cudaError_t run_prim(mstar_ctx* c, int nt) {
  size_t smem = (size_t)c->n * (4 * sizeof(float) + sizeof(int) + sizeof(short));
  cudaError_t e = cudaFuncSetAttribute(k_prim<VPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_prim<VPT><<<1, nt, smem, c->stream>>>(c->n, c->npad, c->d.r, c->d.parent, c->d.level, c->d.order,
                                          c->d.root);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prim(mstar_ctx* c) {
  const int n = c->n;
  const int vpts[] = {1, 2, 3, 4, 6, 8, 10};
  int vpt = 10;
  for (int v : vpts)
    if (v * 1024 >= n) {
      vpt = v;
      break;
    }
  int nt = ((n + vpt - 1) / vpt + 31) / 32 * 32;
  if (nt < 32) nt = 32;
  // up to 96 bodies one warp takes every vertex (up to 3 each): its reductions need no
  // shared-memory stage and no block barrier
  if (n <= 96) {
    vpt = (n + 31) / 32;
    nt = 32;
  }
  switch (vpt) {
    case 1: return run_prim<1>(c, nt);
    case 2: return run_prim<2>(c, nt);
    case 3: return run_prim<3>(c, nt);
    case 4: return run_prim<4>(c, nt);
    case 6: return run_prim<6>(c, nt);
    case 8: return run_prim<8>(c, nt);
    default: return run_prim<10>(c, nt);
  }
}

cudaError_t launch_tree(mstar_ctx* c) {
  size_t smem = (size_t)c->n * 2 * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(k_tree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tree<<<1, 1024, smem, c->stream>>>(c->n, c->npad, c->d.parent, c->d.level, c->d.gp, c->d.child_off,
                                       c->d.child_idx, c->d.bylev);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

}  // namespace mstar
