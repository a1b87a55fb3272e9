// Prim's minimum spanning tree on the GPU (Sec. 3.2) with the indexing of Sec. 3.4.
//
// One CTA builds the whole tree: Prim's N iterations are sequential, and keeping the tree
// inside one SM turns every iteration's global argmin into a block reduction with two
// barriers. Each thread owns up to VPT vertices and keeps their exact FP64 keys (squared
// distance to the tree) in registers; parents, levels and FP32 copies of the positions
// live in shared memory.
//
// Keys must be bit-identical to the CPU definition, so every distance that can change a
// key is computed in FP64 exactly as ((dx*dx)+(dy*dy))+(dz*dz) without contraction. One
// SM issues only ~1.6 FP64 instructions per clock, so an FP32 lower bound of the distance,
// with a rigorous rounding-error allowance, first decides whether the new tree vertex can
// possibly lower a key; only then is the FP64 distance evaluated. The skip test never
// rejects a vertex whose FP64 distance would be strictly below its key (derivation beside
// the code), so the tree, order and levels are those of the plain algorithm.
#include <climits>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

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

template <int VPT>
__global__ void __launch_bounds__(1024, 1)
k_prim(int n, int npad, const double* __restrict__ r, int* __restrict__ parent_out,
       int* __restrict__ level_out, int* __restrict__ order_out, int* __restrict__ root_out) {
  extern __shared__ float sm_f[];
  float* xf = sm_f;
  float* yf = xf + n;
  float* zf = yf + n;
  int* par = reinterpret_cast<int*>(zf + n);
  int* lvl = par + n;
  __shared__ unsigned long long rk[32], wk;
  __shared__ int ri[32], wi;

  const double* X = r;
  const double* Y = r + npad;
  const double* Z = r + 2 * (size_t)npad;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int w = tid; w < n; w += nt) {
    xf[w] = __double2float_rn(X[w]);
    yf[w] = __double2float_rn(Y[w]);
    zf[w] = __double2float_rn(Z[w]);
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

  unsigned long long key[VPT];
  float kf[VPT];  // an upper bound (round-up float) of key, for the FP32 skip test
  unsigned intree = 0;
#pragma unroll
  for (int s = 0; s < VPT; ++s) {
    key[s] = kInfBits;
    kf[s] = __int_as_float(0x7f800000);
    int w = tid + s * nt;
    if (w >= n || w == root) intree |= 1u << s;
  }
  if (tid == 0) {
    order_out[0] = root;
    root_out[0] = root;
  }

  int u = root;
  for (int it = 1; it < n; ++it) {
    const double xu = X[u], yu = Y[u], zu = Z[u];
    const float xfu = xf[u], yfu = yf[u], zfu = zf[u];
    const float axu = fabsf(xfu), ayu = fabsf(yfu), azu = fabsf(zfu);
    bk = ~0ull;
    bi = INT_MAX;
#pragma unroll
    for (int s = 0; s < VPT; ++s) {
      if (intree & (1u << s)) continue;
      const int w = tid + s * nt;
      // Lower bound of |dx| from float copies: |x - fl(x)| <= 2^-24 |fl(x)| and the float
      // subtraction errs by <= 2^-24 |dxf|; 2^-23 doubles that allowance to cover the
      // rounding of the bound itself, 1e-37 covers subnormal coordinates.
      const float xw = xf[w], yw = yf[w], zw = zf[w];
      const float dxf = xfu - xw, dyf = yfu - yw, dzf = zfu - zw;
      const float lx = fmaxf(fabsf(dxf) - (axu + fabsf(xw) + fabsf(dxf)) * 0x1p-23f - 1e-37f, 0.0f);
      const float ly = fmaxf(fabsf(dyf) - (ayu + fabsf(yw) + fabsf(dyf)) * 0x1p-23f - 1e-37f, 0.0f);
      const float lz = fmaxf(fabsf(dzf) - (azu + fabsf(zw) + fabsf(dzf)) * 0x1p-23f - 1e-37f, 0.0f);
      // lx^2+ly^2+lz^2 in float is at most (1+2^-24)^3 too large; scaling by (1-2^-20)
      // leaves a value below the true squared distance by more than the FP64 distance's
      // own relative error (< 2^-50). So lbf >= kf >= key implies d_fp64 >= key.
      const float lbf = ((lx * lx + ly * ly) + lz * lz) * (1.0f - 0x1p-20f);
      if (lbf < kf[s]) {
        const double dx = __dsub_rn(xu, X[w]), dy = __dsub_rn(yu, Y[w]), dz = __dsub_rn(zu, Z[w]);
        const double d = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (d < __longlong_as_double((long long)key[s])) {
          key[s] = key_bits(d);
          kf[s] = __double2float_ru(d);
          par[w] = u;
        }
      }
      argmin_combine(bk, bi, key[s], w);
    }
    block_argmin(bk, bi, rk, ri, &wk, &wi);
    const int nxt = bi;
    if (tid == nxt % nt) {
      intree |= 1u << (nxt / nt);
      int p = par[nxt];
      if (p < 0) {  // only with non-finite positions
        p = root;
        par[nxt] = p;
      }
      lvl[nxt] = lvl[p] + 1;
      order_out[it] = nxt;
    }
    u = nxt;
  }
  __syncthreads();
  for (int w = tid; w < n; w += nt) {
    parent_out[w] = par[w];
    level_out[w] = lvl[w];
  }
}

// Grandparents and the children lists (CSR, each list in ascending index) of the tree.
__global__ void __launch_bounds__(1024, 1)
k_tree(int n, int npad, const int* __restrict__ parent, int* __restrict__ gp, int* __restrict__ child_off,
       int* __restrict__ child_idx) {
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
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < nt; ++t) {
      int x = part[t];
      part[t] = acc;
      acc += x;
    }
    child_off[n] = acc;
  }
  __syncthreads();
  s = part[tid];
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
}

template <int VPT>
cudaError_t run_prim(mstar_ctx* c, int nt) {
  size_t smem = (size_t)c->n * (3 * sizeof(float) + 2 * sizeof(int));
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
  k_tree<<<1, 1024, smem, c->stream>>>(c->n, c->npad, c->d.parent, c->d.gp, c->d.child_off, c->d.child_idx);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

}  // namespace mstar
