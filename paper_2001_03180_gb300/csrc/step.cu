// The O(N) parts of a GBS step: MST coordinates, LogH drift and kick, rebuilding the
// Cartesian state, and the Neville-Aitken extrapolation with its error norm.
//
// All k_fix leapfrog divisions of a step advance together: "slot" k (0-based) holds
// division k+1 with n = 2(k+1) substeps (Deuflhard sequence, Eq. seq-deuflhard); slot
// k_fix holds the step-start state used for the error norm's derivatives. Each kernel
// takes a contiguous slot range in blockIdx.y, so one launch serves every division that
// is active at a given substep level (Sec. 4.2: the divisions are independent).
//
// The drift/kick/rebuild arithmetic uses explicitly rounded FP64 operations (no
// contraction), the same operation order as the CPU reference.
#include <algorithm>
#include <cooperative_groups.h>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

__constant__ double c_fac[kMaxKfix][kMaxKfix];  // 1 / ((n_k / n_{k-j})^2 - 1)

__device__ __forceinline__ double madd(double a, double f, double b) {  // a + f*b, two roundings
  return __dadd_rn(a, __dmul_rn(f, b));
}

// Edge vectors of the step start: X_v = r_v - r_parent(v), V_v likewise (0 at the root and
// in the padding); copies r and X0 into the step-start slot; block sums of m v^2.
__global__ void __launch_bounds__(kBlock)
k_prepare(int n, int npad, int K, const double* __restrict__ m, const int* __restrict__ parent,
          const double* __restrict__ r, const double* __restrict__ v, double* __restrict__ X0,
          double* __restrict__ V0, double* __restrict__ sr, double* __restrict__ sX, double* __restrict__ Tblk,
          int nblk) {
  __shared__ double scratch[32];
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  double t2 = 0.0;
  if (w < npad) {
    const int p = w < n ? parent[w] : -1;
    double* srK = sr + (size_t)K * 3 * npad;
    double* sXK = sX + (size_t)K * 3 * npad;
    double vv[3];
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad;
      const double rw = r[o + w], vw = v[o + w];
      const double x = p >= 0 ? __dsub_rn(rw, r[o + p]) : 0.0;
      const double u = p >= 0 ? __dsub_rn(vw, v[o + p]) : 0.0;
      X0[o + w] = x;
      V0[o + w] = u;
      srK[o + w] = rw;
      sXK[o + w] = x;
      vv[c] = vw;
    }
    if (w < n) t2 = __dmul_rn(m[w], __dadd_rn(__dadd_rn(__dmul_rn(vv[0], vv[0]), __dmul_rn(vv[1], vv[1])),
                                               __dmul_rn(vv[2], vv[2])));
  }
  const double s = block_sum(t2, scratch);
  if (threadIdx.x == 0) Tblk[(size_t)K * nblk + blockIdx.x] = s;
}

// A0_v = a0_v - a0_parent(v) from the step-start slot; block 0 also stores U0 and T0.
__global__ void __launch_bounds__(kBlock)
k_start_derivs(int n, int npad, int K, const int* __restrict__ parent, const double* __restrict__ sa,
               double* __restrict__ A0, const double* __restrict__ Ublk, const double* __restrict__ Tblk,
               int nblk, double* __restrict__ sc, double* __restrict__ res) {
  __shared__ double sU, sT;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const double* aK = sa + (size_t)K * 3 * npad;
  if (w < npad) {
    const int p = w < n ? parent[w] : -1;
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad;
      A0[o + w] = p >= 0 ? __dsub_rn(aK[o + w], aK[o + p]) : 0.0;
    }
  }
  if (blockIdx.x == 0) {
    sum_partials(Ublk + (size_t)K * nblk, nblk, 1, &sU);
    sum_partials(Tblk + (size_t)K * nblk, nblk, 1, &sT);
    if (threadIdx.x == 0) {
      const double T0 = 0.5 * sT;
      res[2] = sU;
      res[3] = T0;
      sc[K * kScal + SC_U] = sU;
      sc[K * kScal + SC_T_KIN] = T0;
    }
  }
}

// First half drift D(h/2n) of every division from the step start (Sec. 2.3):
// X = X0 + f V0, V = V0, t = t0 + f with f = (delta/2) / (T0 + B), delta = H / n_k.
__global__ void __launch_bounds__(kBlock)
k_init_drift(int n, int npad, int K, const double* __restrict__ par, double B, const double* __restrict__ X0,
             const double* __restrict__ V0, double* __restrict__ sX, double* __restrict__ sV,
             double* __restrict__ sc, const double* __restrict__ Tblk, int nblk) {
  __shared__ double sT;
  const double H = par[0], t0 = par[1];  // the attempt's fictitious step and start time
  const int slot = blockIdx.y;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  // T0 as k_start_derivs forms it, from the step start's kinetic partials (the step-start force
  // evaluation, which k_start_derivs ends, may still be running beside the divisions)
  sum_partials(Tblk + (size_t)K * nblk, nblk, 1, &sT);
  const double T0 = 0.5 * sT;
  const double delta = H / (double)(2 * (slot + 1));
  const double f = (0.5 * delta) / (T0 + B);
  if (w < npad) {
    double* X = sX + (size_t)slot * 3 * npad;
    double* V = sV + (size_t)slot * 3 * npad;
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad;
      X[o + w] = madd(X0[o + w], f, V0[o + w]);
      V[o + w] = V0[o + w];
    }
  }
  if (w == 0) {
    sc[slot * kScal + SC_T_PHYS] = t0 + f;
    sc[slot * kScal + SC_T_KIN] = T0;
  }
}

// K(delta): V_v += (delta / U) (a_v - a_parent(v)), delta = H / n_k (Sec. 2.2).
__global__ void __launch_bounds__(kBlock)
k_kick(int n, int npad, int slot_lo, const double* __restrict__ par, const int* __restrict__ parent,
       const double* __restrict__ sa, double* __restrict__ sV, const double* __restrict__ Ublk, int nblk,
       double* __restrict__ sc) {
  __shared__ double sU;
  const double H = par[0];
  const int slot = slot_lo + blockIdx.y;
  sum_partials(Ublk + (size_t)slot * nblk, nblk, 1, &sU);
  const double U = sU;
  const double f = (H / (double)(2 * (slot + 1))) / U;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < n) {
    const int p = parent[w];
    if (p >= 0) {
      const double* a = sa + (size_t)slot * 3 * npad;
      double* V = sV + (size_t)slot * 3 * npad;
      for (int c = 0; c < 3; ++c) {
        const size_t o = (size_t)c * npad;
        V[o + w] = madd(V[o + w], f, __dsub_rn(a[o + w], a[o + p]));
      }
    }
  }
  if (w == 0) sc[slot * kScal + SC_U] = U;
}

// D(h): X += f V, t += f with f = h / (T + B); h = delta, or delta/2 for the last drift.
__global__ void __launch_bounds__(kBlock)
k_drift(int npad, int slot_lo, const double* __restrict__ par, double B, int tau, double* __restrict__ sX,
        const double* __restrict__ sV, const double* __restrict__ Tblk, int nblk, double* __restrict__ sc) {
  __shared__ double sT;
  const double H = par[0];
  const int slot = slot_lo + blockIdx.y;
  sum_partials(Tblk + (size_t)slot * nblk, nblk, 1, &sT);
  const double T = 0.5 * sT;
  const int nk = 2 * (slot + 1);
  const double delta = H / (double)nk;
  const double h = (tau == nk) ? 0.5 * delta : delta;
  const double f = h / (T + B);
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < npad) {
    double* X = sX + (size_t)slot * 3 * npad;
    const double* V = sV + (size_t)slot * 3 * npad;
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad;
      X[o + w] = madd(X[o + w], f, V[o + w]);
    }
  }
  if (w == 0) {
    sc[slot * kScal + SC_T_PHYS] += f;
    sc[slot * kScal + SC_T_KIN] = T;
  }
}

// The three components' block sums of m w (kRebuildComps warps-pairs of kBlock threads, one
// component each) into comblk: each is the sum that block_sum forms over kBlock threads (the
// same shuffle tree in each of the component's two warps, then the two warp sums added).
constexpr int kRebuildComps = 3;
static_assert(kBlock == 64, "the component sums below assume two warps per component");
__device__ __forceinline__ void component_block_sums(double x, double* scratch, double* out3) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = x;
  __syncthreads();
  if (threadIdx.x < kRebuildComps) out3[threadIdx.x] = scratch[2 * threadIdx.x] + scratch[2 * threadIdx.x + 1];
}

// Cartesian vector of every body from edge vectors: the path sum w_v = W_v + W_parent(v)
// + ... up to the root (root: 0), plus block sums of m w for the centre of mass. A CTA takes
// kBlock bodies with one thread per component, so the three walks of a body run side by side
// (each adds in the same order as one thread walking all three); beside pair launches of other
// divisions, which keep the FP64 pipe busy, the walks' share of the pipe grows with their warps.
__global__ void __launch_bounds__(kBlock * kRebuildComps)
k_rebuild(int n, int npad, size_t stride, const int* __restrict__ parent, const int* __restrict__ bylev,
          const double* __restrict__ Wb, double* __restrict__ wb, const double* __restrict__ m,
          double* __restrict__ comblk, int nblk) {
  __shared__ double scratch[2 * kRebuildComps];
  const int slot = blockIdx.y;
  const int comp = threadIdx.x / kBlock, b = threadIdx.x - comp * kBlock;
  const double* W = Wb + slot * stride + (size_t)comp * npad;
  double* wv = wb + slot * stride + (size_t)comp * npad;
  // thread i takes body bylev[i]: the lanes of a warp walk paths of about equal length
  const int i = blockIdx.x * kBlock + b;
  const int v = i < n ? bylev[i] : n;
  double s = 0.0;
  if (v < n) {
    for (int u = v; parent[u] >= 0; u = parent[u]) s = __dadd_rn(s, W[u]);
    wv[v] = s;
  }
  const double mv = v < n ? m[v] : 0.0;
  component_block_sums(__dmul_rn(mv, s), scratch, comblk + ((size_t)slot * nblk + blockIdx.x) * 3);
}

// k_rebuild with the slot's edge vectors (3 planes) and the parents staged in shared memory
// first, for systems whose 28 npad bytes fit: every hop of a root path then costs a
// shared-memory load instead of an L2 round trip. Each thread issues its 16-byte cp.async
// copies back to back and waits for its own; the additions and their order are k_rebuild's.
__global__ void __launch_bounds__(kBlock * kRebuildComps)
k_rebuild_staged(int n, int npad, size_t stride, const int* __restrict__ parent, const int* __restrict__ bylev,
                 const double* __restrict__ Wb, double* __restrict__ wb, const double* __restrict__ m,
                 double* __restrict__ comblk, int nblk) {
  extern __shared__ __align__(16) double sW[];  // 3 npad doubles, then npad parents
  int* sP = reinterpret_cast<int*>(sW + 3 * (size_t)npad);
  __shared__ double scratch[2 * kRebuildComps];
  const int slot = blockIdx.y;
  const double* W = Wb + slot * stride;
  {
    const char* gW = reinterpret_cast<const char*>(W);
    const char* gP = reinterpret_cast<const char*>(parent);
    const unsigned dW = (unsigned)__cvta_generic_to_shared(sW);
    const unsigned dP = (unsigned)__cvta_generic_to_shared(sP);
    const int qW = 3 * npad * 8 / 16, qP = npad * 4 / 16;  // npad is a multiple of 32
    for (int q = threadIdx.x; q < qW; q += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dW + 16 * q), "l"(gW + 16 * (size_t)q)
                   : "memory");
    for (int q = threadIdx.x; q < qP; q += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dP + 16 * q), "l"(gP + 16 * (size_t)q)
                   : "memory");
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
  }
  __syncthreads();
  const int comp = threadIdx.x / kBlock, b = threadIdx.x - comp * kBlock;
  const double* sWc = sW + (size_t)comp * npad;
  double* wv = wb + slot * stride + (size_t)comp * npad;
  const int i = blockIdx.x * kBlock + b;
  const int v = i < n ? bylev[i] : n;
  double s = 0.0;
  if (v < n) {
    for (int u = v; sP[u] >= 0; u = sP[u]) s = __dadd_rn(s, sWc[u]);
    wv[v] = s;
  }
  const double mv = v < n ? m[v] : 0.0;
  component_block_sums(__dmul_rn(mv, s), scratch, comblk + ((size_t)slot * nblk + blockIdx.x) * 3);
}

// Sum over the CTA, returned to every thread (block_sum leaves it in thread 0).
__device__ __forceinline__ double cta_sum(double x, double* scratch, double* out) {
  const double b = block_sum(x, scratch);
  if (threadIdx.x == 0) *out = b;
  __syncthreads();
  return *out;
}

// The Cartesian vectors of the edge vectors in sW (3 planes, shared) by path sums over the
// staged parents sP, shifted to the centre-of-mass frame and written to w_out; returns
// m w^2 of the thread's body (0 for none). One body per thread (blockDim >= n), in tree-level
// order; every thread of the CTA calls it (it holds barriers).
__device__ __forceinline__ double rebuild_cta(int n, int npad, double Mtot, const double* __restrict__ m,
                                              const int* sP, const int* __restrict__ bylev, const double* sW,
                                              double* w_out, double* scratch, double* s_bc) {
  const int tid = threadIdx.x;
  const int v = tid < n ? bylev[tid] : n;
  double q[3] = {0.0, 0.0, 0.0};
  if (v < n)
    for (int u = v; sP[u] >= 0; u = sP[u]) {
      q[0] = __dadd_rn(q[0], sW[u]);
      q[1] = __dadd_rn(q[1], sW[npad + u]);
      q[2] = __dadd_rn(q[2], sW[2 * (size_t)npad + u]);
    }
  const double mv = v < n ? m[v] : 0.0;
  double com[3];
  for (int c = 0; c < 3; ++c) com[c] = cta_sum(__dmul_rn(mv, q[c]), scratch, &s_bc[1 + c]);
  double t2 = 0.0;
  if (v < n) {
    for (int c = 0; c < 3; ++c) {
      q[c] = __dsub_rn(q[c], com[c] / Mtot);
      w_out[(size_t)c * npad + v] = q[c];
    }
    t2 = __dmul_rn(mv, __dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])), __dmul_rn(q[2], q[2])));
  }
  return t2;
}

// One substep level tau of division `slot` on the CTA: the kick K(delta) of k_kick with the
// accelerations a (3 planes) and force function U, the velocities rebuilt by path sums and
// shifted to the centre-of-mass frame with their kinetic energy (k_rebuild, k_shift), the
// drift of k_drift, and, when `pos` (the division kicks again), the positions rebuilt and
// shifted into r_out. Every thread of the CTA calls it; sW is 3 npad doubles of scratch.
__device__ __forceinline__ void level_body(int n, int npad, int slot, bool pos, double H, double B, double Mtot,
                                           int tau, double U, const double* a, const double* __restrict__ m,
                                           const int* sP, const int* __restrict__ bylev, double* V, double* X,
                                           double* sW, double* v_out, double* r_out, double* scratch, double* s_bc,
                                           double* __restrict__ sc) {
  const int tid = threadIdx.x;
  // K(delta): V_w += (delta / U) (a_w - a_parent(w))
  const double fk = (H / (double)(2 * (slot + 1))) / U;
  for (int w = tid; w < npad; w += blockDim.x) {
    const int p = sP[w];
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad + w;
      double x = V[o];
      if (p >= 0) x = madd(x, fk, __dsub_rn(a[o], a[(size_t)c * npad + p]));
      V[o] = x;
      sW[o] = x;
    }
  }
  if (tid == 0) sc[slot * kScal + SC_U] = U;
  __syncthreads();
  const double T = 0.5 * cta_sum(rebuild_cta(n, npad, Mtot, m, sP, bylev, sW, v_out, scratch, s_bc), scratch,
                                 &s_bc[4]);
  // D(h): X += f V, t += f with f = h / (T + B); h = delta, or delta/2 for the last drift
  const int nk = 2 * (slot + 1);
  const double delta = H / (double)nk;
  const double h = (tau == nk) ? 0.5 * delta : delta;
  const double fd = h / (T + B);
  for (int w = tid; w < npad; w += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad + w;
      const double x = madd(X[o], fd, V[o]);
      X[o] = x;
      sW[o] = x;
    }
  if (tid == 0) {
    sc[slot * kScal + SC_T_PHYS] += fd;
    sc[slot * kScal + SC_T_KIN] = T;
  }
  __syncthreads();
  if (pos) rebuild_cta(n, npad, Mtot, m, sP, bylev, sW, r_out, scratch, s_bc);
}

// One substep level of every active division of a system that one CTA holds (npad <= 1024,
// one body per thread; the step uses it up to kLevelCtaMax): level_body with the
// accelerations and force-function partials of the pair kernels - six launches of the
// multi-CTA path in one, with the CTA's barriers in place of the kernel boundaries. The
// edge vectors are staged in shared memory for the walks. The operations are those of the
// multi-CTA kernels; the centre-of-mass and kinetic sums are CTA-wide instead of per 64-body
// block, so they round in another order.
__global__ void __launch_bounds__(1024)
k_level_cta(int n, int npad, int slot_lo, int pos_lo, const double* __restrict__ par, double B, double Mtot,
            int tau, const double* __restrict__ m, const int* __restrict__ parent, const int* __restrict__ bylev,
            const double* __restrict__ sa, double* __restrict__ sV, double* __restrict__ sv, double* __restrict__ sX,
            double* __restrict__ sr, const double* __restrict__ Ublk, int nblk, double* __restrict__ sc) {
  extern __shared__ __align__(16) double lvl_sh[];  // 3 npad staged edge vectors, then npad parents
  double* sW = lvl_sh;
  int* sP = reinterpret_cast<int*>(lvl_sh + 3 * (size_t)npad);
  __shared__ double scratch[32];
  __shared__ double s_bc[8];
  const int slot = slot_lo + blockIdx.x;
  const size_t st = (size_t)3 * npad;
  for (int u = threadIdx.x; u < npad; u += blockDim.x) sP[u] = u < n ? parent[u] : -1;
  sum_partials(Ublk + (size_t)slot * nblk, nblk, 1, &s_bc[0]);  // ends with a barrier
  level_body(n, npad, slot, slot >= pos_lo, par[0], B, Mtot, tau, s_bc[0], sa + slot * st, m, sP, bylev,
             sV + slot * st, sX + slot * st, sW, sv + slot * st, sr + slot * st, scratch, s_bc, sc);
}

// One substep level of a division on a thread-block cluster of C CTAs, for systems too large for
// one CTA (k_level_cta) whose staged edge vectors still fit in shared memory: the kick (k_kick),
// the velocity rebuild and shift with the kinetic energy (k_rebuild, k_shift), the drift
// (k_drift) and, when the division kicks again, the position rebuild and shift - six launches,
// with five cluster barriers in place of the kernel boundaries.
//
// Every operation, and every sum's association, is that of the multi-kernel path, so the
// results are bit-identical to it: the 64-body blocks of those kernels are kept as groups of
// 3 x 64 threads (one thread per component), dealt out over the cluster's CTAs. The blocks of
// the tree walks take the bodies in level order (as k_rebuild), those of the element-wise
// phases in index order (as k_kick, k_shift, k_drift). Each block's partial sums (m w for the
// centre of mass, m w^2 for the kinetic energy) are written into every CTA's shared memory,
// and every CTA then adds the nblk partials in sum_partials' order. The edge vectors that a
// walk needs and the walks' results are exchanged the same way: each value is written by the
// CTA that computes it into every CTA's copy (distributed shared memory).
constexpr int kScGroupThreads = 3 * kBlock;  // a 64-body block, one thread per component
static_assert(kBlock == 64, "the substep cluster's block sums assume two warps per component");

// One CTA's share of a rebuild: the path sums of its level-order blocks over the edge vectors in
// sW, written with the blocks' centre-of-mass partials into every CTA of the cluster.
template <int C>
__device__ __forceinline__ void cluster_walks(int n, int npad, int nblk, int rank, int G, int g, int comp, int b,
                                              const int* __restrict__ bylev, const double* __restrict__ m,
                                              const int* sP, const double* sW, double* sQ, double* sCom,
                                              double* scr) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int t = threadIdx.x - g * kScGroupThreads;
  const int passes = (nblk + C * G - 1) / (C * G);
  for (int it = 0; it < passes; ++it) {
    const int blk = (it * C + rank) * G + g;
    const int i = blk * kBlock + b;
    const int v = (blk < nblk && i < n) ? bylev[i] : n;
    double s = 0.0;
    if (v < n) {
      const double* W = sW + (size_t)comp * npad;
      for (int u = v; sP[u] >= 0; u = sP[u]) s = __dadd_rn(s, W[u]);
      const size_t o = (size_t)comp * npad + v;
#pragma unroll
      for (int r = 0; r < C; ++r) cl.map_shared_rank(sQ, r)[o] = s;
    }
    double x = __dmul_rn(v < n ? m[v] : 0.0, s);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((t & 31) == 0) scr[g * 6 + (t >> 5)] = x;
    __syncthreads();
    if (t < 3 && blk < nblk) {
      const double val = scr[g * 6 + 2 * t] + scr[g * 6 + 2 * t + 1];
#pragma unroll
      for (int r = 0; r < C; ++r) cl.map_shared_rank(sCom, r)[blk * 3 + t] = val;
    }
    __syncthreads();
  }
}

// The centre of mass from the blocks' partials (warp c sums component c in sum_partials' order)
// into s_com[0..2]; holds a barrier.
__device__ __forceinline__ void cluster_com(int nblk, const double* sCom, double* s_com) {
  const int tid = threadIdx.x;
  if (tid < 96) {
    const int c = tid >> 5, lane = tid & 31;
    double s = 0.0;
    for (int bb = lane; bb < nblk; bb += 32) s += sCom[bb * 3 + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) s_com[c] = s;
  }
  __syncthreads();
}

template <int C>
__global__ void __launch_bounds__(kScGroupThreads * 5)
k_substep_cluster(int n, int npad, int nblk, int slot_lo, int pos_lo, int tau, const double* __restrict__ par,
                  double B, double Mtot, const double* __restrict__ m, const int* __restrict__ parent,
                  const int* __restrict__ bylev, const double* __restrict__ sa, double* __restrict__ sV,
                  double* __restrict__ sv, double* __restrict__ sX, double* __restrict__ sr,
                  const double* __restrict__ Ublk, double* __restrict__ Tblk, double* __restrict__ sc) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  // shared: staged edge vectors (3 npad), walk results (3 npad), centre-of-mass partials
  // (3 nblk), kinetic partials (nblk), parents (npad ints)
  extern __shared__ __align__(16) double sub_sh[];
  double* sW = sub_sh;
  double* sQ = sW + 3 * (size_t)npad;
  double* sCom = sQ + 3 * (size_t)npad;
  double* sT = sCom + 3 * (size_t)nblk;
  int* sP = reinterpret_cast<int*>(sT + nblk);
  __shared__ double scr[5 * 6];
  __shared__ double s_sc[4];
  __shared__ double sq3[5][3][kBlock];
  const int rank = (int)cl.block_rank();
  const int slot = slot_lo + (int)blockIdx.x / C;
  const bool pos = slot >= pos_lo;
  const int tid = threadIdx.x;
  const int G = (int)blockDim.x / kScGroupThreads;
  const int g = tid / kScGroupThreads, t = tid - g * kScGroupThreads;
  const int comp = t / kBlock, b = t - comp * kBlock;
  const int passes = (nblk + C * G - 1) / (C * G);
  const size_t st = (size_t)3 * npad;
  const double H = par[0];
  double* V = sV + slot * st;
  double* X = sX + slot * st;
  const double* a = sa + slot * st;

  for (int u = tid; u < npad; u += blockDim.x) sP[u] = u < n ? parent[u] : -1;
  sum_partials(Ublk + (size_t)slot * nblk, nblk, 1, &s_sc[0]);  // ends with a barrier
  const double U = s_sc[0];
  cl.sync();  // every CTA of the cluster runs before any writes into its shared memory
  // K(delta), as k_kick: V_w += (delta / U) (a_w - a_parent(w))
  const double fk = (H / (double)(2 * (slot + 1))) / U;
  for (int it = 0; it < passes; ++it) {
    const int blk = (it * C + rank) * G + g;
    const int w = blk * kBlock + b;
    if (blk < nblk && w < npad) {
      const size_t o = (size_t)comp * npad + w;
      double x = V[o];
      if (w < n) {
        const int p = sP[w];
        if (p >= 0) {
          x = madd(x, fk, __dsub_rn(a[o], a[(size_t)comp * npad + p]));
          V[o] = x;
        }
      }
#pragma unroll
      for (int r = 0; r < C; ++r) cl.map_shared_rank(sW, r)[o] = x;
    }
  }
  if (rank == 0 && tid == 0) sc[slot * kScal + SC_U] = U;
  cl.sync();
  // velocity rebuild (k_rebuild), then the shift and the kinetic partials (k_shift)
  cluster_walks<C>(n, npad, nblk, rank, G, g, comp, b, bylev, m, sP, sW, sQ, sCom, scr);
  cl.sync();
  cluster_com(nblk, sCom, &s_sc[1]);
  double* vout = sv + slot * st;
  for (int it = 0; it < passes; ++it) {
    const int blk = (it * C + rank) * G + g;
    const int w = blk * kBlock + b;
    const bool own = blk < nblk && w < n;
    double q = 0.0;
    if (own) {
      const size_t o = (size_t)comp * npad + w;
      q = __dsub_rn(sQ[o], s_sc[1 + comp] / Mtot);
      vout[o] = q;
    }
    sq3[g][comp][b] = q;
    __syncthreads();
    if (comp == 0) {
      double t2 = 0.0;
      if (own) {
        const double q0 = sq3[g][0][b], q1 = sq3[g][1][b], q2 = sq3[g][2][b];
        t2 = __dmul_rn(m[w], __dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2)));
      }
      for (int o = 16; o > 0; o >>= 1) t2 += __shfl_down_sync(0xffffffffu, t2, o);
      if ((t & 31) == 0) scr[g * 6 + (t >> 5)] = t2;
    }
    __syncthreads();
    if (t == 0 && blk < nblk) {
      const double val = scr[g * 6] + scr[g * 6 + 1];
      Tblk[(size_t)slot * nblk + blk] = val;
#pragma unroll
      for (int r = 0; r < C; ++r) cl.map_shared_rank(sT, r)[blk] = val;
    }
    __syncthreads();
  }
  cl.sync();
  // D(h), as k_drift: X += f V, t += f with f = h / (T + B); h = delta, or delta/2 for the last drift
  if (tid < 32) {
    double s = 0.0;
    for (int bb = tid; bb < nblk; bb += 32) s += sT[bb];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (tid == 0) s_sc[0] = s;
  }
  __syncthreads();
  const double T = 0.5 * s_sc[0];
  const int nk = 2 * (slot + 1);
  const double delta = H / (double)nk;
  const double h = (tau == nk) ? 0.5 * delta : delta;
  const double fd = h / (T + B);
  for (int it = 0; it < passes; ++it) {
    const int blk = (it * C + rank) * G + g;
    const int w = blk * kBlock + b;
    if (blk < nblk && w < npad) {
      const size_t o = (size_t)comp * npad + w;
      const double x = madd(X[o], fd, sW[o]);
      X[o] = x;
      if (pos) {
#pragma unroll
        for (int r = 0; r < C; ++r) cl.map_shared_rank(sW, r)[o] = x;
      }
    }
  }
  if (rank == 0 && tid == 0) {
    sc[slot * kScal + SC_T_PHYS] += fd;
    sc[slot * kScal + SC_T_KIN] = T;
  }
  if (!pos) return;  // nothing of this CTA's shared memory is read by another CTA after the last barrier
  cl.sync();
  // position rebuild and shift (k_rebuild, k_shift)
  cluster_walks<C>(n, npad, nblk, rank, G, g, comp, b, bylev, m, sP, sW, sQ, sCom, scr);
  cl.sync();
  cluster_com(nblk, sCom, &s_sc[1]);
  double* rout = sr + slot * st;
  for (int it = 0; it < passes; ++it) {
    const int blk = (it * C + rank) * G + g;
    const int w = blk * kBlock + b;
    if (blk < nblk && w < n) {
      const size_t o = (size_t)comp * npad + w;
      rout[o] = __dsub_rn(sQ[o], s_sc[1 + comp] / Mtot);
    }
  }
}

// Sum over a warp (lane 0 holds it): a fixed shuffle tree.
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// A whole attempt's divisions, one CTA each (systems with npad <= kDivisionCtaMax): the first
// half drift of k_init_drift, then the division's n_k substeps, each the pair sums of Sec. 3.4
// followed by the kick, velocity rebuild, drift and position rebuild of the multi-kernel path.
// One launch replaces the 3 + 3 n_k launches of the level-by-level path.
//
// The division's state stays in shared memory for the whole attempt. An FP64 instruction
// occupies its SM sub-partition's FP64 unit for about 64 cycles however few of the warp's lanes
// are active, so the serial parts give each warp one component of 32 bodies (thread
// (c, i) = (t / npad, t % npad) for t < 3 npad): the tree walks, kicks, drifts and
// centre-of-mass sums of the three components run on different warps, and the per-warp
// shuffle sums are added in warp order by one thread.
//
// Pair sums: the symmetric tiling of k_pair_tiles inside the CTA. The nb = npad / 32 body tiles
// form nb (nb + 1) / 2 tile pairs (I <= J); each tile pair's partner steps (32, or 16 on the
// diagonal) are split into S chunks, and warp w takes chunk w of the P S tasks. A task's lanes are
// the bodies of tile I; at step k lane l meets body (l + k) mod 32 of tile J, so the 32 partner
// sums are updated without conflicts in the task's shared j-side planes. Each unordered far pair
// is evaluated once, with the integer-pipe scalars of k_pair_tiles. The task also takes its
// share of its bodies' near partners (parent, children, grandparent, grandchildren, siblings for
// N_d = 2, from the edge vectors): partner number k of body i goes to the task of rank k modulo
// the (nb - I) S tasks whose i-side is tile I. A body then adds its tasks' partials in task
// order. The sum of m_j / r is exact within a task (UAcc).
//
// With C > 1 a division runs on a cluster of C CTAs: the tasks are dealt out over the cluster
// (task w to CTA w mod C), each CTA adds its own tasks' partials per body (in task order), and
// after a cluster barrier every CTA reads the C CTAs' sums through distributed shared memory and
// adds them in rank order. Every CTA runs the serial phases on its own copy of the state, which
// stays bit-identical across the cluster; rank 0 writes the results. The per-CTA sums are
// double-buffered by substep, so one cluster barrier per substep orders the writes of a
// substep's sums after every CTA's reads of the ones two substeps before.
template <int C>
__global__ void __launch_bounds__(kDivisionCtaThreads)
k_division_cta(int n, int npad, int K, int n_d, double G, const double* __restrict__ par, double B,
               double Mtot, const double* __restrict__ m, const int* __restrict__ parent, const int* __restrict__ gp,
               const int* __restrict__ child_off, const int* __restrict__ child_idx, const int* __restrict__ bylev,
               const double* __restrict__ X0, const double* __restrict__ V0, double* __restrict__ sX,
               double* __restrict__ sV, double* __restrict__ sc, const double* __restrict__ Tblk, int nblk) {
  // shared: edge positions X and velocities V, Cartesian positions sx, accelerations sA (3 npad
  // each), masses (npad), two buffers of the CTA's tasks' partials (kDivisionCtaThreads / 32
  // tasks x 7 planes of 32: the i-side ax, ay, az, m/r sums, then the j-side sums), two buffers
  // of the CTA's sums per body (4 planes of npad), mass significands (npad), then mass
  // exponents, parents, grandparents, children offsets (npad + 1) and children (npad)
  extern __shared__ __align__(16) double div_sh[];
  double* X = div_sh;
  double* V = X + 3 * (size_t)npad;
  double* sx = V + 3 * (size_t)npad;
  double* sA = sx + 3 * (size_t)npad;
  double* sm = sA + 3 * (size_t)npad;
  double* part = sm + npad;
  unsigned long long* smm =
      reinterpret_cast<unsigned long long*>(part + (size_t)2 * kDivisionCtaTasks * 7 * 32 + (size_t)8 * npad);
  int* sme = reinterpret_cast<int*>(smm + npad);
  int* sP = sme + npad;
  int* sG = sP + npad;
  int* sCo = sG + npad;
  int* sCi = sCo + npad + 1;
  __shared__ double red[kDivisionCtaThreads / 32];
  __shared__ double s_val[4];
  const int slot = blockIdx.x / C, rank = blockIdx.x - (blockIdx.x / C) * C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = npad >> 5;  // warps per component
  const size_t st = (size_t)3 * npad;
  const double H = par[0], t0 = par[1];
  __shared__ double sT0;
  sum_partials(Tblk + (size_t)K * nblk, nblk, 1, &sT0);  // T0 as k_start_derivs forms it
  const double T0 = 0.5 * sT0;
  const int nk = 2 * (slot + 1);
  const double delta = H / (double)nk;
  for (int u = tid; u < npad; u += blockDim.x) {
    const bool body = u < n;
    sP[u] = body ? parent[u] : -1;
    sG[u] = body ? gp[u] : -1;
    sCi[u] = body ? child_idx[u] : 0;
    const double mu = m[u];
    sm[u] = mu;
    const MassSplit ms = mass_split(mu);
    smm[u] = ms.m;
    sme[u] = ms.e;
    if (!body)  // the padding's positions, which no rebuild writes
      for (int c = 0; c < 3; ++c) sx[(size_t)c * npad + u] = 0.0;
  }
  for (int u = tid; u <= npad; u += blockDim.x) sCo[u] = child_off[u < n ? u : n];
  // the serial phases' task: component c of the body v at tree-level rank i
  const bool task = tid < 3 * npad;
  const int c = tid / npad, ti = tid - (tid / npad) * npad;
  const int v = (task && ti < n) ? bylev[ti] : n;
  const double mv = v < n ? m[v] : 0.0;
  // D(delta/2) from the step start (k_init_drift): X = X0 + f V0, V = V0
  const double f0 = (0.5 * delta) / (T0 + B);
  if (task) {
    const size_t o = (size_t)c * npad + ti;
    X[o] = madd(X0[o], f0, V0[o]);
    V[o] = V0[o];
  }
  double t_phys = t0 + f0, T = T0, U = 0.0;
  __syncthreads();

  // Cartesian vectors of the edge vectors W (one component per task) by path sums, shifted to
  // the centre-of-mass frame; returns the task's m v q^2 term (0 for none)
  auto rebuild = [&](const double* W, double* out) {
    double q = 0.0;
    if (v < n)
      for (int u = v; sP[u] >= 0; u = sP[u]) q = __dadd_rn(q, W[(size_t)c * npad + u]);
    if (task) {  // warp-uniform (3 npad is a multiple of 32)
      const double s = warp_sum(__dmul_rn(mv, q));
      if (lane == 0) red[warp] = s;
    }
    __syncthreads();
    if (tid < 3) {
      double com = red[tid * nb];
      for (int w = 1; w < nb; ++w) com += red[tid * nb + w];
      s_val[tid] = com / Mtot;
    }
    __syncthreads();
    double t2 = 0.0;
    if (v < n) {
      q = __dsub_rn(q, s_val[c]);
      if (out) out[(size_t)c * npad + v] = q;
      t2 = __dmul_rn(mv, __dmul_rn(q, q));
    }
    __syncthreads();  // s_val and red are free again
    return t2;
  };
  // T = sum of the tasks' m v^2 terms (warp order) / 2, and the drift factor f = h / (T + B)
  // of substep tau, to every thread (s_val[3], s_val[0])
  auto kinetic = [&](double x, int tau) {
    if (task) {
      const double s = warp_sum(x);
      if (lane == 0) red[warp] = s;
    }
    __syncthreads();
    if (tid == 0) {
      double a = red[0];
      for (int w = 1; w < 3 * nb; ++w) a += red[w];
      const double Tk = 0.5 * a;
      s_val[3] = Tk;
      s_val[0] = ((tau == nk) ? 0.5 * delta : delta) / (Tk + B);
    }
    __syncthreads();
    return s_val[3];
  };

  rebuild(X, sx);
  // the pair-sum tasks: tile pairs (in tile_pair order) times S chunks of partner steps (at most
  // 8 chunks: with 4 or 16 at most, attempts at N = 64 ... 160 took 2-16 % longer), dealt out
  // over the cluster
  const int ntp = nb * (nb + 1) / 2;
  int S = (kDivisionCtaTasks * C) / ntp;
  S = S < 1 ? 1 : (S > 8 ? 8 : S);
  const int ntask = ntp * S;  // <= kDivisionCtaTasks C (ntp <= 15)
  const bool nd1 = n_d >= 1, nd2 = n_d >= 2;
  for (int tau = 1; tau <= nk; ++tau) {
    double* partb = part + (size_t)(tau & 1) * kDivisionCtaTasks * 7 * 32;  // this substep's buffer
    __syncthreads();  // sx holds the rebuilt positions
    const int w = rank + C * warp;  // the warp's task
    if (w < ntask) {
      const int tp = w / S, sc_ = w - (w / S) * S;
      int I, J;
      tile_pair(tp, nb, I, J);
      const bool diag = I == J;
      const int kb = diag ? 1 + (16 * sc_) / S : (32 * sc_) / S;
      const int ke = diag ? 1 + (16 * (sc_ + 1)) / S : (32 * (sc_ + 1)) / S;
      double* pt = partb + (size_t)warp * 7 * 32;  // the task's 7 planes
      double* jx = pt + 4 * 32;
      double* jy = jx + 32;
      double* jz = jy + 32;
      jx[lane] = 0.0;
      jy[lane] = 0.0;
      jz[lane] = 0.0;
      __syncwarp();
      const int i = 32 * I + lane, j0 = 32 * J;
      const double xi = sx[i], yi = sx[npad + i], zi = sx[2 * npad + i];
      const MassSplit msi{smm[i], sme[i]};
      const int pi = sP[i], gpi = sG[i];
      const bool i_pad = i >= n;
      double ax = 0.0, ay = 0.0, az = 0.0;
      UAcc uacc;
      bool ubad = false;
      unsigned long long Rn;
      int eR;
      double sj, si;
      for (int k = kb; k < ke; ++k) {
        const int jl = (lane + k) & 31, j = j0 + jl;
        const int pj = sP[j], gj = sG[j];
        bool masked = i_pad | (j >= n) | (diag & (k == 16) & (lane >= 16));
        masked |= nd1 & ((pi == j) | (pj == i));
        masked |= nd2 & ((gpi == j) | (gj == i) | (pi == pj));
        const double dx = sx[j] - xi, dy = sx[npad + j] - yi, dz = sx[2 * npad + j] - zi;
        const unsigned long long mjm = smm[j];
        const int mje = sme[j];
        pair_scalars_core(dx, dy, dz, MassSplit{mjm, mje}, msi, Rn, eR, sj, si);
        sj = __longlong_as_double(masked ? 0ll : __double_as_longlong(sj));
        si = __longlong_as_double(masked ? 0ll : __double_as_longlong(si));
        ubad |= !masked && Rn == 0ull;
        uacc.add(masked ? 0ull : __umul64hi(mjm, Rn), masked ? uacc.L : mje + eR + 64);
        ax = fma(sj, dx, ax);
        ay = fma(sj, dy, ay);
        az = fma(sj, dz, az);
        // partner sums are kept with the opposite sign and negated once at the end
        jx[jl] = fma(si, dx, jx[jl]);
        jy[jl] = fma(si, dy, jy[jl]);
        jz[jl] = fma(si, dz, jz[jl]);
        __syncwarp();
      }
      // this task's share of body i's near partners: separation d = r_q - r_i from the edge
      // vectors, (+-X_a) + (+-X_b) (no second term for b < 0), signs flipped on the bit patterns
      if (nd1 && !i_pad) {
        const int count = (nb - I) * S, share = (J - I) * S + sc_;
        int kc = 0;  // partners seen so far, mod count
        const double* Xx = X;
        const double* Xy = X + npad;
        const double* Xz = X + 2 * (size_t)npad;
        auto flip = [](double x, bool neg) {
          return neg ? __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull) : x;
        };
        auto near = [&](int q, int a, bool na, int b, bool nb_) {
          const bool mine = kc == share;
          kc = kc + 1 == count ? 0 : kc + 1;
          if (!mine) return;
          double dx = flip(Xx[a], na), dy = flip(Xy[a], na), dz = flip(Xz[a], na);
          if (b >= 0) {
            dx = __dadd_rn(dx, flip(Xx[b], nb_));
            dy = __dadd_rn(dy, flip(Xy[b], nb_));
            dz = __dadd_rn(dz, flip(Xz[b], nb_));
          }
          pair_scalars_core(dx, dy, dz, MassSplit{smm[q], sme[q]}, msi, Rn, eR, sj, si);
          ubad |= Rn == 0ull;
          ax = fma(sj, dx, ax);
          ay = fma(sj, dy, ay);
          az = fma(sj, dz, az);
          if (q > i) uacc.add(__umul64hi(smm[q], Rn), sme[q] + eR + 64);
        };
        if (pi >= 0) near(pi, i, true, -1, false);
        const int c0 = sCo[i], c1 = sCo[i + 1];
        for (int a = c0; a < c1; ++a) {
          const int ch = sCi[a];
          near(ch, ch, false, -1, false);
        }
        if (nd2) {
          if (gpi >= 0) near(gpi, i, true, pi, true);
          for (int a = c0; a < c1; ++a) {
            const int ch = sCi[a];
            for (int b = sCo[ch]; b < sCo[ch + 1]; ++b) {
              const int gc = sCi[b];
              near(gc, gc, false, ch, false);
            }
          }
          if (pi >= 0)
            for (int b = sCo[pi]; b < sCo[pi + 1]; ++b) {
              const int sb = sCi[b];
              if (sb != i) near(sb, sb, false, i, true);
            }
        }
      }
      const double ui = ubad ? __longlong_as_double(0x7ff8000000000000LL) : uacc.value();
      if (diag) {  // both sides belong to tile I's bodies
        pt[lane] = ax - jx[lane];
        pt[32 + lane] = ay - jy[lane];
        pt[64 + lane] = az - jz[lane];
      } else {
        pt[lane] = ax;
        pt[32 + lane] = ay;
        pt[64 + lane] = az;
        const long long sgn = (long long)0x8000000000000000ull;
        jx[lane] = __longlong_as_double(__double_as_longlong(jx[lane]) ^ sgn);
        jy[lane] = __longlong_as_double(__double_as_longlong(jy[lane]) ^ sgn);
        jz[lane] = __longlong_as_double(__double_as_longlong(jz[lane]) ^ sgn);
      }
      pt[96 + lane] = ui;
    }
    __syncthreads();
    // this CTA's sums over its tasks, in task order: component c of body ti's acceleration and,
    // on the c = 0 tasks, the body's sum of m/r
    double a = 0.0, u = 0.0;
    if (task) {
      const int t = ti >> 5, l = ti & 31;
      int wt = 0;
      for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J)
          for (int q = 0; q < S; ++q, ++wt) {
            if ((wt & (C - 1)) != rank || (I != t && J != t)) continue;  // C is a power of two
            const double* pt = partb + (size_t)(wt / C) * 7 * 32;
            if (I == t) {
              a += pt[c * 32 + l];
              if (c == 0) u += pt[96 + l];
            } else {
              a += pt[(4 + c) * 32 + l];
            }
          }
    }
    if constexpr (C > 1) {
      // the cluster's sums: every CTA adds the C CTAs' sums in rank order
      double* loc = part + (size_t)2 * kDivisionCtaTasks * 7 * 32 + (size_t)(tau & 1) * 4 * npad;
      if (task) {
        loc[(size_t)c * npad + ti] = a;
        if (c == 0) loc[3 * (size_t)npad + ti] = u;
      }
      cooperative_groups::this_cluster().sync();  // every CTA's sums of this substep are written
      if (task) {
        double rc[C], ru[C];
#pragma unroll
        for (int r = 0; r < C; ++r) {
          const double* lr = cooperative_groups::this_cluster().map_shared_rank(loc, r);
          rc[r] = lr[(size_t)c * npad + ti];
          ru[r] = c == 0 ? lr[3 * (size_t)npad + ti] : 0.0;
        }
        a = rc[0];
        u = ru[0];
#pragma unroll
        for (int r = 1; r < C; ++r) {
          a += rc[r];
          u += ru[r];
        }
      }
    }
    double um = 0.0;
    if (task) {
      sA[(size_t)c * npad + ti] = G * a;
      if (c == 0 && ti < n) um = sm[ti] * u;
    }
    {
      if (warp < nb) {
        const double s = warp_sum(um);
        if (lane == 0) red[warp] = s;
      }
      __syncthreads();
      if (tid == 0) {
        double a = red[0];
        for (int w = 1; w < nb; ++w) a += red[w];
        const double Ug = G * a;
        s_val[3] = Ug;
        s_val[0] = delta / Ug;
      }
      __syncthreads();
      U = s_val[3];
    }
    // K(delta): V_w += (delta / U) (a_w - a_parent(w))
    if (task) {
      const int p = sP[ti];
      if (p >= 0) {
        const size_t o = (size_t)c * npad;
        V[o + ti] = madd(V[o + ti], s_val[0], __dsub_rn(sA[o + ti], sA[o + p]));
      }
    }
    __syncthreads();
    // velocities rebuilt and shifted; T = sum m v^2 / 2
    // D(h): X += f V, t += f with f = h / (T + B); h = delta, or delta/2 for the last drift
    T = kinetic(rebuild(V, nullptr), tau);
    const double fd = s_val[0];
    if (task) {
      const size_t o = (size_t)c * npad + ti;
      X[o] = madd(X[o], fd, V[o]);
    }
    t_phys += fd;
    __syncthreads();
    if (tau < nk) rebuild(X, sx);
  }
  // the division's final state and scalars for the extrapolation (every CTA of a cluster holds
  // the same; no CTA leaves while another may still read its partials)
  if constexpr (C > 1) {
    cooperative_groups::this_cluster().sync();
    if (rank != 0) return;
  }
  if (task) {
    const size_t o = (size_t)c * npad + ti;
    sX[slot * st + o] = X[o];
    sV[slot * st + o] = V[o];
  }
  if (tid == 0) {
    sc[slot * kScal + SC_T_PHYS] = t_phys;
    sc[slot * kScal + SC_T_KIN] = T;
    sc[slot * kScal + SC_U] = U;
  }
}

// Shift to the centre-of-mass frame: w -= (sum m w) / M; optionally block sums of m w^2.
__global__ void __launch_bounds__(kBlock)
k_shift(int n, int npad, size_t stride, double Mtot, double* __restrict__ wb, const double* __restrict__ m,
        const double* __restrict__ comblk, double* __restrict__ Tblk, int nblk) {
  __shared__ double scratch[32];
  __shared__ double sc3[3];
  const int slot = blockIdx.y;
  sum_partials3(comblk + (size_t)slot * nblk * 3, nblk, sc3);
  double* wv = wb + slot * stride;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double t2 = 0.0;
  if (v < n) {
    double q[3];
    for (int c = 0; c < 3; ++c) {
      q[c] = __dsub_rn(wv[(size_t)c * npad + v], sc3[c] / Mtot);
      wv[(size_t)c * npad + v] = q[c];
    }
    t2 = __dmul_rn(m[v], __dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])), __dmul_rn(q[2], q[2])));
  }
  if (Tblk) {
    const double s = block_sum(t2, scratch);
    if (threadIdx.x == 0) Tblk[(size_t)slot * nblk + blockIdx.x] = s;
  }
}

__device__ __forceinline__ void neville(const double* S, int K, double& tkk, double& tprev) {
  double prev[kMaxKfix], cur[kMaxKfix];
#pragma unroll
  for (int k = 0; k < kMaxKfix; ++k) {
    if (k < K) {
      cur[0] = S[k];
#pragma unroll
      for (int j = 1; j < kMaxKfix; ++j)
        if (j <= k) cur[j] = fma(__dsub_rn(cur[j - 1], prev[j - 1]), c_fac[k][j], cur[j - 1]);
      if (k == K - 2) tprev = cur[k];
#pragma unroll
      for (int j = 0; j < kMaxKfix; ++j) prev[j] = cur[j];
    }
  }
  tkk = prev[K - 1];
}

__device__ __forceinline__ double norm3(double x, double y, double z) {
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
}

// Neville-Aitken extrapolation of every edge vector component and t over the K divisions
// (Sec. 4.2), and the error of Eq. gbs-criterion:
// eps = max_q |T_KK - T_{K-1,K-1}|_q / |S_q(s0) + delta_K S'_q(s0)| over X_v, V_v, t with
// S' = V / (T0 + B) for X, A0 / U0 for V, 1 / (T0 + B) for t, delta_K = H / n_K.
// CTA (b, part) takes the 64 bodies of block b with one thread per component, for the edge
// positions (part 0, which also takes t) or the edge velocities (part 1): the six tableaux of a
// body run on six threads, and the first thread of each body forms its error term. The maximum
// over the CTAs' maxima (k_eps_final) does not depend on their order.
__global__ void __launch_bounds__(3 * kBlock)
k_extrapolate(int n, int npad, int K, const double* __restrict__ par, double B, const int* __restrict__ parent,
              const double* __restrict__ sX, const double* __restrict__ sV, const double* __restrict__ X0,
              const double* __restrict__ V0, const double* __restrict__ A0, const double* __restrict__ sc,
              double* __restrict__ Tkk, double* __restrict__ epsblk, int nblk) {
  __shared__ double scratch[32];
  __shared__ double sd[3][kBlock];
  const double H = par[0], t0 = par[1];
  const int part = blockIdx.y;
  const int comp = threadIdx.x / kBlock, b = threadIdx.x - comp * kBlock;
  const int v = blockIdx.x * kBlock + b;
  const double T0 = sc[K * kScal + SC_T_KIN], U0 = sc[K * kScal + SC_U];
  const double rate = 1.0 / (T0 + B);
  const double delta = H / (double)(2 * K);
  const size_t slot_stride = (size_t)3 * npad;
  double e = 0.0;
  if (v < n) {
    double S[kMaxKfix];
    const double* src = part == 0 ? sX : sV;
    double tkk, tp = 0.0;
    for (int k = 0; k < K; ++k) S[k] = src[k * slot_stride + (size_t)comp * npad + v];
    neville(S, K, tkk, tp);
    Tkk[(size_t)(3 * part + comp) * npad + v] = tkk;
    sd[comp][b] = __dsub_rn(tkk, tp);
  }
  __syncthreads();
  if (comp == 0 && v < n && parent[v] >= 0) {
    double q[3];
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad + v;
      q[c] = part == 0 ? madd(X0[o], delta, __dmul_rn(V0[o], rate)) : madd(V0[o], delta, A0[o] / U0);
    }
    e = norm3(sd[0][b], sd[1][b], sd[2][b]) / fmax(norm3(q[0], q[1], q[2]), 1e-300);
  }
  if (part == 0 && v == 0 && comp == 0) {
    double S[kMaxKfix];
    for (int k = 0; k < K; ++k) S[k] = sc[k * kScal + SC_T_PHYS];
    double tkk, tp = 0.0;
    neville(S, K, tkk, tp);
    Tkk[(size_t)6 * npad] = tkk;
    const double rt = fabs(__dsub_rn(tkk, tp)) / fmax(fabs(madd(t0, delta, rate)), 1e-300);
    e = nanmax(e, rt);
  }
  const double bm = block_nanmax(e, scratch);
  if (threadIdx.x == 0) epsblk[(size_t)part * nblk + blockIdx.x] = bm;
}

__global__ void k_eps_final(int npad, const double* __restrict__ epsblk, int nblk, const double* __restrict__ Tkk,
                            double* __restrict__ res) {
  __shared__ double scratch[32];
  double e = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) e = nanmax(e, epsblk[b]);
  e = block_nanmax(e, scratch);
  if (threadIdx.x == 0) {
    res[0] = e;
    res[1] = Tkk[(size_t)6 * npad];
  }
}

// Block partials of T = sum m v^2 / 2 (stored as sum m v^2), P = sum m v, L = sum m r x v.
__global__ void __launch_bounds__(kBlock)
k_moments(int n, int npad, const double* __restrict__ m, const double* __restrict__ r, const double* __restrict__ v,
          double* __restrict__ mom) {
  __shared__ double scratch[32];
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  double q[7] = {0, 0, 0, 0, 0, 0, 0};
  if (w < n) {
    const double mw = m[w];
    const double x = r[w], y = r[npad + w], z = r[2 * (size_t)npad + w];
    const double vx = v[w], vy = v[npad + w], vz = v[2 * (size_t)npad + w];
    q[0] = mw * ((vx * vx + vy * vy) + vz * vz);
    q[1] = mw * vx;
    q[2] = mw * vy;
    q[3] = mw * vz;
    q[4] = mw * (y * vz - z * vy);
    q[5] = mw * (z * vx - x * vz);
    q[6] = mw * (x * vy - y * vx);
  }
  for (int c = 0; c < 7; ++c) {
    const double s = block_sum(q[c], scratch);
    if (threadIdx.x == 0) mom[(size_t)blockIdx.x * 8 + c] = s;
  }
}

}  // namespace

cudaError_t launch_prepare(mstar_ctx* c) {
  k_prepare<<<c->nblk, kBlock, 0, c->stream>>>(c->n, c->npad, c->K, c->d.m, c->d.parent, c->d.r, c->d.v, c->d.X0,
                                              c->d.V0, c->d.sr, c->d.sX, c->d.Tblk, c->nblk);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_start_derivs(mstar_ctx* c) {
  k_start_derivs<<<c->nblk, kBlock, 0, c->stream>>>(c->n, c->npad, c->K, c->d.parent, c->d.sa, c->d.A0, c->d.Ublk,
                                                   c->d.Tblk, c->nblk, c->d.sc, c->d.res);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

// The Neville factors 1 / ((n_k / n_{k-j})^2 - 1) for every k < kMaxKfix (they do not
// depend on k_fix), once per context.
cudaError_t upload_step_constants(mstar_ctx* c) {
  double fac[kMaxKfix][kMaxKfix] = {};
  for (int k = 0; k < kMaxKfix; ++k)
    for (int j = 1; j <= k; ++j) {
      const double ratio = (double)(2 * (k + 1)) / (double)(2 * (k - j + 1));
      fac[k][j] = 1.0 / (ratio * ratio - 1.0);
    }
  return cudaMemcpyToSymbolAsync(c_fac, fac, sizeof(fac), 0, cudaMemcpyHostToDevice, c->stream);
}

// The attempt's H and start time t into d.res[4], d.res[5] (from pinned host_res[8], [9]);
// the host has synchronised with the previous attempt, so the staging slots are free.
cudaError_t stage_attempt_scalars(mstar_ctx* c, double H) {
  c->host_res[8] = H;
  c->host_res[9] = c->t;
  return cudaMemcpyAsync(c->d.res + 4, c->host_res + 8, 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
}

cudaError_t launch_init_drift(mstar_ctx* c) {
  dim3 grid(c->nblk, c->K);
  k_init_drift<<<grid, kBlock, 0, c->stream>>>(c->n, c->npad, c->K, c->d.res + 4, c->B, c->d.X0, c->d.V0, c->d.sX,
                                              c->d.sV, c->d.sc, c->d.Tblk, c->nblk);
  MSTAR_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t st = (size_t)3 * c->npad;
  return launch_rebuild(c, c->d.sX, c->d.sr, st, c->K, 0, nullptr, c->d.comblk);
}

cudaError_t launch_kick(mstar_ctx* c, int slot_lo, int slot_hi) {
  dim3 grid(c->nblk, slot_hi - slot_lo);
  k_kick<<<grid, kBlock, 0, c->stream>>>(c->n, c->npad, slot_lo, c->d.res + 4, c->d.parent, c->d.sa, c->d.sV,
                                        c->d.Ublk, c->nblk, c->d.sc);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_drift(mstar_ctx* c, int slot_lo, int slot_hi, int tau) {
  dim3 grid(c->nblk, slot_hi - slot_lo);
  k_drift<<<grid, kBlock, 0, c->stream>>>(c->npad, slot_lo, c->d.res + 4, c->B, tau, c->d.sX, c->d.sV, c->d.Tblk,
                                         c->nblk, c->d.sc);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_rebuild(mstar_ctx* c, const double* W, double* w, size_t stride, int nsl, int want_T,
                           double* Tblk_base, double* comblk_base) {
  if (nsl <= 0) return cudaSuccess;
  dim3 grid(c->nblk, nsl);
  const size_t staged = (size_t)c->npad * (3 * sizeof(double) + sizeof(int));
  cudaError_t e;
  if (staged <= c->rebuild_smem) {
    k_rebuild_staged<<<grid, kBlock * kRebuildComps, staged, c->stream>>>(c->n, c->npad, stride, c->d.parent, c->d.bylev, W, w,
                                                           c->d.m, comblk_base, c->nblk);
  } else {
    k_rebuild<<<grid, kBlock * kRebuildComps, 0, c->stream>>>(c->n, c->npad, stride, c->d.parent, c->d.bylev, W, w, c->d.m,
                                              comblk_base, c->nblk);
  }
  MSTAR_LAUNCHED(c);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_shift<<<grid, kBlock, 0, c->stream>>>(c->n, c->npad, stride, c->Mtot, w, c->d.m, comblk_base,
                                         want_T ? Tblk_base : nullptr, c->nblk);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

// Clusters of Cl CTAs of the division kernel that the device can hold at once (0: it cannot
// launch them at all, e.g. when a partition of the GPU has too few SMs per cluster).
template <int Cl>
int division_clusters_resident(const mstar_ctx* c) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->K * Cl);
  cfg.blockDim = dim3(kDivisionCtaThreads);
  cfg.dynamicSmemBytes = division_cta_smem(c->npad);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int num = 0;
  if (cudaOccupancyMaxActiveClusters(&num, k_division_cta<Cl>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

// At context creation: the division kernel's shared memory for this size (above 48 KB needs it),
// and a cluster size the device can launch (halved from the requested one until it can).
cudaError_t prepare_division_cta(mstar_ctx* c) {
  if (c->npad > kDivisionCtaMax) return cudaSuccess;
  const int smem = (int)division_cta_smem(c->npad);
  cudaError_t e = cudaFuncSetAttribute(k_division_cta<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_division_cta<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_division_cta<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_division_cta<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess || !c->div_cta) return e;
  for (;;) {
    int num = 1;
    switch (c->div_cluster) {
      case 8: num = division_clusters_resident<8>(c); break;
      case 4: num = division_clusters_resident<4>(c); break;
      case 2: num = division_clusters_resident<2>(c); break;
      default: return cudaSuccess;
    }
    if (num > 0) return cudaSuccess;
    c->div_cluster /= 2;
  }
}

template <int Cl>
cudaError_t launch_division_cta_c(mstar_ctx* c) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->K * Cl);
  cfg.blockDim = dim3(kDivisionCtaThreads);
  cfg.dynamicSmemBytes = division_cta_smem(c->npad);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_division_cta<Cl>, c->n, c->npad, c->K, c->p.n_d, c->p.G,
                            (const double*)(c->d.res + 4), c->B, c->Mtot, (const double*)c->d.m,
                            (const int*)c->d.parent, (const int*)c->d.gp, (const int*)c->d.child_off,
                            (const int*)c->d.child_idx, (const int*)c->d.bylev, (const double*)c->d.X0,
                            (const double*)c->d.V0, c->d.sX, c->d.sV, c->d.sc, (const double*)c->d.Tblk, c->nblk);
}

// Every division of an attempt, from the first half drift to the last drift, in one launch
// with one CTA, or a cluster of c->div_cluster CTAs, per division (npad <= kDivisionCtaMax).
cudaError_t launch_division_cta(mstar_ctx* c) {
  cudaError_t e;
  switch (c->div_cluster) {
    case 2: e = launch_division_cta_c<2>(c); break;
    case 4: e = launch_division_cta_c<4>(c); break;
    case 8: e = launch_division_cta_c<8>(c); break;
    default: e = launch_division_cta_c<1>(c); break;
  }
  MSTAR_LAUNCHED(c);
  c->force_evals += (long long)c->K * (c->K + 1);  // sum of n_k = 2 (k + 1) over the divisions
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// One substep level (kick, velocity rebuild, drift, position rebuild) of the divisions
// [slot_lo, slot_hi) in one launch, for systems with npad <= kLevelCtaMax.
cudaError_t launch_level_cta(mstar_ctx* c, int slot_lo, int slot_hi, int pos_lo, int tau) {
  const size_t smem = (size_t)c->npad * (3 * sizeof(double) + sizeof(int));
  k_level_cta<<<slot_hi - slot_lo, c->npad, smem, c->stream>>>(c->n, c->npad, slot_lo, pos_lo, c->d.res + 4, c->B,
                                                            c->Mtot, tau, c->d.m, c->d.parent, c->d.bylev, c->d.sa,
                                                            c->d.sV, c->d.sv, c->d.sX, c->d.sr, c->d.Ublk, c->nblk,
                                                            c->d.sc);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

size_t substep_cluster_smem(int npad, int nblk) {
  return (size_t)(6 * (size_t)npad + 4 * (size_t)nblk) * sizeof(double) + (size_t)npad * sizeof(int);
}

template <int Cl>
int substep_clusters_resident(const mstar_ctx* c, int G) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Cl);
  cfg.blockDim = dim3(kScGroupThreads * G);
  cfg.dynamicSmemBytes = substep_cluster_smem(c->npad, c->nblk);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int num = 0;
  if (cudaOccupancyMaxActiveClusters(&num, k_substep_cluster<Cl>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

// At context creation, for kLevelCtaMax < npad <= kSubstepClusterMax: the cluster substep
// kernel's shared memory, and the largest cluster of up to 8 CTAs that the device can launch
// (c->sub_cluster stays 0, and the multi-kernel path serves, if none can).
cudaError_t prepare_substep_cluster(mstar_ctx* c) {
  c->sub_cluster = 0;
  if (c->npad <= kLevelCtaMax || c->npad > kSubstepClusterMax) return cudaSuccess;
  const int smem = (int)substep_cluster_smem(c->npad, c->nblk);
  cudaError_t e = cudaFuncSetAttribute(k_substep_cluster<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_substep_cluster<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_substep_cluster<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  for (int Cl = 8; Cl >= 2; Cl /= 2) {
    const int G = std::min(5, (c->nblk + Cl - 1) / Cl);
    int num = 0;
    switch (Cl) {
      case 8: num = substep_clusters_resident<8>(c, G); break;
      case 4: num = substep_clusters_resident<4>(c, G); break;
      default: num = substep_clusters_resident<2>(c, G); break;
    }
    if (num > 0) {
      c->sub_cluster = Cl;
      c->sub_groups = G;
      return cudaSuccess;
    }
  }
  return cudaSuccess;
}

template <int Cl>
cudaError_t launch_substep_cluster_c(mstar_ctx* c, int slot_lo, int slot_hi, int pos_lo, int tau) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Cl * (slot_hi - slot_lo));
  cfg.blockDim = dim3(kScGroupThreads * c->sub_groups);
  cfg.dynamicSmemBytes = substep_cluster_smem(c->npad, c->nblk);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_substep_cluster<Cl>, c->n, c->npad, c->nblk, slot_lo, pos_lo, tau,
                            (const double*)(c->d.res + 4), c->B, c->Mtot, (const double*)c->d.m,
                            (const int*)c->d.parent, (const int*)c->d.bylev, (const double*)c->d.sa, c->d.sV,
                            c->d.sv, c->d.sX, c->d.sr, (const double*)c->d.Ublk, c->d.Tblk, c->d.sc);
}

// One substep level (kick, velocity rebuild, drift, position rebuild) of the divisions
// [slot_lo, slot_hi) in one launch, a cluster of c->sub_cluster CTAs per division; the
// divisions >= pos_lo get their positions rebuilt.
cudaError_t launch_substep_cluster(mstar_ctx* c, int slot_lo, int slot_hi, int pos_lo, int tau) {
  if (slot_hi <= slot_lo) return cudaSuccess;
  cudaError_t e;
  switch (c->sub_cluster) {
    case 8: e = launch_substep_cluster_c<8>(c, slot_lo, slot_hi, pos_lo, tau); break;
    case 4: e = launch_substep_cluster_c<4>(c, slot_lo, slot_hi, pos_lo, tau); break;
    case 2: e = launch_substep_cluster_c<2>(c, slot_lo, slot_hi, pos_lo, tau); break;
    default: return cudaErrorInvalidValue;
  }
  MSTAR_LAUNCHED(c);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Allows the staged rebuild kernel the shared memory a context of this size needs (at
// context creation, outside any stream capture); larger systems keep k_rebuild.
cudaError_t prepare_rebuild(mstar_ctx* c) {
  const size_t staged = (size_t)c->npad * (3 * sizeof(double) + sizeof(int));
  c->rebuild_smem = 0;
  if (staged > kRebuildStageBytes) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(k_rebuild_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged);
  if (e != cudaSuccess) return e;
  c->rebuild_smem = staged;
  return cudaSuccess;
}

// The largest shared-memory share for the O(N) kernels of an attempt (see
// prefer_shared_pair_kernels in pair.cu).
void prefer_shared_step_kernels() {
  const int sh = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(k_rebuild_staged, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_rebuild, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_kick, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_drift, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_shift, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_init_drift, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_extrapolate, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaFuncSetAttribute(k_eps_final, cudaFuncAttributePreferredSharedMemoryCarveout, sh);
  cudaGetLastError();
}

cudaError_t launch_extrapolate(mstar_ctx* c) {
  k_extrapolate<<<dim3(c->nblk, 2), 3 * kBlock, 0, c->stream>>>(c->n, c->npad, c->K, c->d.res + 4, c->B,
                                                                c->d.parent, c->d.sX, c->d.sV, c->d.X0, c->d.V0,
                                                                c->d.A0, c->d.sc, c->d.Tkk, c->d.epsblk, c->nblk);
  MSTAR_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_eps_final<<<1, kBlock, 0, c->stream>>>(c->npad, c->d.epsblk, 2 * c->nblk, c->d.Tkk, c->d.res);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

// block sums of m w (slot 0 of comblk)
__global__ void __launch_bounds__(kBlock)
k_mw(int n, int npad, const double* __restrict__ m, const double* __restrict__ w, double* __restrict__ comblk) {
  __shared__ double scratch[32];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const double mv = v < n ? m[v] : 0.0;
  for (int c = 0; c < 3; ++c) {
    const double x = v < n ? w[(size_t)c * npad + v] : 0.0;
    const double b = block_sum(__dmul_rn(mv, x), scratch);
    if (threadIdx.x == 0) comblk[(size_t)blockIdx.x * 3 + c] = b;
  }
}

cudaError_t launch_com_shift(mstar_ctx* c, double* w, double* Tblk) {
  k_mw<<<c->nblk, kBlock, 0, c->stream>>>(c->n, c->npad, c->d.m, w, c->d.comblk);
  MSTAR_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_shift<<<dim3(c->nblk, 1), kBlock, 0, c->stream>>>(c->n, c->npad, 0, c->Mtot, w, c->d.m, c->d.comblk, Tblk,
                                                     c->nblk);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

cudaError_t launch_moments(mstar_ctx* c) {
  k_moments<<<c->nblk, kBlock, 0, c->stream>>>(c->n, c->npad, c->d.m, c->d.r, c->d.v, c->d.mom);
  MSTAR_LAUNCHED(c);
  return cudaGetLastError();
}

}  // namespace mstar
