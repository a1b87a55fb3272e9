// The O(N^2) pair loop (Eq. 2) with the near/far separation rule of Sec. 3.4.
//
// Far pairs use Cartesian separations r_j - r_i; near pairs (within N_d tree edges,
// Eq. LCA) use sums of MST edge vectors. The tiled kernel evaluates every unordered far
// pair exactly once and applies the result to both bodies (a_i += m_j d/r^3,
// a_j -= m_i d/r^3), which halves the FP64 work - the resource that bounds this loop on
// GB300. Near pairs are masked out of the tiles with integer compares on parent and
// grandparent indices and summed in a sparse pass with the edge-vector separations.
//
// Per pair the FP64 pipe issues only the separation (3 DADD) and the two force
// accumulations (6 DFMA); r^2, 1/r, 1/r^3 and the mass products run on the integer pipe
// (pair_scalars_core), and so does the force-function sum: m_j / r is a 64-bit product of
// significands added exactly into a 128-bit fixed-point accumulator (UAcc) and rounded to a
// double once per tile.
//
// Tiles: the N bodies form NT tiles of T = 32*W. CTA (I, J), I <= J, owns the I-tile as
// "i" bodies (one per thread, accumulators in registers) and stages the J-tile ("j"
// bodies) in shared memory together with their accumulators. Each warp sweeps the W
// 32-wide sub-tiles in a rotated order; within a sub-tile, lane l pairs with j-slot
// (l + k) mod 32 at step k, so the 32 lanes update 32 distinct j accumulators at every
// step and no atomics are needed. On a diagonal tile only pairs i < j are visited.
//
// Determinism: CTA (I, J) writes its i-side sums into partial slot J of the i bodies and
// its j-side sums into slot I of the j bodies (a diagonal tile writes both into slot I).
// Every body thus receives exactly one write per slot, and the finishing pass adds the
// NT slots in a fixed order.
#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

// Upper-triangle tile pair tp -> (I, J), rows of length NT - I.
__device__ __forceinline__ void tile_pair(int tp, int NT, int& I, int& J) {
  float b = (float)NT + 0.5f;
  int i = (int)floorf(b - sqrtf(fmaxf(b * b - 2.0f * (float)tp, 0.0f)));
  i = max(0, min(i, NT - 1));
  auto start = [NT](int r) { return r * NT - (r * (r - 1)) / 2; };
  while (i > 0 && start(i) > tp) --i;
  while (i + 1 < NT && start(i + 1) <= tp) ++i;
  I = i;
  J = i + (tp - start(i));
}

template <int W>
__global__ void __launch_bounds__(32 * W)
k_pair_tiles(int n, int npad, int NT, int slot_lo, int n_d, const double* __restrict__ m,
             const int* __restrict__ parent, const int* __restrict__ gp, const double* __restrict__ sr,
             double* __restrict__ P) {
  constexpr int T = 32 * W;
  __shared__ double sx[T], sy[T], sz[T], sax[T], say[T], saz[T];
  __shared__ unsigned long long smm[T];
  __shared__ int sp[T], sg[T], sme[T];

  const int slot = slot_lo + blockIdx.y;
  int I, J;
  tile_pair(blockIdx.x, NT, I, J);
  const double* rx = sr + (size_t)slot * 3 * npad;
  const double* ry = rx + npad;
  const double* rz = ry + npad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = J * T;
  sx[tid] = rx[j0 + tid];
  sy[tid] = ry[j0 + tid];
  sz[tid] = rz[j0 + tid];
  {
    const MassSplit ms = mass_split(m[j0 + tid]);
    smm[tid] = ms.m;
    sme[tid] = ms.e;
  }
  sp[tid] = parent[j0 + tid];
  sg[tid] = gp[j0 + tid];
  sax[tid] = 0.0;
  say[tid] = 0.0;
  saz[tid] = 0.0;
  const int i = I * T + tid;
  const double xi = rx[i], yi = ry[i], zi = rz[i];
  const MassSplit msi = mass_split(m[i]);
  const int pi = parent[i], gpi = gp[i];
  const bool i_pad = i >= n;
  const bool nd1 = n_d >= 1, nd2 = n_d >= 2;
  double axi = 0.0, ayi = 0.0, azi = 0.0;
  UAcc uacc;          // sum over j of m_j / r_ij
  bool ubad = false;  // a coincident pair: the force is undefined
  const bool diag = (I == J);
  __syncthreads();

#pragma unroll 1
  for (int s = 0; s < W; ++s) {
    const int sub = (warp + s) & (W - 1);
    const bool self = diag && sub == warp;
    if (!(diag && sub < warp)) {
      const int kbeg = self ? 1 : 0;
      const int kend = self ? 17 : 32;
#pragma unroll 4
      for (int k = kbeg; k < kend; ++k) {
        const int jl = sub * 32 + ((lane + k) & 31);
        const int j = j0 + jl;
        const double xj = sx[jl], yj = sy[jl], zj = sz[jl];
        const int pj = sp[jl], gj = sg[jl];
        bool masked = i_pad | (j >= n) | (self & (k == 16) & (lane >= 16));
        masked |= nd1 & ((pi == j) | (pj == i));
        masked |= nd2 & ((gpi == j) | (gj == i) | (pi == pj));
        double dx = xj - xi, dy = yj - yi, dz = zj - zi;
        // keep the separations in registers: recomputing them for the accumulations would
        // cost three more FP64 instructions per pair
        asm volatile("" : "+d"(dx), "+d"(dy), "+d"(dz));
        unsigned long long Rn;
        int eR;
        double sj, si;
        const unsigned long long mjm = smm[jl];
        const int mje = sme[jl];
        pair_scalars_core(dx, dy, dz, MassSplit{mjm, mje}, msi, Rn, eR, sj, si);
        // masked pairs contribute nothing (integer selects on the bit patterns)
        sj = __longlong_as_double(masked ? 0ll : __double_as_longlong(sj));
        si = __longlong_as_double(masked ? 0ll : __double_as_longlong(si));
        ubad |= !masked && Rn == 0ull;
        // m_j / r = mjm Rn 2^(mje + eR) ~ hi64(mjm Rn) 2^(mje + eR + 64)
        uacc.add(masked ? 0ull : __umul64hi(mjm, Rn), masked ? uacc.L : mje + eR + 64);
        axi = fma(sj, dx, axi);
        ayi = fma(sj, dy, ayi);
        azi = fma(sj, dz, azi);
        // j-side sums are kept with the opposite sign and negated once when written
        sax[jl] = fma(si, dx, sax[jl]);
        say[jl] = fma(si, dy, say[jl]);
        saz[jl] = fma(si, dz, saz[jl]);
        __syncwarp();
      }
    }
    __syncthreads();
  }

  const double ui = ubad ? __longlong_as_double(0x7ff8000000000000LL) : uacc.value();
  double* Ps = P + (size_t)slot * NT * 4 * npad;
  if (diag) {
    double* q = Ps + (size_t)I * 4 * npad + i;
    q[0] = axi - sax[tid];
    q[(size_t)npad] = ayi - say[tid];
    q[2 * (size_t)npad] = azi - saz[tid];
    q[3 * (size_t)npad] = ui;
  } else {
    double* q = Ps + (size_t)J * 4 * npad + i;
    q[0] = axi;
    q[(size_t)npad] = ayi;
    q[2 * (size_t)npad] = azi;
    q[3 * (size_t)npad] = ui;
    double* qj = Ps + (size_t)I * 4 * npad + j0 + tid;
    qj[0] = -sax[tid];
    qj[(size_t)npad] = -say[tid];
    qj[2 * (size_t)npad] = -saz[tid];
    qj[3 * (size_t)npad] = 0.0;
  }
}

struct NearAcc {
  double ax = 0.0, ay = 0.0, az = 0.0, u = 0.0;
  // body p, partner q at separation d = r_q - r_p from edge-vector sums
  __device__ __forceinline__ void add(int p, int q, double dx, double dy, double dz, double mq) {
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double rinv = rsqrt_fp64(r2);
    const double s = mq * ((rinv * rinv) * rinv);
    ax = fma(s, dx, ax);
    ay = fma(s, dy, ay);
    az = fma(s, dz, az);
    if (q > p) u = fma(mq, rinv, u);
  }
};

// Sum of the tile partials plus the near pairs of Sec. 3.4 (N_d <= 2: parent, child,
// grandparent, grandchild, sibling), times G. Writes a (3 planes) and per-block sums of
// m_p * u_p, where u_p sums m_q / r_pq over partners q > p (each unordered pair once).
__global__ void __launch_bounds__(kBlock)
k_pair_finish(int n, int npad, int NT, int slot_lo, int n_d, double G, const double* __restrict__ m,
              const int* __restrict__ parent, const int* __restrict__ gp, const int* __restrict__ child_off,
              const int* __restrict__ child_idx, const double* __restrict__ sX, const double* __restrict__ P,
              double* __restrict__ sa, double* __restrict__ Ublk, int nblk) {
  __shared__ double scratch[32];
  const int slot = slot_lo + blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double um = 0.0;
  if (p < n) {
    const double* Ps = P + (size_t)slot * NT * 4 * npad + p;
    NearAcc acc;
    for (int s = 0; s < NT; ++s) {
      const double* q = Ps + (size_t)s * 4 * npad;
      acc.ax += q[0];
      acc.ay += q[(size_t)npad];
      acc.az += q[2 * (size_t)npad];
      acc.u += q[3 * (size_t)npad];
    }
    if (n_d >= 1) {
      const double* Xx = sX + (size_t)slot * 3 * npad;
      const double* Xy = Xx + npad;
      const double* Xz = Xy + npad;
      const int pp = parent[p];
      const double xp = Xx[p], yp = Xy[p], zp = Xz[p];
      if (pp >= 0) acc.add(p, pp, -xp, -yp, -zp, m[pp]);
      const int c0 = child_off[p], c1 = child_off[p + 1];
      for (int a = c0; a < c1; ++a) {
        const int c = child_idx[a];
        acc.add(p, c, Xx[c], Xy[c], Xz[c], m[c]);
      }
      if (n_d >= 2) {
        const int g = gp[p];
        if (g >= 0) acc.add(p, g, -(xp + Xx[pp]), -(yp + Xy[pp]), -(zp + Xz[pp]), m[g]);
        for (int a = c0; a < c1; ++a) {
          const int c = child_idx[a];
          const double xc = Xx[c], yc = Xy[c], zc = Xz[c];
          for (int b = child_off[c]; b < child_off[c + 1]; ++b) {
            const int gc = child_idx[b];
            acc.add(p, gc, Xx[gc] + xc, Xy[gc] + yc, Xz[gc] + zc, m[gc]);
          }
        }
        if (pp >= 0) {
          for (int b = child_off[pp]; b < child_off[pp + 1]; ++b) {
            const int sib = child_idx[b];
            if (sib != p) acc.add(p, sib, Xx[sib] - xp, Xy[sib] - yp, Xz[sib] - zp, m[sib]);
          }
        }
      }
    }
    double* a = sa + (size_t)slot * 3 * npad + p;
    a[0] = G * acc.ax;
    a[(size_t)npad] = G * acc.ay;
    a[2 * (size_t)npad] = G * acc.az;
    um = m[p] * acc.u;
  }
  const double s = block_sum(um, scratch);
  if (threadIdx.x == 0) Ublk[(size_t)slot * nblk + blockIdx.x] = G * s;
}

template <int W>
cudaError_t run_tiles(mstar_ctx* c, int slot_lo, int nsl, int n_d) {
  dim3 grid(c->ntp, nsl);
  if (c->prof) prof_begin(c);
  k_pair_tiles<W><<<grid, 32 * W, 0, c->stream>>>(c->n, c->npad, c->NT, slot_lo, n_d, c->d.m, c->d.parent,
                                                  c->d.gp, c->d.sr, c->d.P);
  MSTAR_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->prof) prof_end(c, nsl);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_forces(mstar_ctx* c, int slot_lo, int slot_hi, int n_d) {
  const int nsl = slot_hi - slot_lo;
  if (nsl <= 0) return cudaSuccess;
  cudaError_t e;
  switch (c->W) {
    case 1: e = run_tiles<1>(c, slot_lo, nsl, n_d); break;
    case 2: e = run_tiles<2>(c, slot_lo, nsl, n_d); break;
    default: e = run_tiles<4>(c, slot_lo, nsl, n_d); break;
  }
  if (e != cudaSuccess) return e;
  dim3 grid(c->nblk, nsl);
  k_pair_finish<<<grid, kBlock, 0, c->stream>>>(c->n, c->npad, c->NT, slot_lo, n_d, c->p.G, c->d.m, c->d.parent,
                                                c->d.gp, c->d.child_off, c->d.child_idx, c->d.sX, c->d.P,
                                                c->d.sa, c->d.Ublk, c->nblk);
  MSTAR_LAUNCHED(c);
  c->force_evals += nsl;
  return cudaGetLastError();
}

}  // namespace mstar
