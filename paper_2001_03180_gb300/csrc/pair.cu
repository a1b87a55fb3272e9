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
// Every body thus receives exactly one write per slot, and the NT slots are added in a
// fixed order.
//
// Reduction on chip: every tile receives exactly NT contributions (CTAs (t, J >= t) and
// (I < t, t)). After writing its partials, a CTA counts itself in for its tiles; the CTA
// that brings a tile's count to NT adds that tile's NT slots (ascending) while they are
// still in L2, writes the 4 sums per body, resets the count and discards the partials'
// L2 lines, so that they are never written back to DRAM. Nothing waits: the last CTA to
// arrive finds everything it needs already written. The division slots of a launch run one
// after another (blockIdx.y), so a slot's last tiles are summed while later slots' CTAs
// compute. The trailing slots - those whose CTAs can still be resident together at the end
// of the launch, or all whose partials fit in L2 anyway - are left to the finishing pass,
// which reads their partials from L2 right after, so that no reduction trails the launch.
#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

// Sum of tile t's NT partial slots (ascending s) for its T bodies, one per thread of the
// first T of the CTA's NTH threads, into Pt (4 planes); then its count is reset and the
// partials' lines dropped from L2. Every thread of the CTA calls it (it holds a barrier).
template <int T, int NTH = T>
__device__ __forceinline__ void finish_tile(int t, int npad, int NT, const double* Ps, double* Pt, int* cnt) {
  const int tid = threadIdx.x;
  if (NTH == T || tid < T) {
    const double* q = Ps + (size_t)t * T + tid;
    double ax = 0.0, ay = 0.0, az = 0.0, u = 0.0;
    // L2 loads (the slots were written by other CTAs after this SM's L1 could have seen
    // them), four slots at a time ahead of their additions, which keep the ascending order
    int s = 0;
    for (; s + 4 <= NT; s += 4) {
      double b[4][4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double* qs = q + (size_t)(s + k) * 4 * npad;
        b[k][0] = __ldcg(qs);
        b[k][1] = __ldcg(qs + npad);
        b[k][2] = __ldcg(qs + 2 * (size_t)npad);
        b[k][3] = __ldcg(qs + 3 * (size_t)npad);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ax += b[k][0];
        ay += b[k][1];
        az += b[k][2];
        u += b[k][3];
      }
    }
    for (; s < NT; ++s) {
      const double* qs = q + (size_t)s * 4 * npad;
      ax += __ldcg(qs);
      ay += __ldcg(qs + npad);
      az += __ldcg(qs + 2 * (size_t)npad);
      u += __ldcg(qs + 3 * (size_t)npad);
    }
    double* o = Pt + (size_t)t * T + tid;
    o[0] = ax;
    o[(size_t)npad] = ay;
    o[2 * (size_t)npad] = az;
    o[3 * (size_t)npad] = u;
  }
  __syncthreads();  // every thread has read the tile's slots
  // the slots of tile t: NT x 4 runs of T doubles, each starting on a 256-byte boundary
  // (npad and t T are multiples of T >= 32); T / 16 lines of 128 bytes per run
  constexpr int kLinesPerRun = T / 16;
  for (int l = tid; l < NT * 4 * kLinesPerRun; l += NTH) {
    const int run = l / kLinesPerRun, line = l - run * kLinesPerRun;
    const double* a = Ps + (size_t)run * npad + (size_t)t * T + 16 * line;
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
  }
  if (tid == 0) cnt[t] = 0;
}

// The near pairs of Sec. 3.4 (N_d <= 2) of the CTA's bodies, one per thread, into Nb (4 planes:
// ax, ay, az and the sum of m/r over partners of higher index). They depend on the slot's edge
// vectors alone, so the pair launches take them in CTAs of their own ahead of the tile pairs,
// and the finishing pass adds them to the tile sums instead of walking the near partners itself.
__device__ __forceinline__ void near_block(int n, int npad, int slot, int n_d, const double* __restrict__ m,
                                           const int* __restrict__ parent, const int* __restrict__ gp,
                                           const int* __restrict__ child_off, const int* __restrict__ child_idx,
                                           const double* __restrict__ sX, double* __restrict__ Nb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  NearAcc acc;
  near_terms(p, npad, n_d, sX + (size_t)slot * 3 * npad, m, parent, gp, child_off, child_idx, acc);
  double* o = Nb + (size_t)slot * 4 * npad + p;
  o[0] = acc.ax;
  o[(size_t)npad] = acc.ay;
  o[2 * (size_t)npad] = acc.az;
  o[3 * (size_t)npad] = acc.u;
}

template <int W>
__global__ void __launch_bounds__(32 * W)
k_pair_tiles(int n, int npad, int NT, int slot_lo, int n_d, const double* __restrict__ m,
             const int* __restrict__ parent, const int* __restrict__ gp, const double* __restrict__ sr,
             double* __restrict__ P, double* __restrict__ Pt, int* __restrict__ tcnt, int keep_from,
             const int* __restrict__ child_off, const int* __restrict__ child_idx, const double* __restrict__ sX,
             double* __restrict__ Nb, int nnear) {
  constexpr int T = 32 * W;
  __shared__ double sx[T], sy[T], sz[T], sax[T], say[T], saz[T];
  __shared__ unsigned long long smm[T];
  __shared__ int sp[T], sg[T], sme[T];

  const int slot = slot_lo + blockIdx.y;
  if ((int)blockIdx.x < nnear) {
    near_block(n, npad, slot, n_d, m, parent, gp, child_off, child_idx, sX, Nb);
    return;
  }
  int I, J;
  tile_pair((int)blockIdx.x - nnear, NT, I, J);
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

  // count this CTA in for tiles I and J; the last of a tile's NT contributors sums it (the
  // trailing slots from keep_from on are summed by the finishing pass)
  if ((int)blockIdx.y >= keep_from) return;
  __shared__ int s_last[2];
  __threadfence();  // this CTA's partials are visible device-wide before it is counted
  __syncthreads();
  if (tid == 0) {
    int* cnt = tcnt + (size_t)slot * NT;
    s_last[0] = atomicAdd(&cnt[I], 1) == NT - 1;
    s_last[1] = diag ? 0 : atomicAdd(&cnt[J], 1) == NT - 1;
    __threadfence();  // the counts seen before the other contributors' partials are read
  }
  __syncthreads();
  if (s_last[0] | s_last[1]) {
    int* cnt = tcnt + (size_t)slot * NT;
    double* Pts = Pt + (size_t)slot * 4 * npad;
    if (s_last[0]) finish_tile<T>(I, npad, NT, Ps, Pts, cnt);
    if (s_last[1]) {
      __syncthreads();
      finish_tile<T>(J, npad, NT, Ps, Pts, cnt);
    }
  }
}

// The pair loop of small systems: the tiling and per-pair arithmetic of k_pair_tiles<1>
// (32-body tiles), with the 32 partner steps of a tile pair split over S warps (S divides
// 16). Warp w takes steps [32 w / S, 32 (w + 1) / S) of an off-diagonal pair and
// [1 + 16 w / S, 1 + 16 (w + 1) / S) of a diagonal one, keeping its own i-side sums and its
// own copy of the partner sums; the S copies are added in warp order at the end. At N ~ 10^2
// a tile pair's 32 dependent steps in one warp bind the launch; S warps shorten them S-fold.
template <int S>
__global__ void __launch_bounds__(32 * S)
k_pair_tiles_ks(int n, int npad, int NT, int slot_lo, int n_d, const double* __restrict__ m,
                const int* __restrict__ parent, const int* __restrict__ gp, const double* __restrict__ sr,
                double* __restrict__ P, double* __restrict__ Pt, int* __restrict__ tcnt, int keep_from,
                const int* __restrict__ child_off, const int* __restrict__ child_idx,
                const double* __restrict__ sX, double* __restrict__ Nb, int nnear) {
  constexpr int T = 32;
  __shared__ double sx[T], sy[T], sz[T];
  __shared__ double sax[S][T], say[S][T], saz[S][T];     // partner sums, one copy per warp
  __shared__ double rax[S][T], ray[S][T], raz[S][T], rau[S][T];  // i-side sums per warp
  __shared__ unsigned long long smm[T];
  __shared__ int sp[T], sg[T], sme[T];
  const int slot = slot_lo + blockIdx.y;
  if ((int)blockIdx.x < nnear) {
    near_block(n, npad, slot, n_d, m, parent, gp, child_off, child_idx, sX, Nb);
    return;
  }
  int I, J;
  tile_pair((int)blockIdx.x - nnear, NT, I, J);
  const double* rx = sr + (size_t)slot * 3 * npad;
  const double* ry = rx + npad;
  const double* rz = ry + npad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = J * T;
  if (warp == 0) {
    sx[lane] = rx[j0 + lane];
    sy[lane] = ry[j0 + lane];
    sz[lane] = rz[j0 + lane];
    const MassSplit ms = mass_split(m[j0 + lane]);
    smm[lane] = ms.m;
    sme[lane] = ms.e;
    sp[lane] = parent[j0 + lane];
    sg[lane] = gp[j0 + lane];
  }
  sax[warp][lane] = 0.0;
  say[warp][lane] = 0.0;
  saz[warp][lane] = 0.0;
  const int i = I * T + lane;
  const double xi = rx[i], yi = ry[i], zi = rz[i];
  const MassSplit msi = mass_split(m[i]);
  const int pi = parent[i], gpi = gp[i];
  const bool i_pad = i >= n;
  const bool nd1 = n_d >= 1, nd2 = n_d >= 2;
  double axi = 0.0, ayi = 0.0, azi = 0.0;
  UAcc uacc;
  bool ubad = false;
  const bool diag = (I == J);
  const int kbeg = diag ? 1 + 16 * warp / S : 32 * warp / S;
  const int kend = diag ? 1 + 16 * (warp + 1) / S : 32 * (warp + 1) / S;
  __syncthreads();
#pragma unroll 4
  for (int k = kbeg; k < kend; ++k) {
    const int jl = (lane + k) & 31;
    const int j = j0 + jl;
    const double xj = sx[jl], yj = sy[jl], zj = sz[jl];
    const int pj = sp[jl], gj = sg[jl];
    bool masked = i_pad | (j >= n) | (diag & (k == 16) & (lane >= 16));
    masked |= nd1 & ((pi == j) | (pj == i));
    masked |= nd2 & ((gpi == j) | (gj == i) | (pi == pj));
    double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    asm volatile("" : "+d"(dx), "+d"(dy), "+d"(dz));
    unsigned long long Rn;
    int eR;
    double sj, si;
    const unsigned long long mjm = smm[jl];
    const int mje = sme[jl];
    pair_scalars_core(dx, dy, dz, MassSplit{mjm, mje}, msi, Rn, eR, sj, si);
    sj = __longlong_as_double(masked ? 0ll : __double_as_longlong(sj));
    si = __longlong_as_double(masked ? 0ll : __double_as_longlong(si));
    ubad |= !masked && Rn == 0ull;
    uacc.add(masked ? 0ull : __umul64hi(mjm, Rn), masked ? uacc.L : mje + eR + 64);
    axi = fma(sj, dx, axi);
    ayi = fma(sj, dy, ayi);
    azi = fma(sj, dz, azi);
    sax[warp][jl] = fma(si, dx, sax[warp][jl]);
    say[warp][jl] = fma(si, dy, say[warp][jl]);
    saz[warp][jl] = fma(si, dz, saz[warp][jl]);
    __syncwarp();
  }
  rax[warp][lane] = axi;
  ray[warp][lane] = ayi;
  raz[warp][lane] = azi;
  rau[warp][lane] = ubad ? __longlong_as_double(0x7ff8000000000000LL) : uacc.value();
  __syncthreads();
  double* Ps = P + (size_t)slot * NT * 4 * npad;
  if (warp == 0) {
    double ax = rax[0][lane], ay = ray[0][lane], az = raz[0][lane], u = rau[0][lane];
    double jx = sax[0][lane], jy = say[0][lane], jz = saz[0][lane];
#pragma unroll
    for (int w = 1; w < S; ++w) {
      ax += rax[w][lane];
      ay += ray[w][lane];
      az += raz[w][lane];
      u += rau[w][lane];
      jx += sax[w][lane];
      jy += say[w][lane];
      jz += saz[w][lane];
    }
    if (diag) {
      double* q = Ps + (size_t)I * 4 * npad + i;
      q[0] = ax - jx;
      q[(size_t)npad] = ay - jy;
      q[2 * (size_t)npad] = az - jz;
      q[3 * (size_t)npad] = u;
    } else {
      double* q = Ps + (size_t)J * 4 * npad + i;
      q[0] = ax;
      q[(size_t)npad] = ay;
      q[2 * (size_t)npad] = az;
      q[3 * (size_t)npad] = u;
      double* qj = Ps + (size_t)I * 4 * npad + j0 + lane;
      qj[0] = -jx;
      qj[(size_t)npad] = -jy;
      qj[2 * (size_t)npad] = -jz;
      qj[3 * (size_t)npad] = 0.0;
    }
  }
  // the on-chip reduction of k_pair_tiles (the first 32 threads sum a tile)
  if ((int)blockIdx.y >= keep_from) return;
  __shared__ int s_last[2];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    int* cnt = tcnt + (size_t)slot * NT;
    s_last[0] = atomicAdd(&cnt[I], 1) == NT - 1;
    s_last[1] = diag ? 0 : atomicAdd(&cnt[J], 1) == NT - 1;
    __threadfence();
  }
  __syncthreads();
  if (s_last[0] | s_last[1]) {
    int* cnt = tcnt + (size_t)slot * NT;
    double* Pts = Pt + (size_t)slot * 4 * npad;
    if (s_last[0]) finish_tile<T, 32 * S>(I, npad, NT, Ps, Pts, cnt);
    if (s_last[1]) {
      __syncthreads();
      finish_tile<T, 32 * S>(J, npad, NT, Ps, Pts, cnt);
    }
  }
}

// The tile sums plus the near pairs of Sec. 3.4 (N_d <= 2: parent, child, grandparent,
// grandchild, sibling), times G. Writes a (3 planes) and per-block sums of m_p * u_p, where
// u_p sums m_q / r_pq over partners q > p (each unordered pair once). The trailing slots
// (blockIdx.y >= keep_from) sum their NT partial slots here (ascending, as the tile kernel does
// for the other slots).
//
// A CTA takes kBlock bodies with kFinishPlanes threads each: thread (c, b) sums plane c (ax, ay,
// az, u) of body b over the slots, so the four sums run side by side (each in the same order
// as one thread summing all four), and the first kBlock threads finish the bodies. Where the
// pass runs beside pair launches of other divisions, which keep the FP64 pipe busy, its share
// of the pipe grows with its warps.
constexpr int kFinishPlanes = 4;
__global__ void __launch_bounds__(kBlock * kFinishPlanes)
k_pair_finish(int n, int npad, int NT, int slot_lo, int n_d, double G, const double* __restrict__ m,
              const double* __restrict__ Nb, const double* __restrict__ P, const double* __restrict__ Pt,
              double* __restrict__ sa, double* __restrict__ Ublk, int nblk, int keep_from) {
  __shared__ double scratch[32];
  __shared__ double splane[kFinishPlanes][kBlock];
  const int slot = slot_lo + blockIdx.y;
  const int plane = threadIdx.x / kBlock, b = threadIdx.x - plane * kBlock;
  const int p = blockIdx.x * kBlock + b;
  const bool deferred = (int)blockIdx.y >= keep_from;
  if (deferred) {
    double acc = 0.0;
    if (p < n) {
      const double* q = P + (size_t)slot * NT * 4 * npad + (size_t)plane * npad + p;
      int s = 0;
      for (; s + 4 <= NT; s += 4) {
        double t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = q[(size_t)(s + k) * 4 * npad];
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += t[k];
      }
      for (; s < NT; ++s) acc += q[(size_t)s * 4 * npad];
    }
    splane[plane][b] = acc;
    // the block's bodies' partials are read: drop their L2 lines, so that they are not
    // written back to DRAM when later launches' partials evict them (every slot is written
    // again before it is next read). NT x 4 runs of kBlock doubles, each starting on a
    // 512-byte boundary; a line is dropped only where it lies below npad.
    __syncthreads();
    constexpr int kLinesPerRun = kBlock / 16;
    const int b0 = blockIdx.x * kBlock;
    const double* base = P + (size_t)slot * NT * 4 * npad + b0;
    for (int l = threadIdx.x; l < NT * 4 * kLinesPerRun; l += blockDim.x) {
      const int run = l / kLinesPerRun, line = l - run * kLinesPerRun;
      if (b0 + 16 * line < npad) {
        const double* a = base + (size_t)run * npad + 16 * line;
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
      }
    }
  }
  double um = 0.0;
  if (plane == 0 && p < n) {
    NearAcc acc;
    if (deferred) {
      acc.ax = splane[0][b];
      acc.ay = splane[1][b];
      acc.az = splane[2][b];
      acc.u = splane[3][b];
    } else {
      const double* q = Pt + (size_t)slot * 4 * npad + p;
      acc.ax = q[0];
      acc.ay = q[(size_t)npad];
      acc.az = q[2 * (size_t)npad];
      acc.u = q[3 * (size_t)npad];
    }
    if (n_d >= 1) {  // the near pairs, from the pair launch's near CTAs
      const double* nb = Nb + (size_t)slot * 4 * npad + p;
      acc.ax += nb[0];
      acc.ay += nb[(size_t)npad];
      acc.az += nb[2 * (size_t)npad];
      acc.u += nb[3 * (size_t)npad];
    }
    double* a = sa + (size_t)slot * 3 * npad + p;
    a[0] = G * acc.ax;
    a[(size_t)npad] = G * acc.ay;
    a[2 * (size_t)npad] = G * acc.az;
    um = m[p] * acc.u;
  }
  // the other planes' threads add zeros after the first kBlock threads' sum, so the block sum
  // is that of the kBlock bodies alone
  const double s = block_sum(um, scratch);
  if (threadIdx.x == 0) Ublk[(size_t)slot * nblk + blockIdx.x] = G * s;
}

// Partial bytes that the trailing slots of a launch may leave in L2 for the finishing pass.
constexpr double kDeferL2Bytes = 48.0 * 1024 * 1024;

// Trailing slots of a launch left to the finishing pass: the slots whose CTAs can be resident
// together at the end of the launch (plus one), and at least as many as fit in the L2 budget.
template <typename K>
int defer_slots(const mstar_ctx* c, K kernel, int threads) {
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    return 1 << 20;  // unknown: every slot is summed by the finishing pass
  }
  const long long resident = (long long)per_sm * sms;
  const int d_wave = (int)((resident + c->ntp - 1) / c->ntp) + 1;
  const double slot_bytes = (double)c->NT * 4.0 * c->npad * sizeof(double);
  const int d_l2 = (int)(kDeferL2Bytes / slot_bytes);
  return d_wave > d_l2 ? d_wave : d_l2;
}

template <int W, int S>
cudaError_t run_tiles(mstar_ctx* c, int slot_lo, int nsl, int n_d, int keep_from) {
  constexpr int threads = S == 1 ? 32 * W : 32 * S;
  const int nnear = n_d >= 1 ? (c->n + threads - 1) / threads : 0;  // the near CTAs come first
  dim3 grid(nnear + c->ntp, nsl);
  if (c->prof) prof_begin(c);
  if constexpr (S == 1)
    k_pair_tiles<W><<<grid, 32 * W, 0, c->stream>>>(c->n, c->npad, c->NT, slot_lo, n_d, c->d.m, c->d.parent,
                                                    c->d.gp, c->d.sr, c->d.P, c->d.Pt, c->d.tcnt, keep_from,
                                                    c->d.child_off, c->d.child_idx, c->d.sX, c->d.Nb, nnear);
  else
    k_pair_tiles_ks<S><<<grid, 32 * S, 0, c->stream>>>(c->n, c->npad, c->NT, slot_lo, n_d, c->d.m, c->d.parent,
                                                       c->d.gp, c->d.sr, c->d.P, c->d.Pt, c->d.tcnt, keep_from,
                                                       c->d.child_off, c->d.child_idx, c->d.sX, c->d.Nb, nnear);
  MSTAR_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->prof) prof_end(c, nsl);
  return cudaSuccess;
}

}  // namespace

// The pair launches run beside the small kernels of other divisions (a stream per division),
// several of which take tens of KB of shared memory (the staged rebuild). An SM runs CTAs of
// kernels together only under one split of its on-chip memory between L1 and shared memory, so
// every kernel of an attempt asks for the largest shared-memory share: the small kernels' CTAs
// can then start on SMs that hold pair CTAs (GBS steps at N = 2050 2.4 % faster). A hint: a
// device that ignores it loses nothing else.
void prefer_shared_pair_kernels() {
  cudaFuncSetAttribute(k_pair_tiles<1>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pair_tiles<2>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pair_tiles<4>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pair_tiles_ks<2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pair_tiles_ks<4>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pair_tiles_ks<8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pair_finish, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaGetLastError();
}

cudaError_t launch_forces(mstar_ctx* c, int slot_lo, int slot_hi, int n_d) {
  const int nsl = slot_hi - slot_lo;
  if (nsl <= 0) return cudaSuccess;
  if (c->pair_defer < 0) {
    if (c->W == 1) {
      switch (c->S) {
        case 2: c->pair_defer = defer_slots(c, k_pair_tiles_ks<2>, 64); break;
        case 4: c->pair_defer = defer_slots(c, k_pair_tiles_ks<4>, 128); break;
        case 8: c->pair_defer = defer_slots(c, k_pair_tiles_ks<8>, 256); break;
        default: c->pair_defer = defer_slots(c, k_pair_tiles<1>, 32); break;
      }
    } else {
      c->pair_defer = c->W == 2 ? defer_slots(c, k_pair_tiles<2>, 64) : defer_slots(c, k_pair_tiles<4>, 128);
    }
  }
  const int keep_from = nsl - c->pair_defer;  // slots below this index are summed on chip
  cudaError_t e;
  if (c->W == 1) {
    switch (c->S) {
      case 2: e = run_tiles<1, 2>(c, slot_lo, nsl, n_d, keep_from); break;
      case 4: e = run_tiles<1, 4>(c, slot_lo, nsl, n_d, keep_from); break;
      case 8: e = run_tiles<1, 8>(c, slot_lo, nsl, n_d, keep_from); break;
      default: e = run_tiles<1, 1>(c, slot_lo, nsl, n_d, keep_from); break;
    }
  } else {
    e = c->W == 2 ? run_tiles<2, 1>(c, slot_lo, nsl, n_d, keep_from) : run_tiles<4, 1>(c, slot_lo, nsl, n_d, keep_from);
  }
  if (e != cudaSuccess) return e;
  dim3 grid(c->nblk, nsl);
  k_pair_finish<<<grid, kBlock * kFinishPlanes, 0, c->stream>>>(c->n, c->npad, c->NT, slot_lo, n_d, c->p.G,
                                                                c->d.m, c->d.Nb, c->d.P, c->d.Pt, c->d.sa,
                                                                c->d.Ublk, c->nblk, keep_from);
  MSTAR_LAUNCHED(c);
  c->force_evals += nsl;
  return cudaGetLastError();
}

}  // namespace mstar
