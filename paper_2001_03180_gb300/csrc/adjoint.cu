// Reverse-mode adjoint of a fixed-step run: gradients of a loss of the final state
// (positions, velocities and energy) with respect to the masses, positions and velocities
// given to mstar_init.
//
// The forward is the ordinary GBS step (MST, edge coordinates, k_fix leapfrog divisions,
// Aitken-Neville extrapolation; Sec. 2-4) with a fixed fictitious step H and every attempt
// accepted. In real arithmetic the MST-coordinate step equals the Cartesian LogH leapfrog:
// the edge vectors are a linear change of variables, their near-pair sums equal r_j - r_i,
// and the rebuild is the inverse map plus a shift that is the identity on the
// centre-of-mass frame. The reverse sweep therefore applies the transposed Jacobians of
// the Cartesian substeps of Sec. 2.1-2.2,
//   D(h): f = h / (T + B),  r' = r + f v,        T = sum m |v|^2 / 2
//   K(h): g = h / U,        v' = v + g a(r; m),  U = G sum_{i<j} m_i m_j / |r_ij|
// around the trajectory that the forward computed (recorded by the attempt), and of the
// extrapolation, which is linear: the result is sum_k c_k S_k with the Lagrange weights
// c_k of the nodes (1/n_k)^2 at 0. The MST topology is piecewise constant and has no
// derivative. B = U0 - T0 of the initial state and the initial centre-of-mass shift
// carry their own terms.
//
// Reverse recurrences of one division (adjoints lr, lv of r, v; lm of m; lB of B):
//   D:  lf = lr . v;  lv += f lr;  lT = -lf h / (T + B)^2;  lB += lT;
//       lv += lT m v;  lm += lT |v|^2 / 2
//   K:  lg = lv . a;  lU = -lg h / U^2;  la = g lv;
//       lr += J_a^T la + lU m a   (grad_r U = m a),   lm += (da/dm)^T la + lU phi
// with (J_a^T la)_i = G sum_j M_ij (m_i la_j - m_j la_i), M_ij = I/r^3 - 3 d d^T / r^5,
// ((da/dm)^T la)_i = -G sum_j la_j . d_ij / r^3 and phi_i = G sum_j m_j / r_ij.
//
// Memory: (r, v) every `checkpoint_every` steps; the steps of one segment are recomputed
// from its checkpoint with their trajectories recorded, then swept backwards.
#include <cmath>
#include <new>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

constexpr int kAdjI = 32;    // bodies i per CTA of the VJP pair loop
constexpr int kAdjZMax = 16; // partner ranges (grid z): ceil(n / 32) up to 16, each a multiple of kAdjI

// Partner range length for n bodies: at most kAdjZMax ranges of at least kAdjI partners.
int adj_jchunk(int n) {
  int nz = (n + kAdjI - 1) / kAdjI;
  if (nz > kAdjZMax) nz = kAdjZMax;
  const int per = (n + nz - 1) / nz;
  return (per + kAdjI - 1) / kAdjI * kAdjI;
}

struct Weights {
  double c[kMaxKfix];
};

// lr_s = c_s lrf, lv_s = c_s lvf for every division slot s.
__global__ void __launch_bounds__(kBlock)
k_adj_init(int npad, Weights cw, const double* __restrict__ lrf, const double* __restrict__ lvf,
           double* __restrict__ lr, double* __restrict__ lv) {
  const int s = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  const size_t st = (size_t)3 * npad;
  for (int c = 0; c < 3; ++c) {
    const size_t o = (size_t)c * npad + i;
    lr[s * st + o] = cw.c[s] * lrf[o];
    lv[s * st + o] = cw.c[s] * lvf[o];
  }
}

// Per-block partial sums of X_s . Y_s over the bodies, for slots slot_lo + blockIdx.y.
__global__ void __launch_bounds__(kBlock)
k_adj_dot(int n, int npad, int slot_lo, const double* __restrict__ X, size_t xs, const double* __restrict__ Y,
          size_t ys, double* __restrict__ part, int nblk) {
  __shared__ double scratch[32];
  const int s = slot_lo + blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    const double* x = X + s * xs;
    const double* y = Y + s * ys;
    for (int c = 0; c < 3; ++c) acc += x[(size_t)c * npad + i] * y[(size_t)c * npad + i];
  }
  acc = block_sum(acc, scratch);
  if (threadIdx.x == 0) part[(size_t)s * nblk + blockIdx.x] = acc;
}

// Transposed drift of level tau (tau = 0: the first half drift) for each active slot,
// then per-block partials of lv . a for the transposed kick of the same level (A != null).
__global__ void __launch_bounds__(kBlock)
k_adj_drift(int n, int npad, int slot_lo, int tau, double H, double B, const double* __restrict__ m,
            const double* __restrict__ lr, double* __restrict__ lv, const double* __restrict__ V, size_t vs,
            const double* __restrict__ SC, const double* __restrict__ pf, int nblk, double* __restrict__ lm,
            double* __restrict__ lB, const double* __restrict__ A, double* __restrict__ pg) {
  __shared__ double s_lf;
  __shared__ double scratch[32];
  const int s = slot_lo + blockIdx.y;
  sum_partials(pf + (size_t)s * nblk, nblk, 1, &s_lf);
  const double T = SC[s * kScal + SC_T_KIN];
  const int nk = 2 * (s + 1);
  const double delta = H / (double)nk;
  const double h = (tau == 0 || tau == nk) ? 0.5 * delta : delta;
  const double den = T + B;
  const double f = h / den;
  const double lT = -s_lf * h / (den * den);
  const size_t st = (size_t)3 * npad;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    const double* v = V + s * vs;
    const double* r_ = lr + s * st;
    double* l = lv + s * st;
    double v2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * npad + i;
      const double vc = v[o];
      const double nl = l[o] + f * r_[o] + lT * m[i] * vc;
      l[o] = nl;
      v2 += vc * vc;
      if (A) acc += nl * A[s * st + o];
    }
    lm[(size_t)s * npad + i] += lT * 0.5 * v2;
  }
  if (A) {
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) pg[(size_t)s * nblk + blockIdx.x] = acc;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) lB[s] += lT;
}

// VJP pair loop. For body i of slot s against partners j in [z jchunk, (z+1) jchunk):
//   mu_i  = G g sum_j [ w / r^3 - 3 d (d . w) / r^5 ],  w = m_i L_j - m_j L_i
//   nu_i  = -G g sum_j (L_j . d) / r^3
//   phi_i = G sum_j m_j / r,   a_i = G sum_j m_j d / r^3,   d = r_j - r_i
// with L the slot's velocity adjoint and g = delta / U of the slot's kick (L == null: mu and
// nu are skipped). Partial results per z; the consumer adds the nz partials in order.
__global__ void __launch_bounds__(kAdjI)
k_adj_pair(int n, int npad, int slot_lo, double G, double H, const double* __restrict__ m,
           const double* __restrict__ Rb, size_t rs, const double* __restrict__ Lb, size_t ls,
           const double* __restrict__ SC, int nz, int jchunk, double* __restrict__ mu, double* __restrict__ nu,
           double* __restrict__ phi, double* __restrict__ aout) {
  __shared__ double sx[kAdjI], sy[kAdjI], sz[kAdjI], sm[kAdjI], slx[kAdjI], sly[kAdjI], slz[kAdjI];
  const int s = slot_lo + blockIdx.y;
  const int z = blockIdx.z;
  const double* R = Rb + s * rs;
  const double* L = Lb ? Lb + s * ls : nullptr;
  const double g = SC ? (H / (double)(2 * (s + 1))) / SC[s * kScal + SC_U] : 1.0;
  const int i = blockIdx.x * kAdjI + threadIdx.x;
  const bool live = i < n;
  const double xi = live ? R[i] : 0.0, yi = live ? R[npad + i] : 0.0, zi = live ? R[2 * (size_t)npad + i] : 0.0;
  const double mi = live ? m[i] : 0.0;
  const double lxi = (live && L) ? L[i] : 0.0, lyi = (live && L) ? L[npad + i] : 0.0,
               lzi = (live && L) ? L[2 * (size_t)npad + i] : 0.0;
  double mux = 0.0, muy = 0.0, muz = 0.0, nuv = 0.0, ph = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
  const int jend = min(n, (z + 1) * jchunk);
  for (int j0 = z * jchunk; j0 < jend; j0 += kAdjI) {
    const int j = j0 + threadIdx.x;
    const bool jl = j < jend;
    sx[threadIdx.x] = jl ? R[j] : 0.0;
    sy[threadIdx.x] = jl ? R[npad + j] : 0.0;
    sz[threadIdx.x] = jl ? R[2 * (size_t)npad + j] : 0.0;
    sm[threadIdx.x] = jl ? m[j] : 0.0;
    slx[threadIdx.x] = (jl && L) ? L[j] : 0.0;
    sly[threadIdx.x] = (jl && L) ? L[npad + j] : 0.0;
    slz[threadIdx.x] = (jl && L) ? L[2 * (size_t)npad + j] : 0.0;
    __syncthreads();
    const int cnt = min(kAdjI, jend - j0);
    if (live) {
      for (int q = 0; q < cnt; ++q) {
        if (j0 + q == i) continue;
        const double dx = sx[q] - xi, dy = sy[q] - yi, dz = sz[q] - zi;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double ri = rsqrt_fp64(r2);
        const double ri2 = ri * ri, ri3 = ri2 * ri;
        const double mj = sm[q];
        ph = fma(mj, ri, ph);
        const double s3 = mj * ri3;
        ax = fma(s3, dx, ax);
        ay = fma(s3, dy, ay);
        az = fma(s3, dz, az);
        if (L) {
          const double wx = mi * slx[q] - mj * lxi, wy = mi * sly[q] - mj * lyi, wz = mi * slz[q] - mj * lzi;
          const double dw = fma(dz, wz, fma(dy, wy, dx * wx));
          const double t = 3.0 * dw * ri3 * ri2;
          mux += wx * ri3 - t * dx;
          muy += wy * ri3 - t * dy;
          muz += wz * ri3 - t * dz;
          nuv -= fma(slz[q], dz, fma(sly[q], dy, slx[q] * dx)) * ri3;
        }
      }
    }
    __syncthreads();
  }
  if (!live) return;
  const size_t zo = (size_t)s * nz + z;
  if (L) {
    const double gg = G * g;
    double* muo = mu + zo * 3 * npad;
    muo[i] = gg * mux;
    muo[npad + i] = gg * muy;
    muo[2 * (size_t)npad + i] = gg * muz;
    nu[zo * npad + i] = gg * nuv;
  }
  phi[zo * npad + i] = G * ph;
  if (aout) {
    double* ao = aout + zo * 3 * npad;
    ao[i] = G * ax;
    ao[npad + i] = G * ay;
    ao[2 * (size_t)npad + i] = G * az;
  }
}

// The same VJP sums over every unordered pair once, in the tiling of the forward pair loop:
// CTA (I, J), I <= J, holds tile I's bodies in registers and stages tile J's positions,
// masses, adjoints and accumulators in shared memory; at step k of a 32-wide sub-tile lane l
// pairs with partner (l + k) mod 32, so the lanes update distinct partner accumulators. For
// d = r_j - r_i and w = m_i L_j - m_j L_i the pair gives
//   u = w / r^3 - 3 d (d . w) / r^5:   mu_i += u, mu_j -= u   (M_ij = M_ji, w_ji = -w_ij)
//   nu_i -= (L_j . d) / r^3,  nu_j += (L_i . d) / r^3,  phi_i += m_j / r,  phi_j += m_i / r,
// about half the FP64 work of visiting each ordered pair. CTA (I, J) writes tile I's sums to
// partial slot J and tile J's to slot I (a diagonal CTA writes both into slot I), so each
// body receives one write per slot; the consumer adds the NT slots in order.
template <int W>
__global__ void __launch_bounds__(32 * W)
k_adj_pair_sym(int n, int npad, int NT, int slot_lo, double G, double H, const double* __restrict__ m,
               const double* __restrict__ Rb, size_t rs, const double* __restrict__ Lb, size_t ls,
               const double* __restrict__ SC, double* __restrict__ mu, double* __restrict__ nu,
               double* __restrict__ phi) {
  constexpr int T = 32 * W;
  __shared__ double sx[T], sy[T], sz[T], sm[T], slx[T], sly[T], slz[T];
  __shared__ double smx[T], smy[T], smz[T], snu[T], sph[T];
  const int s = slot_lo + blockIdx.y;
  int I, J;
  tile_pair(blockIdx.x, NT, I, J);
  const double* R = Rb + s * rs;
  const double* L = Lb + s * ls;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = J * T;
  sx[tid] = R[j0 + tid];
  sy[tid] = R[npad + j0 + tid];
  sz[tid] = R[2 * (size_t)npad + j0 + tid];
  sm[tid] = m[j0 + tid];
  slx[tid] = L[j0 + tid];
  sly[tid] = L[npad + j0 + tid];
  slz[tid] = L[2 * (size_t)npad + j0 + tid];
  smx[tid] = 0.0;
  smy[tid] = 0.0;
  smz[tid] = 0.0;
  snu[tid] = 0.0;
  sph[tid] = 0.0;
  const int i = I * T + tid;
  const double xi = R[i], yi = R[npad + i], zi = R[2 * (size_t)npad + i];
  const double mi = m[i];
  const double lxi = L[i], lyi = L[npad + i], lzi = L[2 * (size_t)npad + i];
  const bool i_pad = i >= n;
  const bool diag = (I == J);
  double mux = 0.0, muy = 0.0, muz = 0.0, nui = 0.0, phi_i = 0.0;
  __syncthreads();
#pragma unroll 1
  for (int sb = 0; sb < W; ++sb) {
    const int sub = (warp + sb) & (W - 1);
    const bool self = diag && sub == warp;
    if (!(diag && sub < warp)) {
      const int kbeg = self ? 1 : 0;
      const int kend = self ? 17 : 32;
#pragma unroll 2
      for (int k = kbeg; k < kend; ++k) {
        const int jl = sub * 32 + ((lane + k) & 31);
        const bool masked = i_pad | (j0 + jl >= n) | (self & (k == 16) & (lane >= 16));
        const double dx = sx[jl] - xi, dy = sy[jl] - yi, dz = sz[jl] - zi;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        double ri = rsqrt_fp64(r2);
        // masked pairs contribute nothing (an integer select on the bit pattern)
        ri = __longlong_as_double(masked ? 0ll : __double_as_longlong(ri));
        const double ri2 = ri * ri, ri3 = ri2 * ri, ri5 = ri3 * ri2;
        const double mj = sm[jl], ljx = slx[jl], ljy = sly[jl], ljz = slz[jl];
        const double wx = fma(mi, ljx, -mj * lxi), wy = fma(mi, ljy, -mj * lyi), wz = fma(mi, ljz, -mj * lzi);
        const double t = 3.0 * fma(dz, wz, fma(dy, wy, dx * wx)) * ri5;
        const double ux = fma(wx, ri3, -t * dx), uy = fma(wy, ri3, -t * dy), uz = fma(wz, ri3, -t * dz);
        mux += ux;
        muy += uy;
        muz += uz;
        smx[jl] -= ux;
        smy[jl] -= uy;
        smz[jl] -= uz;
        nui = fma(-fma(ljz, dz, fma(ljy, dy, ljx * dx)), ri3, nui);
        snu[jl] = fma(fma(lzi, dz, fma(lyi, dy, lxi * dx)), ri3, snu[jl]);
        phi_i = fma(mj, ri, phi_i);
        sph[jl] = fma(mi, ri, sph[jl]);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  const double gg = G * (H / (double)(2 * (s + 1))) / SC[s * kScal + SC_U];
  const size_t st = (size_t)3 * npad;
  auto put = [&](int slot_of, int body, double ax_, double ay_, double az_, double n_, double p_) {
    const size_t zo = (size_t)s * NT + slot_of;
    double* muo = mu + zo * st;
    muo[body] = gg * ax_;
    muo[npad + body] = gg * ay_;
    muo[2 * (size_t)npad + body] = gg * az_;
    nu[zo * npad + body] = gg * n_;
    phi[zo * npad + body] = G * p_;
  };
  if (diag) {
    put(I, i, mux + smx[tid], muy + smy[tid], muz + smz[tid], nui + snu[tid], phi_i + sph[tid]);
  } else {
    put(J, i, mux, muy, muz, nui, phi_i);
    put(I, j0 + tid, smx[tid], smy[tid], smz[tid], snu[tid], sph[tid]);
  }
}

// k_adj_pair_sym with 32-body tiles and a tile pair's 32 partner steps split over S warps (S
// divides 16), as in the forward pair loop of small systems: each warp keeps its own i-side
// sums and its own copy of the partner sums, added in warp order at the end.
template <int S>
__global__ void __launch_bounds__(32 * S)
k_adj_pair_sym_ks(int n, int npad, int NT, int slot_lo, double G, double H, const double* __restrict__ m,
                  const double* __restrict__ Rb, size_t rs, const double* __restrict__ Lb, size_t ls,
                  const double* __restrict__ SC, double* __restrict__ mu, double* __restrict__ nu,
                  double* __restrict__ phi) {
  constexpr int T = 32;
  __shared__ double sx[T], sy[T], sz[T], sm[T], slx[T], sly[T], slz[T];
  __shared__ double smx[S][T], smy[S][T], smz[S][T], snu[S][T], sph[S][T];  // partner sums per warp
  __shared__ double rmx[S][T], rmy[S][T], rmz[S][T], rnu[S][T], rph[S][T];  // i-side sums per warp
  const int s = slot_lo + blockIdx.y;
  int I, J;
  tile_pair(blockIdx.x, NT, I, J);
  const double* R = Rb + s * rs;
  const double* L = Lb + s * ls;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = J * T;
  if (warp == 0) {
    sx[lane] = R[j0 + lane];
    sy[lane] = R[npad + j0 + lane];
    sz[lane] = R[2 * (size_t)npad + j0 + lane];
    sm[lane] = m[j0 + lane];
    slx[lane] = L[j0 + lane];
    sly[lane] = L[npad + j0 + lane];
    slz[lane] = L[2 * (size_t)npad + j0 + lane];
  }
  smx[warp][lane] = 0.0;
  smy[warp][lane] = 0.0;
  smz[warp][lane] = 0.0;
  snu[warp][lane] = 0.0;
  sph[warp][lane] = 0.0;
  const int i = I * T + lane;
  const double xi = R[i], yi = R[npad + i], zi = R[2 * (size_t)npad + i];
  const double mi = m[i];
  const double lxi = L[i], lyi = L[npad + i], lzi = L[2 * (size_t)npad + i];
  const bool i_pad = i >= n;
  const bool diag = (I == J);
  const int kbeg = diag ? 1 + 16 * warp / S : 32 * warp / S;
  const int kend = diag ? 1 + 16 * (warp + 1) / S : 32 * (warp + 1) / S;
  double mux = 0.0, muy = 0.0, muz = 0.0, nui = 0.0, phi_i = 0.0;
  __syncthreads();
#pragma unroll 2
  for (int k = kbeg; k < kend; ++k) {
    const int jl = (lane + k) & 31;
    const bool masked = i_pad | (j0 + jl >= n) | (diag & (k == 16) & (lane >= 16));
    const double dx = sx[jl] - xi, dy = sy[jl] - yi, dz = sz[jl] - zi;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    double ri = rsqrt_fp64(r2);
    ri = __longlong_as_double(masked ? 0ll : __double_as_longlong(ri));
    const double ri2 = ri * ri, ri3 = ri2 * ri, ri5 = ri3 * ri2;
    const double mj = sm[jl], ljx = slx[jl], ljy = sly[jl], ljz = slz[jl];
    const double wx = fma(mi, ljx, -mj * lxi), wy = fma(mi, ljy, -mj * lyi), wz = fma(mi, ljz, -mj * lzi);
    const double t = 3.0 * fma(dz, wz, fma(dy, wy, dx * wx)) * ri5;
    const double ux = fma(wx, ri3, -t * dx), uy = fma(wy, ri3, -t * dy), uz = fma(wz, ri3, -t * dz);
    mux += ux;
    muy += uy;
    muz += uz;
    smx[warp][jl] -= ux;
    smy[warp][jl] -= uy;
    smz[warp][jl] -= uz;
    nui = fma(-fma(ljz, dz, fma(ljy, dy, ljx * dx)), ri3, nui);
    snu[warp][jl] = fma(fma(lzi, dz, fma(lyi, dy, lxi * dx)), ri3, snu[warp][jl]);
    phi_i = fma(mj, ri, phi_i);
    sph[warp][jl] = fma(mi, ri, sph[warp][jl]);
    __syncwarp();
  }
  rmx[warp][lane] = mux;
  rmy[warp][lane] = muy;
  rmz[warp][lane] = muz;
  rnu[warp][lane] = nui;
  rph[warp][lane] = phi_i;
  __syncthreads();
  if (warp != 0) return;
  double ax = rmx[0][lane], ay = rmy[0][lane], az = rmz[0][lane], an = rnu[0][lane], ap = rph[0][lane];
  double bx = smx[0][lane], by = smy[0][lane], bz = smz[0][lane], bn = snu[0][lane], bp = sph[0][lane];
#pragma unroll
  for (int w = 1; w < S; ++w) {
    ax += rmx[w][lane];
    ay += rmy[w][lane];
    az += rmz[w][lane];
    an += rnu[w][lane];
    ap += rph[w][lane];
    bx += smx[w][lane];
    by += smy[w][lane];
    bz += smz[w][lane];
    bn += snu[w][lane];
    bp += sph[w][lane];
  }
  const double gg = G * (H / (double)(2 * (s + 1))) / SC[s * kScal + SC_U];
  const size_t st = (size_t)3 * npad;
  auto put = [&](int slot_of, int body, double ax_, double ay_, double az_, double n_, double p_) {
    const size_t zo = (size_t)s * NT + slot_of;
    double* muo = mu + zo * st;
    muo[body] = gg * ax_;
    muo[npad + body] = gg * ay_;
    muo[2 * (size_t)npad + body] = gg * az_;
    nu[zo * npad + body] = gg * n_;
    phi[zo * npad + body] = G * p_;
  };
  if (diag) {
    put(I, i, ax + bx, ay + by, az + bz, an + bn, ap + bp);
  } else {
    put(J, i, ax, ay, az, an, ap);
    put(I, j0 + lane, bx, by, bz, bn, bp);
  }
}

// Transposed kick of level tau: lU from the lv . a partials, then lr += mu + lU m a and
// lm += nu + lU phi (mu, nu, phi summed over their nz partial slots in order).
__global__ void __launch_bounds__(kBlock)
k_adj_kick(int n, int npad, int slot_lo, double H, const double* __restrict__ m, const double* __restrict__ A,
           const double* __restrict__ SC, const double* __restrict__ pg, int nblk, const double* __restrict__ mu,
           const double* __restrict__ nu, const double* __restrict__ phi, int nz, double* __restrict__ lr,
           double* __restrict__ lm) {
  __shared__ double s_lg;
  const int s = slot_lo + blockIdx.y;
  sum_partials(pg + (size_t)s * nblk, nblk, 1, &s_lg);
  const double U = SC[s * kScal + SC_U];
  const double delta = H / (double)(2 * (s + 1));
  const double lU = -s_lg * delta / (U * U);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t st = (size_t)3 * npad;
  double mc[3] = {0.0, 0.0, 0.0}, nv = 0.0, ph = 0.0;
  for (int z = 0; z < nz; ++z) {
    const size_t zo = (size_t)s * nz + z;
    for (int c = 0; c < 3; ++c) mc[c] += mu[zo * st + (size_t)c * npad + i];
    nv += nu[zo * npad + i];
    ph += phi[zo * npad + i];
  }
  for (int c = 0; c < 3; ++c) {
    const size_t o = s * st + (size_t)c * npad + i;
    lr[o] += mc[c] + lU * m[i] * A[o];
  }
  lm[(size_t)s * npad + i] += nv + lU * ph;
}

// lrf = sum_s lr_s, lvf = sum_s lv_s (ascending s).
__global__ void __launch_bounds__(kBlock)
k_adj_sum(int npad, int K, const double* __restrict__ lr, const double* __restrict__ lv, double* __restrict__ lrf,
          double* __restrict__ lvf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  const size_t st = (size_t)3 * npad;
  for (int c = 0; c < 3; ++c) {
    const size_t o = (size_t)c * npad + i;
    double a = 0.0, b = 0.0;
    for (int s = 0; s < K; ++s) {
      a += lr[s * st + o];
      b += lv[s * st + o];
    }
    lrf[o] = a;
    lvf[o] = b;
  }
}

// Energy term of the loss, E = T - U at the final state: lrf -= gE m a, lvf += gE m v,
// lm_0 += gE (|v|^2 / 2 - phi); a and phi from k_adj_pair (slot 0, nz partials).
__global__ void __launch_bounds__(kBlock)
k_adj_eterm(int n, int npad, double gE, const double* __restrict__ m, const double* __restrict__ v,
            const double* __restrict__ aout, const double* __restrict__ phi, int nz, double* __restrict__ lrf,
            double* __restrict__ lvf, double* __restrict__ lm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t st = (size_t)3 * npad;
  double ph = 0.0, v2 = 0.0;
  for (int z = 0; z < nz; ++z) ph += phi[(size_t)z * npad + i];
  for (int c = 0; c < 3; ++c) {
    double a = 0.0;
    for (int z = 0; z < nz; ++z) a += aout[z * st + (size_t)c * npad + i];
    const size_t o = (size_t)c * npad + i;
    lrf[o] -= gE * m[i] * a;
    lvf[o] += gE * m[i] * v[o];
    v2 += v[o] * v[o];
  }
  lm[i] += gE * (0.5 * v2 - ph);
}

// B = U0 - T0 of the initial state: lr0 += lB m a0, lv0 -= lB m v0, and the mass adjoint
// total lmt = sum_s lm_s + lB (phi0 - |v0|^2 / 2), with lB = sum_s lB_s. Per-block partials
// of sum lr0 and sum lv0 (6 values) for the centre-of-mass shift.
__global__ void __launch_bounds__(kBlock)
k_adj_bterm(int n, int npad, int K, const double* __restrict__ m, const double* __restrict__ v0,
            const double* __restrict__ aout, const double* __restrict__ phi, int nz, const double* __restrict__ lB,
            const double* __restrict__ lm, double* __restrict__ lr0, double* __restrict__ lv0,
            double* __restrict__ lmt, double* __restrict__ pc) {
  __shared__ double scratch[32];
  double B = 0.0;
  for (int s = 0; s < K; ++s) B += lB[s];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t st = (size_t)3 * npad;
  double part[6] = {0, 0, 0, 0, 0, 0};
  if (i < n) {
    double ph = 0.0, v2 = 0.0, lms = 0.0;
    for (int z = 0; z < nz; ++z) ph += phi[(size_t)z * npad + i];
    for (int s = 0; s < K; ++s) lms += lm[(size_t)s * npad + i];
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int z = 0; z < nz; ++z) a += aout[z * st + (size_t)c * npad + i];
      const size_t o = (size_t)c * npad + i;
      const double vc = v0[o];
      lr0[o] += B * m[i] * a;
      lv0[o] -= B * m[i] * vc;
      v2 += vc * vc;
      part[c] = lr0[o];
      part[3 + c] = lv0[o];
    }
    lmt[i] = lms + B * (ph - 0.5 * v2);
  }
  for (int q = 0; q < 6; ++q) {
    const double t = block_sum(part[q], scratch);
    if (threadIdx.x == 0) pc[(size_t)blockIdx.x * 6 + q] = t;
  }
}

// Initial centre-of-mass shift r0 = r_in - sum m r_in / M (and v): out_r = lr0 - m Sr / M,
// out_v = lv0 - m Sv / M, out_m = lmt - (Sr . r0 + Sv . v0) / M with Sr = sum lr0,
// Sv = sum lv0.
__global__ void __launch_bounds__(kBlock)
k_adj_com(int n, int npad, double M, const double* __restrict__ m, const double* __restrict__ r0,
          const double* __restrict__ v0, const double* __restrict__ pc, int nblk, const double* __restrict__ lr0,
          const double* __restrict__ lv0, const double* __restrict__ lmt, double* __restrict__ out_r,
          double* __restrict__ out_v, double* __restrict__ out_m) {
  __shared__ double S[6];
  for (int q = 0; q < 6; ++q) sum_partials(pc + q, nblk, 6, &S[q]);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  double dot = 0.0;
  for (int c = 0; c < 3; ++c) {
    const size_t o = (size_t)c * npad + i;
    out_r[o] = i < n ? lr0[o] - m[i] * S[c] / M : 0.0;
    out_v[o] = i < n ? lv0[o] - m[i] * S[3 + c] / M : 0.0;
    dot += S[c] * r0[o] + S[3 + c] * v0[o];
  }
  out_m[i] = i < n ? lmt[i] - dot / M : 0.0;
}

}  // namespace
}  // namespace mstar

using namespace mstar;

struct mstar_adjoint {
  mstar_ctx* c = nullptr;
  int nsteps = 0, every = 0, nck = 0, nz = 0, jchunk = 0;
  double H = 0.0;
  void* mem = nullptr;
  double* ck = nullptr;              // nck x (r planes, v planes)
  std::vector<double> tck;           // time of each checkpoint
  double* fin = nullptr;             // final (r planes, v planes)
  double t_final = 0.0;
  std::vector<AdjTraj> tr;           // one per step of a segment
  int tr_seg = -1;                   // the segment whose trajectories tr holds (-1: none)
  double *lr = nullptr, *lv = nullptr, *lrf = nullptr, *lvf = nullptr, *lm = nullptr, *lB = nullptr;
  double *mu = nullptr, *nu = nullptr, *phi = nullptr, *aout = nullptr, *pf = nullptr, *pg = nullptr;
  double *lmt = nullptr, *pc = nullptr, *outr = nullptr, *outv = nullptr, *outm = nullptr;
  Weights cw{};
  // the reverse substeps of step q of a segment, captured once as a graph (see bw_step)
  std::vector<cudaGraphExec_t> bw_exec;
  bool bw_off = false;
  long long bw_launches = 0;
};

namespace {

int blocks_of(int n) { return (n + kBlock - 1) / kBlock; }

struct ACarve {
  char* base;
  size_t off = 0;
  explicit ACarve(void* b) : base(static_cast<char*>(b)) {}
  double* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    double* p = base ? reinterpret_cast<double*>(base + off) : nullptr;
    off += count * sizeof(double);
    return p;
  }
};

size_t adj_carve(mstar_adjoint* a, void* base) {
  mstar_ctx* c = a->c;
  const size_t st = (size_t)3 * c->npad, np = c->npad, K = c->K, nb = c->nblk;
  const size_t lvl = K * st, nsc = (K + 1) * kScal;
  ACarve cv(base);
  a->ck = cv.take((size_t)a->nck * 2 * st);
  a->fin = cv.take(2 * st);
  for (auto& t : a->tr) {
    t.R = cv.take(2 * K * lvl);
    t.A = cv.take(2 * K * lvl);
    t.Vv = cv.take(2 * K * lvl);
    t.SC = cv.take((2 * K + 1) * nsc);
    t.v0 = cv.take(st);
  }
  a->lr = cv.take(K * st);
  a->lv = cv.take(K * st);
  a->lrf = cv.take(st);
  a->lvf = cv.take(st);
  a->lm = cv.take(K * np);
  a->lB = cv.take(K);
  // partials of the VJP pair loops: nz partner ranges (the state's a and phi) or NT tile slots
  const size_t nzp = (size_t)(a->nz > c->NT ? a->nz : c->NT);
  a->mu = cv.take(K * nzp * st);
  a->nu = cv.take(K * nzp * np);
  a->phi = cv.take(K * nzp * np);
  a->aout = cv.take((size_t)a->nz * st);
  a->pf = cv.take(K * nb);
  a->pg = cv.take(K * nb);
  a->lmt = cv.take(np);
  a->pc = cv.take(nb * 6);
  a->outr = cv.take(st);
  a->outv = cv.take(st);
  a->outm = cv.take(np);
  return cv.off;
}

#define ACK(call)                          \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) return MSTAR_ERR_CUDA; \
  } while (0)

// One fixed step from the context's state: MST, attempt at H, accept.
int fixed_step(mstar_ctx* c, double H) {
  double U0, T0, eps, tn;
  int rc = step_prepare(c, &U0, &T0);
  if (!rc) rc = step_attempt(c, H, &eps, &tn);
  if (!rc) rc = step_accept(c);
  if (!rc) c->t = tn;
  return rc;
}

int set_planes(mstar_ctx* c, const double* rv, double t) {
  const size_t st = (size_t)3 * c->npad;
  ACK(cudaMemcpyAsync(c->d.r, rv, sizeof(double) * st, cudaMemcpyDeviceToDevice, c->stream));
  ACK(cudaMemcpyAsync(c->d.v, rv + st, sizeof(double) * st, cudaMemcpyDeviceToDevice, c->stream));
  c->t = t;
  c->mst_valid = false;
  return MSTAR_OK;
}

int save_planes(mstar_ctx* c, double* rv) {
  const size_t st = (size_t)3 * c->npad;
  ACK(cudaMemcpyAsync(rv, c->d.r, sizeof(double) * st, cudaMemcpyDeviceToDevice, c->stream));
  ACK(cudaMemcpyAsync(rv + st, c->d.v, sizeof(double) * st, cudaMemcpyDeviceToDevice, c->stream));
  return MSTAR_OK;
}

// a(r) and phi(r) of the state whose positions are the planes R, into aout / phi slot 0.
int pair_state(mstar_ctx* c, mstar_adjoint* a, const double* R) {
  const dim3 grid((c->n + kAdjI - 1) / kAdjI, 1, a->nz);
  k_adj_pair<<<grid, kAdjI, 0, c->stream>>>(c->n, c->npad, 0, c->p.G, a->H, c->d.m, R, 0, nullptr, 0, nullptr,
                                             a->nz, a->jchunk, a->mu, a->nu, a->phi, a->aout);
  MSTAR_LAUNCHED(c);
  ACK(cudaGetLastError());
  return MSTAR_OK;
}

// Reverse sweep of one step: lrf, lvf (adjoint of the step's output state) become the
// adjoint of its start state; lm, lB accumulate.
int backward_step(mstar_ctx* c, mstar_adjoint* a, const AdjTraj& t) {
  const int K = c->K, n = c->n, np = c->npad, nb = c->nblk;
  const size_t st = (size_t)3 * np, lvl = (size_t)K * st, nsc = (size_t)(K + 1) * kScal;
  cudaStream_t s = c->stream;
  k_adj_init<<<dim3(blocks_of(np), K), kBlock, 0, s>>>(np, a->cw, a->lrf, a->lvf, a->lr, a->lv);
  MSTAR_LAUNCHED(c);
  for (int tau = 2 * K; tau >= 0; --tau) {
    const int lo = tau > 0 ? (tau + 1) / 2 - 1 : 0;
    const int nsl = K - lo;
    const double* V = tau > 0 ? t.Vv + (tau - 1) * lvl : t.v0;
    const size_t vs = tau > 0 ? st : 0;
    const double* SC = t.SC + tau * nsc;
    const double* A = tau > 0 ? t.A + (tau - 1) * lvl : nullptr;
    k_adj_dot<<<dim3(nb, nsl), kBlock, 0, s>>>(n, np, lo, a->lr, st, V, vs, a->pf, nb);
    k_adj_drift<<<dim3(nb, nsl), kBlock, 0, s>>>(n, np, lo, tau, a->H, c->B, c->d.m, a->lr, a->lv, V, vs, SC, a->pf,
                                                  nb, a->lm, a->lB, A, a->pg);
    c->launches += 2;
    if (tau > 0) {
      const dim3 grid(c->ntp, nsl);
      const double* R = t.R + (tau - 1) * lvl;
      switch (c->W == 1 ? (c->S > 1 ? -c->S : 1) : c->W) {
        case -2:
          k_adj_pair_sym_ks<2><<<grid, 64, 0, s>>>(n, np, c->NT, lo, c->p.G, a->H, c->d.m, R, st, a->lv, st, SC,
                                                   a->mu, a->nu, a->phi);
          break;
        case -4:
          k_adj_pair_sym_ks<4><<<grid, 128, 0, s>>>(n, np, c->NT, lo, c->p.G, a->H, c->d.m, R, st, a->lv, st, SC,
                                                    a->mu, a->nu, a->phi);
          break;
        case -8:
          k_adj_pair_sym_ks<8><<<grid, 256, 0, s>>>(n, np, c->NT, lo, c->p.G, a->H, c->d.m, R, st, a->lv, st, SC,
                                                    a->mu, a->nu, a->phi);
          break;
        case 1:
          k_adj_pair_sym<1><<<grid, 32, 0, s>>>(n, np, c->NT, lo, c->p.G, a->H, c->d.m, R, st, a->lv, st, SC, a->mu,
                                                a->nu, a->phi);
          break;
        case 2:
          k_adj_pair_sym<2><<<grid, 64, 0, s>>>(n, np, c->NT, lo, c->p.G, a->H, c->d.m, R, st, a->lv, st, SC, a->mu,
                                                a->nu, a->phi);
          break;
        default:
          k_adj_pair_sym<4><<<grid, 128, 0, s>>>(n, np, c->NT, lo, c->p.G, a->H, c->d.m, R, st, a->lv, st, SC,
                                                 a->mu, a->nu, a->phi);
          break;
      }
      k_adj_kick<<<dim3(nb, nsl), kBlock, 0, s>>>(n, np, lo, a->H, c->d.m, A, SC, a->pg, nb, a->mu, a->nu, a->phi,
                                                   c->NT, a->lr, a->lm);
      c->launches += 2;
    }
  }
  k_adj_sum<<<blocks_of(np), kBlock, 0, s>>>(np, K, a->lr, a->lv, a->lrf, a->lvf);
  MSTAR_LAUNCHED(c);
  ACK(cudaGetLastError());
  return MSTAR_OK;
}

// backward_step for step q of a segment, as one graph launch: its launches depend only on
// the adjoint's buffers and step q's trajectory record, so the graph captured the first
// time serves every segment. A failed capture falls back to direct launches.
int bw_step(mstar_ctx* c, mstar_adjoint* a, int q) {
  if (a->bw_exec.size() != a->tr.size()) a->bw_exec.assign(a->tr.size(), nullptr);
  if (!a->bw_exec[q] && !a->bw_off) {
    cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    cudaGraph_t g = nullptr;
    bool ok = c->cap || cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
      c->stream = c->cap;
      ok = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const int rc = backward_step(c, a, a->tr[q]);
        ok = cudaStreamEndCapture(c->cap, &g) == cudaSuccess && rc == MSTAR_OK && g;
      }
      c->stream = user;
    }
    a->bw_launches = c->launches - l0;
    c->launches = l0;
    if (ok) ok = cudaGraphInstantiate(&a->bw_exec[q], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      a->bw_exec[q] = nullptr;
      a->bw_off = true;
    }
  }
  if (!a->bw_exec[q]) return backward_step(c, a, a->tr[q]);
  if (cudaGraphLaunch(a->bw_exec[q], c->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
  c->launches += a->bw_launches;
  return MSTAR_OK;
}

}  // namespace

extern "C" {

void mstar_adjoint_free(mstar_adjoint* a) {
  if (!a) return;
  if (a->c && a->c->stream) cudaStreamSynchronize(a->c->stream);
  if (a->c) mstar::drop_traj_graphs(a->c);
  for (cudaGraphExec_t e : a->bw_exec)
    if (e) cudaGraphExecDestroy(e);
  if (a->mem) cudaFree(a->mem);
  delete a;
}

int mstar_adjoint_forward(mstar_ctx* c, double H, int nsteps, int checkpoint_every, mstar_adjoint** out) {
  if (!out) return MSTAR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!c || !std::isfinite(H) || H == 0.0 || nsteps < 1 || checkpoint_every < 1) return MSTAR_ERR_INVALID_ARG;
  if (!c->at_init) return MSTAR_ERR_INVALID_ARG;
  mstar_adjoint* a = new (std::nothrow) mstar_adjoint();
  if (!a) return MSTAR_ERR_NOMEM;
  a->c = c;
  a->H = H;
  a->nsteps = nsteps;
  a->every = checkpoint_every < nsteps ? checkpoint_every : nsteps;
  a->nck = (nsteps + a->every - 1) / a->every;
  a->jchunk = adj_jchunk(c->n);
  a->nz = (c->n + a->jchunk - 1) / a->jchunk;
  a->tr.resize(a->every);
  a->tck.resize(a->nck);
  // Lagrange weights of the extrapolation to 0 over the nodes x_k = (1/n_k)^2
  for (int k = 0; k < c->K; ++k) {
    const double xk = 1.0 / (double)((2 * (k + 1)) * (2 * (k + 1)));
    double w = 1.0;
    for (int j = 0; j < c->K; ++j) {
      if (j == k) continue;
      const double xj = 1.0 / (double)((2 * (j + 1)) * (2 * (j + 1)));
      w *= xj / (xj - xk);
    }
    a->cw.c[k] = w;
  }
  const size_t bytes = adj_carve(a, nullptr);
  if (cudaMalloc(&a->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete a;
    return MSTAR_ERR_NOMEM;
  }
  adj_carve(a, a->mem);
  int rc = cudaMemsetAsync(a->mem, 0, bytes, c->stream) == cudaSuccess ? MSTAR_OK : MSTAR_ERR_CUDA;
  const size_t st = (size_t)3 * c->npad;
  // the steps of the last segment record their trajectories on the way, so that the reverse
  // sweep starts without recomputing that segment
  const int last_first = (a->nck - 1) * a->every;
  for (int i = 0; i < nsteps && !rc; ++i) {
    if (i % a->every == 0) {
      a->tck[i / a->every] = c->t;
      rc = save_planes(c, a->ck + (size_t)(i / a->every) * 2 * st);
    }
    if (!rc) {
      // every step level by level: the reverse sweep's recomputations, which record
      // trajectories, then reproduce the checkpoints bit for bit
      c->traj = i >= last_first ? &a->tr[i - last_first] : nullptr;
      c->levelled = true;
      rc = fixed_step(c, H);
      c->levelled = false;
      c->traj = nullptr;
    }
  }
  if (!rc) a->tr_seg = a->nck - 1;
  if (!rc) rc = save_planes(c, a->fin);
  a->t_final = c->t;
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = MSTAR_ERR_CUDA;
  if (rc) {
    mstar_adjoint_free(a);
    return rc;
  }
  *out = a;
  return MSTAR_OK;
}

int mstar_step_adjoint(mstar_ctx* c, mstar_adjoint* a, const double* g_r, const double* g_v, double g_E, double* d_r,
                       double* d_v, double* d_m) {
  if (!c || !a || a->c != c || !std::isfinite(g_E)) return MSTAR_ERR_INVALID_ARG;
  const int n = c->n, np = c->npad, nb = c->nblk;
  const size_t st = (size_t)3 * np;
  cudaStream_t s = c->stream;
  int rc = MSTAR_OK;
  // adjoint of the final state from the loss: the given gradients plus the energy term
  ACK(cudaMemsetAsync(a->lrf, 0, sizeof(double) * st, s));
  ACK(cudaMemsetAsync(a->lvf, 0, sizeof(double) * st, s));
  ACK(cudaMemsetAsync(a->lm, 0, sizeof(double) * (size_t)c->K * np, s));
  ACK(cudaMemsetAsync(a->lB, 0, sizeof(double) * c->K, s));
  if (g_r && (rc = vectors_in(c, g_r, a->lrf))) return rc;
  if (g_v && (rc = vectors_in(c, g_v, a->lvf))) return rc;
  if (g_E != 0.0) {
    if ((rc = pair_state(c, a, a->fin))) return rc;
    k_adj_eterm<<<blocks_of(n), kBlock, 0, s>>>(n, np, g_E, c->d.m, a->fin + st, a->aout, a->phi, a->nz, a->lrf,
                                                 a->lvf, a->lm);
    MSTAR_LAUNCHED(c);
  }
  // segments from the last: recompute with trajectories, then sweep the steps backwards
  for (int seg = a->nck - 1; seg >= 0 && !rc; --seg) {
    const int first = seg * a->every;
    const int cnt = (a->nsteps - first) < a->every ? (a->nsteps - first) : a->every;
    if (a->tr_seg != seg) {  // recompute the segment from its checkpoint, recording it
      a->tr_seg = -1;
      rc = set_planes(c, a->ck + (size_t)seg * 2 * st, a->tck[seg]);
      for (int q = 0; q < cnt && !rc; ++q) {
        c->traj = &a->tr[q];
        c->levelled = true;
        rc = fixed_step(c, a->H);
        c->levelled = false;
        c->traj = nullptr;
      }
      if (!rc) a->tr_seg = seg;
    }
    for (int q = cnt - 1; q >= 0 && !rc; --q) rc = bw_step(c, a, q);
  }
  // B = U0 - T0 and the centre-of-mass shift of the initial state, then the outputs
  if (!rc) rc = pair_state(c, a, a->ck);
  if (!rc) {
    k_adj_bterm<<<nb, kBlock, 0, s>>>(n, np, c->K, c->d.m, a->ck + st, a->aout, a->phi, a->nz, a->lB, a->lm, a->lrf,
                                      a->lvf, a->lmt, a->pc);
    k_adj_com<<<blocks_of(np), kBlock, 0, s>>>(n, np, c->Mtot, c->d.m, a->ck, a->ck + st, a->pc, nb, a->lrf, a->lvf,
                                               a->lmt, a->outr, a->outv, a->outm);
    c->launches += 2;
    if (cudaGetLastError() != cudaSuccess) rc = MSTAR_ERR_CUDA;
  }
  if (!rc && d_r) rc = vectors_out(c, a->outr, d_r);
  if (!rc && d_v) rc = vectors_out(c, a->outv, d_v);
  if (!rc && d_m) {
    if (cudaMemcpyAsync(d_m, a->outm, sizeof(double) * n, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = MSTAR_ERR_CUDA;
  }
  // the context ends at the run's final state, as after the forward
  const int rc2 = set_planes(c, a->fin, a->t_final);
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = MSTAR_ERR_CUDA;
  return rc ? rc : rc2;
}

}  // extern "C"
