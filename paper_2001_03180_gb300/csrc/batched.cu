// Batched GBS steps for many independent small systems (Sec. 4.2 notes the method extends to
// integrating multiple independent N-body systems simultaneously).
//
// One graph launch advances every unfinished system by one GBS step attempt. Each system is
// one CTA of four division groups of G warps (G = 1, 2 or 4, chosen per size class):
//  - the whole CTA builds the system's MST (Prim, exact FP64 keys, Sec. 3.2 / 3.4), the
//    edge coordinates and the derivative information of the step start;
//  - the k_fix leapfrog divisions are spread over the four groups with the paper's greedy
//    recipe (largest n_k first, to the least-loaded group, lowest index on ties; Sec. 4.2);
//    a group runs its divisions with group-level barriers only, its G warps splitting the
//    pair loop by 32 x 32 blocks and the O(N) work by body;
//  - the whole CTA then extrapolates (Aitken-Neville), evaluates the error of Eq.
//    gbs-criterion and applies the step control of Sec. 2.3-2.4 for its system.
// Systems of the same G form one kernel node of the graph (largest system first); the
// nodes are independent, so the schedules run side by side on the GPU.
//
// The pair loop inside a warp uses the same symmetric rotation as the large-N kernel: lane
// l owns body i of a 32-block and pairs with body (l + k) mod 32 of the partner block at
// step k, so every unordered pair is visited once and the 32 partner accumulators are
// updated by distinct lanes. Each warp accumulates into its own partial acceleration
// buffer; the group adds the G partials in a fixed order, so results do not depend on
// timing. Near pairs (N_d <= 2) are masked out and summed from edge vectors afterwards,
// exactly as in the large-N path.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

constexpr int kGroups = 4;        // division groups per system
constexpr int kMaxG = 4;          // warps per group of the widest schedule
constexpr int kBMaxN = 512;       // largest system of a batch
constexpr int kNumClasses = 7;    // size classes of the schedule table

// Size class of a system of n bodies: [2,8], [9,16], [17,32], ..., [257,512].
__host__ __device__ __forceinline__ int size_class(int n) {
  int c = 0;
  while (c < kNumClasses - 1 && n > (8 << c)) ++c;
  return c;
}

// Per-system scalars in device memory.
struct SysScalars {
  double t, B, H, M, U0, T0, eps, Ha;  // Ha: the fictitious step of the current attempt
  long long accepted, rejected, force_evals;
  int status;      // 0 running, 1 reached t_end, 2 time-iteration limit, -3 no convergence
  int halvings, time_iters, go;  // go: the current attempt runs (1) or the system stopped (0)
};

// Per-body storage (doubles), offsets in units of n doubles (a 3-vector field spans 3).
enum : int {
  B_R = 0, B_V = 3, B_X0 = 6, B_V0 = 9, B_A0 = 12, B_TKK = 15,
  B_GRP = 21,                          // per group: X 3, V 3, r 3, v 3, kMaxG partial a x 3
  kGrpStride = 12 + 3 * kMaxG,
  B_END = B_GRP + kGroups * kGrpStride,  // k_fix division end states x (X 3, V 3)
};
constexpr int kBodyDoublesBase = B_END;  // + 6 * k_fix

__constant__ double c_bfac[kMaxKfix][kMaxKfix];  // 1 / ((n_k / n_{k-j})^2 - 1)

struct BatchParams {
  double eta, a_gbs, fac_min, fac_max, q_first, t_tol, G;
  int k_fix, n_d, max_halvings, max_time_iter;
  int body_doubles;
};

// Position of a thread within its division group.
struct GI {
  int g;     // group 0..3
  int w;     // warp within the group
  int lane;
  int t;     // thread within the group
};

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double madd(double a, double f, double b) { return __dadd_rn(a, __dmul_rn(f, b)); }

// S / M from rM = 1/M (rounded) and one residual correction (Markstein's method): three FP64
// instructions instead of a full division, and the correctly rounded quotient except in rare
// cases next to a rounding boundary, where it is one unit in the last place away.
__device__ __forceinline__ double quot(double S, double M, double rM) {
  const double q = S * rM;
  return fma(fma(-q, M, S), rM, q);
}

// Barrier over the 32 G threads of group g (named barrier g + 1; 0 is __syncthreads).
template <int G>
__device__ __forceinline__ void gsync(int g) {
  if constexpr (G == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(32 * G) : "memory");
  }
}

// Sum of one value over the group, added warp by warp in a fixed order.
template <int G>
__device__ __forceinline__ double gsum1(double a, const GI& gi, double (*red)[kMaxG][3]) {
  a = warp_sum(a);
  if constexpr (G > 1) {
    if (gi.lane == 0) red[gi.g][gi.w][0] = a;
    gsync<G>(gi.g);
    a = red[gi.g][0][0];
    for (int q = 1; q < G; ++q) a += red[gi.g][q][0];
    gsync<G>(gi.g);
  }
  return a;
}

// Sums of three values over the group, added warp by warp in a fixed order.
template <int G>
__device__ __forceinline__ void gsum3(double& a, double& b, double& c, const GI& gi, double (*red)[kMaxG][3]) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if constexpr (G > 1) {
    if (gi.lane == 0) {
      red[gi.g][gi.w][0] = a;
      red[gi.g][gi.w][1] = b;
      red[gi.g][gi.w][2] = c;
    }
    gsync<G>(gi.g);
    a = red[gi.g][0][0];
    b = red[gi.g][0][1];
    c = red[gi.g][0][2];
    for (int q = 1; q < G; ++q) {
      a += red[gi.g][q][0];
      b += red[gi.g][q][1];
      c += red[gi.g][q][2];
    }
    gsync<G>(gi.g);
  }
}

// Path sums from edge vectors (w_v = W_v + W_parent(v) + ...), then the COM shift; returns
// sum m |w|^2 after the shift when want_T. Group-level; ends with the group synchronised.
// The path walks take the bodies in order of tree level (bylev), so that the lanes of a
// warp walk paths of about equal length.
template <int G>
__device__ double grebuild(int n, const double* __restrict__ m, const int* __restrict__ parent,
                           const int* __restrict__ bylev, const double* W, double* w, double Mtot, double rM,
                           bool want_T, const GI& gi, double (*red)[kMaxG][3]) {
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  for (int i = gi.t; i < n; i += 32 * G) {
    const int v = bylev[i];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int u = v; parent[u] >= 0; u = parent[u]) {
      s0 = __dadd_rn(s0, W[3 * u]);
      s1 = __dadd_rn(s1, W[3 * u + 1]);
      s2 = __dadd_rn(s2, W[3 * u + 2]);
    }
    w[3 * v] = s0;
    w[3 * v + 1] = s1;
    w[3 * v + 2] = s2;
    c0 += __dmul_rn(m[v], s0);
    c1 += __dmul_rn(m[v], s1);
    c2 += __dmul_rn(m[v], s2);
  }
  gsum3<G>(c0, c1, c2, gi, red);
  c0 = quot(c0, Mtot, rM);
  c1 = quot(c1, Mtot, rM);
  c2 = quot(c2, Mtot, rM);
  double t2 = 0.0;
  for (int v = gi.t; v < n; v += 32 * G) {
    const double q0 = __dsub_rn(w[3 * v], c0), q1 = __dsub_rn(w[3 * v + 1], c1), q2 = __dsub_rn(w[3 * v + 2], c2);
    w[3 * v] = q0;
    w[3 * v + 1] = q1;
    w[3 * v + 2] = q2;
    if (want_T) t2 += __dmul_rn(m[v], __dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2)));
  }
  gsync<G>(gi.g);
  if (!want_T) return 0.0;
  return gsum1<G>(t2, gi, red);
}

// x with its sign bit flipped when neg (an integer operation: no FP64 issue slot).
__device__ __forceinline__ double flip(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}

// The near partners of body p (tree distance <= n_d <= 2, Sec. 3.4) in the order parent,
// children, grandparent, grandchildren (by child), siblings, each with the edges whose
// vectors give the separation r_q - r_p: q = parent: -X_p; child: X_q; grandparent:
// -(X_p + X_parent(p)); grandchild: X_q + X_parent(q); sibling: X_q - X_p. Integer work only.
struct NearWalk {
  int p, pp, g, stage, c, cend, ch, gc, gcend, sb, send;
  __device__ __forceinline__ NearWalk(int p_, int n_d, const int* parent, const int* gp, const int* coff)
      : p(p_), pp(parent[p_]), g(n_d >= 2 ? gp[p_] : -1), stage(0), c(coff[p_]), cend(coff[p_ + 1]), ch(-1),
        gc(0), gcend(0), sb(0), send(0) {
    if (n_d < 2) stage = 10;  // parent and children only
  }
  // next partner q and separation edges (ea with sign na, eb >= 0 with sign nb, or eb = -1)
  __device__ __forceinline__ bool next(const int* cidx, const int* coff, int& q, int& ea, bool& na, int& eb, bool& nb) {
    for (;;) {
      switch (stage) {
        case 0:
        case 10:
          stage += 1;
          if (pp >= 0) {
            q = pp; ea = p; na = true; eb = -1; nb = false;
            return true;
          }
          break;
        case 1:
        case 11:
          if (c < cend) {
            q = cidx[c++]; ea = q; na = false; eb = -1; nb = false;
            return true;
          }
          if (stage == 11) return false;
          stage = 2;
          break;
        case 2:
          stage = 3;
          c = coff[p];
          if (g >= 0) {
            q = g; ea = p; na = true; eb = pp; nb = true;
            return true;
          }
          break;
        case 3:
          while (gc == gcend && c < cend) {
            ch = cidx[c++];
            gc = coff[ch];
            gcend = coff[ch + 1];
          }
          if (gc < gcend) {
            q = cidx[gc++]; ea = q; na = false; eb = ch; nb = false;
            return true;
          }
          stage = 4;
          if (pp >= 0) {
            sb = coff[pp];
            send = coff[pp + 1];
          }
          break;
        default:
          while (sb < send && cidx[sb] == p) ++sb;
          if (sb < send) {
            q = cidx[sb++]; ea = q; na = false; eb = p; nb = true;
            return true;
          }
          return false;
      }
    }
  }
};

// One 32-block of partners and their accumulators, per warp.
struct WarpShared {
  double x[32], y[32], z[32], mm[32], ax[32], ay[32], az[32];
  unsigned long long ms[32];
  int me[32], p[32], g[32];
};

// Pair loop of one system by one group: accelerations (3-vectors, times G) into a0 (the
// group's first partial buffer; partial w at a0 + 3 n w) and the return value U. Ends with
// the group synchronised and a0 complete.
template <int G>
__device__ double gforces(int n, int n_d, double Gc, const double* __restrict__ m, const int* __restrict__ parent,
                          const int* __restrict__ gp, const int* __restrict__ coff, const int* __restrict__ cidx,
                          const double* r, const double* X, double* a0, WarpShared& sh, const GI& gi,
                          double (*red)[kMaxG][3]) {
  const int lane = gi.lane;
  double* a = a0 + (size_t)3 * n * gi.w;
  for (int v = lane; v < n; v += 32) {
    a[3 * v] = 0.0;
    a[3 * v + 1] = 0.0;
    a[3 * v + 2] = 0.0;
  }
  __syncwarp();
  const int nb = (n + 31) >> 5;
  const bool nd1 = n_d >= 1, nd2 = n_d >= 2;
  double usum = 0.0;
  int q = 0;
  for (int I = 0; I < nb; ++I) {
    for (int J = I; J < nb; ++J, ++q) {
      if ((q & (G - 1)) != gi.w) continue;
      const int i = I * 32 + lane;
      const bool ipad = i >= n;
      const double xi = ipad ? 0.0 : r[3 * i], yi = ipad ? 0.0 : r[3 * i + 1], zi = ipad ? 0.0 : r[3 * i + 2];
      const MassSplit msi = mass_split(ipad ? 1.0 : m[i]);
      const double mi = ipad ? 0.0 : m[i];
      const int pi = ipad ? -3 : parent[i], gpi = ipad ? -3 : gp[i];
      double axi = 0.0, ayi = 0.0, azi = 0.0, ui = 0.0;
      const int jb = J * 32 + lane;
      const bool jpad = jb >= n;
      sh.x[lane] = jpad ? 0.0 : r[3 * jb];
      sh.y[lane] = jpad ? 0.0 : r[3 * jb + 1];
      sh.z[lane] = jpad ? 0.0 : r[3 * jb + 2];
      sh.mm[lane] = jpad ? 0.0 : m[jb];
      const MassSplit ms = mass_split(jpad ? 1.0 : m[jb]);
      sh.ms[lane] = ms.m;
      sh.me[lane] = ms.e;
      sh.p[lane] = jpad ? -3 : parent[jb];
      sh.g[lane] = jpad ? -3 : gp[jb];
      sh.ax[lane] = 0.0;
      sh.ay[lane] = 0.0;
      sh.az[lane] = 0.0;
      __syncwarp();
      // A partner block with t < 32 bodies (the last one) is swept at width Wb = the power of
      // two >= t: lane l pairs with slot (l + k) mod Wb, Wb steps (Wb/2 + 1 on the diagonal),
      // and the 32 / Wb lane groups keep separate partner accumulators (added below in group
      // order), so that no two lanes update the same accumulator at a step.
      const bool self = (I == J);
      const int tail = n - J * 32;
      const int Wb = tail >= 32 ? 32 : (1 << (32 - __clz(tail - 1)));
      const int cb = lane & ~(Wb - 1);
      const int kbeg = self ? 1 : 0, kend = self ? Wb / 2 + 1 : Wb;
      for (int k = kbeg; k < kend; ++k) {
        const int jl = (lane + k) & (Wb - 1);
        const int ja = cb + jl;
        const int j = J * 32 + jl;
        bool masked = ipad | (j >= n) | (self & (k == Wb / 2) & ((lane & (Wb - 1)) >= Wb / 2));
        const int pj = sh.p[jl], gj = sh.g[jl];
        masked |= nd1 & ((pi == j) | (pj == i));
        masked |= nd2 & ((gpi == j) | (gj == i) | (pi == pj));
        double dx = sh.x[jl] - xi, dy = sh.y[jl] - yi, dz = sh.z[jl] - zi;
        asm volatile("" : "+d"(dx), "+d"(dy), "+d"(dz));
        double rinv, sj, si;
        if (!masked) {
          pair_scalars_int(dx, dy, dz, MassSplit{sh.ms[jl], sh.me[jl]}, msi, rinv, sj, si);
        } else {
          rinv = sj = si = 0.0;
        }
        axi = fma(sj, dx, axi);
        ayi = fma(sj, dy, ayi);
        azi = fma(sj, dz, azi);
        ui = fma(sh.mm[jl], rinv, ui);
        sh.ax[ja] = fma(si, dx, sh.ax[ja]);
        sh.ay[ja] = fma(si, dy, sh.ay[ja]);
        sh.az[ja] = fma(si, dz, sh.az[ja]);
        __syncwarp();
      }
      // body jb and body i of this item are only ever touched by this lane of this warp
      if (!jpad) {  // partner sums were kept with the opposite sign
        double sx = sh.ax[lane], sy = sh.ay[lane], sz = sh.az[lane];
        for (int c = Wb; c < 32; c += Wb) {
          sx += sh.ax[c + lane];
          sy += sh.ay[c + lane];
          sz += sh.az[c + lane];
        }
        a[3 * jb] -= sx;
        a[3 * jb + 1] -= sy;
        a[3 * jb + 2] -= sz;
      }
      if (!ipad) {
        a[3 * i] += axi;
        a[3 * i + 1] += ayi;
        a[3 * i + 2] += azi;
      }
      usum += mi * ui;
      __syncwarp();
    }
  }
  // near pairs from edge vectors: parent, children, grandparent, grandchildren, siblings,
  // walked as one list per body (NearWalk) so that the FP64 part of a warp's loop runs as
  // many times as its longest list, with the pair scalars on the integer pipe.
  // Body p goes to thread p mod 32G, i.e. lane p mod 32 of this warp: the same lane that
  // updated it in the loop above.
  if (n_d >= 1) {
    for (int p = gi.t; p < n; p += 32 * G) {
      double ax = 0.0, ay = 0.0, az = 0.0, u = 0.0;
      NearWalk nw(p, n_d, parent, gp, coff);
      int q, ea, eb;
      bool na, nb;
      while (nw.next(cidx, coff, q, ea, na, eb, nb)) {
        // d = r_q - r_p = (+/-) X_ea (+/-) X_eb, one rounding per component (as the
        // edge-vector sums of the reference order: j side summed upward, minus the i side)
        const double dx = __dadd_rn(flip(X[3 * ea], na), eb >= 0 ? flip(X[3 * eb], nb) : 0.0);
        const double dy = __dadd_rn(flip(X[3 * ea + 1], na), eb >= 0 ? flip(X[3 * eb + 1], nb) : 0.0);
        const double dz = __dadd_rn(flip(X[3 * ea + 2], na), eb >= 0 ? flip(X[3 * eb + 2], nb) : 0.0);
        const double mq = m[q];
        const MassSplit ms = mass_split(mq);
        double rinv, sq, unused;
        pair_scalars_int(dx, dy, dz, ms, ms, rinv, sq, unused);
        ax = fma(sq, dx, ax);
        ay = fma(sq, dy, ay);
        az = fma(sq, dz, az);
        if (q > p) u = fma(mq, rinv, u);
      }
      a[3 * p] += ax;
      a[3 * p + 1] += ay;
      a[3 * p + 2] += az;
      usum += m[p] * u;
    }
  }
  gsync<G>(gi.g);
  // a0 = G_const x (partial 0 + partial 1 + ...), fixed order
  for (int v = gi.t; v < n; v += 32 * G) {
    for (int c = 0; c < 3; ++c) {
      double s = a0[3 * v + c];
      for (int w = 1; w < G; ++w) s += a0[(size_t)3 * n * w + 3 * v + c];
      a0[3 * v + c] = s * Gc;
    }
  }
  gsync<G>(gi.g);
  return Gc * gsum1<G>(usum, gi, red);
}

template <int NW>
__device__ __forceinline__ void block_argmin(unsigned long long& k, int& i, unsigned long long* rk, int* ri) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_down_sync(0xffffffffu, k, o);
    const int i2 = __shfl_down_sync(0xffffffffu, i, o);
    if (k2 < k || (k2 == k && i2 < i)) {
      k = k2;
      i = i2;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    rk[warp] = k;
    ri[warp] = i;
  }
  __syncthreads();
  k = rk[0];
  i = ri[0];
  for (int w = 1; w < NW; ++w)
    if (rk[w] < k || (rk[w] == k && ri[w] < i)) {
      k = rk[w];
      i = ri[w];
    }
}

__device__ __forceinline__ double d2x(const double* r, int u, int v) {
  const double dx = __dsub_rn(r[3 * u], r[3 * v]), dy = __dsub_rn(r[3 * u + 1], r[3 * v + 1]),
               dz = __dsub_rn(r[3 * u + 2], r[3 * v + 2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Sec. 2.4: the fictitious step of this attempt -- the first step ds = q U dt, later the
// controller's step, clamped so that t + H/U does not pass t_end (with the time-iteration
// count) -- or true when the system stops here (t_end reached, iterations exhausted).
__device__ bool choose_step(SysScalars* S, const BatchParams& P, double t_end, double t0, double U0, double* Hs_out) {
  const double dt = t_end - t0;
  double Hs = 0.0;
  bool abort_ = false;
  if (fabs(dt) <= P.t_tol * fabs(t_end)) {
    S->status = 1;
    abort_ = true;
  } else {
    Hs = (S->H == 0.0) ? P.q_first * U0 * dt : fabs(S->H) * (dt < 0 ? -1.0 : 1.0);
    if (fabs(Hs / U0) >= fabs(dt)) {
      Hs = U0 * dt;
      if (S->halvings == 0) {
        if (S->time_iters >= P.max_time_iter) {
          S->status = 2;
          abort_ = true;
        } else {
          S->time_iters++;
        }
      }
    }
  }
  *Hs_out = Hs;
  return abort_;
}

// Sec. 2.3 and Eq. hnext: accept (new H from eps, time of the extrapolated state) or halve H.
__device__ bool accept_or_halve(SysScalars* S, const BatchParams& P, int K, double eps, double H, double tkk_t) {
  S->eps = eps;
  S->force_evals += 2 * K * (K + 1) / 2 + 1;
  if (eps <= P.eta) {
    double fc = (eps > 0.0) ? P.a_gbs * pow(P.eta / eps, 1.0 / (2 * K - 1)) : P.fac_max;
    fc = fmin(fmax(fc, P.fac_min), P.fac_max);
    S->H = fc * H;
    S->t = tkk_t;
    S->accepted++;
    S->halvings = 0;
    return true;
  }
  S->rejected++;
  S->H = 0.5 * H;
  if (++S->halvings > P.max_halvings) S->status = -3;
  return false;
}

// Per-system view of the batch storage: body-major blocks of 3-vectors (field f of body v
// at bd[f * n + 3 v + c]) and the integer tree arrays.
struct SysView {
  int n;
  const double* m;
  double* bd;
  int *parent, *gp, *coff, *cidx;  // coff: n + 1 entries, cidx: n - 1 entries
  int* bylev;                        // the bodies by tree level (ascending), then index
  __device__ __forceinline__ double* F(int field) const { return bd + (size_t)field * n; }
};

__device__ __forceinline__ SysView sys_view(int s, const int* __restrict__ off, const double* __restrict__ mass,
                                            double* body, int* ibody, int body_doubles) {
  SysView V;
  const int o = off[s];
  V.n = off[s + 1] - o;
  V.m = mass + o;
  V.bd = body + (size_t)o * body_doubles;
  int* ib = ibody + (size_t)o * 5;
  V.parent = ib;
  V.gp = ib + V.n;
  V.coff = ib + 2 * V.n;
  V.cidx = ib + 3 * V.n + 1;
  V.bylev = ib + 4 * V.n;
  return V;
}

// Start of an attempt, by a CTA of 128 G threads: the MST (Prim with exact FP64 keys) and
// its children lists, the edge coordinates of the step start, the derivative information
// (one force evaluation by group 0) and the step size. Leaves U0, T0, the attempt's H (Ha)
// and go = 0 (system stops) or 1 in S; the caller synchronises before reading them.
template <int G>
__device__ void attempt_begin(const SysView& V, SysScalars* S, const BatchParams& P, double t_end, WarpShared* wsh,
                              unsigned long long* rk, int* ri, int* s_cnt, int* s_lev, double (*s_gred)[kMaxG][3]) {
  constexpr int NT = 128 * G, NW = 4 * G, VPT = kBMaxN / NT;
  const int n = V.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const GI gi{warp / G, warp % G, lane, (warp % G) * 32 + lane};
  const double* m = V.m;
  double* R = V.F(B_R);
  double* Vs = V.F(B_V);
  double* X0 = V.F(B_X0);
  double* V0 = V.F(B_V0);
  double* A0 = V.F(B_A0);
  int* parent = V.parent;
  int* gp = V.gp;
  int* coff = V.coff;
  int* cidx = V.cidx;
  const double t0 = S->t;

  // ---- MST (Prim with exact FP64 keys, one CTA) and the children lists
  {
    unsigned long long key[VPT];
    bool intree[VPT];
    unsigned long long bk = ~0ull;
    int bi = INT_MAX;
    for (int q = 0; q < VPT; ++q) {
      const int v = tid + q * NT;
      intree[q] = v >= n;
      key[q] = 0x7ff0000000000000ull;
      if (v < n) {
        const double x = R[3 * v], y = R[3 * v + 1], z = R[3 * v + 2];
        const unsigned long long d = key_bits(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
        if (d < bk) {
          bk = d;
          bi = v;
        }
        parent[v] = -1;
      }
    }
    block_argmin<NW>(bk, bi, rk, ri);
    const int root = bi;
    for (int q = 0; q < VPT; ++q)
      if (tid + q * NT == root) intree[q] = true;
    int u = root;
    for (int it = 1; it < n; ++it) {
      bk = ~0ull;
      bi = INT_MAX;
      for (int q = 0; q < VPT; ++q) {
        if (intree[q]) continue;
        const int v = tid + q * NT;
        const double d = d2x(R, u, v);
        if (d < __longlong_as_double((long long)key[q])) {
          key[q] = key_bits(d);
          parent[v] = u;
        }
        if (key[q] < bk) {
          bk = key[q];
          bi = v;
        }
      }
      block_argmin<NW>(bk, bi, rk, ri);
      const int nxt = bi;
      if ((nxt % NT) == tid) {
        intree[nxt / NT] = true;
        if (parent[nxt] < 0) parent[nxt] = root;
      }
      u = nxt;
    }
    __syncthreads();
    // grandparents and children CSR (ascending child index)
    for (int v = tid; v <= n; v += NT) s_cnt[v] = 0;
    __syncthreads();
    for (int v = tid; v < n; v += NT) {
      const int p = parent[v];
      gp[v] = p >= 0 ? parent[p] : -1;
      if (p >= 0) atomicAdd(&s_cnt[p], 1);
    }
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int v = 0; v < n; ++v) {
        const int c = s_cnt[v];
        coff[v] = acc;
        s_cnt[v] = acc;
        acc += c;
      }
      coff[n] = acc;
      // n <= 512: a sequential fill keeps every list in ascending order
      for (int v = 0; v < n; ++v) {
        const int p = parent[v];
        if (p >= 0) cidx[s_cnt[p]++] = v;
      }
    }
    __syncthreads();
    // bodies by tree level (counting sort; ascending index within a level)
    for (int v = tid; v < n; v += NT) {
      int d = 0;
      for (int w = parent[v]; w >= 0; w = parent[w]) ++d;
      s_lev[v] = d;
    }
    for (int v = tid; v <= n; v += NT) s_cnt[v] = 0;
    __syncthreads();
    for (int v = tid; v < n; v += NT) atomicAdd(&s_cnt[s_lev[v]], 1);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int l = 0; l < n; ++l) {
        const int c = s_cnt[l];
        s_cnt[l] = acc;
        acc += c;
      }
      for (int v = 0; v < n; ++v) V.bylev[s_cnt[s_lev[v]]++] = v;
    }
    __syncthreads();
  }

  // ---- edge coordinates of the step start
  for (int v = tid; v < n; v += NT) {
    const int p = parent[v];
    for (int c = 0; c < 3; ++c) {
      X0[3 * v + c] = p >= 0 ? __dsub_rn(R[3 * v + c], R[3 * p + c]) : 0.0;
      V0[3 * v + c] = p >= 0 ? __dsub_rn(Vs[3 * v + c], Vs[3 * p + c]) : 0.0;
    }
  }
  __syncthreads();
  // ---- derivative information of the step start (group 0) and the step size
  if (gi.g == 0) {
    double* ga = V.F(B_GRP) + 12 * n;
    const double U0 = gforces<G>(n, P.n_d, P.G, m, parent, gp, coff, cidx, R, X0, ga, wsh[warp], gi, s_gred);
    double t2 = 0.0;
    for (int v = gi.t; v < n; v += 32 * G) {
      const double q0 = Vs[3 * v], q1 = Vs[3 * v + 1], q2 = Vs[3 * v + 2];
      t2 += __dmul_rn(m[v], __dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2)));
      const int p = parent[v];
      for (int c = 0; c < 3; ++c) A0[3 * v + c] = p >= 0 ? __dsub_rn(ga[3 * v + c], ga[3 * p + c]) : 0.0;
    }
    const double T0 = 0.5 * gsum1<G>(t2, gi, s_gred);
    if (gi.t == 0) {
      double Hs = 0.0;
      const bool abort_ = choose_step(S, P, t_end, t0, U0, &Hs);
      S->U0 = U0;
      S->T0 = T0;
      S->Ha = Hs;
      S->go = abort_ ? 0 : 1;
    }
  }
}

// The divisions of group gi.g (greedy longest-first assignment of the k_fix divisions to
// the four groups, Sec. 4.2), by the group's G warps with group-level barriers only.
template <int G>
__device__ void attempt_divisions(const SysView& V, const SysScalars* S, const BatchParams& P, const GI& gi,
                                  WarpShared& wsh, double (*s_gred)[kMaxG][3], double* tdiv_s) {
  const int n = V.n, K = P.k_fix;
  const double* m = V.m;
  const double* X0 = V.F(B_X0);
  const double* V0 = V.F(B_V0);
  const int* parent = V.parent;
  double* gX = V.F(B_GRP + gi.g * kGrpStride);
  double* gV = gX + 3 * n;
  double* gr = gX + 6 * n;
  double* gv = gX + 9 * n;
  double* ga = gX + 12 * n;
  const double t0 = S->t, B = S->B, Mtot = S->M, T0 = S->T0, H = S->Ha, rM = 1.0 / Mtot;
  int load[kGroups] = {0, 0, 0, 0};
  for (int k = K; k >= 1; --k) {
    int gsel = 0;
    for (int w = 1; w < kGroups; ++w)
      if (load[w] < load[gsel]) gsel = w;
    load[gsel] += 2 * k;
    if (gsel != gi.g) continue;
    const int nk = 2 * k;
    const double delta = H / (double)nk;
    double f = (0.5 * delta) / (T0 + B);
    for (int v = gi.t; v < n; v += 32 * G)
      for (int c = 0; c < 3; ++c) {
        gX[3 * v + c] = madd(X0[3 * v + c], f, V0[3 * v + c]);
        gV[3 * v + c] = V0[3 * v + c];
      }
    double t = t0 + f;
    gsync<G>(gi.g);
    grebuild<G>(n, m, parent, V.bylev, gX, gr, Mtot, rM, false, gi, s_gred);
    for (int tau = 1; tau <= nk; ++tau) {
      const double U = gforces<G>(n, P.n_d, P.G, m, parent, V.gp, V.coff, V.cidx, gr, gX, ga, wsh, gi, s_gred);
      const double fk = delta / U;
      for (int v = gi.t; v < n; v += 32 * G) {
        const int p = parent[v];
        if (p >= 0)
          for (int c = 0; c < 3; ++c) gV[3 * v + c] = madd(gV[3 * v + c], fk, __dsub_rn(ga[3 * v + c], ga[3 * p + c]));
      }
      gsync<G>(gi.g);
      const double T = 0.5 * grebuild<G>(n, m, parent, V.bylev, gV, gv, Mtot, rM, true, gi, s_gred);
      f = ((tau == nk) ? 0.5 * delta : delta) / (T + B);
      for (int v = gi.t; v < n; v += 32 * G)
        for (int c = 0; c < 3; ++c) gX[3 * v + c] = madd(gX[3 * v + c], f, gV[3 * v + c]);
      t += f;
      gsync<G>(gi.g);
      if (tau < nk) grebuild<G>(n, m, parent, V.bylev, gX, gr, Mtot, rM, false, gi, s_gred);
    }
    double* E = V.F(B_END + 6 * (k - 1));
    for (int v = gi.t; v < n; v += 32 * G)
      for (int c = 0; c < 3; ++c) {
        E[3 * v + c] = gX[3 * v + c];
        E[3 * n + 3 * v + c] = gV[3 * v + c];
      }
    if (gi.t == 0) tdiv_s[k - 1] = t;
    gsync<G>(gi.g);
  }
}

// End of an attempt, by a CTA of 128 G threads: Aitken-Neville extrapolation of the
// division end states, the error of Eq. gbs-criterion, the step control and, when the
// attempt is accepted, the deconstruction of the extrapolated edge vectors.
template <int G>
__device__ void attempt_finish(const SysView& V, SysScalars* S, const BatchParams& P, const double* tdiv_s,
                               double* s_red, int* s_flag, double (*s_gred)[kMaxG][3]) {
  constexpr int NT = 128 * G, NW = 4 * G;
  const int n = V.n, K = P.k_fix;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const GI gi{warp / G, warp % G, lane, (warp % G) * 32 + lane};
  const double* X0 = V.F(B_X0);
  const double* V0 = V.F(B_V0);
  const double* A0 = V.F(B_A0);
  double* TKK = V.F(B_TKK);
  const double t0 = S->t, B = S->B, Mtot = S->M;
  const double H = S->Ha, T0 = S->T0, U0 = S->U0;
  const double rate = 1.0 / (T0 + B), delta = H / (double)(2 * K);
  auto neville = [&](const double* Sv, double& tkk, double& tprev) {
    double prev[kMaxKfix], cur[kMaxKfix];
    for (int k = 0; k < K; ++k) {
      cur[0] = Sv[k];
      for (int j = 1; j <= k; ++j) cur[j] = fma(__dsub_rn(cur[j - 1], prev[j - 1]), c_bfac[k][j], cur[j - 1]);
      if (k == K - 2) tprev = cur[k];
      for (int j = 0; j <= k; ++j) prev[j] = cur[j];
    }
    tkk = prev[K - 1];
  };
  double e = 0.0;
  for (int v = tid; v < n; v += NT) {
    double Sv[kMaxKfix], dX[3], dV[3];
    for (int c = 0; c < 3; ++c) {
      double tkk, tp = 0.0;
      for (int k = 0; k < K; ++k) Sv[k] = V.F(B_END + 6 * k)[3 * v + c];
      neville(Sv, tkk, tp);
      TKK[3 * v + c] = tkk;
      dX[c] = __dsub_rn(tkk, tp);
      for (int k = 0; k < K; ++k) Sv[k] = V.F(B_END + 6 * k)[3 * n + 3 * v + c];
      neville(Sv, tkk, tp);
      TKK[3 * n + 3 * v + c] = tkk;
      dV[c] = __dsub_rn(tkk, tp);
    }
    if (V.parent[v] >= 0) {
      double q[3], g[3];
      for (int c = 0; c < 3; ++c) {
        q[c] = madd(X0[3 * v + c], delta, __dmul_rn(V0[3 * v + c], rate));
        g[c] = madd(V0[3 * v + c], delta, A0[3 * v + c] / U0);
      }
      auto nrm = [](const double* w) {
        return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(w[0], w[0]), __dmul_rn(w[1], w[1])), __dmul_rn(w[2], w[2])));
      };
      e = nanmax(e, nanmax(nrm(dX) / fmax(nrm(q), 1e-300), nrm(dV) / fmax(nrm(g), 1e-300)));
    }
  }
  double tkk_t = 0.0;
  if (tid == 0) {
    double Sv[kMaxKfix], tp = 0.0;
    for (int k = 0; k < K; ++k) Sv[k] = tdiv_s[k];
    neville(Sv, tkk_t, tp);
    e = nanmax(e, fabs(__dsub_rn(tkk_t, tp)) / fmax(fabs(madd(t0, delta, rate)), 1e-300));
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) e = nanmax(e, __shfl_xor_sync(0xffffffffu, e, o2));
  if (lane == 0) s_red[warp] = e;
  __syncthreads();
  if (tid == 0) {
    double eps = s_red[0];
    for (int w = 1; w < NW; ++w) eps = nanmax(eps, s_red[w]);
    *s_flag = accept_or_halve(S, P, K, eps, H, tkk_t) ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag == 0) return;
  // ---- accept: deconstruct the extrapolated edge vectors into the Cartesian state
  if (gi.g < 2) {
    double* dst = gi.g == 0 ? V.F(B_R) : V.F(B_V);
    const double* src = gi.g == 0 ? TKK : TKK + 3 * n;
    grebuild<G>(n, V.m, V.parent, V.bylev, src, dst, Mtot, 1.0 / Mtot, false, gi, s_gred);
  }
}

// All batched-step kernels take the same arguments, so that one argument list serves every
// node of the graph.
#define MSTAR_BSTEP_ARGS                                                                                    \
  int count, const int *__restrict__ order, const int *__restrict__ off, BatchParams P,                     \
      const double *__restrict__ tend, const double *__restrict__ mass, double *__restrict__ body,          \
      int *__restrict__ ibody, SysScalars *__restrict__ sys, double *__restrict__ tdiv

// One GBS step attempt for each of the `count` systems order[0 .. count-1], one CTA per
// system: the whole CTA starts the attempt, its four groups run the divisions, the whole CTA
// finishes it.
template <int G>
__global__ void __launch_bounds__(128 * G) k_batched_step(MSTAR_BSTEP_ARGS) {
  __shared__ WarpShared wsh[4 * G];
  __shared__ unsigned long long rk[4 * G];
  __shared__ int ri[4 * G];
  __shared__ int s_cnt[kBMaxN + 1];
  __shared__ int s_lev[kBMaxN];
  __shared__ double s_red[4 * G];
  __shared__ double s_gred[kGroups][kMaxG][3];
  __shared__ int s_flag;
  if ((int)blockIdx.x >= count) return;
  const int s = order[blockIdx.x];
  SysScalars* S = sys + s;
  if (S->status != 0) return;
  const SysView V = sys_view(s, off, mass, body, ibody, P.body_doubles);
  attempt_begin<G>(V, S, P, *tend, wsh, rk, ri, s_cnt, s_lev, s_gred);
  __syncthreads();
  if (S->go == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GI gi{warp / G, warp % G, lane, (warp % G) * 32 + lane};
  attempt_divisions<G>(V, S, P, gi, wsh[warp], s_gred, tdiv + (size_t)s * kMaxKfix);
  __syncthreads();
  attempt_finish<G>(V, S, P, tdiv + (size_t)s * kMaxKfix, s_red, &s_flag, s_gred);
}

// The same attempt as three graph nodes, so that one system's four division groups run as
// four CTAs (on up to four SMs) instead of one: the start (one CTA per system), the
// divisions (one CTA of G warps per system and group; CTA 4 i + g runs group g of system
// order[i]) and the finish (one CTA per system).
template <int G>
__global__ void __launch_bounds__(128 * G) k_bsplit_begin(MSTAR_BSTEP_ARGS) {
  __shared__ WarpShared wsh[4 * G];
  __shared__ unsigned long long rk[4 * G];
  __shared__ int ri[4 * G];
  __shared__ int s_cnt[kBMaxN + 1];
  __shared__ int s_lev[kBMaxN];
  __shared__ double s_gred[kGroups][kMaxG][3];
  if ((int)blockIdx.x >= count) return;
  const int s = order[blockIdx.x];
  SysScalars* S = sys + s;
  if (S->status != 0) return;
  const SysView V = sys_view(s, off, mass, body, ibody, P.body_doubles);
  attempt_begin<G>(V, S, P, *tend, wsh, rk, ri, s_cnt, s_lev, s_gred);
}

template <int G>
__global__ void __launch_bounds__(32 * G) k_bsplit_div(MSTAR_BSTEP_ARGS) {
  __shared__ WarpShared wsh[G];
  __shared__ double s_gred[kGroups][kMaxG][3];
  const int item = (int)(blockIdx.x >> 2), g = (int)(blockIdx.x & 3);
  if (item >= count) return;
  const int s = order[item];
  const SysScalars* S = sys + s;
  if (S->status != 0 || S->go == 0) return;
  const SysView V = sys_view(s, off, mass, body, ibody, P.body_doubles);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GI gi{g, warp, lane, warp * 32 + lane};
  attempt_divisions<G>(V, S, P, gi, wsh[warp], s_gred, tdiv + (size_t)s * kMaxKfix);
}

template <int G>
__global__ void __launch_bounds__(128 * G) k_bsplit_finish(MSTAR_BSTEP_ARGS) {
  __shared__ double s_red[4 * G];
  __shared__ double s_gred[kGroups][kMaxG][3];
  __shared__ int s_flag;
  if ((int)blockIdx.x >= count) return;
  const int s = order[blockIdx.x];
  SysScalars* S = sys + s;
  if (S->status != 0 || S->go == 0) return;
  const SysView V = sys_view(s, off, mass, body, ibody, P.body_doubles);
  attempt_finish<G>(V, S, P, tdiv + (size_t)s * kMaxKfix, s_red, &s_flag, s_gred);
}

// ---------------------------------------------------------------------------- segment schedules
//
// Systems of at most WD bodies (WD = 8: size class 0, WD = 16: class 1): one system per
// 4 x WD threads, four division groups of WD lanes, lane l of a group holding body l of
// the group's division state in registers. The pair loop is the symmetric rotation of the
// CTA schedules inside the group's lanes (partner (l + k) mod WD at step k, exchanged by
// shuffles, the partner's share returned to its lane the same way); near pairs take their
// separation from edge vectors; rebuilds sum edge vectors up the tree by shuffles.
constexpr int kSegThreads = 128;

template <int WD>
struct Seg {
  int g, l, base;       // group, lane in the group, first lane of the group within the warp
  unsigned mask;        // the group's lanes
  __device__ __forceinline__ double get(double x, int src) const { return __shfl_sync(mask, x, src, WD); }
  __device__ __forceinline__ int get(int x, int src) const { return __shfl_sync(mask, x, src, WD); }
  __device__ __forceinline__ double sum(double x) const {
    for (int o = WD / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, WD);
    return x;
  }
};

// Barrier over the 4 WD threads of one system (a warp, or named barrier 1 + system slot).
template <int WD>
__device__ __forceinline__ void sys_sync(int slot) {
  if constexpr (4 * WD == 32) {
    __syncwarp();
  } else if constexpr (4 * WD < 32) {  // two or more systems per warp: the system's lanes
    __syncwarp(((1u << (4 * WD)) - 1u) << ((threadIdx.x & 31) & ~(4 * WD - 1)));
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(4 * WD) : "memory");
  }
}

// Path sums of the edge vectors W up the tree (vertex first, root excluded), then the
// centre-of-mass shift; returns sum m |w|^2 of the group's bodies after the shift.
template <int WD>
__device__ double seg_rebuild(const Seg<WD>& sg, bool live, double mv, int par, int depth, const double W[3],
                              double w[3], double Mtot, double rM) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  int u = live ? sg.l : -1;
  for (int it = 0; it < depth; ++it) {  // depth: the tree's largest level
    const int su = u >= 0 ? u : 0;
    const double w0 = sg.get(W[0], su), w1 = sg.get(W[1], su), w2 = sg.get(W[2], su);
    const int pu = sg.get(par, su);
    if (u >= 0 && pu >= 0) {
      s0 = __dadd_rn(s0, w0);
      s1 = __dadd_rn(s1, w1);
      s2 = __dadd_rn(s2, w2);
    }
    u = (u >= 0) ? pu : -1;
  }
  const double c0 = quot(sg.sum(live ? __dmul_rn(mv, s0) : 0.0), Mtot, rM),
               c1 = quot(sg.sum(live ? __dmul_rn(mv, s1) : 0.0), Mtot, rM),
               c2 = quot(sg.sum(live ? __dmul_rn(mv, s2) : 0.0), Mtot, rM);
  w[0] = __dsub_rn(s0, c0);
  w[1] = __dsub_rn(s1, c1);
  w[2] = __dsub_rn(s2, c2);
  const double t2 =
      live ? __dmul_rn(mv, __dadd_rn(__dadd_rn(__dmul_rn(w[0], w[0]), __dmul_rn(w[1], w[1])), __dmul_rn(w[2], w[2])))
           : 0.0;
  return sg.sum(t2);
}

// The pair loop of one group: a (times G) of the lane's body and the return value U.
template <int WD>
__device__ double seg_forces(const Seg<WD>& sg, int n, int n_d, double Gc, double mv, int par, int gpar,
                             const double r[3], const double X[3], double a[3]) {
  const bool live = sg.l < n;
  const MassSplit ms = mass_split(live ? mv : 1.0);
  const double Xp0 = sg.get(X[0], par >= 0 ? par : 0), Xp1 = sg.get(X[1], par >= 0 ? par : 0),
               Xp2 = sg.get(X[2], par >= 0 ? par : 0);  // X of this body's parent
  const bool nd1 = n_d >= 1, nd2 = n_d >= 2;
  double ax = 0.0, ay = 0.0, az = 0.0, ui = 0.0;
  const int msh = (int)(ms.m >> 32), msl = (int)(ms.m & 0xffffffffu);
  for (int k = 1; k <= WD / 2; ++k) {
    const int jl = (sg.l + k) & (WD - 1);
    const double xj = sg.get(r[0], jl), yj = sg.get(r[1], jl), zj = sg.get(r[2], jl);
    const double Xj0 = sg.get(X[0], jl), Xj1 = sg.get(X[1], jl), Xj2 = sg.get(X[2], jl);
    const double Xpj0 = sg.get(Xp0, jl), Xpj1 = sg.get(Xp1, jl), Xpj2 = sg.get(Xp2, jl);
    const double mj = sg.get(mv, jl);
    const int pj = sg.get(par, jl), gj = sg.get(gpar, jl);
    const int mjh = sg.get(msh, jl), mjl = sg.get(msl, jl), mje = sg.get(ms.e, jl);
    const int i = sg.l, j = jl;
    const bool valid = live && j < n && !(k == WD / 2 && sg.l >= WD / 2);
    double dx, dy, dz;
    if (nd1 && par == j) {                 // j is the parent of i
      dx = -X[0]; dy = -X[1]; dz = -X[2];
    } else if (nd1 && pj == i) {           // i is the parent of j
      dx = Xj0; dy = Xj1; dz = Xj2;
    } else if (nd2 && gpar == j) {         // j is the grandparent of i
      dx = -(X[0] + Xp0); dy = -(X[1] + Xp1); dz = -(X[2] + Xp2);
    } else if (nd2 && gj == i) {           // i is the grandparent of j
      dx = Xj0 + Xpj0; dy = Xj1 + Xpj1; dz = Xj2 + Xpj2;
    } else if (nd2 && par >= 0 && par == pj) {  // siblings
      dx = Xj0 - X[0]; dy = Xj1 - X[1]; dz = Xj2 - X[2];
    } else {
      dx = xj - r[0]; dy = yj - r[1]; dz = zj - r[2];
    }
    double rinv = 0.0, sj = 0.0, si = 0.0;
    if (valid) {
      const MassSplit msj{((unsigned long long)(unsigned)mjh << 32) | (unsigned)mjl, mje};
      pair_scalars_int(dx, dy, dz, msj, ms, rinv, sj, si);
    }
    ax = fma(sj, dx, ax);
    ay = fma(sj, dy, ay);
    az = fma(sj, dz, az);
    ui = fma(valid ? mj : 0.0, rinv, ui);
    // the partner's share, -si d, goes back to its lane
    const int from = (sg.l - k) & (WD - 1);
    const double bx = sg.get(-si * dx, from), by = sg.get(-si * dy, from), bz = sg.get(-si * dz, from);
    ax += bx;
    ay += by;
    az += bz;
  }
  a[0] = Gc * ax;
  a[1] = Gc * ay;
  a[2] = Gc * az;
  return Gc * sg.sum(live ? mv * ui : 0.0);
}

template <int WD>
__global__ void __launch_bounds__(kSegThreads)
k_batched_seg(int count, const int* __restrict__ order, const int* __restrict__ off, BatchParams P,
              const double* __restrict__ tend, const double* __restrict__ mass, double* __restrict__ body,
              int* __restrict__ ibody, SysScalars* __restrict__ sys, double* __restrict__ tdiv) {
  constexpr int PER = kSegThreads / (4 * WD);  // systems per CTA
  __shared__ int s_par[PER][WD];
  __shared__ double s_E[PER][kMaxKfix][6][WD];
  __shared__ double s_T[PER][6][WD];
  __shared__ double s_t[PER][kMaxKfix];
  __shared__ double s_scal[PER][4];
  __shared__ double s_err[PER][4 * WD >= 32 ? 4 * WD / 32 : 1];
  __shared__ int s_dep[PER];
  const int slot = threadIdx.x / (4 * WD), lt = threadIdx.x % (4 * WD);
  Seg<WD> sg;
  sg.g = lt / WD;
  sg.l = lt % WD;
  sg.base = (threadIdx.x & 31) & ~(WD - 1);
  sg.mask = (WD == 32 ? 0xffffffffu : ((1u << WD) - 1u)) << sg.base;
  const int q = blockIdx.x * PER + slot;
  if (q >= count) return;  // whole systems leave together
  const int s = order[q];
  SysScalars* S = sys + s;
  if (S->status != 0) return;
  const double t_end = *tend;
  const int o = off[s], n = off[s + 1] - o;
  const int K = P.k_fix;
  const double* m = mass + o;
  double* bd = body + (size_t)o * P.body_doubles;
  double* Rg = bd + (size_t)B_R * n;
  double* Vg = bd + (size_t)B_V * n;
  const double t0 = S->t, B = S->B, Mtot = S->M, rM = 1.0 / Mtot;
  const int l = sg.l;
  const bool live = l < n;
  const double mv = live ? m[l] : 0.0;
  double R[3], Vs[3];
  for (int c = 0; c < 3; ++c) {
    R[c] = live ? Rg[3 * l + c] : 0.0;
    Vs[c] = live ? Vg[3 * l + c] : 0.0;
  }
  // ---- MST by one thread (Prim with exact keys, lowest index on ties)
  if (lt == 0) {
    unsigned long long key[WD];
    bool in[WD];
    int root = 0;
    unsigned long long best = ~0ull;
    for (int w = 0; w < n; ++w) {
      const double x = Rg[3 * w], y = Rg[3 * w + 1], z = Rg[3 * w + 2];
      const unsigned long long d = key_bits(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
      if (d < best) {
        best = d;
        root = w;
      }
      key[w] = 0x7ff0000000000000ull;
      in[w] = false;
      s_par[slot][w] = -1;
    }
    in[root] = true;
    int u = root;
    for (int it = 1; it < n; ++it) {
      int nx = -1;
      for (int w = 0; w < n; ++w) {
        if (in[w]) continue;
        const unsigned long long d = key_bits(d2x(Rg, u, w));
        if (d < key[w]) {
          key[w] = d;
          s_par[slot][w] = u;
        }
        if (nx < 0 || key[w] < key[nx]) nx = w;
      }
      in[nx] = true;
      if (s_par[slot][nx] < 0) s_par[slot][nx] = root;
      u = nx;
    }
    int dep = 0;
    for (int w = 0; w < n; ++w) {
      int d = 0;
      for (int x = s_par[slot][w]; x >= 0; x = s_par[slot][x]) ++d;
      dep = d > dep ? d : dep;
    }
    s_dep[slot] = dep;
  }
  sys_sync<WD>(slot);
  const int depth = s_dep[slot];
  const int par = live ? s_par[slot][l] : -3;
  const int gpar = par >= 0 ? s_par[slot][par] : (live ? -1 : -3);
  // ---- edge coordinates and derivative information of the step start (every group)
  double X0[3], V0[3], A0[3], a[3];
  for (int c = 0; c < 3; ++c) {
    const double Rp = sg.get(R[c], par >= 0 ? par : 0), Vp = sg.get(Vs[c], par >= 0 ? par : 0);
    X0[c] = par >= 0 ? __dsub_rn(R[c], Rp) : 0.0;
    V0[c] = par >= 0 ? __dsub_rn(Vs[c], Vp) : 0.0;
  }
  const double U0 = seg_forces<WD>(sg, n, P.n_d, P.G, mv, par, gpar, R, X0, a);
  for (int c = 0; c < 3; ++c) {
    const double ap = sg.get(a[c], par >= 0 ? par : 0);
    A0[c] = par >= 0 ? __dsub_rn(a[c], ap) : 0.0;
  }
  const double T0 = 0.5 * sg.sum(live ? __dmul_rn(mv, __dadd_rn(__dadd_rn(__dmul_rn(Vs[0], Vs[0]),
                                                                         __dmul_rn(Vs[1], Vs[1])),
                                                                __dmul_rn(Vs[2], Vs[2])))
                                      : 0.0);
  if (lt == 0) {
    double Hs = 0.0;
    const bool ab = choose_step(S, P, t_end, t0, U0, &Hs);
    s_scal[slot][0] = Hs;
    s_scal[slot][1] = ab ? 1.0 : 0.0;
  }
  sys_sync<WD>(slot);
  const double H = s_scal[slot][0];
  if (s_scal[slot][1] != 0.0) return;
  // ---- this group's divisions (greedy longest-first assignment to the four groups), run
  // as one sequence of substeps so that the four groups of a warp stay in step: a division
  // that ends is followed at once by the group's next one (its first half drift folded in)
  int mydiv[kMaxKfix], nmy = 0;
  int load[kGroups] = {0, 0, 0, 0};
  for (int k = K; k >= 1; --k) {
    int gsel = 0;
    for (int w = 1; w < kGroups; ++w)
      if (load[w] < load[gsel]) gsel = w;
    load[gsel] += 2 * k;
    if (gsel == sg.g) mydiv[nmy++] = k;
  }
  int steps = 0;
  for (int w = 0; w < kGroups; ++w) steps = load[w] > steps ? load[w] : steps;
  const int mine = load[sg.g];
  {
    int di = 0, k = mydiv[0], nk = 2 * k, sub = 0;
    double delta = H / (double)nk;
    double f = (0.5 * delta) / (T0 + B);
    double X[3], V[3], r[3], v[3];
    for (int c = 0; c < 3; ++c) {
      X[c] = madd(X0[c], f, V0[c]);
      V[c] = V0[c];
    }
    double t = t0 + f;
    seg_rebuild<WD>(sg, live, mv, par, depth, X, r, Mtot, rM);
    for (int step = 0; step < steps; ++step) {
      const bool active = step < mine;
      const double U = seg_forces<WD>(sg, n, P.n_d, P.G, mv, par, gpar, r, X, a);
      const double fk = delta / U;
      for (int c = 0; c < 3; ++c) {
        const double ap = sg.get(a[c], par >= 0 ? par : 0);
        if (par >= 0) V[c] = madd(V[c], fk, __dsub_rn(a[c], ap));
      }
      const double T = 0.5 * seg_rebuild<WD>(sg, live, mv, par, depth, V, v, Mtot, rM);
      const bool last = sub == nk - 1;
      f = (last ? 0.5 * delta : delta) / (T + B);
      for (int c = 0; c < 3; ++c) X[c] = madd(X[c], f, V[c]);
      t += f;
      if (active && last) {
        for (int c = 0; c < 3; ++c) {
          s_E[slot][k - 1][c][l] = X[c];
          s_E[slot][k - 1][3 + c][l] = V[c];
        }
        if (l == 0) s_t[slot][k - 1] = t;
      }
      if (last) {
        sub = 0;
        if (++di < nmy) {
          k = mydiv[di];
          nk = 2 * k;
          delta = H / (double)nk;
          f = (0.5 * delta) / (T0 + B);
          for (int c = 0; c < 3; ++c) {
            X[c] = madd(X0[c], f, V0[c]);
            V[c] = V0[c];
          }
          t = t0 + f;
        }
      } else {
        ++sub;
      }
      if (step + 1 < steps) seg_rebuild<WD>(sg, live, mv, par, depth, X, r, Mtot, rM);
    }
  }
  sys_sync<WD>(slot);
  // ---- Aitken-Neville extrapolation and the error of Eq. gbs-criterion: group 0 takes X,
  // group 1 takes V of its lane's body, group 2 (lane 0) takes t
  const double rate = 1.0 / (T0 + B), delta = H / (double)(2 * K);
  auto neville = [&](const double* Sv, double& tkk, double& tprev) {
    double prev[kMaxKfix], cur[kMaxKfix];
    for (int k = 0; k < K; ++k) {
      cur[0] = Sv[k];
      for (int j = 1; j <= k; ++j) cur[j] = fma(__dsub_rn(cur[j - 1], prev[j - 1]), c_bfac[k][j], cur[j - 1]);
      if (k == K - 2) tprev = cur[k];
      for (int j = 0; j <= k; ++j) prev[j] = cur[j];
    }
    tkk = prev[K - 1];
  };
  double e = 0.0, tkk_t = 0.0;
  auto nrm = [](const double* x) {
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x[0], x[0]), __dmul_rn(x[1], x[1])), __dmul_rn(x[2], x[2])));
  };
  if (sg.g < 2 && live) {
    double Sv[kMaxKfix], dd[3];
    for (int c = 0; c < 3; ++c) {
      double tkk, tp = 0.0;
      for (int k = 0; k < K; ++k) Sv[k] = s_E[slot][k][3 * sg.g + c][l];
      neville(Sv, tkk, tp);
      s_T[slot][3 * sg.g + c][l] = tkk;
      dd[c] = __dsub_rn(tkk, tp);
    }
    if (par >= 0) {
      double qv[3];
      for (int c = 0; c < 3; ++c)
        qv[c] = sg.g == 0 ? madd(X0[c], delta, __dmul_rn(V0[c], rate)) : madd(V0[c], delta, A0[c] / U0);
      e = nrm(dd) / fmax(nrm(qv), 1e-300);
    }
  }
  if (sg.g == 2 && l == 0) {
    double Sv[kMaxKfix], tp = 0.0;
    for (int k = 0; k < K; ++k) Sv[k] = s_t[slot][k];
    neville(Sv, tkk_t, tp);
    e = fabs(__dsub_rn(tkk_t, tp)) / fmax(fabs(madd(t0, delta, rate)), 1e-300);
    s_scal[slot][2] = tkk_t;
  }
  if constexpr (4 * WD >= 32) {
    for (int o = 16; o > 0; o >>= 1) e = nanmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) s_err[slot][lt / 32] = e;
  } else {  // the system's 4 WD lanes of a shared warp
    const unsigned smask = ((1u << (4 * WD)) - 1u) << ((threadIdx.x & 31) & ~(4 * WD - 1));
    for (int o = 2 * WD; o > 0; o >>= 1) e = nanmax(e, __shfl_xor_sync(smask, e, o));
    if (lt == 0) s_err[slot][0] = e;
  }
  sys_sync<WD>(slot);
  if (lt == 0) {
    double eps = s_err[slot][0];
    for (int w = 1; w < 4 * WD / 32; ++w) eps = nanmax(eps, s_err[slot][w]);
    s_scal[slot][3] = accept_or_halve(S, P, K, eps, H, s_scal[slot][2]) ? 1.0 : 0.0;
  }
  sys_sync<WD>(slot);
  if (s_scal[slot][3] == 0.0) return;
  // ---- accept: deconstruct the extrapolated edge vectors into the Cartesian state
  if (sg.g < 2) {
    double W[3], w[3];
    for (int c = 0; c < 3; ++c) W[c] = live ? s_T[slot][3 * sg.g + c][l] : 0.0;
    seg_rebuild<WD>(sg, live, mv, par, depth, W, w, Mtot, rM);
    if (live)
      for (int c = 0; c < 3; ++c) (sg.g ? Vg : Rg)[3 * l + c] = w[c];
  }
}

// Initial COM shift, B = U - T and M per system (one warp each).
__global__ void __launch_bounds__(32)
k_batched_init(int nsys, const int* __restrict__ off, BatchParams P, const double* __restrict__ mass,
               double* __restrict__ body, int* __restrict__ ibody, SysScalars* __restrict__ sys) {
  __shared__ WarpShared wsh;
  const int s = blockIdx.x;
  const int o = off[s], n = off[s + 1] - o;
  const int lane = threadIdx.x;
  const GI gi{0, 0, lane, lane};
  const double* m = mass + o;
  double* bd = body + (size_t)o * P.body_doubles;
  double* R = bd + (size_t)B_R * n;
  double* Vs = bd + (size_t)B_V * n;
  double M = 0.0;
  if (lane == 0)
    for (int v = 0; v < n; ++v) M += m[v];
  M = __shfl_sync(0xffffffffu, M, 0);
  for (int w = 0; w < 2; ++w) {
    double* q = w == 0 ? R : Vs;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    for (int v = lane; v < n; v += 32) {
      c0 += __dmul_rn(m[v], q[3 * v]);
      c1 += __dmul_rn(m[v], q[3 * v + 1]);
      c2 += __dmul_rn(m[v], q[3 * v + 2]);
    }
    c0 = warp_sum(c0) / M;
    c1 = warp_sum(c1) / M;
    c2 = warp_sum(c2) / M;
    for (int v = lane; v < n; v += 32) {
      q[3 * v] = __dsub_rn(q[3 * v], c0);
      q[3 * v + 1] = __dsub_rn(q[3 * v + 1], c1);
      q[3 * v + 2] = __dsub_rn(q[3 * v + 2], c2);
    }
    __syncwarp();
  }
  // U with every pair Cartesian (Eq. 1), T
  int* ib = ibody + (size_t)o * 5;
  double* a = bd + (size_t)B_GRP * n + 12 * (size_t)n;
  const double U = gforces<1>(n, 0, P.G, m, ib, ib + n, ib + 2 * n, ib + 3 * n + 1, R, R, a, wsh, gi, nullptr);
  double t2 = 0.0;
  for (int v = lane; v < n; v += 32) {
    const double q0 = Vs[3 * v], q1 = Vs[3 * v + 1], q2 = Vs[3 * v + 2];
    t2 += __dmul_rn(m[v], __dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2)));
  }
  const double T = 0.5 * warp_sum(t2);
  if (lane == 0) {
    SysScalars& S = sys[s];
    S.M = M;
    S.B = U - T;
  }
}

}  // namespace
}  // namespace mstar

using mstar::SysScalars;
using mstar::BatchParams;
using mstar::kBodyDoublesBase;
using mstar::kMaxKfix;
using mstar::kBMaxN;
using mstar::kNumClasses;
using mstar::B_R;
using mstar::B_V;

static_assert(kNumClasses == MSTAR_BATCH_NUM_CLASSES, "size classes of the schedule table");
static_assert(kBMaxN == MSTAR_BATCH_MAX_N, "largest system of a batch");

struct mstar_batch {
  int nsys = 0, nbody = 0;
  mstar_params p{};
  cudaStream_t stream = nullptr;
  bool own_ws = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int *off = nullptr, *order = nullptr, *ibody = nullptr;
  double *mass = nullptr, *body = nullptr, *tdiv = nullptr, *stage = nullptr, *tend = nullptr;
  SysScalars* sys = nullptr;
  BatchParams bp{};
  std::vector<int> off_h;
  long long launches = 0;
  // schedule: warps per division group for each size class, the systems of each schedule
  // (largest first) as consecutive segments of `order`, and the graph of one launch
  int sched[kNumClasses] = {};
  // node kinds: one CTA per system with G = 1, 2, 4; the 8- and 16-lane segment kernels; the
  // split attempt (start, divisions, finish) with G = 1, 2, 4
  int seg_begin[9] = {}, seg_count[9] = {};
  cudaGraphExec_t exec = nullptr;
  int graph_nodes = 0;
  double tend_h = NAN;
};

namespace mstar_batch_detail {

struct BCarve {
  char* base;
  size_t off = 0;
  explicit BCarve(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

size_t bcarve(int nsys, int nbody, int K, void* base, mstar_batch* b) {
  BCarve c(base);
  const int bdbl = kBodyDoublesBase + 6 * K;
  int* off = c.take<int>(nsys + 1);
  int* order = c.take<int>(nsys);
  int* ibody = c.take<int>((size_t)nbody * 5);
  double* mass = c.take<double>(nbody);
  double* body = c.take<double>((size_t)nbody * bdbl);
  double* tdiv = c.take<double>((size_t)nsys * kMaxKfix);
  double* stage = c.take<double>((size_t)nbody * 3);
  SysScalars* sys = c.take<SysScalars>(nsys);
  double* tend = c.take<double>(1);
  if (b) {
    b->off = off;
    b->order = order;
    b->ibody = ibody;
    b->mass = mass;
    b->body = body;
    b->tdiv = tdiv;
    b->stage = stage;
    b->sys = sys;
    b->tend = tend;
  }
  return (c.off + 255) & ~size_t(255);
}

bool batch_sizes_ok(int nsys, const int* off, int* nbody) {
  if (nsys < 1 || !off || off[0] != 0) return false;
  for (int s = 0; s < nsys; ++s) {
    const int n = off[s + 1] - off[s];
    if (n < 2 || n > kBMaxN) return false;
  }
  *nbody = off[nsys];
  return true;
}

__global__ void k_scatter_vec(int nbody, const int* __restrict__ off, int nsys, int bdbl, int field,
                              const double* __restrict__ src, double* __restrict__ body, int to_body) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbody) return;
  int lo = 0, hi = nsys;  // system of body i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  const int o = off[lo], n = off[lo + 1] - o, v = i - o;
  double* dst = body + (size_t)o * bdbl + (size_t)field * n + 3 * v;
  for (int c = 0; c < 3; ++c) {
    if (to_body) dst[c] = src[3 * (size_t)i + c];
    else const_cast<double*>(src)[3 * (size_t)i + c] = dst[c];
  }
}

// Schedule values: 1, 2, 4 warps per division group (one CTA per system); -1, -2, -4 for the
// same groups with the attempt split into three nodes (one CTA per division group); 0 for
// the size classes of at most 16 bodies: groups of 8 (class 0; 4 for systems of at most 4
// bodies) or 16 (class 1) lanes, one body per lane. Node kind: 0, 1, 2 for G = 1, 2, 4; 3
// and 4 for the 8- and 16-lane kernels; 5, 6, 7 for the split attempt with G = 1, 2, 4; 8
// for the 4-lane kernel.
constexpr int kNodeKinds = 9;
int sched_index(int cls, int G) {
  if (G == 0) return cls == 0 ? 3 : (cls == 1 ? 4 : -1);
  if (G < 0) return G == -1 ? 5 : (G == -2 ? 6 : (G == -4 ? 7 : -1));
  return G == 1 ? 0 : (G == 2 ? 1 : (G == 4 ? 2 : -1));
}
bool sched_ok(int cls, int G) { return sched_index(cls, G) >= 0; }

// Warps per division group by size class before any tuning: wider groups for larger systems.
void default_schedule(int* sched) {
  static const int d[kNumClasses] = {0, 0, 1, 1, 1, 2, 4};
  for (int c = 0; c < kNumClasses; ++c) sched[c] = d[c];
}

void destroy_graph(mstar_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_nodes = 0;
}

// Order the systems by node kind, largest pair work first within a kind, upload the order
// and build the graph: one independent kernel node per nonempty kind (a chain of three for
// the split attempt), the widest groups at the highest priority.
int apply_schedule(mstar_batch* b, const int* sched) {
  for (int c = 0; c < kNumClasses; ++c)
    if (!sched_ok(c, sched[c])) return MSTAR_ERR_INVALID_ARG;
  std::vector<int> ord(b->nsys);
  for (int s = 0; s < b->nsys; ++s) ord[s] = s;
  auto n_of = [&](int s) { return b->off_h[s + 1] - b->off_h[s]; };
  auto g_of = [&](int s) {
    const int c = mstar::size_class(n_of(s));
    const int k = sched_index(c, sched[c]);
    return (k == 3 && n_of(s) <= 4) ? 8 : k;  // the 4-lane kernel for systems of at most 4 bodies
  };
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const int gx = g_of(x), gy = g_of(y);
    if (gx != gy) return gx < gy;
    return (long long)n_of(x) * n_of(x) > (long long)n_of(y) * n_of(y);
  });
  int begin[kNodeKinds] = {}, count[kNodeKinds] = {};
  for (int s = 0; s < b->nsys; ++s) count[g_of(s)]++;
  for (int q = 1; q < kNodeKinds; ++q) begin[q] = begin[q - 1] + count[q - 1];
  if (cudaMemcpyAsync(b->order, ord.data(), sizeof(int) * b->nsys, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return MSTAR_ERR_CUDA;
  destroy_graph(b);
  cudaGraph_t graph = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return MSTAR_ERR_CUDA;
  int lo_prio = 0, hi_prio = 0;
  cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  bool ok = true;
  int nodes = 0;
  static const int node_order[kNodeKinds] = {7, 2, 6, 1, 5, 0, 4, 3, 8};  // widest groups first
  auto add_node = [&](void* func, dim3 grid, dim3 block, void** args, const cudaGraphNode_t* dep, int prio,
                      cudaGraphNode_t* node) {
    cudaKernelNodeParams kp{};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &kp) != cudaSuccess) return false;
    cudaLaunchAttributeValue pv{};
    pv.priority = prio;
    cudaGraphKernelNodeSetAttribute(*node, cudaLaunchAttributePriority, &pv);  // a hint; failure is harmless
    nodes++;
    return true;
  };
  for (int t = 0; t < kNodeKinds && ok; ++t) {
    const int qi = node_order[t];
    if (!count[qi]) continue;
    int cnt = count[qi];
    const int* ordp = b->order + begin[qi];
    void* args[] = {&cnt, (void*)&ordp, (void*)&b->off, (void*)&b->bp, (void*)&b->tend, (void*)&b->mass,
                    (void*)&b->body, (void*)&b->ibody, (void*)&b->sys, (void*)&b->tdiv};
    const int G = qi >= 5 ? 1 << (qi - 5) : 1 << qi;  // warps per division group (not used for 3, 4)
    const int prio = G == 4 ? hi_prio : (G == 2 ? (hi_prio + lo_prio) / 2 : lo_prio);
    cudaGraphNode_t n0, n1, n2;
    if (qi == 3 || qi == 4 || qi == 8) {
      const int wd = qi == 8 ? 4 : (qi == 3 ? 8 : 16);
      const int per = mstar::kSegThreads / (4 * wd);
      void* f = qi == 8 ? (void*)mstar::k_batched_seg<4>
                        : (qi == 3 ? (void*)mstar::k_batched_seg<8> : (void*)mstar::k_batched_seg<16>);
      ok = add_node(f, dim3((cnt + per - 1) / per), dim3(mstar::kSegThreads), args, nullptr, lo_prio, &n0);
    } else if (qi < 3) {
      void* f = G == 1 ? (void*)mstar::k_batched_step<1> : (G == 2 ? (void*)mstar::k_batched_step<2>
                                                                   : (void*)mstar::k_batched_step<4>);
      ok = add_node(f, dim3(cnt), dim3(128 * G), args, nullptr, prio, &n0);
    } else {
      void* fb = G == 1 ? (void*)mstar::k_bsplit_begin<1> : (G == 2 ? (void*)mstar::k_bsplit_begin<2>
                                                                    : (void*)mstar::k_bsplit_begin<4>);
      void* fd = G == 1 ? (void*)mstar::k_bsplit_div<1> : (G == 2 ? (void*)mstar::k_bsplit_div<2>
                                                                  : (void*)mstar::k_bsplit_div<4>);
      void* ff = G == 1 ? (void*)mstar::k_bsplit_finish<1> : (G == 2 ? (void*)mstar::k_bsplit_finish<2>
                                                                     : (void*)mstar::k_bsplit_finish<4>);
      ok = add_node(fb, dim3(cnt), dim3(128 * G), args, nullptr, prio, &n0) &&
           add_node(fd, dim3(4 * cnt), dim3(32 * G), args, &n0, prio, &n1) &&
           add_node(ff, dim3(cnt), dim3(128 * G), args, &n1, prio, &n2);
    }
  }
  cudaGetLastError();
  if (ok) ok = cudaGraphInstantiate(&b->exec, graph, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
  cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    b->exec = nullptr;
    return MSTAR_ERR_CUDA;
  }
  b->graph_nodes = nodes;
  for (int c = 0; c < kNumClasses; ++c) b->sched[c] = sched[c];
  for (int q = 0; q < kNodeKinds; ++q) {
    b->seg_begin[q] = begin[q];
    b->seg_count[q] = count[q];
  }
  return MSTAR_OK;
}

int set_tend(mstar_batch* b, double t_end) {
  if (b->tend_h == t_end) return MSTAR_OK;
  b->tend_h = t_end;
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  return cudaMemcpyAsync(b->tend, &b->tend_h, sizeof(double), cudaMemcpyHostToDevice, b->stream) == cudaSuccess
             ? MSTAR_OK
             : MSTAR_ERR_CUDA;
}

int launch_graph(mstar_batch* b, int launches) {
  for (int l = 0; l < launches; ++l) {
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
    b->launches += b->graph_nodes;
  }
  return MSTAR_OK;
}

}  // namespace mstar_batch_detail

using namespace mstar_batch_detail;

extern "C" {

size_t mstar_batch_workspace_bytes(int nsys, const int* offsets, const mstar_params* p) {
  mstar_params d;
  if (!p) {
    mstar_default_params(&d);
    p = &d;
  }
  int nbody = 0;
  if (!batch_sizes_ok(nsys, offsets, &nbody) || p->k_fix < 2 || p->k_fix > kMaxKfix) return 0;
  return bcarve(nsys, nbody, p->k_fix, nullptr, nullptr);
}

void mstar_batch_free(mstar_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  destroy_graph(b);
  if (b->own_ws && b->ws) cudaFree(b->ws);
  delete b;
}

int mstar_batch_init(mstar_batch** out, int nsys, const int* offsets, const double* m, const double* r,
                     const double* v, const mstar_params* p, void* workspace, size_t workspace_bytes,
                     void* cuda_stream) {
  if (!out) return MSTAR_ERR_INVALID_ARG;
  *out = nullptr;
  mstar_params pd;
  if (!p) {
    mstar_default_params(&pd);
    p = &pd;
  }
  int nbody = 0;
  if (!offsets || !m || !r || !v) return MSTAR_ERR_INVALID_ARG;
  if (nsys < 1 || offsets[0] != 0) return MSTAR_ERR_INVALID_ARG;
  for (int s = 0; s < nsys; ++s)
    if (offsets[s + 1] - offsets[s] > kBMaxN) return MSTAR_ERR_UNSUPPORTED;
  if (!batch_sizes_ok(nsys, offsets, &nbody)) return MSTAR_ERR_INVALID_ARG;
  if (p->k_fix < 2 || p->k_fix > kMaxKfix || p->n_d < 0 || p->n_d > 2 || !(p->eta_gbs > 0.0) ||
      !(p->G > 0.0) || !(p->a_gbs > 0.0 && p->a_gbs <= 1.0) || !(p->fac_min > 0.0 && p->fac_min <= p->fac_max))
    return MSTAR_ERR_INVALID_ARG;
  mstar_batch* b = new (std::nothrow) mstar_batch();
  if (!b) return MSTAR_ERR_NOMEM;
  b->nsys = nsys;
  b->nbody = nbody;
  b->p = *p;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t need = bcarve(nsys, nbody, p->k_fix, nullptr, nullptr);
  if (workspace) {
    if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
      delete b;
      return MSTAR_ERR_NOMEM;
    }
    b->ws = workspace;
  } else {
    if (cudaMalloc(&b->ws, need) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return MSTAR_ERR_NOMEM;
    }
    b->own_ws = true;
  }
  b->ws_bytes = need;
  bcarve(nsys, nbody, p->k_fix, b->ws, b);
  b->bp = BatchParams{p->eta_gbs, p->a_gbs, p->fac_min, p->fac_max, p->q_first, p->t_tol, p->G,
                      p->k_fix, p->n_d, p->max_halvings, p->max_time_iter, kBodyDoublesBase + 6 * p->k_fix};
  b->off_h.assign(offsets, offsets + nsys + 1);
  // host-side validation of the inputs (copied to the host when they live on the device)
  std::vector<double> mh(nbody), rh(3 * (size_t)nbody), vh(3 * (size_t)nbody);
  auto fetch = [&](double* dst, const double* src, size_t count) {
    return cudaMemcpy(dst, src, sizeof(double) * count, cudaMemcpyDefault) == cudaSuccess;
  };
  if (!fetch(mh.data(), m, nbody) || !fetch(rh.data(), r, 3 * (size_t)nbody) || !fetch(vh.data(), v, 3 * (size_t)nbody)) {
    mstar_batch_free(b);
    return MSTAR_ERR_CUDA;
  }
  for (int i = 0; i < nbody; ++i) {
    if (!std::isfinite(mh[i])) { mstar_batch_free(b); return MSTAR_ERR_NONFINITE; }
    if (!(mh[i] > 0.0)) { mstar_batch_free(b); return MSTAR_ERR_INVALID_ARG; }
    for (int c = 0; c < 3; ++c) {
      if (!std::isfinite(rh[3 * i + c]) || !std::isfinite(vh[3 * i + c])) { mstar_batch_free(b); return MSTAR_ERR_NONFINITE; }
      if (std::fabs(rh[3 * i + c]) >= 1e15) { mstar_batch_free(b); return MSTAR_ERR_UNSUPPORTED; }
    }
  }
  cudaStream_t st = b->stream;
  double fac[kMaxKfix][kMaxKfix] = {};
  for (int k = 0; k < p->k_fix; ++k)
    for (int j = 1; j <= k; ++j) {
      const double ratio = (double)(2 * (k + 1)) / (double)(2 * (k - j + 1));
      fac[k][j] = 1.0 / (ratio * ratio - 1.0);
    }
  bool ok = cudaMemcpyToSymbol(mstar::c_bfac, fac, sizeof(fac)) == cudaSuccess &&
            cudaMemsetAsync(b->ws, 0, need, st) == cudaSuccess &&
            cudaMemcpyAsync(b->off, offsets, sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(b->mass, mh.data(), sizeof(double) * nbody, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(b->stage, rh.data(), sizeof(double) * 3 * nbody, cudaMemcpyHostToDevice, st) == cudaSuccess;
  const int nb = (nbody + 255) / 256;
  if (ok) {
    k_scatter_vec<<<nb, 256, 0, st>>>(nbody, b->off, nsys, b->bp.body_doubles, B_R, b->stage, b->body, 1);
    ok = cudaMemcpyAsync(b->stage, vh.data(), sizeof(double) * 3 * nbody, cudaMemcpyHostToDevice, st) == cudaSuccess;
  }
  if (ok) {
    k_scatter_vec<<<nb, 256, 0, st>>>(nbody, b->off, nsys, b->bp.body_doubles, B_V, b->stage, b->body, 1);
    mstar::k_batched_init<<<nsys, 32, 0, st>>>(nsys, b->off, b->bp, b->mass, b->body, b->ibody, b->sys);
    b->launches += 3;
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  }
  if (!ok) {
    mstar_batch_free(b);
    return MSTAR_ERR_CUDA;
  }
  int sched[kNumClasses];
  default_schedule(sched);
  const int rc = apply_schedule(b, sched);
  if (rc) {
    mstar_batch_free(b);
    return rc;
  }
  *out = b;
  return MSTAR_OK;
}

int mstar_step_batched(mstar_batch* b, double t_end, int launches, mstar_batch_stats* out) {
  if (!b || !std::isfinite(t_end) || launches < 0) return MSTAR_ERR_INVALID_ARG;
  int rc = set_tend(b, t_end);
  if (!rc) rc = launch_graph(b, launches);
  if (rc) return rc;
  if (out) {
    std::vector<SysScalars> h(b->nsys);
    if (cudaMemcpyAsync(h.data(), b->sys, sizeof(SysScalars) * b->nsys, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return MSTAR_ERR_CUDA;
    mstar_batch_stats st{};
    for (const auto& s : h) {
      st.accepted += s.accepted;
      st.rejected += s.rejected;
      st.force_evals += s.force_evals;
      if (s.status != 0) st.finished++;
      if (s.status < 0) st.failed++;
    }
    *out = st;
  } else if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    return MSTAR_ERR_CUDA;
  }
  return MSTAR_OK;
}

int mstar_batch_set_schedule(mstar_batch* b, const int* schedule) {
  if (!b || !schedule) return MSTAR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
  return apply_schedule(b, schedule);
}

int mstar_batch_get_schedule(const mstar_batch* b, int* schedule) {
  if (!b || !schedule) return MSTAR_ERR_INVALID_ARG;
  for (int c = 0; c < kNumClasses; ++c) schedule[c] = b->sched[c];
  return MSTAR_OK;
}

int mstar_batch_autotune(mstar_batch* b, double t_end, int repeats, int* schedule_out, double* ms_out) {
  if (!b || !std::isfinite(t_end) || repeats < 1) return MSTAR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
  // the trials run on the real state: snapshot the workspace and put it back before each
  void* snap = nullptr;
  if (cudaMalloc(&snap, b->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    return MSTAR_ERR_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MSTAR_OK;
  const double tend_saved = b->tend_h;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemcpyAsync(snap, b->ws, b->ws_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
    rc = MSTAR_ERR_CUDA;
  auto restore = [&]() {
    return cudaMemcpyAsync(b->ws, snap, b->ws_bytes, cudaMemcpyDeviceToDevice, b->stream) == cudaSuccess &&
                   cudaStreamSynchronize(b->stream) == cudaSuccess
               ? MSTAR_OK
               : MSTAR_ERR_CUDA;
  };
  // time of one graph launch under schedule `sc` (the order segments are re-uploaded after
  // each restore, since the snapshot holds the order of the schedule current at the call)
  auto trial = [&](const int* sc, double* ms) {
    double best = INFINITY;
    for (int r = 0; r <= repeats; ++r) {  // r = 0 warms up (module load, caches)
      int q = restore();
      if (!q) q = apply_schedule(b, sc);
      b->tend_h = NAN;
      if (!q) q = set_tend(b, t_end);
      if (q) return q;
      if (cudaEventRecord(e0, b->stream) != cudaSuccess) return (int)MSTAR_ERR_CUDA;
      if ((q = launch_graph(b, 1))) return q;
      if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        return (int)MSTAR_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) best = std::min(best, (double)t);
    }
    *ms = best;
    return (int)MSTAR_OK;
  };
  int present[kNumClasses] = {};
  for (int s = 0; s < b->nsys; ++s) present[mstar::size_class(b->off_h[s + 1] - b->off_h[s])] = 1;
  int cur[kNumClasses];
  for (int c = 0; c < kNumClasses; ++c) cur[c] = b->sched[c];
  double cur_ms = 0.0;
  if (!rc) rc = trial(cur, &cur_ms);
  // two passes of coordinate descent, largest class first: each class keeps the schedule
  // that gave the shortest launch with the other classes fixed
  static const int widths[7] = {1, 2, 4, 0, -1, -2, -4};
  for (int pass = 0; pass < 2 * kNumClasses && !rc; ++pass) {
    const int c = kNumClasses - 1 - pass % kNumClasses;
    if (!present[c]) continue;
    for (int q = 0; q < 7 && !rc; ++q) {
      if (widths[q] == cur[c] || !sched_ok(c, widths[q])) continue;
      int cand[kNumClasses];
      for (int x = 0; x < kNumClasses; ++x) cand[x] = cur[x];
      cand[c] = widths[q];
      double ms = 0.0;
      rc = trial(cand, &ms);
      if (!rc && ms < cur_ms) {
        cur_ms = ms;
        cur[c] = widths[q];
      }
    }
  }
  if (!rc) rc = restore();
  if (!rc) rc = apply_schedule(b, cur);
  b->tend_h = NAN;
  if (!rc && std::isfinite(tend_saved)) rc = set_tend(b, tend_saved);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(snap);
  if (rc) return rc;
  if (schedule_out)
    for (int c = 0; c < kNumClasses; ++c) schedule_out[c] = cur[c];
  if (ms_out) *ms_out = cur_ms;
  return MSTAR_OK;
}

int mstar_batch_get_state(mstar_batch* b, double* t, double* r, double* v, double* eps, int* status) {
  if (!b) return MSTAR_ERR_INVALID_ARG;
  std::vector<SysScalars> h(b->nsys);
  if (cudaMemcpyAsync(h.data(), b->sys, sizeof(SysScalars) * b->nsys, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return MSTAR_ERR_CUDA;
  const int nb = (b->nbody + 255) / 256;
  for (int w = 0; w < 2; ++w) {
    double* dst = w == 0 ? r : v;
    if (!dst) continue;
    k_scatter_vec<<<nb, 256, 0, b->stream>>>(b->nbody, b->off, b->nsys, b->bp.body_doubles, w == 0 ? B_R : B_V,
                                             b->stage, b->body, 0);
    b->launches++;
    if (cudaMemcpyAsync(dst, b->stage, sizeof(double) * 3 * b->nbody, cudaMemcpyDefault, b->stream) != cudaSuccess)
      return MSTAR_ERR_CUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
  for (int s = 0; s < b->nsys; ++s) {
    if (t) t[s] = h[s].t;
    if (eps) eps[s] = h[s].eps;
    if (status) status[s] = h[s].status;
  }
  return MSTAR_OK;
}

int mstar_batch_set_H(mstar_batch* b, const double* H) {
  if (!b || !H) return MSTAR_ERR_INVALID_ARG;
  std::vector<SysScalars> h(b->nsys);
  if (cudaMemcpyAsync(h.data(), b->sys, sizeof(SysScalars) * b->nsys, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return MSTAR_ERR_CUDA;
  for (int s = 0; s < b->nsys; ++s) h[s].H = H[s];
  if (cudaMemcpyAsync(b->sys, h.data(), sizeof(SysScalars) * b->nsys, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return MSTAR_ERR_CUDA;
  return MSTAR_OK;
}

long long mstar_batch_launch_count(const mstar_batch* b) { return b ? b->launches : 0; }

}  // extern "C"
