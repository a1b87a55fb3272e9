// Device helpers shared by the libmstar kernels.
//
// GB300 executes FP64 instructions at about 1/75 of the FP32 rate (about 500 G FP64
// instructions/s over the chip), and double<->float conversions cost as much as an FP64
// instruction. The helpers here therefore build FP32 seeds with integer bit operations
// and keep every non-essential operation off the FP64 pipe.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mstar {

// float from the leading bits of a normal double, or 0 when the magnitude is below the
// float range. Truncates the mantissa (relative error < 2^-20); integer pipe only.
__device__ __forceinline__ float approx_float_of(double x) {
  int hi = __double2hiint(x);
  int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  unsigned m = ((unsigned)hi & 0xfffffu) << 3;
  unsigned bits = ((unsigned)hi & 0x80000000u) | ((unsigned)e << 23) | m;
  return (e > 0 && e < 255) ? __uint_as_float(bits) : 0.0f;
}

// Exact double of a normal, non-negative float (0 for zero/subnormal); integer pipe only.
__device__ __forceinline__ double double_of_nonneg_float(float f) {
  unsigned b = __float_as_uint(f);
  int e = (int)((b >> 23) & 0xff);
  unsigned m = b & 0x7fffffu;
  int hi = ((e - 127 + 1023) << 20) | (int)(m >> 3);
  unsigned lo = m << 29;
  return e > 0 ? __hiloint2double(hi, (int)lo) : 0.0;
}

// Upper-triangle tile pair tp -> (I, J), I <= J < NT, rows of length NT - I (the tiled pair
// loops: forces and their vector-Jacobian products).
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

// 1/sqrt(x) to double precision for a normal x > 0, with four FP64 instructions.
//
// Seed: x = 2^(2k) * mx with mx in [1, 4) assembled as a float from x's bits; CUDA's
// rsqrtf(mx) (relative error about 2^-23) is scaled back by 2^-k into an exact double y.
// Refinement: with e = 1 - x y^2 (exact enough from one FMA, since y^2 is exact), the
// binomial series gives x^(-1/2) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + O(e^3)).
// |e| < 2^-20, so the e^3 term is below 2^-62 and the e^2 term needs only float
// precision. x = 0 yields NaN (y^2 overflows), like 0 * (1/sqrt(0)) would.
__device__ __forceinline__ double rsqrt_fp64(double x) {
  int hi = __double2hiint(x);
  unsigned lo = (unsigned)__double2loint(x);
  int E = ((hi >> 20) & 0x7ff) - 1023;
  int k = E >> 1;                      // floor(E / 2)
  int fe = E - 2 * k;                  // 0 or 1
  unsigned mant = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
  float mx = __uint_as_float(((unsigned)(127 + fe) << 23) | mant);
  float yf = rsqrtf(mx);               // in (0.5, 1]
  unsigned yb = __float_as_uint(yf);
  int ye = (int)((yb >> 23) & 0xff) - 127 + 1023 - k;
  unsigned ym = yb & 0x7fffffu;
  double y = __hiloint2double((ye << 20) | (int)(ym >> 3), (int)(ym << 29));
  double y2 = y * y;                   // exact: y has 24 significant bits
  double e = fma(-x, y2, 1.0);
  float ef = approx_float_of(e);
  double c2 = double_of_nonneg_float(0.375f * ef * ef);
  double c = fma(0.5, e, c2);
  return fma(y, c, y);
}

// ---------------------------------------------------------------------------------------
// Pair scalars on the integer pipe.
//
// For a separation (dx, dy, dz) the pair loop needs 1/r and m/r^3. Evaluated with FP64
// instructions these cost 11 of the loop's 21 FP64 issue slots per pair, while the integer
// pipe (which runs beside the FP64 pipe at a far higher rate) sits idle. Here r^2, 1/r,
// 1/r^3 and the mass products are computed in exact 64-bit integer arithmetic on the
// binary64 significands:
//   r^2  = sum of the squared significands aligned to the largest exponent (62 bits kept);
//   1/r  = y (1 + e/2 + 3e^2/8) with y the float seed of the reciprocal square root and
//          e = 1 - r^2 y^2 formed exactly in 62-bit fixed point (|e| < 2^-20);
//   1/r^3, m/r^3 from 64-bit products of the normalised significands.
// Each result is rounded to the nearest double from about 60 correct bits, so it lies
// within one unit in the last place of the exact value (validated against 60-digit
// arithmetic for separations 1e-60 ... 1e12 and any component ratio). Valid while 1/r and
// m/r^3 are normal doubles.

struct MassSplit {  // mass = m * 2^e with m in [2^63, 2^64)
  unsigned long long m;
  int e;
};

__device__ __forceinline__ MassSplit mass_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return MassSplit{((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11, (int)((b >> 52) & 0x7ff) - 1075 - 11};
}

// Sn * 2^e2 with Sn in [2^63, 2^64) to the nearest double (halfway cases rounded up).
__device__ __forceinline__ double u64_to_double(unsigned long long Sn, int e2) {
  unsigned long long mant = (Sn >> 11) + ((Sn >> 10) & 1ull);
  int ex = e2 + 11;
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  return __longlong_as_double((long long)(((unsigned long long)(ex + 1075) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// (m^2 >> 42) >> sh for a significand m < 2^53.
__device__ __forceinline__ unsigned long long sq_top(unsigned long long m, int sh) {
  const unsigned long long hi = __umul64hi(m, m), lo = m * m;
  const unsigned long long T = (hi << 22) | (lo >> 42);
  return sh < 64 ? (T >> sh) : 0ull;
}

// Significand (with the hidden bit; 0 for zero/subnormal) and biased exponent of |x|, built
// from the two 32-bit halves so that no FP64 instruction is involved.
__device__ __forceinline__ unsigned long long sig_of(double x, int& e) {
  const unsigned hi = (unsigned)__double2hiint(x) & 0x7FFFFFFFu;
  const unsigned lo = (unsigned)__double2loint(x);
  e = (int)(hi >> 20);
  const unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  return e ? m : 0ull;
}

// The core of the pair scalars: 1/r as Rn 2^eR (Rn in [2^63, 2^64), about 60 correct bits)
// and the two mass scalings rounded to doubles. Coincident bodies (r = 0, force undefined)
// give Rn = 0 and NaN scalings.
__device__ __forceinline__ void pair_scalars_core(double dx, double dy, double dz, const MassSplit& mj,
                                                  const MassSplit& mi, unsigned long long& Rn_out, int& eR_out,
                                                  double& sj, double& si) {
  int ex, ey, ez;
  const unsigned long long mx = sig_of(dx, ex), my = sig_of(dy, ey), mz = sig_of(dz, ez);
  const int E = max(ex, max(ey, ez));
  // r^2 = F * 2^(2E - 2106); each aligned square is below 2^62, so F < 2^64
  const unsigned long long F = sq_top(mx, 2 + 2 * (E - ex)) + sq_top(my, 2 + 2 * (E - ey)) + sq_top(mz, 2 + 2 * (E - ez));
  if (F == 0ull) {  // coincident bodies: the force is undefined
    sj = si = __longlong_as_double(0x7ff8000000000000LL);
    Rn_out = 0ull;
    eR_out = 0;
    return;
  }
  const int z = __clzll((long long)F);
  const unsigned long long M = F << z;                    // r^2 = (M / 2^63) 2^Er
  const int Er = 2 * E - 2043 - z;
  const int k = Er >> 1, p = Er & 1;                      // r^2 = 2^(2k) * mx, mx in [1, 4)
  const float yf = rsqrtf(__uint_as_float(((unsigned)(127 + p) << 23) | (unsigned)((M >> 40) & 0x7FFFFFull)));
  const unsigned yb = __float_as_uint(yf);
  const int eyf = (int)((yb >> 23) & 0xff);
  const unsigned long long myf = (unsigned long long)((yb & 0x7FFFFFu) | 0x800000u);  // yf = myf 2^(eyf-150)
  const unsigned long long Y2 = myf * myf;                // < 2^48, exact
  // P = r^2 y^2 = (M Y2) 2^-S ~ 1 with S = 363 - p - 2 eyf (109..111); keep 62 fraction bits
  const int sh = 301 - p - 2 * eyf;
  const unsigned long long qh = __umul64hi(M, Y2), ql = M * Y2;
  const unsigned long long Pfix = (qh << (64 - sh)) | (ql >> sh);
  const long long efix = (long long)((1ull << 62) - Pfix);  // e 2^62, |e| < 2^-20
  const long long et = efix >> 20;                           // e 2^42
  const long long cfix = (efix >> 1) + ((3 * et * et) >> 25); // (e/2 + 3e^2/8) 2^62
  const unsigned long long Rm = (unsigned long long)((1ll << 62) + cfix);
  // R = myf (2^62 + cfix) < 2^87; 1/r = R 2^(eyf - 212 - k)
  const unsigned long long Rh = __umul64hi(myf, Rm), Rl = myf * Rm;
  const int zR = __clzll((long long)Rh);                   // 41..43
  const unsigned long long Rn = (Rh << zR) | (Rl >> (64 - zR));
  const int eR = 64 - zR + eyf - 212 - k;                  // 1/r = Rn 2^eR
  Rn_out = Rn;
  eR_out = eR;
  const unsigned long long R2 = __umul64hi(Rn, Rn);        // [2^62, 2^64)
  const unsigned long long R3 = __umul64hi(R2, Rn);        // [2^61, 2^64); 1/r^3 = R3 2^(3 eR + 128)
  unsigned long long S = __umul64hi(mj.m, R3);
  int zs = __clzll((long long)S);
  sj = u64_to_double(S << zs, mj.e + 3 * eR + 192 - zs);
  S = __umul64hi(mi.m, R3);
  zs = __clzll((long long)S);
  si = u64_to_double(S << zs, mi.e + 3 * eR + 192 - zs);
}

__device__ __forceinline__ void pair_scalars_int(double dx, double dy, double dz, const MassSplit& mj,
                                                 const MassSplit& mi, double& rinv, double& sj, double& si) {
  unsigned long long Rn;
  int eR;
  pair_scalars_core(dx, dy, dz, mj, mi, Rn, eR, sj, si);
  rinv = Rn ? u64_to_double(Rn, eR) : __longlong_as_double(0x7ff8000000000000LL);
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

// The near pairs of body p (Sec. 3.4, N_d <= 2: parent, children, grandparent, grandchildren,
// siblings), each from the edge vectors X (3 planes) summed along the tree path between the
// two bodies, added to acc.
__device__ __forceinline__ void near_terms(int p, int npad, int n_d, const double* __restrict__ X,
                                           const double* __restrict__ m, const int* __restrict__ parent,
                                           const int* __restrict__ gp, const int* __restrict__ child_off,
                                           const int* __restrict__ child_idx, NearAcc& acc) {
  if (n_d < 1) return;
  const double* Xx = X;
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
  if (n_d < 2) return;
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

// ---------------------------------------------------------------------------------------
// Exact sums of positive terms on the integer pipe.
//
// Each term is P 2^e with P < 2^64 (a truncated 64-bit product of significands). The sum is
// kept as a 128-bit integer A times 2^L. The window follows the largest term: a term would
// land above bit 120 slides it up (A shifted right, L raised), so the largest term sits at
// bits 56..119 and 256 terms cannot overflow. Terms more than 2^120 below the largest lose
// their low bits, far below a binary64 rounding of the sum.
struct UAcc {
  unsigned long long a0 = 0ull, a1 = 0ull;
  int L = -(1 << 29);  // no term yet: the first one slides the window to it

  __device__ __forceinline__ void add(unsigned long long P, int e) {
    int s = e - L;
    if (s > 56) {
      const int d = s - 56;
      if (d >= 128) {
        a0 = 0ull;
        a1 = 0ull;
      } else if (d >= 64) {
        a0 = a1 >> (d - 64);
        a1 = 0ull;
      } else {
        a0 = (a0 >> d) | (a1 << (64 - d));
        a1 >>= d;
      }
      L += d;
      s = 56;
    }
    unsigned long long lo, hi;
    if (s >= 0) {
      lo = P << s;
      hi = s ? P >> (64 - s) : 0ull;
    } else {
      lo = s > -64 ? P >> (-s) : 0ull;
      hi = 0ull;
    }
    a0 += lo;
    a1 += hi + (a0 < lo ? 1ull : 0ull);
  }

  // the sum to a double: the top 64 bits rounded by u64_to_double (about 2^-64 relative)
  __device__ __forceinline__ double value() const {
    if (a1) {
      const int z = __clzll((long long)a1);
      const unsigned long long top = z ? (a1 << z) | (a0 >> (64 - z)) : a1;
      return u64_to_double(top, L + 64 - z);
    }
    if (a0) {
      const int z = __clzll((long long)a0);
      return u64_to_double(a0 << z, L - z);
    }
    return 0.0;
  }
};

// Non-negative doubles order like their bit patterns.
__device__ __forceinline__ unsigned long long key_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// Deterministic block sum (fixed shuffle tree for a fixed blockDim). All threads must
// call it; the result is valid in thread 0. scratch: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double x, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = x;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? scratch[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// NaN-propagating maximum of non-negative values.
__device__ __forceinline__ double nanmax(double a, double b) {
  if (a != a || b != b) return __longlong_as_double(0x7ff8000000000000LL);
  return a > b ? a : b;
}

__device__ __forceinline__ double block_nanmax(double x, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) x = nanmax(x, __shfl_down_sync(0xffffffffu, x, o));
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = x;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? scratch[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = nanmax(s, __shfl_down_sync(0xffffffffu, s, o));
  }
  return s;
}

// sum_partials for three interleaved components (part[b * 3 + c], c = 0, 1, 2) at once, each in
// sum_partials' order: the three chains overlap instead of running one after another.
__device__ __forceinline__ void sum_partials3(const double* part, int nb, double* out3) {
  if (threadIdx.x < 32) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) {
      s0 += part[(size_t)b * 3];
      s1 += part[(size_t)b * 3 + 1];
      s2 += part[(size_t)b * 3 + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, o);
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) {
      out3[0] = s0;
      out3[1] = s1;
      out3[2] = s2;
    }
  }
  __syncthreads();
}

// Exclusive prefix sum of one int per thread over the block (blockDim a multiple of 32, at most
// 1024): shuffle scans within the warps, then of the warp totals in warp 0. *total receives the
// block's sum. Every thread must call it (it holds barriers); ws: 32 ints of shared memory.
__device__ __forceinline__ int block_exclusive_scan(int x, int* ws, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    ws[lane] = w;  // inclusive totals of the warps
  }
  __syncthreads();
  const int before = warp > 0 ? ws[warp - 1] : 0;
  *total = ws[nw - 1];
  return before + incl - x;
}

// Sum of nb per-block partials in a fixed order, computed by warp 0 of every block that
// needs it (so every block obtains bit-identical values); result broadcast via *out.
__device__ __forceinline__ void sum_partials(const double* part, int nb, int stride, double* out) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += part[(size_t)b * stride];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
  __syncthreads();
}

}  // namespace mstar
