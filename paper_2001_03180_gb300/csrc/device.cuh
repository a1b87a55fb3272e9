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
