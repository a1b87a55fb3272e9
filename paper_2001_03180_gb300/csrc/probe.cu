// FP64 FMA throughput probe: the denominator of the pair loop's roofline.
//
// The pair loop is bound by the FP64 pipe, whose rate on this part is far below the
// tensor and FP32 rates and is not among the measured peaks, so the library
// measures it on the device it runs on: every thread runs 8 independent DFMA chains,
// the grid fills every SM with 8 CTAs of 8 warps, and the rate is timed with CUDA events
// over a ~30 ms launch that follows a launch of the same size (so that the clocks have
// ramped up under this load).
#include "internal.h"

namespace {

__global__ void __launch_bounds__(256) k_dfma_chains(double* out, double b, double c, int iters) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" MSTAR_API int mstar_fp64_fma_rate(double* fma_per_second, void* cuda_stream) {
  if (!fma_per_second) return MSTAR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MSTAR_ERR_CUDA;
  const int grid = sms * 8, block = 256, iters = 512;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MSTAR_ERR_CUDA;
  float ms = 0.0f;
  if (cudaMalloc(&out, sizeof(double) * grid * block) != cudaSuccess) return MSTAR_ERR_NOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  k_dfma_chains<<<grid, block, 0, s>>>(out, 0.9999999, 1e-9, iters);  // warm-up
  cudaEventRecord(e0, s);
  k_dfma_chains<<<grid, block, 0, s>>>(out, 0.9999999, 1e-9, iters);
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) goto done;
  *fma_per_second = (double)grid * block * iters * 16.0 * 8.0 / (ms * 1e-3);
  rc = MSTAR_OK;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
