// mstar_accelerations_noalloc: the Cartesian pair loop for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc: a sub-integrator embedded in a larger code whose
// memory manager owns the whole device heap (and would see a private allocation as a leak
// or a fragmentation hazard), or a host loop that cannot afford cudaMalloc's implicit
// device synchronisation. This entry point needs no context and allocates nothing: its
// scratch (the SoA copy of the inputs and the per-tile partial sums) is one file-scope
// static __device__ array of fixed size, which every GPU that loads the library keeps for
// the life of the process. The caller passes inputs and outputs.
//
// Consequences documented in include/mstar.h: every call shares that array, so calls that
// overlap on the GPU (on different streams, or from different host threads) race; each
// call clears the parts that must start at zero; sizes above MSTAR_NOALLOC_MAX_N are
// rejected. The first call on a device looks up the array's device address.
#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace {

constexpr int kNaW = 4;                  // warps per CTA
constexpr int kNaT = 32 * kNaW;          // tile
constexpr int kNaMax = MSTAR_NOALLOC_MAX_N;
constexpr int kNaNT = kNaMax / kNaT;     // tiles at the maximum size
constexpr int kNaBlk = mstar::kBlock;
constexpr int kNaNblk = kNaMax / kNaBlk;

// Scratch layout (doubles): x, y, z, m planes (4 * kNaMax), partials kNaNT*4*kNaMax,
// per-block force-function sums kNaNblk.
constexpr size_t kNaPlanes = 4 * (size_t)kNaMax;
constexpr size_t kNaPartials = (size_t)kNaNT * 4 * kNaMax;
constexpr size_t kNaDoubles = kNaPlanes + kNaPartials + kNaNblk;

static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

struct DevAddr {
  double* ptr = nullptr;
  bool done = false;
};
std::mutex g_mu;
DevAddr g_addr[64];

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MSTAR_ERR_CUDA;
  if (dev < 0 || dev >= 64) return MSTAR_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev].done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return MSTAR_ERR_CUDA;
    g_addr[dev].ptr = static_cast<double*>(p);
    g_addr[dev].done = true;
  }
  *out = g_addr[dev].ptr;
  return MSTAR_OK;
}

__global__ void k_na_load(int n, int npad, const double* __restrict__ m, const double* __restrict__ r_aos,
                          double* __restrict__ planes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  const bool real = i < n;
  planes[i] = real ? r_aos[3 * (size_t)i] : 0.0;
  planes[(size_t)npad + i] = real ? r_aos[3 * (size_t)i + 1] : 0.0;
  planes[2 * (size_t)npad + i] = real ? r_aos[3 * (size_t)i + 2] : 0.0;
  planes[3 * (size_t)npad + i] = real ? m[i] : 0.0;
}

__device__ __forceinline__ void na_tile_pair(int tp, int NT, int& I, int& J) {
  int i = 0;
  int start = 0;
  while (start + (NT - i) <= tp) {
    start += NT - i;
    ++i;
  }
  I = i;
  J = i + (tp - start);
}

// Symmetric tiled pair loop over Cartesian separations (every pair far), the same tiling
// and partial-slot scheme as the context path's loop with N_d = 0.
__global__ void __launch_bounds__(kNaT) k_na_tiles(int n, int npad, int NT, const double* __restrict__ planes,
                                                   double* __restrict__ P) {
  __shared__ double sx[kNaT], sy[kNaT], sz[kNaT], sm[kNaT], sax[kNaT], say[kNaT], saz[kNaT];
  int I, J;
  na_tile_pair(blockIdx.x, NT, I, J);
  const double* rx = planes;
  const double* ry = planes + npad;
  const double* rz = planes + 2 * (size_t)npad;
  const double* mm = planes + 3 * (size_t)npad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = J * kNaT;
  sx[tid] = rx[j0 + tid];
  sy[tid] = ry[j0 + tid];
  sz[tid] = rz[j0 + tid];
  sm[tid] = mm[j0 + tid];
  sax[tid] = 0.0;
  say[tid] = 0.0;
  saz[tid] = 0.0;
  const int i = I * kNaT + tid;
  const double xi = rx[i], yi = ry[i], zi = rz[i], mi = mm[i];
  const bool i_pad = i >= n;
  double axi = 0.0, ayi = 0.0, azi = 0.0, ui = 0.0;
  const bool diag = (I == J);
  __syncthreads();
  for (int s = 0; s < kNaW; ++s) {
    const int sub = (warp + s) & (kNaW - 1);
    const bool self = diag && sub == warp;
    if (!(diag && sub < warp)) {
      const int kbeg = self ? 1 : 0, kend = self ? 17 : 32;
      for (int k = kbeg; k < kend; ++k) {
        const int jl = sub * 32 + ((lane + k) & 31);
        const int j = j0 + jl;
        const bool masked = i_pad | (j >= n) | (self & (k == 16) & (lane >= 16));
        const double dx = sx[jl] - xi, dy = sy[jl] - yi, dz = sz[jl] - zi;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        double rinv = mstar::rsqrt_fp64(r2);
        rinv = masked ? 0.0 : rinv;
        const double rinv3 = (rinv * rinv) * rinv;
        const double sj = sm[jl] * rinv3, si = mi * rinv3;
        axi = fma(sj, dx, axi);
        ayi = fma(sj, dy, ayi);
        azi = fma(sj, dz, azi);
        ui = fma(sm[jl], rinv, ui);
        sax[jl] = fma(-si, dx, sax[jl]);
        say[jl] = fma(-si, dy, say[jl]);
        saz[jl] = fma(-si, dz, saz[jl]);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (diag) {
    double* q = P + (size_t)I * 4 * npad + i;
    q[0] = axi + sax[tid];
    q[(size_t)npad] = ayi + say[tid];
    q[2 * (size_t)npad] = azi + saz[tid];
    q[3 * (size_t)npad] = ui;
  } else {
    double* q = P + (size_t)J * 4 * npad + i;
    q[0] = axi;
    q[(size_t)npad] = ayi;
    q[2 * (size_t)npad] = azi;
    q[3 * (size_t)npad] = ui;
    double* qj = P + (size_t)I * 4 * npad + j0 + tid;
    qj[0] = sax[tid];
    qj[(size_t)npad] = say[tid];
    qj[2 * (size_t)npad] = saz[tid];
    qj[3 * (size_t)npad] = 0.0;
  }
}

__global__ void __launch_bounds__(kNaBlk) k_na_finish(int n, int npad, int NT, double G,
                                                      const double* __restrict__ planes,
                                                      const double* __restrict__ P, double* __restrict__ a_aos,
                                                      double* __restrict__ Ublk) {
  __shared__ double scratch[32];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double um = 0.0;
  if (p < n) {
    double ax = 0.0, ay = 0.0, az = 0.0, u = 0.0;
    for (int s = 0; s < NT; ++s) {
      const double* q = P + (size_t)s * 4 * npad + p;
      ax += q[0];
      ay += q[(size_t)npad];
      az += q[2 * (size_t)npad];
      u += q[3 * (size_t)npad];
    }
    a_aos[3 * (size_t)p] = G * ax;
    a_aos[3 * (size_t)p + 1] = G * ay;
    a_aos[3 * (size_t)p + 2] = G * az;
    um = planes[3 * (size_t)npad + p] * u;
  }
  const double s = mstar::block_sum(um, scratch);
  if (threadIdx.x == 0) Ublk[blockIdx.x] = G * s;
}

__global__ void k_na_usum(const double* __restrict__ Ublk, int nblk, double* __restrict__ U) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += Ublk[b];
    *U = s;
  }
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" MSTAR_API int mstar_accelerations_noalloc(int n, const double* m, const double* r, double G,
                                                     double* a, double* U, void* cuda_stream) {
  if (n < 2 || !m || !r || !a || !U || !(G > 0.0)) return MSTAR_ERR_INVALID_ARG;
  if (n > MSTAR_NOALLOC_MAX_N) return MSTAR_ERR_UNSUPPORTED;
  if (!is_device_pointer(m) || !is_device_pointer(r) || !is_device_pointer(a) || !is_device_pointer(U))
    return MSTAR_ERR_INVALID_ARG;
  double* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MSTAR_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int npad = (n + kNaT - 1) / kNaT * kNaT;
  const int NT = npad / kNaT;
  const int nblk = (npad + kNaBlk - 1) / kNaBlk;
  double* planes = base;
  double* P = base + kNaPlanes;
  double* Ublk = P + kNaPartials;
  // planes are rewritten in full (padding zeroed) on every call; every partial slot of
  // [0, npad) is written exactly once by the tile kernel, and every Ublk entry it reads
  // [0, nblk) by the finish kernel, so nothing else needs clearing.
  k_na_load<<<(npad + kNaBlk - 1) / kNaBlk, kNaBlk, 0, s>>>(n, npad, m, r, planes);
  k_na_tiles<<<NT * (NT + 1) / 2, kNaT, 0, s>>>(n, npad, NT, planes, P);
  k_na_finish<<<nblk, kNaBlk, 0, s>>>(n, npad, NT, G, planes, P, a, Ublk);
  k_na_usum<<<1, 32, 0, s>>>(Ublk, nblk, U);
  if (cudaGetLastError() != cudaSuccess) return MSTAR_ERR_CUDA;
  return MSTAR_OK;
}
