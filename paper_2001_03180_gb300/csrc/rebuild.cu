// The rebuild test of Sec. 3.5 on the GPU: for each job (one system, one coordinate system,
// one deconstruction rule) repeat, `cycles` times, building the relative coordinates from
// the Cartesian state and deconstructing them back, and record the energy at given cycles.
//
// One CTA per job; the state, the edge vectors and the tree live in shared memory.
// - coordinate systems: the MST (Prim, Sec. 3.2, root closest to the centre of mass) or the
//   chain (Sec. 2.2: the shortest pair first, then the particle closest to either end, the
//   tail on a tie), written as a path tree rooted at the tail;
// - building: X_v = w_v - w_parent(v) (0 at the root);
// - deconstruction: per-vertex path sums X_v + X_parent(v) + ... up to the root, then either
//   the centre-of-mass shift (as the integrator's rebuild) or the root's kept position; or
//   from the root outwards (w_v = w_parent(v) + X_v, parents first) with the root kept, then
//   optionally the centre-of-mass shift;
// - the topology is rebuilt every `topo_every` cycles and compared with the previous one;
// - energies E = T - U with Neumaier-compensated sums of the FP64 terms in index order.
// Every operation is the CPU definition's, in its order (the sums that are sequential there
// are done by one thread), so the results are bit-identical to it.
#include <climits>
#include <cmath>
#include <new>

#include "device.cuh"
#include "internal.h"

namespace mstar {
namespace {

constexpr int kRbThreads = 512;

struct RbArgs {
  int n, cycles, topo_every, nsample;
  const int* sample_at;
  const double *m, *r, *v;  // per job: n, 3n, 3n
  const int *coords, *decon;
  double *E_out, *r_out, *v_out, *mean_level;
  int* topo_changes;
};

__device__ __forceinline__ double norm2_of(const double* x) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x[0], x[0]), __dmul_rn(x[1], x[1])), __dmul_rn(x[2], x[2]));
}

__device__ __forceinline__ double w2_of(const double* r, int u, int v) {
  const double dx = __dsub_rn(r[3 * u], r[3 * v]), dy = __dsub_rn(r[3 * u + 1], r[3 * v + 1]),
               dz = __dsub_rn(r[3 * u + 2], r[3 * v + 2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

struct Neu {
  double s, c;
};

__device__ __forceinline__ void neu_add(Neu& a, double x) {
  const double t = __dadd_rn(a.s, x);
  if (fabs(a.s) >= fabs(x)) a.c = __dadd_rn(a.c, __dadd_rn(__dsub_rn(a.s, t), x));
  else a.c = __dadd_rn(a.c, __dadd_rn(__dsub_rn(x, t), a.s));
  a.s = t;
}

// Lexicographic minimum (key bits, a, b) over the CTA; every thread gets the result.
struct Arg3 {
  unsigned long long k;
  int a, b;
};

__device__ __forceinline__ bool arg3_less(const Arg3& x, const Arg3& y) {
  if (x.k != y.k) return x.k < y.k;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

__device__ Arg3 cta_argmin(Arg3 v, Arg3* red) {
  for (int o = 16; o > 0; o >>= 1) {
    Arg3 c;
    c.k = __shfl_xor_sync(0xffffffffu, v.k, o);
    c.a = __shfl_xor_sync(0xffffffffu, v.a, o);
    c.b = __shfl_xor_sync(0xffffffffu, v.b, o);
    if (arg3_less(c, v)) v = c;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = red[0];
  for (int w = 1; w < kRbThreads / 32; ++w)
    if (arg3_less(red[w], v)) v = red[w];
  return v;
}

// E = T - U with compensated sums, the terms and the order of the CPU definition: the terms
// of a row are computed by all threads, thread 0 adds them in index order.
__device__ double energy_comp(int n, const double* m, const double* r, const double* v, double* row, double* out) {
  Neu T{0.0, 0.0}, U{0.0, 0.0};
  if (threadIdx.x == 0)
    for (int i = 0; i < n; ++i) neu_add(T, __dmul_rn(0.5, __dmul_rn(m[i], norm2_of(v + 3 * i))));
  for (int i = 0; i < n; ++i) {
    __syncthreads();
    for (int j = i + 1 + threadIdx.x; j < n; j += kRbThreads)
      row[j] = __ddiv_rn(__dmul_rn(1.0, __dmul_rn(m[i], m[j])), __dsqrt_rn(w2_of(r, i, j)));
    __syncthreads();
    if (threadIdx.x == 0)
      for (int j = i + 1; j < n; ++j) neu_add(U, row[j]);
  }
  if (threadIdx.x == 0) *out = __dsub_rn(__dadd_rn(T.s, T.c), __dadd_rn(U.s, U.c));
  __syncthreads();
  return *out;
}

// Prim's MST (exact keys; root closest to the origin, lowest index on ties).
__device__ void cta_prim(int n, const double* r, int* parent, int* level, int* order, unsigned long long* key,
                         unsigned char* in, Arg3* red) {
  Arg3 b{~0ull, INT_MAX, 0};
  for (int i = threadIdx.x; i < n; i += kRbThreads) {
    const Arg3 c{key_bits(norm2_of(r + 3 * i)), i, 0};
    if (arg3_less(c, b)) b = c;
    key[i] = 0x7ff0000000000000ull;
    parent[i] = -1;
    in[i] = 0;
  }
  b = cta_argmin(b, red);
  const int root = b.a;
  __syncthreads();
  if (threadIdx.x == 0) {
    in[root] = 1;
    level[root] = 0;
    order[0] = root;
  }
  __syncthreads();
  int u = root;
  for (int it = 1; it < n; ++it) {
    b = Arg3{~0ull, INT_MAX, 0};
    for (int w = threadIdx.x; w < n; w += kRbThreads) {
      if (in[w]) continue;
      const unsigned long long d = key_bits(w2_of(r, u, w));
      if (d < key[w]) {
        key[w] = d;
        parent[w] = u;
      }
      const Arg3 c{key[w], w, 0};
      if (arg3_less(c, b)) b = c;
    }
    b = cta_argmin(b, red);
    u = b.a;
    if (threadIdx.x == 0) {
      in[u] = 1;
      order[it] = u;
      if (parent[u] < 0) parent[u] = root;
      level[u] = level[parent[u]] + 1;
    }
    __syncthreads();
  }
}

// The chain as a path tree rooted at its tail.
__device__ void cta_chain(int n, const double* r, int* parent, int* level, int* order, int* dq, unsigned char* in,
                          Arg3* red) {
  // the shortest pair (lowest (i, j) on ties)
  Arg3 b{~0ull, INT_MAX, INT_MAX};
  for (int i = 0; i < n - 1; ++i)
    for (int j = i + 1 + threadIdx.x; j < n; j += kRbThreads) {
      const Arg3 c{key_bits(w2_of(r, i, j)), i, j};
      if (arg3_less(c, b)) b = c;
    }
  for (int i = threadIdx.x; i < n; i += kRbThreads) in[i] = 0;
  b = cta_argmin(b, red);
  __shared__ int s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = n;
    s_hi = n + 1;
    dq[n] = b.a;
    dq[n + 1] = b.b;
    in[b.a] = 1;
    in[b.b] = 1;
  }
  __syncthreads();
  for (int added = 2; added < n; ++added) {
    const int tail = dq[s_lo], head = dq[s_hi];
    Arg3 c0{~0ull, INT_MAX, 0};
    for (int p = threadIdx.x; p < n; p += kRbThreads) {
      if (in[p]) continue;
      const double dt = w2_of(r, p, tail), dh = w2_of(r, p, head);
      const int end = dh < dt ? 1 : 0;
      const Arg3 c{key_bits(end ? dh : dt), p, end};
      if (arg3_less(c, c0)) c0 = c;
    }
    c0 = cta_argmin(c0, red);
    if (threadIdx.x == 0) {
      in[c0.a] = 1;
      if (c0.b) dq[++s_hi] = c0.a;
      else dq[--s_lo] = c0.a;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += kRbThreads) {
    const int p = dq[s_lo + k];
    order[k] = p;
    parent[p] = k ? dq[s_lo + k - 1] : -1;
    level[p] = k;
  }
  __syncthreads();
}

// One deconstruction of w (3 components per body) from edge vectors W: per-vertex path
// sums, then the centre-of-mass shift (decon 0) or the kept root position (decon 1); or from
// the root outwards, w_v = w_parent(v) + W_v in insertion order with the root kept (decon 2),
// then the centre-of-mass shift (decon 3).
__device__ void deconstruct(int n, const double* m, const int* parent, const int* order, const double* W, double* w,
                            int decon, double* sc) {
  const int root = order[0];
  __syncthreads();
  if (decon >= 2) {
    // one thread per component walks the insertion order: every parent before its children
    if (threadIdx.x < 3) {
      const int c = threadIdx.x;
      for (int k = 0; k < n; ++k) {
        const int v = order[k], p = parent[v];
        if (p >= 0) w[3 * v + c] = __dadd_rn(w[3 * p + c], W[3 * v + c]);
      }
    }
    __syncthreads();
    if (decon == 2) return;
  } else {
    if (threadIdx.x == 0)
      for (int k = 0; k < 3; ++k) sc[k] = w[3 * root + k];
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += kRbThreads) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int u = v; parent[u] >= 0; u = parent[u]) {
        s0 = __dadd_rn(s0, W[3 * u]);
        s1 = __dadd_rn(s1, W[3 * u + 1]);
        s2 = __dadd_rn(s2, W[3 * u + 2]);
      }
      if (decon) {
        s0 = __dadd_rn(s0, sc[0]);
        s1 = __dadd_rn(s1, sc[1]);
        s2 = __dadd_rn(s2, sc[2]);
      }
      w[3 * v] = s0;
      w[3 * v + 1] = s1;
      w[3 * v + 2] = s2;
    }
    __syncthreads();
    if (decon) return;
  }
  if (threadIdx.x == 0) {
    double M = 0.0, c[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
      M = __dadd_rn(M, m[i]);
      for (int k = 0; k < 3; ++k) c[k] = __dadd_rn(c[k], __dmul_rn(m[i], w[3 * i + k]));
    }
    for (int k = 0; k < 3; ++k) sc[3 + k] = __ddiv_rn(c[k], M);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * n; t += kRbThreads) w[t] = __dsub_rn(w[t], sc[3 + t % 3]);
}

__global__ void __launch_bounds__(kRbThreads, 1) k_rebuild_jobs(RbArgs A) {
  extern __shared__ double smem[];
  __shared__ Arg3 red[kRbThreads / 32];
  __shared__ double sc[8];
  const int job = blockIdx.x, n = A.n;
  double* m = smem;
  double* r = m + n;
  double* v = r + 3 * n;
  double* X = v + 3 * n;
  double* V = X + 3 * n;
  double* row = V + 3 * n;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(row + n);
  int* parent = reinterpret_cast<int*>(key + n);
  int* prev = parent + n;
  int* level = prev + n;
  int* order = level + n;
  int* dq = order + n;                                 // 2n + 2
  unsigned char* in = reinterpret_cast<unsigned char*>(dq + 2 * n + 2);
  const int coords = A.coords[job], decon = A.decon[job];
  for (int i = threadIdx.x; i < n; i += kRbThreads) m[i] = A.m[(size_t)job * n + i];
  for (int t = threadIdx.x; t < 3 * n; t += kRbThreads) {
    r[t] = A.r[(size_t)job * 3 * n + t];
    v[t] = A.v[(size_t)job * 3 * n + t];
  }
  __syncthreads();
  int s = 0, changes = 0, builds = 0;
  double lsum = 0.0;
  double* E = A.E_out + (size_t)job * A.nsample;
  while (s < A.nsample && A.sample_at[s] == 0) {
    energy_comp(n, m, r, v, row, &sc[6]);
    if (threadIdx.x == 0) E[s] = sc[6];
    ++s;
  }
  for (int c = 1; c <= A.cycles; ++c) {
    if ((c - 1) % A.topo_every == 0) {
      if (coords == 0) cta_prim(n, r, parent, level, order, key, in, red);
      else cta_chain(n, r, parent, level, order, dq, in, red);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (builds)
          for (int i = 0; i < n; ++i)
            if (parent[i] != prev[i]) {
              ++changes;
              break;
            }
        for (int i = 0; i < n; ++i) {
          prev[i] = parent[i];
          lsum += level[i];
        }
      }
      ++builds;
      __syncthreads();
    }
    for (int w = threadIdx.x; w < n; w += kRbThreads) {
      const int p = parent[w];
      for (int k = 0; k < 3; ++k) {
        X[3 * w + k] = p < 0 ? 0.0 : __dsub_rn(r[3 * w + k], r[3 * p + k]);
        V[3 * w + k] = p < 0 ? 0.0 : __dsub_rn(v[3 * w + k], v[3 * p + k]);
      }
    }
    deconstruct(n, m, parent, order, X, r, decon, sc);
    deconstruct(n, m, parent, order, V, v, decon, sc);
    __syncthreads();
    while (s < A.nsample && A.sample_at[s] == c) {
      energy_comp(n, m, r, v, row, &sc[6]);
      if (threadIdx.x == 0) E[s] = sc[6];
      ++s;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * n; t += kRbThreads) {
    A.r_out[(size_t)job * 3 * n + t] = r[t];
    A.v_out[(size_t)job * 3 * n + t] = v[t];
  }
  if (threadIdx.x == 0) {
    A.topo_changes[job] = changes;
    A.mean_level[job] = builds ? lsum / ((double)builds * n) : 0.0;
  }
}

size_t rb_smem(int n) {
  return sizeof(double) * (size_t)(n + 12 * n + n) + 8 * (size_t)n + sizeof(int) * (size_t)(4 * n + 2 * n + 2) +
         (size_t)n + 16;
}

}  // namespace
}  // namespace mstar

extern "C" int mstar_rebuild_test(int njobs, int n, const double* m, const double* r, const double* v,
                                  const int* coords, const int* deconstruct, int cycles, int topo_every, int nsample,
                                  const int* sample_at, double* E_out, double* r_out, double* v_out, int* topo_changes,
                                  double* mean_level, void* cuda_stream) {
  using namespace mstar;
  if (njobs < 1 || n < 2 || n > MSTAR_REBUILD_MAX_N || cycles < 0 || topo_every < 1 || nsample < 0 || !m || !r ||
      !v || !coords || !deconstruct || (nsample && (!sample_at || !E_out)))
    return MSTAR_ERR_INVALID_ARG;
  for (int j = 0; j < njobs; ++j)
    if ((coords[j] != 0 && coords[j] != 1) || deconstruct[j] < 0 || deconstruct[j] > 3)
      return MSTAR_ERR_INVALID_ARG;
  for (int s = 0; s < nsample; ++s)
    if (sample_at[s] < 0 || sample_at[s] > cycles || (s && sample_at[s] < sample_at[s - 1]))
      return MSTAR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t nm = (size_t)njobs * n, n3 = 3 * nm;
  const size_t bytes = sizeof(double) * (nm + 4 * n3 + (size_t)njobs * nsample + 2 * njobs) +
                       sizeof(int) * (size_t)(2 * njobs + nsample + njobs) + 1024;
  char* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MSTAR_ERR_NOMEM;
  }
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (off + 15) & ~size_t(15);
    char* p = buf + off;
    off += b;
    return p;
  };
  RbArgs A{};
  A.n = n;
  A.cycles = cycles;
  A.topo_every = topo_every;
  A.nsample = nsample;
  double* dm = reinterpret_cast<double*>(take(sizeof(double) * nm));
  double* dr = reinterpret_cast<double*>(take(sizeof(double) * n3));
  double* dv = reinterpret_cast<double*>(take(sizeof(double) * n3));
  double* dro = reinterpret_cast<double*>(take(sizeof(double) * n3));
  double* dvo = reinterpret_cast<double*>(take(sizeof(double) * n3));
  double* dE = reinterpret_cast<double*>(take(sizeof(double) * ((size_t)njobs * nsample + 1)));
  double* dml = reinterpret_cast<double*>(take(sizeof(double) * njobs));
  int* dco = reinterpret_cast<int*>(take(sizeof(int) * njobs));
  int* dde = reinterpret_cast<int*>(take(sizeof(int) * njobs));
  int* dsa = reinterpret_cast<int*>(take(sizeof(int) * (nsample + 1)));
  int* dtc = reinterpret_cast<int*>(take(sizeof(int) * njobs));
  int rc = MSTAR_OK;
  auto cp = [&](void* dst, const void* src, size_t b) {
    if (!rc && cudaMemcpyAsync(dst, src, b, cudaMemcpyDefault, st) != cudaSuccess) rc = MSTAR_ERR_CUDA;
  };
  cp(dm, m, sizeof(double) * nm);
  cp(dr, r, sizeof(double) * n3);
  cp(dv, v, sizeof(double) * n3);
  cp(dco, coords, sizeof(int) * njobs);
  cp(dde, deconstruct, sizeof(int) * njobs);
  if (nsample) cp(dsa, sample_at, sizeof(int) * nsample);
  if (!rc) {
    A.m = dm;
    A.r = dr;
    A.v = dv;
    A.coords = dco;
    A.decon = dde;
    A.sample_at = dsa;
    A.E_out = dE;
    A.r_out = dro;
    A.v_out = dvo;
    A.mean_level = dml;
    A.topo_changes = dtc;
    const size_t smem = rb_smem(n);
    if (cudaFuncSetAttribute(k_rebuild_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      rc = MSTAR_ERR_CUDA;
    if (!rc) {
      k_rebuild_jobs<<<njobs, kRbThreads, smem, st>>>(A);
      if (cudaGetLastError() != cudaSuccess) rc = MSTAR_ERR_CUDA;
    }
  }
  if (nsample) cp(E_out, dE, sizeof(double) * (size_t)njobs * nsample);
  if (r_out) cp(r_out, dro, sizeof(double) * n3);
  if (v_out) cp(v_out, dvo, sizeof(double) * n3);
  if (topo_changes) cp(topo_changes, dtc, sizeof(int) * njobs);
  if (mean_level) cp(mean_level, dml, sizeof(double) * njobs);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = MSTAR_ERR_CUDA;
  cudaFree(buf);
  return rc;
}
