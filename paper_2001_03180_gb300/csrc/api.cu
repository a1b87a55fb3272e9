// C ABI of libmstar (include/mstar.h): contexts, workspace layout, and the host-side
// control of the GBS integrator (Sec. 2.3-2.4). Every vector operation of the path runs
// in the kernels of prim.cu, pair.cu and step.cu; the host only holds scalars (t, B, H)
// and makes the accept/reject and step-size decisions from the few values it reads back.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "device.cuh"
#include "internal.h"

using namespace mstar;

namespace {

#define CK(call)                         \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) return fail(e_); \
  } while (0)

int fail(cudaError_t e) {
  (void)e;
  return MSTAR_ERR_CUDA;
}

// --------------------------------------------------------------------------- layout

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Shape {
  int n, npad, K, S, W, T, NT, nblk;
  size_t dcb;  // divide-and-conquer tree scratch (0 unless that builder is selected)
};

Shape shape_of(int n, const mstar_params& p) {
  Shape s{};
  s.n = n;
  s.W = p.pair_tile ? p.pair_tile / 32 : choose_tile_warps(n);
  s.T = 32 * s.W;
  s.npad = (n + s.T - 1) / s.T * s.T;
  s.K = p.k_fix;
  s.S = p.k_fix + 1;
  s.NT = s.npad / s.T;
  s.nblk = (s.npad + kBlock - 1) / kBlock;
  s.dcb = p.mst_method == 1 ? dc_scratch_bytes(n, p.mst_nsub) : 0;
  return s;
}

// Assigns every device array of a context (base == nullptr: only measures). Returns bytes.
size_t carve(const Shape& s, void* base, Dev* d, double** stage) {
  Carver c(base);
  const size_t np = s.npad, n3 = 3 * np, S = s.S;
  Dev t{};
  t.m = c.take<double>(np);
  t.r = c.take<double>(n3);
  t.v = c.take<double>(n3);
  t.parent = c.take<int>(np);
  t.gp = c.take<int>(np);
  t.level = c.take<int>(np);
  t.order = c.take<int>(np);
  t.root = c.take<int>(1);
  t.child_off = c.take<int>(np + 1);
  t.child_idx = c.take<int>(np);
  t.bylev = c.take<int>(np);
  t.X0 = c.take<double>(n3);
  t.V0 = c.take<double>(n3);
  t.A0 = c.take<double>(n3);
  t.sX = c.take<double>(S * n3);
  t.sV = c.take<double>(S * n3);
  t.sr = c.take<double>(S * n3);
  t.sv = c.take<double>(S * n3);
  t.sa = c.take<double>(S * n3);
  t.P = c.take<double>(S * (size_t)s.NT * 4 * np);
  t.Pt = c.take<double>(S * 4 * np);
  t.Nb = c.take<double>(S * 4 * np);
  t.tcnt = c.take<int>(S * (size_t)s.NT);
  t.Ublk = c.take<double>(S * s.nblk);
  t.Tblk = c.take<double>(S * s.nblk);
  t.comblk = c.take<double>(S * s.nblk * 3);
  t.sc = c.take<double>(S * kScal);
  t.Tkk = c.take<double>(6 * np + 1);
  t.epsblk = c.take<double>(2 * (size_t)s.nblk);
  t.res = c.take<double>(8);
  t.mom = c.take<double>((size_t)s.nblk * 8);
  t.dc = s.dcb ? c.take<char>(s.dcb) : nullptr;
  double* st = c.take<double>(2 * n3);
  if (d) *d = t;
  if (stage) *stage = st;
  return (c.off + 255) & ~size_t(255);
}

bool valid_params(const mstar_params* p) {
  if (!p) return false;
  if (!(p->eta_gbs > 0.0) || !std::isfinite(p->eta_gbs)) return false;
  if (!(p->a_gbs > 0.0 && p->a_gbs <= 1.0)) return false;
  if (!(p->fac_min > 0.0 && p->fac_min <= p->fac_max) || !std::isfinite(p->fac_max)) return false;
  if (!(p->q_first > 0.0) || !std::isfinite(p->q_first)) return false;
  if (!(p->t_tol >= 0.0) || !std::isfinite(p->t_tol)) return false;
  if (!(p->G > 0.0) || !std::isfinite(p->G)) return false;
  if (p->k_fix < 2 || p->k_fix > kMaxKfix) return false;
  if (p->n_d < 0 || p->n_d > 2) return false;
  if (p->max_halvings < 0 || p->max_time_iter < 0) return false;
  if (p->mst_method < 0 || p->mst_method > 1 || p->mst_nsub < 0 || p->mst_nsub > kDcMaxSub) return false;
  if (p->pair_tile != 0 && p->pair_tile != 32 && p->pair_tile != 64 && p->pair_tile != 128) return false;
  if (p->pair_split != 0 && p->pair_split != 1 && p->pair_split != 2 && p->pair_split != 4 && p->pair_split != 8)
    return false;
  if (p->division_schedule < 0 || p->division_schedule > 3) return false;
  if (p->division_cluster != 0 && p->division_cluster != 1 && p->division_cluster != 2 && p->division_cluster != 4 &&
      p->division_cluster != 8)
    return false;
  return true;
}

// --------------------------------------------------------------------------- small kernels

__global__ void k_aos_to_soa(int n, int npad, const double* __restrict__ aos, double* __restrict__ soa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    for (int c = 0; c < 3; ++c) soa[(size_t)c * npad + i] = aos[3 * (size_t)i + c];
}

__global__ void k_soa_to_aos(int n, int npad, const double* __restrict__ soa, double* __restrict__ aos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    for (int c = 0; c < 3; ++c) aos[3 * (size_t)i + c] = soa[(size_t)c * npad + i];
}

// flag bit 0: a non-finite value; bit 1: a mass <= 0; bit 2: |coordinate| >= 1e15
__global__ void k_validate(int n, const double* __restrict__ m, const double* __restrict__ r,
                           const double* __restrict__ v, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  const double mi = m[i];
  if (!isfinite(mi)) f |= 1;
  if (!(mi > 0.0)) f |= 2;
  for (int c = 0; c < 3; ++c) {
    const double x = r[3 * (size_t)i + c], u = v[3 * (size_t)i + c];
    if (!isfinite(x) || !isfinite(u)) f |= 1;
    if (fabs(x) >= 1e15) f |= 4;
  }
  if (f) atomicOr(flag, f);
}

__global__ void k_fill_int(int* __restrict__ p, int count, int value) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = value;
}

struct Staging {
  double* dev = nullptr;
};

int blocks_for(int n) { return (n + kBlock - 1) / kBlock; }

// Copy an n x 3 array (host or device) into the context's AoS staging area, then into
// three SoA planes.
int load_vectors(mstar_ctx* c, double* stage, const double* src, double* dst_planes) {
  CK(cudaMemcpyAsync(stage, src, sizeof(double) * 3 * (size_t)c->n, cudaMemcpyDefault, c->stream));
  k_aos_to_soa<<<blocks_for(c->n), kBlock, 0, c->stream>>>(c->n, c->npad, stage, dst_planes);
  MSTAR_LAUNCHED(c);
  CK(cudaGetLastError());
  return MSTAR_OK;
}

int store_vectors(mstar_ctx* c, double* stage, const double* src_planes, double* dst) {
  k_soa_to_aos<<<blocks_for(c->n), kBlock, 0, c->stream>>>(c->n, c->npad, src_planes, stage);
  MSTAR_LAUNCHED(c);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(dst, stage, sizeof(double) * 3 * (size_t)c->n, cudaMemcpyDefault, c->stream));
  return MSTAR_OK;
}

double* stage_of(mstar_ctx* c) {
  double* st = nullptr;
  Shape s = shape_of(c->n, c->p);
  carve(s, c->ws, nullptr, &st);
  return st;
}

int sync_read_res(mstar_ctx* c) {
  CK(cudaMemcpyAsync(c->host_res, c->d.res, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return MSTAR_OK;
}

void prof_flush(mstar_ctx* c) {
  for (size_t i = 0; i < c->prof_used; ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->prof_pool[i].a, c->prof_pool[i].b) == cudaSuccess) {
      const int nsl = c->prof_pool[i].nsl;
      c->prof_ms += ms;
      c->prof_launches += 1;
      c->prof_evals += nsl;
      c->prof_pairs += (double)nsl * 0.5 * (double)c->n * (double)(c->n - 1);
    }
  }
  c->prof_used = 0;
}

// --------------------------------------------------------------------------- the GBS step

// MST of the current positions and the edge coordinates (with the step start's kinetic
// partials), issued without reading anything back (the MST builders may synchronise for their
// own checks).
int issue_tree_and_edges(mstar_ctx* c) {
  if (!c->mst_valid) {
    if (c->p.mst_method == 1) {
      CK(launch_mst_dc(c));
    } else {
      bool tied = true;
      if (c->n >= kBoruvkaMinN) CK(launch_mst_boruvka(c, &tied));
      if (tied) CK(launch_prim(c));
    }
    CK(launch_tree(c));
    c->mst_valid = true;
  }
  CK(launch_prepare(c));
  return MSTAR_OK;
}

// The step-start force evaluation and the derivative information it gives (A0; U0 and T0 into
// d.res[2], d.res[3] and the step-start slot's scalars).
int issue_start_eval(mstar_ctx* c) {
  CK(launch_forces(c, c->K, c->K + 1, c->p.n_d));
  CK(launch_start_derivs(c));
  return MSTAR_OK;
}

// issue_tree_and_edges, then issue_start_eval.
int issue_prepare(mstar_ctx* c) {
  int rc = issue_tree_and_edges(c);
  if (rc) return rc;
  return issue_start_eval(c);
}

// issue_prepare, then U0 and T0 read back.
int prepare_step(mstar_ctx* c, double* U0, double* T0) {
  int rc = issue_prepare(c);
  if (rc) return rc;
  rc = sync_read_res(c);
  if (rc) return rc;
  prof_flush(c);
  *U0 = c->host_res[2];
  *T0 = c->host_res[3];
  return MSTAR_OK;
}

// One attempt with fictitious step H: all divisions level by level, then the
// extrapolation; reads eps and the extrapolated time back.
// The launches of one attempt after the staging of H and t: all divisions level by level
// (the divisions with n_k >= tau kick and drift at level tau), then the extrapolation.
// With a trajectory record the states of every level are saved on the way.
int issue_attempt_branched(mstar_ctx* c);

// With c->att_start: the step-start force evaluation on st_stream, forked from the context's
// stream before anything of the attempt, and joined before the extrapolation.
int fork_start_eval(mstar_ctx* c) {
  if (!c->att_start) return MSTAR_OK;
  cudaStream_t main_stream = c->stream;
  CK(cudaEventRecord(c->st_fork, main_stream));
  CK(cudaStreamWaitEvent(c->st_stream, c->st_fork, 0));
  c->stream = c->st_stream;
  int rc = issue_start_eval(c);
  if (!rc && cudaEventRecord(c->st_join, c->stream) != cudaSuccess) rc = MSTAR_ERR_CUDA;
  c->stream = main_stream;
  return rc;
}

int join_start_eval(mstar_ctx* c) {
  if (c->att_start) CK(cudaStreamWaitEvent(c->stream, c->st_join, 0));
  return MSTAR_OK;
}

int issue_attempt(mstar_ctx* c) {
  // attempts that record a trajectory, time the pair kernel or serve the adjoint go level by level
  const bool plain = !c->traj && !c->prof && !c->levelled;
  int rc = fork_start_eval(c);
  if (rc) return rc;
  if (plain && c->div_cta) {
    CK(launch_division_cta(c));
    if ((rc = join_start_eval(c))) return rc;
    CK(launch_extrapolate(c));
    return MSTAR_OK;
  }
  if (plain && c->branched) return issue_attempt_branched(c);
  const int K = c->K;
  const size_t st = (size_t)3 * c->npad;
  AdjTraj* tr = c->traj;
  const size_t lvl = (size_t)K * st, nsc = (size_t)(K + 1) * kScal;
  auto save = [&](double* dst, const double* src, size_t count) {
    return cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToDevice, c->stream);
  };
  CK(launch_init_drift(c));
  if (tr) {
    CK(save(tr->SC, c->d.sc, nsc));
    CK(save(tr->v0, c->d.v, st));
  }
  for (int tau = 1; tau <= 2 * K; ++tau) {
    const int lo = (tau + 1) / 2 - 1;  // divisions with n_k >= tau kick and drift
    CK(launch_forces(c, lo, K, c->p.n_d));
    if (tr) {
      CK(save(tr->R + (tau - 1) * lvl + lo * st, c->d.sr + lo * st, (K - lo) * st));
      CK(save(tr->A + (tau - 1) * lvl + lo * st, c->d.sa + lo * st, (K - lo) * st));
    }
    const int lo2 = tau / 2;  // divisions with n_k > tau need positions for the next kick
    if (c->npad <= kLevelCtaMax) {
      // one CTA per division: the whole level in one launch (the position rebuild leaves the
      // velocities and scalars that the trajectory record takes below as they were)
      CK(launch_level_cta(c, lo, K, lo2, tau));
      if (tr) {
        CK(save(tr->Vv + (tau - 1) * lvl + lo * st, c->d.sv + lo * st, (K - lo) * st));
        CK(save(tr->SC + tau * nsc, c->d.sc, nsc));
      }
      continue;
    }
    if (c->sub_cluster) {
      CK(launch_substep_cluster(c, lo, K, lo2, tau));
      if (tr) {
        CK(save(tr->Vv + (tau - 1) * lvl + lo * st, c->d.sv + lo * st, (K - lo) * st));
        CK(save(tr->SC + tau * nsc, c->d.sc, nsc));
      }
      continue;
    }
    CK(launch_kick(c, lo, K));
    CK(launch_rebuild(c, c->d.sV + lo * st, c->d.sv + lo * st, st, K - lo, 1, c->d.Tblk + (size_t)lo * c->nblk,
                      c->d.comblk + (size_t)lo * c->nblk * 3));
    CK(launch_drift(c, lo, K, tau));
    if (tr) {
      CK(save(tr->Vv + (tau - 1) * lvl + lo * st, c->d.sv + lo * st, (K - lo) * st));
      CK(save(tr->SC + tau * nsc, c->d.sc, nsc));
    }
    if (lo2 < K)
      CK(launch_rebuild(c, c->d.sX + lo2 * st, c->d.sr + lo2 * st, st, K - lo2, 0, nullptr,
                        c->d.comblk + (size_t)lo2 * c->nblk * 3));
  }
  if ((rc = join_start_eval(c))) return rc;
  CK(launch_extrapolate(c));
  return MSTAR_OK;
}

// The attempt with each division on its own stream: after the first half drift of every
// division (on the context's stream), division k runs its n_k kicks and drifts as one chain on
// stream k, and the extrapolation waits for all of them. A division's launches are those of
// the level order restricted to its slot, so the results are the same; the chains overlap one
// division's small kernels with another's pair loop. Every buffer these launches touch is
// indexed by slot, so the chains share nothing.
int issue_attempt_branched(mstar_ctx* c) {
  const int K = c->K;
  const size_t st = (size_t)3 * c->npad;
  cudaStream_t main_stream = c->stream;
  if (!c->br_fork) return MSTAR_ERR_CUDA;  // created with the context
  CK(launch_init_drift(c));
  CK(cudaEventRecord(c->br_fork, main_stream));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    c->stream = c->br_stream[k];
    e = cudaStreamWaitEvent(c->stream, c->br_fork, 0);
    const int nk = 2 * (k + 1);
    for (int tau = 1; tau <= nk && e == cudaSuccess; ++tau) {
      e = launch_forces(c, k, k + 1, c->p.n_d);
      const int pos = tau < nk ? k : k + 1;  // positions for the next kick, unless this was the last
      if (e == cudaSuccess && c->npad <= kLevelCtaMax) {
        e = launch_level_cta(c, k, k + 1, pos, tau);
        continue;
      }
      if (e == cudaSuccess) e = launch_kick(c, k, k + 1);
      if (e == cudaSuccess)
        e = launch_rebuild(c, c->d.sV + k * st, c->d.sv + k * st, st, 1, 1, c->d.Tblk + (size_t)k * c->nblk,
                           c->d.comblk + (size_t)k * c->nblk * 3);
      if (e == cudaSuccess) e = launch_drift(c, k, k + 1, tau);
      if (e == cudaSuccess && pos == k)
        e = launch_rebuild(c, c->d.sX + k * st, c->d.sr + k * st, st, 1, 0, nullptr,
                           c->d.comblk + (size_t)k * c->nblk * 3);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->br_join[k], c->stream);
  }
  c->stream = main_stream;
  CK(e);
  for (int k = 0; k < K; ++k) CK(cudaStreamWaitEvent(main_stream, c->br_join[k], 0));
  const int rc = join_start_eval(c);
  if (rc) return rc;
  CK(launch_extrapolate(c));
  return MSTAR_OK;
}

// Stream priority of division k's chain: the longer a division (n_k = 2 (k + 1) substeps), the
// higher, so that the longest chain, which bounds the attempt, is served first where the
// divisions' kernels compete for SMs.
int division_priority(int k, int K) {
  int lo = 0, hi = 0;  // least and greatest priority (greatest is the numerically smallest)
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int levels = lo - hi + 1;
  return lo - (int)((long long)k * levels / K);
}

// Capture issue_attempt once on a private stream and instantiate it. The launches depend
// only on the context's sizes and buffers and on the trajectory record (H and t are read
// from device memory), so the graph serves every later attempt with the same record. Any
// failure turns the graph path off for the context.
cudaGraphExec_t build_attempt_graph(mstar_ctx* c) {
  cudaStream_t user = c->stream;
  const long long l0 = c->launches, f0 = c->force_evals;
  cudaGraph_t g = nullptr;
  bool ok = c->cap || cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) {
    c->stream = c->cap;
    ok = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int rc = issue_attempt(c);
      ok = cudaStreamEndCapture(c->cap, &g) == cudaSuccess && rc == MSTAR_OK && g;
    }
    c->stream = user;
  }
  c->att_launches = c->launches - l0;
  c->att_evals = c->force_evals - f0;
  c->launches = l0;
  c->force_evals = f0;
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiateWithFlags(&exec, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    c->att_graph_off = true;
    return nullptr;
  }
  c->att_graphs.push_back({c->traj, c->levelled, c->att_start, exec, c->att_launches, c->att_evals});
  return exec;
}

// One attempt with fictitious step H; reads eps and the extrapolated time back. Without
// profiling the attempt is one graph launch. With start, the attempt also runs the step-start
// force evaluation (issue_start_eval) beside its divisions; U0 and T0 are then read back with
// eps and t.
int run_attempt(mstar_ctx* c, double H, double* eps, double* tnew, bool start = false) {
  CK(stage_attempt_scalars(c, H));
  c->att_start = start;
  cudaGraphExec_t exec = nullptr;
  long long g_launches = 0, g_evals = 0;
  if (!c->prof && !c->att_graph_off) {
    for (const auto& ag : c->att_graphs)
      if (ag.traj == c->traj && ag.levelled == c->levelled && ag.start == start) {
        exec = ag.exec;
        g_launches = ag.launches;
        g_evals = ag.evals;
      }
    if (!exec && (exec = build_attempt_graph(c))) {
      g_launches = c->att_launches;
      g_evals = c->att_evals;
    }
  }
  int rc = MSTAR_OK;
  if (exec) {
    if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) rc = MSTAR_ERR_CUDA;
    c->launches += g_launches;
    c->force_evals += g_evals;
  } else {
    rc = issue_attempt(c);
  }
  c->att_start = false;
  if (rc) return rc;
  rc = sync_read_res(c);
  if (rc) return rc;
  prof_flush(c);
  *eps = c->host_res[0];
  *tnew = c->host_res[1];
  return MSTAR_OK;
}

// The extrapolated MST coordinates become the Cartesian state (COM frame).
int accept_state(mstar_ctx* c) {
  const size_t n3 = (size_t)3 * c->npad;
  if (c->d.v == c->d.r + n3) {  // positions and velocities in one launch (two slots n3 apart)
    CK(launch_rebuild(c, c->d.Tkk, c->d.r, n3, 2, 0, nullptr, c->d.comblk));
  } else {
    CK(launch_rebuild(c, c->d.Tkk, c->d.r, 0, 1, 0, nullptr, c->d.comblk));
    CK(launch_rebuild(c, c->d.Tkk + n3, c->d.v, 0, 1, 0, nullptr, c->d.comblk));
  }
  c->mst_valid = false;
  return MSTAR_OK;
}

int extract_out(mstar_ctx* c, double* r_out, double* v_out, const double* Xsrc, const double* Vsrc) {
  // rebuild into the step-start slot's r/v buffers (free after the attempt) and copy out
  const size_t n3 = (size_t)3 * c->npad;
  double* rr = c->d.sr + (size_t)c->K * n3;
  double* vv = c->d.sv + (size_t)c->K * n3;
  CK(launch_rebuild(c, Xsrc, rr, 0, 1, 0, nullptr, c->d.comblk));
  CK(launch_rebuild(c, Vsrc, vv, 0, 1, 0, nullptr, c->d.comblk));
  double* stage = stage_of(c);
  int rc;
  if (r_out && (rc = store_vectors(c, stage, rr, r_out))) return rc;
  if (v_out && (rc = store_vectors(c, stage + n3, vv, v_out))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return MSTAR_OK;
}

}  // namespace

// --------------------------------------------------------------------------- internals

namespace mstar {

void drop_traj_graphs(mstar_ctx* c) {
  std::vector<mstar_ctx::AttGraph> keep;
  for (const auto& ag : c->att_graphs) {
    if (ag.traj) cudaGraphExecDestroy(ag.exec);
    else keep.push_back(ag);
  }
  c->att_graphs.swap(keep);
}


int step_prepare(mstar_ctx* c, double* U0, double* T0) { return prepare_step(c, U0, T0); }
int step_attempt(mstar_ctx* c, double H, double* eps, double* tnew) { return run_attempt(c, H, eps, tnew); }
int step_accept(mstar_ctx* c) {
  c->at_init = false;
  return accept_state(c);
}
int vectors_in(mstar_ctx* c, const double* src, double* planes) { return load_vectors(c, stage_of(c), src, planes); }
int vectors_out(mstar_ctx* c, const double* planes, double* dst) {
  const int rc = store_vectors(c, stage_of(c), planes, dst);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return MSTAR_OK;
}

// Pair tile of 32 W bodies by system size, from a sweep of full GBS steps on Plummer spheres
// (pair-forces/s): below ~4000 bodies the 32-body tiles give the most CTAs per slot (+18 %
// at N = 2050 over 128-body tiles); up to ~8000 the 64-body tiles; above, the 128-body
// tiles keep the partial sums (slots x tiles x 4 x npad doubles) a quarter as large at the
// same speed.
int choose_tile_warps(int n) { return n <= 4096 ? 1 : (n <= 8192 ? 2 : 4); }

size_t workspace_bytes(int n, const mstar_params& p, int* npad_out, int* W_out) {
  Shape s = shape_of(n, p);
  if (npad_out) *npad_out = s.npad;
  if (W_out) *W_out = s.W;
  return carve(s, nullptr, nullptr, nullptr);
}

void prof_begin(mstar_ctx* c) {
  if (c->prof_used == c->prof_pool.size()) {
    mstar_prof_rec r{};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
      c->prof = false;
      return;
    }
    c->prof_pool.push_back(r);
  }
  cudaEventRecord(c->prof_pool[c->prof_used].a, c->stream);
}

void prof_end(mstar_ctx* c, int nsl) {
  if (!c->prof || c->prof_used >= c->prof_pool.size()) return;
  cudaEventRecord(c->prof_pool[c->prof_used].b, c->stream);
  c->prof_pool[c->prof_used].nsl = nsl;
  c->prof_used++;
}

}  // namespace mstar

// --------------------------------------------------------------------------- C ABI

extern "C" {

void mstar_default_params(mstar_params* p) {
  if (!p) return;
  p->eta_gbs = 1e-12;
  p->a_gbs = 0.9;
  p->fac_min = 0.2;
  p->fac_max = 2.0;
  p->q_first = 0.1;
  p->t_tol = 1e-10;
  p->G = 1.0;
  p->k_fix = 8;
  p->n_d = 2;
  p->max_halvings = 30;
  p->max_time_iter = 8;
  p->mst_method = 0;
  p->mst_nsub = 0;
  p->pair_tile = 0;
  p->pair_split = 0;
  p->division_schedule = 0;
  p->division_cluster = 0;
}

size_t mstar_workspace_bytes(int n, const mstar_params* p) {
  mstar_params d;
  if (!p) {
    mstar_default_params(&d);
    p = &d;
  }
  if (n < 2 || n > MSTAR_MAX_N || !valid_params(p)) return 0;
  return workspace_bytes(n, *p);
}

const char* mstar_strerror(int code) {
  switch (code) {
    case MSTAR_OK: return "ok";
    case MSTAR_ERR_INVALID_ARG: return "invalid argument";
    case MSTAR_ERR_NONFINITE: return "non-finite input";
    case MSTAR_ERR_NO_CONVERGENCE: return "GBS step did not converge within max_halvings";
    case MSTAR_ERR_TIMEOUT: return "device wait timed out";
    case MSTAR_ERR_CUDA: return "CUDA runtime error";
    case MSTAR_ERR_UNSUPPORTED: return "unsupported size";
    case MSTAR_ERR_NOMEM: return "workspace too small or allocation failed";
    default: return "unknown error";
  }
}

void mstar_free(mstar_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& r : c->prof_pool) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto& ag : c->att_graphs) cudaGraphExecDestroy(ag.exec);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (int k = 0; k < kMaxKfix; ++k) {
    if (c->br_stream[k]) cudaStreamDestroy(c->br_stream[k]);
    if (c->br_join[k]) cudaEventDestroy(c->br_join[k]);
  }
  if (c->br_fork) cudaEventDestroy(c->br_fork);
  if (c->st_stream) cudaStreamDestroy(c->st_stream);
  if (c->st_fork) cudaEventDestroy(c->st_fork);
  if (c->st_join) cudaEventDestroy(c->st_join);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  if (c->host_res) cudaFreeHost(c->host_res);
  if (c->host_buf) cudaFreeHost(c->host_buf);
  delete c;
}

int mstar_init(mstar_ctx** out, int n, const double* m, const double* r, const double* v, const mstar_params* p,
               void* workspace, size_t workspace_bytes, void* cuda_stream) {
  if (!out) return MSTAR_ERR_INVALID_ARG;
  *out = nullptr;
  mstar_params pd;
  if (!p) {
    mstar_default_params(&pd);
    p = &pd;
  }
  if (!m || !r || !v || !valid_params(p)) return MSTAR_ERR_INVALID_ARG;
  if (n < 2) return MSTAR_ERR_INVALID_ARG;
  if (n > MSTAR_MAX_N) return MSTAR_ERR_UNSUPPORTED;
  mstar_ctx* c = new (std::nothrow) mstar_ctx();
  if (!c) return MSTAR_ERR_NOMEM;
  c->p = *p;
  c->n = n;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  Shape s = shape_of(n, *p);
  c->npad = s.npad;
  c->K = s.K;
  c->nslots = s.S;
  c->W = s.W;
  c->T = s.T;
  c->NT = s.NT;
  c->ntp = s.NT * (s.NT + 1) / 2;
  c->S = s.W != 1 ? 1 : (p->pair_split ? p->pair_split : (n <= 512 ? 4 : 1));
  // how an attempt's divisions are issued: one CTA per division (pair sums included) for small
  // systems, else a stream per division from 1000 bodies, else level by level
  const int ds = p->division_schedule;
  c->div_cta = (ds == 3 && c->npad <= kDivisionCtaMax) || (ds == 0 && c->npad <= kDivisionCtaRule);
  c->div_cluster = p->division_cluster ? p->division_cluster : (c->npad <= 32 ? 4 : 8);
  c->branched = ds == 2 || ((ds == 0 || ds == 3) && !c->div_cta && n >= 1000);
  c->nblk = s.nblk;
  const size_t need = carve(s, nullptr, nullptr, nullptr);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return MSTAR_ERR_CUDA;
  }
  if (workspace) {
    if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
      delete c;
      return MSTAR_ERR_NOMEM;
    }
    c->ws = workspace;
  } else {
    if (cudaMalloc(&c->ws, need) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return MSTAR_ERR_NOMEM;
    }
    c->own_ws = true;
  }
  c->ws_bytes = need;
  double* stage = nullptr;
  carve(s, c->ws, &c->d, &stage);
  if (cudaMallocHost(&c->host_res, 16 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->host_buf, (size_t)c->nblk * 8 * sizeof(double) + 64) != cudaSuccess) {
    cudaGetLastError();
    mstar_free(c);
    return MSTAR_ERR_NOMEM;
  }
  auto bail = [&](int code) {
    mstar_free(c);
    return code;
  };
  prefer_shared_pair_kernels();
  prefer_shared_step_kernels();
  if (cudaMemsetAsync(c->ws, 0, need, c->stream) != cudaSuccess || upload_step_constants(c) != cudaSuccess ||
      prepare_rebuild(c) != cudaSuccess || prepare_division_cta(c) != cudaSuccess ||
      prepare_substep_cluster(c) != cudaSuccess)
    return bail(MSTAR_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&c->st_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->st_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->st_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(MSTAR_ERR_CUDA);
  if (c->branched) {  // the streams and events of the per-division attempt graph
    if (cudaEventCreateWithFlags(&c->br_fork, cudaEventDisableTiming) != cudaSuccess) return bail(MSTAR_ERR_CUDA);
    for (int k = 0; k < c->K; ++k)
      if (cudaStreamCreateWithPriority(&c->br_stream[k], cudaStreamNonBlocking, division_priority(k, c->K)) !=
              cudaSuccess ||
          cudaEventCreateWithFlags(&c->br_join[k], cudaEventDisableTiming) != cudaSuccess)
        return bail(MSTAR_ERR_CUDA);
  }
  k_fill_int<<<blocks_for(c->npad), kBlock, 0, c->stream>>>(c->d.parent, c->npad, -1);
  k_fill_int<<<blocks_for(c->npad), kBlock, 0, c->stream>>>(c->d.gp, c->npad, -1);
  c->launches += 2;
  // inputs -> device (masses straight, vectors via the AoS staging area)
  const size_t n3 = (size_t)3 * c->npad;
  if (cudaMemcpyAsync(c->d.m, m, sizeof(double) * n, cudaMemcpyDefault, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(stage, r, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(stage + n3, v, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream) != cudaSuccess)
    return bail(MSTAR_ERR_CUDA);
  int* flag = reinterpret_cast<int*>(c->d.res + 4);
  k_validate<<<blocks_for(n), kBlock, 0, c->stream>>>(n, c->d.m, stage, stage + n3, flag);
  k_aos_to_soa<<<blocks_for(n), kBlock, 0, c->stream>>>(n, c->npad, stage, c->d.r);
  k_aos_to_soa<<<blocks_for(n), kBlock, 0, c->stream>>>(n, c->npad, stage + n3, c->d.v);
  c->launches += 3;
  if (cudaGetLastError() != cudaSuccess) return bail(MSTAR_ERR_CUDA);
  // masses to the host for M (sequential sum) and the validation flag
  std::vector<double> mh(n);
  if (cudaMemcpyAsync(mh.data(), c->d.m, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->host_res, c->d.res, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(MSTAR_ERR_CUDA);
  int f = 0;
  std::memcpy(&f, reinterpret_cast<const char*>(c->host_res) + 4 * sizeof(double), sizeof(int));
  if (f & 1) return bail(MSTAR_ERR_NONFINITE);
  if (f & 2) return bail(MSTAR_ERR_INVALID_ARG);
  if (f & 4) return bail(MSTAR_ERR_UNSUPPORTED);
  double M = 0.0;
  for (int i = 0; i < n; ++i) M += mh[i];
  c->Mtot = M;
  // centre-of-mass frame, then B = U - T with the Cartesian force function (Eq. 1)
  if (launch_com_shift(c, c->d.r, nullptr) != cudaSuccess) return bail(MSTAR_ERR_CUDA);
  if (launch_com_shift(c, c->d.v, c->d.Tblk) != cudaSuccess) return bail(MSTAR_ERR_CUDA);
  if (cudaMemcpyAsync(c->d.sr + (size_t)c->K * n3, c->d.r, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                      c->stream) != cudaSuccess)
    return bail(MSTAR_ERR_CUDA);
  if (launch_forces(c, c->K, c->K + 1, 0) != cudaSuccess) return bail(MSTAR_ERR_CUDA);
  if (cudaMemcpyAsync(c->host_buf, c->d.Ublk + (size_t)c->K * c->nblk, sizeof(double) * c->nblk,
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->host_buf + c->nblk, c->d.Tblk, sizeof(double) * c->nblk, cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(MSTAR_ERR_CUDA);
  double U = 0.0, T2 = 0.0;
  for (int b = 0; b < c->nblk; ++b) {
    U += c->host_buf[b];
    T2 += c->host_buf[c->nblk + b];
  }
  c->B = U - 0.5 * T2;
  c->t = 0.0;
  c->H = 0.0;
  c->force_evals = 0;
  c->mst_valid = false;
  c->at_init = true;
  *out = c;
  return MSTAR_OK;
}

int mstar_set_H(mstar_ctx* c, double H) {
  if (!c || !std::isfinite(H)) return MSTAR_ERR_INVALID_ARG;
  c->H = H;
  return MSTAR_OK;
}

int mstar_get_state(mstar_ctx* c, double* t, double* r, double* v) {
  if (!c) return MSTAR_ERR_INVALID_ARG;
  if (t) *t = c->t;
  double* stage = stage_of(c);
  int rc;
  if (r && (rc = store_vectors(c, stage, c->d.r, r))) return rc;
  if (v && (rc = store_vectors(c, stage + 3 * (size_t)c->npad, c->d.v, v))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return MSTAR_OK;
}

int mstar_set_state(mstar_ctx* c, double t, const double* r, const double* v) {
  if (!c || !r || !v || !std::isfinite(t)) return MSTAR_ERR_INVALID_ARG;
  double* stage = stage_of(c);
  int rc;
  if ((rc = load_vectors(c, stage, r, c->d.r))) return rc;
  if ((rc = load_vectors(c, stage + 3 * (size_t)c->npad, v, c->d.v))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->t = t;
  c->mst_valid = false;
  c->at_init = false;
  return MSTAR_OK;
}

int mstar_get_mst(mstar_ctx* c, int* root, int* parent, int* level, int* order) {
  if (!c) return MSTAR_ERR_INVALID_ARG;
  if (c->p.mst_method == 1) {
    // the divide-and-conquer tree; its order is the breadth-first walk of the build
    if (!c->mst_valid) {
      CK(launch_mst_dc(c));
      CK(launch_tree(c));
      c->mst_valid = true;
    }
  } else if (order) {
    // Prim's kernel records the insertion order; it builds the same tree as the step's
    // MST builder, so the step buffers stay valid.
    CK(launch_prim(c));
    CK(launch_tree(c));
    c->mst_valid = true;
  } else if (!c->mst_valid) {
    bool tied = true;
    if (c->n >= kBoruvkaMinN) CK(launch_mst_boruvka(c, &tied));
    if (tied) CK(launch_prim(c));
    CK(launch_tree(c));
    c->mst_valid = true;
  }
  const size_t b = sizeof(int) * c->n;
  if (root) CK(cudaMemcpyAsync(root, c->d.root, sizeof(int), cudaMemcpyDefault, c->stream));
  if (parent) CK(cudaMemcpyAsync(parent, c->d.parent, b, cudaMemcpyDefault, c->stream));
  if (level) CK(cudaMemcpyAsync(level, c->d.level, b, cudaMemcpyDefault, c->stream));
  if (order) CK(cudaMemcpyAsync(order, c->d.order, b, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return MSTAR_OK;
}

int mstar_accelerations(mstar_ctx* c, double* a, double* U) {
  if (!c) return MSTAR_ERR_INVALID_ARG;
  double U0, T0;
  int rc = prepare_step(c, &U0, &T0);
  if (rc) return rc;
  if (U) *U = U0;
  if (a && (rc = store_vectors(c, stage_of(c), c->d.sa + (size_t)c->K * 3 * c->npad, a))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return MSTAR_OK;
}

int mstar_attempt(mstar_ctx* c, double H, double* eps, double* r_out, double* v_out, double* t_out) {
  if (!c || !std::isfinite(H) || H == 0.0) return MSTAR_ERR_INVALID_ARG;
  double U0, T0, e, tn;
  int rc = prepare_step(c, &U0, &T0);
  if (rc) return rc;
  if ((rc = run_attempt(c, H, &e, &tn))) return rc;
  if (eps) *eps = e;
  if (t_out) *t_out = tn;
  if (r_out || v_out) {
    const size_t n3 = (size_t)3 * c->npad;
    if ((rc = extract_out(c, r_out, v_out, c->d.Tkk, c->d.Tkk + n3))) return rc;
  }
  return MSTAR_OK;
}

int mstar_tune_pair_tile(int n, const double* m, const double* r, const double* v, const mstar_params* p,
                         int repeats, int* tile_out, int* split_out, double* ms_out, void* cuda_stream) {
  if (!tile_out || !split_out || repeats < 1) return MSTAR_ERR_INVALID_ARG;
  mstar_params q;
  if (p) q = *p;
  else mstar_default_params(&q);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return MSTAR_ERR_CUDA;
  }
  // the tiles serve the multi-kernel attempt (one CTA per division has no tiles): that is the
  // one timed, on streams from 1000 bodies unless the parameters ask for levels
  if (q.division_schedule != 1 && q.division_schedule != 2) q.division_schedule = n >= 1000 ? 2 : 1;
  const int tiles[4] = {32, 32, 64, 128}, splits[4] = {4, 1, 1, 1};
  double best = 0.0;
  int best_k = -1, rc = MSTAR_OK;
  for (int k = 0; k < 4 && !rc; ++k) {
    q.pair_tile = tiles[k];
    q.pair_split = splits[k];
    mstar_ctx* c = nullptr;
    rc = mstar_init(&c, n, m, r, v, &q, nullptr, 0, cuda_stream);
    if (rc) break;
    double U0, T0, e, tn;
    rc = prepare_step(c, &U0, &T0);
    const double H = 1e-6 * U0;
    if (!rc) rc = run_attempt(c, H, &e, &tn);  // untimed: captures the attempt's graph
    float ms = 0.0f;
    if (!rc) {
      cudaEventRecord(e0, c->stream);
      for (int i = 0; i < repeats && !rc; ++i) rc = run_attempt(c, H, &e, &tn);
      cudaEventRecord(e1, c->stream);
      if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = MSTAR_ERR_CUDA;
    }
    mstar_free(c);
    if (rc) break;
    const double per = (double)ms / repeats;
    if (ms_out) ms_out[k] = per;
    if (best_k < 0 || per < best) {
      best = per;
      best_k = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) {
    *tile_out = tiles[best_k];
    *split_out = splits[best_k];
  }
  return rc;
}

int mstar_step(mstar_ctx* c, double t_end, int max_gbs_steps, mstar_stats* out) {
  if (!c || !std::isfinite(t_end) || max_gbs_steps < 0) return MSTAR_ERR_INVALID_ARG;
  const mstar_params& p = c->p;
  mstar_stats st{};
  const long long fe0 = c->force_evals;
  int rc = MSTAR_OK;
  const double tol = p.t_tol * std::fabs(t_end);
  while (st.accepted < max_gbs_steps) {
    if (std::fabs(t_end - c->t) <= tol) break;
    double U0, T0;
    const double dt = t_end - c->t;
    double eps = 0.0, tn = c->t;
    // With the controller's step known (c->H != 0), the first attempt is issued right behind
    // the step's preparation, with no read-back between them, and U0 is read with its result.
    // The clamp below depends on U0 alone, so when it applies, that attempt is discarded and
    // the clamped one run: the steps taken are the same as with U0 read first.
    bool have_attempt = false;
    if (c->H != 0.0) {
      // the step-start force evaluation runs inside the attempt, beside its divisions, where the
      // attempt replays as a graph (profiled attempts keep it ahead of the attempt)
      const bool beside = !c->prof && !c->att_graph_off && c->st_stream;
      if ((rc = beside ? issue_tree_and_edges(c) : issue_prepare(c))) break;
      if ((rc = run_attempt(c, std::fabs(c->H) * (dt < 0 ? -1.0 : 1.0), &eps, &tn, beside))) break;
      U0 = c->host_res[2];
      T0 = c->host_res[3];
      have_attempt = true;
    } else if ((rc = prepare_step(c, &U0, &T0))) {
      break;
    }
    (void)T0;
    // Sec. 2.4: first step ds = q U dt, then the controller's step clamped so that the
    // estimated end time t + ds/U does not pass t_end; past t_end, steps head back.
    double Hs = (c->H == 0.0) ? p.q_first * U0 * dt : std::fabs(c->H) * (dt < 0 ? -1.0 : 1.0);
    bool clamped = false;
    if (std::fabs(Hs / U0) >= std::fabs(dt)) {
      Hs = U0 * dt;
      clamped = true;
    }
    if (clamped) {
      if (st.time_iters >= p.max_time_iter) break;
      st.time_iters++;
      have_attempt = false;
    }
    int halvings = 0;
    for (;;) {
      if (have_attempt) {
        have_attempt = false;
      } else if ((rc = run_attempt(c, Hs, &eps, &tn))) {
        goto done;
      }
      if (eps <= p.eta_gbs) break;
      st.rejected++;
      if (++halvings > p.max_halvings) {
        rc = MSTAR_ERR_NO_CONVERGENCE;
        goto done;
      }
      Hs *= 0.5;
    }
    if ((rc = accept_state(c))) break;
    c->at_init = false;
    c->t = tn;
    {
      // Eq. hnext with k = k_fix
      double fac = (eps > 0.0) ? p.a_gbs * std::pow(p.eta_gbs / eps, 1.0 / (2 * c->K - 1)) : p.fac_max;
      if (fac < p.fac_min) fac = p.fac_min;
      if (fac > p.fac_max) fac = p.fac_max;
      c->H = fac * Hs;
    }
    st.accepted++;
    st.eps_last = eps;
  }
done:
  if (rc == MSTAR_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = MSTAR_ERR_CUDA;
  st.force_evals = c->force_evals - fe0;
  st.H = c->H;
  st.t = c->t;
  if (out) *out = st;
  return rc;
}

int mstar_energy(mstar_ctx* c, double* E, double* T, double* U, double P[3], double L[3]) {
  if (!c) return MSTAR_ERR_INVALID_ARG;
  const size_t n3 = (size_t)3 * c->npad;
  CK(cudaMemcpyAsync(c->d.sr + (size_t)c->K * n3, c->d.r, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                     c->stream));
  CK(launch_forces(c, c->K, c->K + 1, 0));
  CK(launch_moments(c));
  CK(cudaMemcpyAsync(c->host_buf, c->d.Ublk + (size_t)c->K * c->nblk, sizeof(double) * c->nblk,
                     cudaMemcpyDeviceToHost, c->stream));
  std::vector<double> mom((size_t)c->nblk * 8);
  CK(cudaMemcpyAsync(mom.data(), c->d.mom, sizeof(double) * mom.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  prof_flush(c);
  double u = 0.0, q[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < c->nblk; ++b) {
    u += c->host_buf[b];
    for (int k = 0; k < 7; ++k) q[k] += mom[(size_t)b * 8 + k];
  }
  const double t = 0.5 * q[0];
  if (T) *T = t;
  if (U) *U = u;
  if (E) *E = t - u;
  if (P)
    for (int k = 0; k < 3; ++k) P[k] = q[1 + k];
  if (L)
    for (int k = 0; k < 3; ++k) L[k] = q[4 + k];
  // the step-start slot buffers were used as scratch; the MST is unaffected
  return MSTAR_OK;
}

long long mstar_launch_count(const mstar_ctx* c) { return c ? c->launches : 0; }

int mstar_profile_enable(mstar_ctx* c, int on) {
  if (!c) return MSTAR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
  prof_flush(c);
  c->prof = on != 0;
  c->prof_used = 0;
  c->prof_launches = c->prof_evals = 0;
  c->prof_ms = c->prof_pairs = 0.0;
  return MSTAR_OK;
}

int mstar_profile_read(mstar_ctx* c, mstar_profile* out) {
  if (!c || !out) return MSTAR_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return MSTAR_ERR_CUDA;
  prof_flush(c);
  out->pair_launches = c->prof_launches;
  out->pair_ms = c->prof_ms;
  out->pair_interactions = c->prof_pairs;
  out->force_evals = c->prof_evals;
  return MSTAR_OK;
}

}  // extern "C"
