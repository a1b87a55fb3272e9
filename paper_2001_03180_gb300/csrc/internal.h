// Host-side declarations shared by the translation units of libmstar (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/mstar.h"

namespace mstar {

constexpr int kBlock = 64;        // threads of the O(N) kernels (more CTAs per slot: their FP64 work spreads over more SMs)
constexpr int kMaxKfix = 12;      // divisions supported (n_k = 2k <= 24)
constexpr int kScal = 8;          // per-slot device scalars
// Largest shared-memory staging of the rebuild walk: a slot's edge vectors and the parents,
// 28 bytes per body (npad up to 7168).
constexpr size_t kRebuildStageBytes = 200 * 1024;

// Per-slot device scalars (sc[slot * kScal + i]).
enum { SC_T_PHYS = 0, SC_T_KIN = 1, SC_U = 2 };

// Device layout of one context. Every array of length npad (a multiple of the pair tile)
// is zero-padded; vectors are three consecutive planes x[npad], y[npad], z[npad].
struct Dev {
  double* m;        // masses (0 in the padding)
  double* r;        // current state positions, COM frame (3 planes)
  double* v;        // current state velocities, COM frame
  int* parent;      // MST parent (-1 root, -3 padding)
  int* gp;          // grandparent (-1 if none, -3 padding)
  int* level;
  int* order;
  int* root;        // [1]
  int* child_off;   // [npad + 1] CSR of children
  int* child_idx;   // [npad]
  int* bylev;       // [npad] the bodies in order of tree level, then index (path-sum order)
  double* X0;       // edge vectors of the step start (3 planes)
  double* V0;
  double* A0;       // relative accelerations a_v - a_parent(v) at the step start
  // per slot: slots 0..K-1 are the divisions (n_k = 2(k+1)), slot K is the step start
  double* sX;       // slots x 3 planes
  double* sV;
  double* sr;
  double* sv;
  double* sa;
  double* P;        // pair partials: slots x NT x 4 x npad
  double* Pt;       // their sums per body: slots x 4 x npad (ax, ay, az, sum of m/r)
  double* Nb;       // the near pairs' sums per body: slots x 4 x npad (written by the pair launches)
  int* tcnt;        // per slot and tile, the tile-pair CTAs counted in (0 between launches)
  double* Ublk;     // slots x nblk
  double* Tblk;     // slots x nblk
  double* comblk;   // slots x nblk x 3
  double* sc;       // slots x kScal scalars
  double* Tkk;      // extrapolated (X 3 planes, V 3 planes, t)
  double* epsblk;   // 2 nblk: the edge-position and edge-velocity maxima per block
  double* res;      // small results read by the host: [0] eps, [1] t, [2] U0, [3] T0
  double* mom;      // nblk x 8 block partials of T, P, L
  char* dc;         // divide-and-conquer tree scratch (mst_method 1 only)
};

}  // namespace mstar

struct mstar_prof_rec {
  cudaEvent_t a, b;
  int nsl;
};

namespace mstar {
// Device buffers that receive one GBS attempt's trajectory when a context's `traj` is set
// (the reverse sweep of the fixed-step adjoint linearises around it). Level tau = 1..2K
// of the attempt has slots lo(tau) = ceil(tau/2) - 1 .. K-1 active (slot s: n = 2(s+1)).
struct AdjTraj {
  double* R;   // [2K][K][3 npad] Cartesian positions at which the forces of level tau act
  double* A;   // [2K][K][3 npad] those accelerations (G included)
  double* Vv;  // [2K][K][3 npad] Cartesian velocities after the kick of level tau
  double* SC;  // [2K + 1][(K + 1) kScal] slot scalars after the drift of level tau (0: first drift)
  double* v0;  // [3 npad] Cartesian velocity of the step start
};
}  // namespace mstar

struct mstar_ctx {
  int n = 0, npad = 0, K = 0, nslots = 0;
  int W = 0, T = 0, NT = 0, ntp = 0;  // pair tiling: warps/CTA, tile, tiles, tile pairs
  int S = 1;                          // warps sharing a tile pair's partner steps (32-body tiles)
  bool div_cta = false;               // attempts run each division in one CTA, in one launch
  int div_cluster = 1;                // ... or in a cluster of this many CTAs (1, 2 or 4)
  bool branched = false;              // attempts issue each division on its own stream
  bool levelled = false;              // attempts go level by level (the adjoint's forward runs)
  cudaStream_t br_stream[mstar::kMaxKfix] = {};  // those streams (created with the context)
  cudaEvent_t br_fork = nullptr, br_join[mstar::kMaxKfix] = {};
  int pair_defer = -1;  // trailing slots of a pair launch summed by the finishing pass (-1: unset)
  size_t rebuild_smem = 0;  // shared memory of the staged rebuild (0: the plain kernel is used)
  int sub_cluster = 0;      // CTAs of the cluster that runs a division's substep level (0: the multi-kernel path)
  int sub_groups = 0;       // 64-body blocks per CTA of that cluster
  int nblk = 0;
  mstar_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  mstar::Dev d{};
  double* host_res = nullptr;  // pinned: [0..7] mirror of d.res, [8..9] staging of the attempt's H and t
  double* host_buf = nullptr;  // pinned staging (nblk * 8 doubles)
  // host-side scalar state (the step control of Sec. 2.3-2.4 runs on the host)
  double t = 0.0, B = 0.0, H = 0.0, Mtot = 0.0;
  bool mst_valid = false;  // the MST/edge buffers describe the current state
  int mst_rounds = 0;      // Boruvka rounds the last exact-MST build ran (issued before its first check)
  bool at_init = false;    // the state is still the one mstar_init set up (no step taken)
  mstar::AdjTraj* traj = nullptr;  // when set, run_attempt records its trajectory here
  long long launches = 0;
  long long force_evals = 0;
  // profiling of the tiled pair kernel: event pairs recorded around each launch, read
  // back after the next host synchronisation
  bool prof = false;
  // an attempt's launches (without profiling) captured as a graph on a private stream and
  // replayed on `stream`: one graph per trajectory record in use (nullptr: none)
  struct AttGraph {
    const mstar::AdjTraj* traj;
    bool levelled;
    bool start;  // the graph also runs the step-start force evaluation, beside the divisions
    cudaGraphExec_t exec;
    long long launches, evals;  // kernel launches and force evaluations per replay
  };
  // attempts issued with att_start run the step-start force evaluation (and the derivatives that
  // end it) on st_stream beside the divisions, joined before the extrapolation, the only kernel
  // of an attempt that reads its results
  bool att_start = false;
  cudaStream_t st_stream = nullptr;
  cudaEvent_t st_fork = nullptr, st_join = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<AttGraph> att_graphs;
  bool att_graph_off = false;  // capture failed once: launch directly
  long long att_launches = 0, att_evals = 0;
  std::vector<mstar_prof_rec> prof_pool;
  size_t prof_used = 0;
  long long prof_launches = 0, prof_evals = 0;
  double prof_ms = 0.0, prof_pairs = 0.0;
};

namespace mstar {

// Layout helpers
size_t workspace_bytes(int n, const mstar_params& p, int* npad_out = nullptr, int* W_out = nullptr);
int choose_tile_warps(int n);

// prim.cu
cudaError_t launch_prim(mstar_ctx* c);      // MST of d.r -> parent, level, order, root
cudaError_t launch_tree(mstar_ctx* c);      // grandparents and children CSR
// boruvka.cu: exact MST by Boruvka rounds; *tied = true asks for the Prim kernel instead
cudaError_t launch_mst_boruvka(mstar_ctx* c, bool* tied);
constexpr int kBoruvkaMinN = 512;           // below this Prim in one CTA is as fast
// BFS orientation of an undirected spanning tree from Prim's root (boruvka.cu)
cudaError_t launch_orient(mstar_ctx* c, const int* eu, const int* ev, int* adj_off, int* adj, int* queue);
// dcmst.cu: divide-and-conquer spanning tree of d.r (Sec. 3.3) into parent/level/root/order
cudaError_t launch_mst_dc(mstar_ctx* c);
size_t dc_scratch_bytes(int n, int nsub);    // device scratch the builder needs
constexpr int kDcMaxSub = 1024;              // largest subgraph count the GPU builder accepts

// pair.cu: slots [slot_lo, slot_hi) -> sa, Ublk. n_d as in params (0 = all Cartesian).
cudaError_t launch_forces(mstar_ctx* c, int slot_lo, int slot_hi, int n_d);
// at context creation: every kernel of an attempt prefers the largest shared-memory share, so that
// the CTAs of different kernels can share an SM (a hint; nothing fails without it)
void prefer_shared_pair_kernels();
void prefer_shared_step_kernels();

// step.cu
cudaError_t launch_prepare(mstar_ctx* c);   // X0, V0, slot K copies, T0 partials
cudaError_t launch_start_derivs(mstar_ctx* c);  // A0 and U0, T0 into d.res
// d.res[4] = H and d.res[5] = t of the attempt (written by stage_attempt_scalars) are read
// by the drift, kick and extrapolation kernels, so that an attempt can be replayed as a graph
cudaError_t upload_step_constants(mstar_ctx* c);
// forget the attempt graphs that record into trajectory buffers (their owner is being freed)
void drop_traj_graphs(mstar_ctx* c);
cudaError_t stage_attempt_scalars(mstar_ctx* c, double H);
cudaError_t launch_init_drift(mstar_ctx* c);
cudaError_t launch_kick(mstar_ctx* c, int slot_lo, int slot_hi);
cudaError_t launch_drift(mstar_ctx* c, int slot_lo, int slot_hi, int tau);
cudaError_t launch_rebuild(mstar_ctx* c, const double* W, double* w, size_t stride, int nsl,
                           int want_T, double* Tblk_base, double* comblk_base);
cudaError_t prepare_rebuild(mstar_ctx* c);  // at context creation: the staged rebuild's shared memory
// kick, velocity rebuild, drift and position rebuild of one level in one CTA per division
// (systems with npad <= kLevelCtaMax: up to 256 bodies, where it beats the multi-CTA path by
// launches saved; above, one SM per division binds its path sums); the divisions >= pos_lo get
// their positions rebuilt
constexpr int kLevelCtaMax = 256;
cudaError_t launch_level_cta(mstar_ctx* c, int slot_lo, int slot_hi, int pos_lo, int tau);
// the same level of a division on a thread-block cluster (kLevelCtaMax < npad <= kSubstepClusterMax),
// in the level-by-level schedule: bit-identical to the multi-kernel kick, rebuild, shift and drift
// launches it replaces. Level-by-level steps of Plummer spheres with a central binary took 5-7 %
// less time with it from 260 to 500 bodies, and 1-2 % more at 640 and 800; beside the pair loops
// of other divisions (a stream per division) the clusters wait for whole SMs and slow those loops
constexpr int kSubstepClusterMax = 576;
cudaError_t prepare_substep_cluster(mstar_ctx* c);  // at context creation; sets sub_cluster
cudaError_t launch_substep_cluster(mstar_ctx* c, int slot_lo, int slot_hi, int pos_lo, int tau);
// a whole attempt's divisions in one launch, one CTA of kDivisionCtaThreads threads each (pair
// sums included): systems with npad <= kDivisionCtaMax (three tasks of 32 bodies per warp, at
// most 15 tile pairs of 32 bodies)
constexpr int kDivisionCtaThreads = 512;
constexpr int kDivisionCtaTasks = kDivisionCtaThreads / 32;
constexpr int kDivisionCtaMax = 160;
constexpr int kDivisionCtaRule = 160;  // the size rule's limit (division_schedule 0)
constexpr size_t division_cta_smem(int npad) {
  return (size_t)npad * (13 * sizeof(double) + sizeof(unsigned long long) + 5 * sizeof(int)) + sizeof(int) +
         (size_t)2 * kDivisionCtaTasks * 7 * 32 * sizeof(double) + (size_t)8 * npad * sizeof(double);
}
// at context creation: the division kernel's shared memory for this size (above 48 KB needs it),
// and the largest cluster size up to the requested one that the device can launch
cudaError_t prepare_division_cta(mstar_ctx* c);
cudaError_t launch_division_cta(mstar_ctx* c);

cudaError_t launch_extrapolate(mstar_ctx* c);
cudaError_t launch_moments(mstar_ctx* c);   // T, P, L partials of the state into d.mom
// w (3 planes of the state) -= centre of mass; optionally T partials into Tblk slot 0
cudaError_t launch_com_shift(mstar_ctx* c, double* w, double* Tblk);

// api.cu
void prof_begin(mstar_ctx* c);
// The pieces of one GBS step (MSTAR_OK or an MSTAR_ERR_* code): the MST and derivative
// information of the step start, one attempt with fictitious step H (records the
// trajectory when c->traj is set), and the acceptance of the extrapolated state.
int step_prepare(mstar_ctx* c, double* U0, double* T0);
int step_attempt(mstar_ctx* c, double H, double* eps, double* tnew);
int step_accept(mstar_ctx* c);
// n x 3 arrays (host or device) to and from three SoA planes of length npad.
int vectors_in(mstar_ctx* c, const double* src, double* planes);
int vectors_out(mstar_ctx* c, const double* planes, double* dst);
void prof_end(mstar_ctx* c, int nsl);

}  // namespace mstar

#define MSTAR_LAUNCHED(c) ((c)->launches++)
