/*
 * mstar.h - C ABI of the GB300 (sm_103a) FP64 implementation of the MSTAR hot path:
 * one GBS extrapolation step of the algorithmically regularised integrator with
 * minimum-spanning-tree (MST) coordinates (Rantala, Pihajoki, Mannerkoski, Johansson &
 * Naab, "MSTAR - a fast parallelised algorithmically regularised integrator with minimum
 * spanning tree coordinates", MNRAS 2020).
 *
 * Problem (Sec. 2.1, Eq. 1-2): N point masses m_i with positions r_i and velocities v_i,
 * Newtonian gravity with constant G, H = T - U. The integrator uses the logarithmic
 * Hamiltonian time transformation (triplet (1,0,0), Eq. ttl): dt/ds = 1/(T+B),
 * dr/ds = v/(T+B), dv/ds = a/U with B = -H. One GBS step over a fictitious interval H
 * builds the MST with Prim's algorithm (Sec. 3.2), switches to MST edge coordinates
 * (Sec. 3.4), runs k_fix leapfrog divisions with n_k = 2k substeps (Eq. seq-deuflhard,
 * Sec. 2.3) concurrently (Sec. 4.2), extrapolates them with the Aitken-Neville
 * polynomial scheme (Sec. 4.2) and tests convergence (Eq. gbs-criterion). Steps are
 * halved on failure, grown by Eq. hnext on success, and clamped to reach an exact end
 * time (Sec. 2.4).
 *
 * Conventions for every entry point:
 *  - All arithmetic is IEEE binary64 (FP64). G defaults to 1.
 *  - Arrays of vectors are n x 3 row-major doubles (x0 y0 z0 x1 ...).
 *  - Array arguments may be host or device pointers; the library detects which with
 *    cudaPointerGetAttributes. The caller owns every array it passes; inputs are copied,
 *    outputs are written before the call returns (the call synchronises its stream).
 *  - A context owns its device memory: either the caller-provided workspace (at least
 *    mstar_workspace_bytes() bytes, 256-byte aligned, owned by the caller and kept alive
 *    until mstar_free) or, when workspace is NULL, memory the library allocates itself.
 *  - All GPU work of a context runs on the CUDA stream given at init (NULL = legacy
 *    default stream). Contexts are not thread-safe; distinct contexts are independent.
 *  - Return value: MSTAR_OK (0) or a negative MSTAR_ERR_* code. No call throws.
 *    After MSTAR_ERR_CUDA the context must be freed.
 */
#ifndef MSTAR_H
#define MSTAR_H

#include <stddef.h>

#if defined(__GNUC__)
#define MSTAR_API __attribute__((visibility("default")))
#else
#define MSTAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MSTAR_OK 0
#define MSTAR_ERR_INVALID_ARG (-1)    /* bad size, pointer, parameter, mass <= 0 */
#define MSTAR_ERR_NONFINITE (-2)      /* non-finite input value */
#define MSTAR_ERR_NO_CONVERGENCE (-3) /* more than max_halvings step rejections */
#define MSTAR_ERR_TIMEOUT (-4)        /* a bounded device wait gave up */
#define MSTAR_ERR_CUDA (-5)           /* a CUDA runtime call failed */
#define MSTAR_ERR_UNSUPPORTED (-6)    /* outside the sizes this build supports */
#define MSTAR_ERR_NOMEM (-7)          /* workspace too small or allocation failed */

/* Largest system a single context accepts (the one-CTA Prim kernel keeps the tree in
   shared memory and registers). */
#define MSTAR_MAX_N 10240

typedef struct mstar_ctx mstar_ctx;

/* Parameters; mstar_default_params() fills the defaults given beside each field. */
typedef struct {
  double eta_gbs;    /* GBS tolerance eta_GBS of Eq. gbs-criterion. 1e-12 */
  double a_gbs;      /* safety factor a_GBS in (0,1] of Eq. hnext. 0.9 */
  double fac_min;    /* lower clamp of the step-growth factor of Eq. hnext. 0.2 */
  double fac_max;    /* upper clamp of the step-growth factor. 2.0 */
  double q_first;    /* first step ds = q U dt (Sec. 2.4), dt = t_end - t. 0.1 */
  double t_tol;      /* relative end-time tolerance |t - t_end| <= t_tol |t_end|. 1e-10 */
  double G;          /* gravitational constant. 1.0 */
  int k_fix;         /* number of substep divisions, n_k = 2k, 2 <= k_fix <= 12. 8 */
  int n_d;           /* near-pair tree distance N_d of Eq. LCA, 0 <= n_d <= 2. 2 */
  int max_halvings;  /* rejections of one step before MSTAR_ERR_NO_CONVERGENCE. 30 */
  int max_time_iter; /* end-time-clamped steps per mstar_step call (Sec. 2.4). 8 */
  int mst_method;    /* spanning tree of each step: 0 Prim's MST (Sec. 3.2), 1 the divide-and-conquer
                        tree of Sec. 3.3 (octree subgraphs, their MSTs joined by the meta-graph's
                        MST; a few per cent longer than the MST). Batches always use 0. 0 */
  int mst_nsub;      /* subgraphs of the divide-and-conquer octree, 0 = ceil(sqrt(n)), at most
                        1024. 0 */
  int pair_tile;     /* bodies per tile of the pair loop: 32, 64 or 128, or 0 for the size rule
                        (32 up to 4096 bodies, 64 up to 8192, 128 above); mstar_tune_pair_tile
                        times the choices on a given system. 0 */
  int pair_split;    /* warps that share the 32 partner steps of a tile pair, with 32-body tiles:
                        1, 2, 4 or 8, or 0 for the size rule (4 up to 512 bodies, else 1); the
                        other tiles take 1. Partial sums are added in warp order, so results
                        differ from the unsplit loop by rounding only. 0 */
  int division_schedule; /* how an attempt's k_fix divisions are issued: 1 level by level (the
                        kernels of a substep level for every division active at it: one CTA per
                        division for up to 256 padded bodies, a thread-block cluster per division
                        for up to 576, else one launch per kernel; all bit-identical), 2 each
                        division on its own stream (longer divisions at higher priority), so that
                        one division's small kernels overlap another's pair loop, 3 each division
                        on one CTA, or a cluster of them (division_cluster), from its first drift
                        to its last, pair sums included, all divisions in one launch (systems of at
                        most 160 padded bodies; larger ones take the size rule), 0 for the size
                        rule (3 up to 160 padded bodies, 2 from 1000 bodies, else 1). 1 and 2
                        give bit-identical results; 3 sums the pair forces in another order, so
                        its results differ from theirs by rounding. Attempts that record an
                        adjoint trajectory or time the pair kernel, and the forward runs of the
                        adjoint, use 1. 0 */
  int division_cluster; /* CTAs per division under division_schedule 3: 1, or 2, 4 or 8 as a
                        thread-block cluster that shares out the pair sums and reads the partials
                        through distributed shared memory, or 0 for the size rule (4 up to 32
                        padded bodies, else 8; halved at context creation while the device cannot
                        launch it). The pair sums are chunked by the cluster size, so results
                        differ between sizes by rounding. 0 */
} mstar_params;

/* Counters of one mstar_step call, and the state after it. */
typedef struct {
  long long accepted;    /* accepted GBS steps */
  long long rejected;    /* rejected attempts (each halved H) */
  long long force_evals; /* pair-loop evaluations (73 per attempt at k_fix = 8) */
  long long time_iters;  /* steps whose H was clamped to land on t_end */
  double eps_last;       /* error of the last accepted step (Eq. gbs-criterion) */
  double H;              /* fictitious step proposed for the next step (Eq. hnext) */
  double t;              /* physical time reached */
} mstar_stats;

MSTAR_API void mstar_default_params(mstar_params* p);

/* Device bytes a context for n bodies needs under p (for a caller-provided workspace). */
MSTAR_API size_t mstar_workspace_bytes(int n, const mstar_params* p);

/* Create a context: copies m[n] (> 0), r[n x 3], v[n x 3], shifts them to the centre-of-
   mass frame, and computes B = U - T (B = -H, Sec. 2.1). The physical time starts at 0
   and the next fictitious step is unset (the first mstar_step uses ds = q U dt).
   n must be in [2, MSTAR_MAX_N]. cuda_stream is a cudaStream_t (NULL: default stream).
   Errors: INVALID_ARG, NONFINITE, UNSUPPORTED, NOMEM, CUDA. On error *out is NULL. */
MSTAR_API int mstar_init(mstar_ctx** out, int n, const double* m, const double* r, const double* v,
               const mstar_params* p, void* workspace, size_t workspace_bytes, void* cuda_stream);

/* Take accepted GBS steps towards t_end (Sec. 2.3-2.4) until |t - t_end| <= t_tol |t_end|,
   or max_gbs_steps steps were accepted, or max_time_iter clamped steps were taken.
   Each step: MST (Prim), edge coordinates, one pair-loop evaluation at the step start
   (for the error norm's S'), k_fix concurrent leapfrog divisions, Neville-Aitken
   extrapolation, the convergence test; rejected steps are retried with H/2. Once the
   controller's step is known, a step's first attempt is issued right behind the MST and edge
   coordinates, runs the step-start evaluation beside its divisions, and U0 is read back with
   that attempt's result; when the clamp to t_end then applies, that attempt is discarded and
   the clamped one taken, so the steps are those of reading U0 first.
   out (may be NULL) receives the counters of this call. Errors: NO_CONVERGENCE, CUDA. */
MSTAR_API int mstar_step(mstar_ctx* ctx, double t_end, int max_gbs_steps, mstar_stats* out);

/* One GBS step attempt with fictitious step H > 0 (or < 0) from the current state,
   without step control; the state is not changed. Writes the error eps of Eq.
   gbs-criterion and the extrapolated state (r_out, v_out: n x 3, COM frame; t_out);
   any output pointer may be NULL. */
MSTAR_API int mstar_attempt(mstar_ctx* ctx, double H, double* eps, double* r_out, double* v_out,
                  double* t_out);

/* Energy diagnostics of the current state (Eq. 1): E = T - U with the Cartesian pair
   sum, total momentum P and angular momentum L about the origin. NULL outputs skipped. */
MSTAR_API int mstar_energy(mstar_ctx* ctx, double* E, double* T, double* U, double P[3], double L[3]);

/* Read / replace the current state (t, r[n x 3], v[n x 3]). get_state returns the state in
   the centre-of-mass frame; any output may be NULL. set_state keeps B and H and takes r and v
   as given: the caller keeps them in the centre-of-mass frame (as get_state returns them);
   a non-finite state makes the next step fail with NO_CONVERGENCE. Errors: INVALID_ARG (NULL
   ctx; for set_state also NULL r or v, or a non-finite t), CUDA. */
MSTAR_API int mstar_get_state(mstar_ctx* ctx, double* t, double* r, double* v);
MSTAR_API int mstar_set_state(mstar_ctx* ctx, double t, const double* r, const double* v);

/* Set the next fictitious step H (0 = unset: the next mstar_step uses ds = q U dt).
   Errors: INVALID_ARG (NULL ctx or a non-finite H). */
MSTAR_API int mstar_set_H(mstar_ctx* ctx, double H);

/* Prim's MST of the current positions (Sec. 3.2) and its indexing (Sec. 3.4): root
   (closest to the centre of mass, lowest index on ties), parent[n] (-1 at the root),
   level[n], order[n] (insertion order). Ties: argmin takes the lowest index, keys are
   replaced only by strictly smaller squared distances. Any output may be NULL.
   With order == NULL the tree comes from the builder the GBS step uses (Boruvka rounds for
   n >= 512, which yield Prim's tree whenever no two deciding distances are equal, and
   Prim's kernel otherwise); with order != NULL Prim's kernel runs and reports the order. */
MSTAR_API int mstar_get_mst(mstar_ctx* ctx, int* root, int* parent, int* level, int* order);

/* One pair-loop evaluation on the current state (Eq. 2 with the near/far separation rule
   of Sec. 3.4 on the current MST): accelerations a[n x 3] and force function U. */
MSTAR_API int mstar_accelerations(mstar_ctx* ctx, double* a, double* U);

/* Tuner with no counterpart in the paper: for the system (n, m, r, v) under p, creates a
   context for each of four pair loops - 32-body tiles with the partner steps split over 4
   warps, and unsplit tiles of 32, 64 and 128 bodies - (allocating and freeing its
   workspace), times `repeats` GBS step attempts of each with CUDA events on cuda_stream after
   one untimed attempt, and returns the fastest as *tile_out and *split_out, with the mean
   attempt time of each in ms_out[4] (in that order; may be NULL). The attempts are those of
   the multi-kernel schedules (division_schedule 1, or 2 from 1000 bodies, unless p asks for 1
   or 2): one CTA per division has no tiles. The attempts change no
   state; the caller sets p.pair_tile and p.pair_split to the result for its own context. An
   attempt's work does not depend on its fictitious step, which is set to 1e-6 U. Errors as
   mstar_init. */
MSTAR_API int mstar_tune_pair_tile(int n, const double* m, const double* r, const double* v, const mstar_params* p,
                                   int repeats, int* tile_out, int* split_out, double* ms_out, void* cuda_stream);

MSTAR_API void mstar_free(mstar_ctx* ctx);
MSTAR_API const char* mstar_strerror(int code);

/* Kernel launches the context has issued since init (for launch accounting). */
MSTAR_API long long mstar_launch_count(const mstar_ctx* ctx);

/* Device timing of the pair-loop kernel (the dominant kernel), for roofline reporting.
   While enabled, every launch of the tiled pair kernel is bracketed by CUDA events on the
   context's stream; mstar_profile_read sums their elapsed times. Enabling resets the
   counters. */
typedef struct {
  long long pair_launches;    /* tiled pair-kernel launches timed */
  double pair_ms;             /* summed device time of those launches */
  double pair_interactions;   /* unordered pair interactions they evaluated (N(N-1)/2
                                 per force evaluation, near pairs included) */
  long long force_evals;      /* force evaluations those launches covered */
} mstar_profile;
MSTAR_API int mstar_profile_enable(mstar_ctx* ctx, int on);
MSTAR_API int mstar_profile_read(mstar_ctx* ctx, mstar_profile* out);

/* Diagnostic with no counterpart in the paper: measures the FP64 FMA issue rate of the
   current device (FMAs per second over all SMs, 8 independent chains per thread) on the
   given stream, for reporting the pair loop against the chip's measured FP64 roofline.
   Allocates and frees a small device buffer. */
MSTAR_API int mstar_fp64_fma_rate(double* fma_per_second, void* cuda_stream);

/* ---- Batched independent systems (Sec. 4.2: the parallel method extends to many
   independent N-body systems integrated simultaneously). */

/* Largest system of a batch (one CTA builds its MST with at most 4 keys per thread). */
#define MSTAR_BATCH_MAX_N 512

/* Size classes of the batch schedule: n in [2,8], [9,16], [17,32], [33,64], [65,128],
   [129,256], [257,512]. */
#define MSTAR_BATCH_NUM_CLASSES 7

typedef struct mstar_batch mstar_batch;

typedef struct {
  long long accepted;    /* accepted GBS steps, summed over the systems */
  long long rejected;    /* rejected attempts (each halved that system's H) */
  long long force_evals; /* pair-loop evaluations */
  int finished;          /* systems that reached t_end or stopped (status != 0) */
  int failed;            /* systems stopped by an error (status < 0) */
} mstar_batch_stats;

/* Device bytes a batch needs (0 if the sizes or parameters are invalid). */
MSTAR_API size_t mstar_batch_workspace_bytes(int nsys, const int* offsets, const mstar_params* p);

/* Create a batch of nsys independent systems. offsets[nsys + 1] (host) is a CSR over the
   concatenated bodies: system s owns bodies offsets[s] .. offsets[s+1]-1, each system has
   2 .. MSTAR_BATCH_MAX_N bodies. m[nbody], r[nbody x 3], v[nbody x 3] (host or device) are
   copied; each system is shifted to its own centre-of-mass frame and gets its own B = U - T,
   time 0 and unset step. Workspace as for mstar_init (NULL: allocated by the library).
   Errors: INVALID_ARG, NONFINITE, UNSUPPORTED (a system above MSTAR_BATCH_MAX_N or a
   coordinate >= 1e15), NOMEM, CUDA. */
MSTAR_API int mstar_batch_init(mstar_batch** out, int nsys, const int* offsets, const double* m, const double* r,
                               const double* v, const mstar_params* p, void* workspace, size_t workspace_bytes,
                               void* cuda_stream);

/* `launches` launches of the batch's CUDA graph; each advances every unfinished system by
   one GBS step attempt towards t_end (accepted: the state and time advance and H grows by
   Eq. hnext; rejected: H halves for the next launch; Sec. 2.3-2.4 as in mstar_step, per
   system). A system stops at |t - t_end| <= t_tol |t_end|, after max_time_iter
   end-time-clamped steps, or (status -3) after more than max_halvings successive
   rejections. Each system runs four division groups of G warps (G from the schedule, by
   size class), in one CTA or split over four CTAs; its k_fix divisions go to the groups by
   the greedy longest-first recipe of Sec. 4.2. The graph holds one independent kernel node
   per schedule in use (a chain of three for a split schedule). Synchronises the stream; out
   may be NULL. */
MSTAR_API int mstar_step_batched(mstar_batch* b, double t_end, int launches, mstar_batch_stats* out);

/* Per-system time t[nsys], state r, v (nbody x 3, host or device), last error eps[nsys]
   and status[nsys] (0 running, 1 at t_end, 2 time-iteration limit, -3 no convergence). Any
   output may be NULL. */
MSTAR_API int mstar_batch_get_state(mstar_batch* b, double* t, double* r, double* v, double* eps, int* status);

/* Set every system's next fictitious step (host array H[nsys]; 0 = unset). */
MSTAR_API int mstar_batch_set_H(mstar_batch* b, const double* H);

/* Schedule of the batch, for each of the MSTAR_BATCH_NUM_CLASSES size classes:
     1, 2, 4     G warps per division group, one CTA of 4 G warps per system;
     -1, -2, -4  G = |value| warps per division group, the attempt split into three graph
                 nodes: the start (MST, derivative information, step size; one CTA per
                 system), the divisions (one CTA of G warps per system and group, so that
                 a system's groups run on up to four SMs) and the finish (extrapolation,
                 error, step control; one CTA per system);
     0           for the classes of at most 16 bodies: four division groups of 8 (class 0;
                 4 for systems of at most 4 bodies, two systems per warp) or 16 (class 1)
                 lanes per system, one body per lane, the group's state in registers and the
                 pair rotation and tree sums done by warp shuffles.
   A new schedule rebuilds the graph (INVALID_ARG for any other value). The default is 0, 0,
   1, 1, 1, 2, 4. The schedule changes only the work split, not the arithmetic of a system
   beyond the order in which partial sums are added (a split schedule gives the same results
   as the one-CTA schedule of the same G). */
MSTAR_API int mstar_batch_set_schedule(mstar_batch* b, const int* schedule);
MSTAR_API int mstar_batch_get_schedule(const mstar_batch* b, int* schedule);

/* Autotuner with no counterpart in the paper (its GPU analogue of choosing how many
   processes work on one force loop, Sec. 4.3): two passes of coordinate descent over the
   size classes present, largest first, timing one graph launch towards t_end (best of
   `repeats`, after a warm-up) for each allowed schedule with the other classes fixed, and
   keeping the fastest. Trials run on a snapshot of the batch, which is put back: the
   systems' state, time and step sizes are unchanged. Allocates a temporary device copy of
   the workspace (NOMEM if that fails). Sets and returns the schedule (schedule_out may be
   NULL) and the launch time it measured in ms (ms_out may be NULL). */
MSTAR_API int mstar_batch_autotune(mstar_batch* b, double t_end, int repeats, int* schedule_out, double* ms_out);

/* Kernel launches issued so far (graph kernel nodes count one each per graph launch). */
MSTAR_API long long mstar_batch_launch_count(const mstar_batch* b);
MSTAR_API void mstar_batch_free(mstar_batch* b);

/* Largest n that mstar_accelerations_noalloc accepts. Its scratch is a fixed static device
   array of about 1.1 MB (positions, masses and the per-tile partial sums for 2048 bodies). */
#define MSTAR_NOALLOC_MAX_N 2048

/* No counterpart in the paper: an allocation-free form of the pair loop, for callers that
   may not allocate device memory - for example a sub-integrator living inside a larger code
   whose memory manager owns the whole device heap, or a host loop that cannot afford the
   device synchronisation cudaMalloc implies. It needs no context and calls no allocating
   routine (no cudaMalloc/cudaFree, no allocating library call).
   Computes, with every pair taken as far (Cartesian separations, as n_d = 0), the
   accelerations a_i = G sum_j m_j (r_j - r_i)/|r_j - r_i|^3 and the force function
   U = G sum_{i<j} m_i m_j / |r_j - r_i|. Its own kernel (128-body tiles, an FP64 reciprocal
   square root, a plain FP64 sum of U) is not the context's pair kernel: the results agree
   with mstar_accelerations on a context created with n_d = 0 to rounding (1e-13 relative),
   not bit for bit, since the reduction order and the scalar arithmetic differ.
   Arguments: n in [2, MSTAR_NOALLOC_MAX_N] (larger n: MSTAR_ERR_UNSUPPORTED); m[n] and
   r[n x 3] (row-major) inputs, a[n x 3] and U[1] outputs - all four DEVICE (or managed)
   pointers owned by the caller (host pointers: MSTAR_ERR_INVALID_ARG); G > 0. The work is
   queued on cuda_stream and the call returns without waiting for it.
   Scratch: one file-scope static __device__ array that every GPU loading the library holds
   until the process exits. Every call uses the same array and overwrites what the previous
   call left there (each call rewrites all it reads), so calls that overlap on the GPU - on
   different streams or from different threads - race and must be serialised by the caller.
   The first call on each device looks up the array's device address (cudaGetSymbolAddress);
   make that first call before capturing a stream into a graph. */
MSTAR_API int mstar_accelerations_noalloc(int n, const double* m, const double* r, double G, double* a,
                                          double* U, void* cuda_stream);


/* ---- Adjoint of a fixed-step run (no counterpart in the paper; reverse-mode derivative
   of the method of Sec. 2-4 with the step control switched off). */

typedef struct mstar_adjoint mstar_adjoint;

/* Forward pass: nsteps GBS steps of fixed fictitious step H (k_fix divisions each, every
   attempt accepted: no error test, no step-size control or end-time clamp) from the state
   that mstar_init set up; the context must not have been stepped or given a new state
   since (INVALID_ARG otherwise). Keeps (r, v) of every `checkpoint_every`-th step start in
   device memory owned by *out (NOMEM if it cannot be allocated), and the trajectories of
   the last segment's steps, which the reverse sweep needs first. The context ends at the
   final state. Errors as mstar_step; on error *out is NULL. */
MSTAR_API int mstar_adjoint_forward(mstar_ctx* c, double H, int nsteps, int checkpoint_every, mstar_adjoint** out);

/* Reverse sweep of the run recorded by `a` for the loss L whose gradients with respect to
   the final state are g_r = dL/dr_f, g_v = dL/dv_f (n x 3, host or device; NULL = 0) and
   g_E = dL/dE_f (E_f = T - U of the final state, Eq. 1). Writes dL/dm (n), dL/dr, dL/dv
   (n x 3) with respect to the masses, positions and velocities given to mstar_init,
   through the centre-of-mass shift and B = U0 - T0 (any output may be NULL). Each segment
   of checkpoint_every steps whose trajectories are not already held (the last one, after
   the forward) is recomputed from its checkpoint with its trajectory recorded; the
   transposed substeps then run in reverse, one VJP pair loop per kick. The
   MST of each step is held fixed (its topology is piecewise constant). The context ends at
   the final state of the run. May be called again with other loss gradients. */
MSTAR_API int mstar_step_adjoint(mstar_ctx* c, mstar_adjoint* a, const double* g_r, const double* g_v, double g_E,
                                 double* d_r, double* d_v, double* d_m);
MSTAR_API void mstar_adjoint_free(mstar_adjoint* a);


/* ---- The rebuild test of Sec. 3.5 (a numerical experiment on the coordinate systems). */

/* Largest system of mstar_rebuild_test (one CTA holds a job's state in shared memory). */
#define MSTAR_REBUILD_MAX_N 1024

/* njobs independent runs of the rebuild test of Sec. 3.5 on systems of n bodies: each job
   builds its coordinate system from the Cartesian state and deconstructs it back `cycles`
   times, and records E = T - U (Eq. 1, Neumaier-compensated sums in index order) after
   sample_at[s] cycles (ascending; 0 = the start) in E_out[job * nsample + s].
   coords[job]: 0 the MST (Prim, Sec. 3.2; root closest to the centre of mass), 1 the chain
   of Sec. 2.2 (shortest pair first, then the particle closest to either end, the tail on a
   tie), as a path tree rooted at its tail. Building: X_v = w_v - w_parent(v). Deconstruction:
   deconstruct[job] 0: per-vertex sums of the edge vectors from the vertex up to the root,
   then the centre-of-mass shift (the integrator's rebuild); 1: the same sums plus the root's
   kept position; 2: from the root outwards, w_v = w_parent(v) + X_v with every parent before
   its children, from the root's kept position; 3: as 2, then the centre-of-mass shift.
   The topology is rebuilt every topo_every cycles; topo_changes[job] counts rebuilds that
   changed it and mean_level[job] is the mean level <L> of the trees built. m (njobs x n),
   r and v (njobs x n x 3), outputs: host or device; r_out, v_out, topo_changes, mean_level
   may be NULL. The operations and their order are those of the CPU
   definition, so the results are bit-identical to it. Allocates and frees device scratch;
   synchronises the stream. Errors: INVALID_ARG (n outside [2, MSTAR_REBUILD_MAX_N], other
   bad arguments), NOMEM, CUDA. */
MSTAR_API int mstar_rebuild_test(int njobs, int n, const double* m, const double* r, const double* v,
                                 const int* coords, const int* deconstruct, int cycles, int topo_every, int nsample,
                                 const int* sample_at, double* E_out, double* r_out, double* v_out, int* topo_changes,
                                 double* mean_level, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MSTAR_H */
