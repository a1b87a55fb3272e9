/*
 * MSTAR oracle: a plain, slow, obviously correct FP64 CPU implementation of one
 * GBS extrapolation step of the algorithmically regularised integrator with
 * minimum-spanning-tree (MST) coordinates, and of the driver that takes such steps
 * to an exact end time (Rantala, Pihajoki, Mannerkoski, Johansson & Naab, "MSTAR").
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the benchmark's CPU
 * baseline load this library; the product (the CUDA library behind include/mstar.h)
 * never does, and the two share no code.
 *
 * Conventions: positions/velocities are n x 3 row-major doubles; G is a parameter.
 * Edge vectors of the MST are stored at the child vertex: W[3*v] = w_v - w_parent(v),
 * zero at the root. Built with -ffp-contract=off, so a*b+c always rounds twice.
 *
 * Parity status of each function is stated beside it: "pinned" functions are checked
 * by CPU tests against facts the paper or mathematics fix. The constants the paper leaves
 * open (a_GBS = 0.9, the growth clamp [0.2, 2], q = 0.1, t_tol = 1e-10) are "parity
 * unpinned": only oracle <-> GPU agreement is checked for them.
 */
#ifndef MSTAR_ORACLE_H
#define MSTAR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double eta;        /* GBS tolerance eta_GBS (Eq. gbs-criterion) */
  double a_gbs;      /* safety factor a_GBS in (0,1] (Eq. hnext) */
  double fac_min;    /* clamp of the step-growth factor (reading; unpinned) */
  double fac_max;
  double q_first;    /* first step ds = q U dt (Sec. 2.4) */
  double t_tol;      /* relative end-time tolerance (Sec. 2.4) */
  double G;          /* gravitational constant */
  int k_fix;         /* number of substep divisions, n_k = 2k (Eq. seq-deuflhard) */
  int n_d;           /* near-pair tree distance N_d (Eq. LCA) */
  int max_halvings;  /* step rejections before giving up (Sec. 2.3) */
  int max_time_iter; /* extra steps towards the end time (Sec. 2.4) */
  int mst_method;    /* 0: Prim's MST (Sec. 3.2); 1: divide-and-conquer tree (Sec. 3.3) */
  int mst_nsub;      /* subgraphs of the divide-and-conquer octree (0: ceil(sqrt(n))) */
} orc_params;

typedef struct {
  long long accepted, rejected, force_evals, time_iters;
  double eps_last, H, t;
} orc_stats;

typedef struct orc_system orc_system;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NONFINITE = -2, ORC_ERR_NO_CONVERGENCE = -3 };

void orc_params_default(orc_params* p);

/* Eq. 1: kinetic energy T and force function U (Cartesian separations). */
double orc_kinetic(int n, const double* m, const double* v);
double orc_potential(int n, const double* m, const double* r, double G);
/* Shift w (n x 3) so that sum m w = 0 (centre-of-mass frame). */
void orc_com_shift(int n, const double* m, double* w);

/* Prim's algorithm (Sec. 3.2) with the indexing of Sec. 3.4. r must be in the COM frame.
   Returns the root; fills parent (-1 at root), level, order (insertion order). Pinned. */
int orc_prim(int n, const double* r, int* parent, int* level, int* order);
/* Chained coordinates (Sec. 2.2): the shortest inter-particle vector starts the chain
   (its lower index is the tail); then the particle closest to the tail or the head joins
   at that end (the tail on a tie, then the lowest index), until all are chained. Written
   as a tree rooted at the final tail: parent[c_k] = c_{k-1}, level[c_k] = k, order = the
   chain from tail to head, so the edge-vector transforms below apply unchanged. Returns
   the tail. Pinned: a Hamiltonian path whose first link is the shortest pair, no shorter
   than the MST; a hand-computed case; <L_chain>/<L_MST> in the paper's range. */
int orc_chain(int n, const double* r, int* parent, int* level, int* order);
/* E = T - U (Eq. 1) with Neumaier-compensated sums. */
double orc_energy_comp(int n, const double* m, const double* r, const double* v, double G);
/* The rebuild test of Sec. 3.5: `cycles` times build the coordinate system (coords 0: the
   MST, 1: the chain) from (r, v), i.e. the edge vectors X, V, and deconstruct them back to
   (r, v) by per-vertex path sums from the vertex up to the root, then either
   (deconstruct 0) the centre-of-mass shift, as the integrator does after every drift and
   kick, or (deconstruct 1) adding the root's kept position; or from the root outwards,
   w_v = w_parent(v) + X_v in insertion order from the root's kept position (deconstruct 2),
   then the centre-of-mass shift (deconstruct 3). The topology is rebuilt every
   `topo_every` cycles (the state moves only by rounding); topo_changes counts rebuilds
   that changed it. E_out[s] = the compensated energy after sample_at[s] cycles (sample_at
   ascending; 0 = the start). mean_level = the mean <L> of the topologies built. */
int orc_rebuild_run(int n, const double* m, double* r, double* v, int coords, int deconstruct, int cycles,
                    int topo_every, int nsample, const int* sample_at, double* E_out, int* topo_changes,
                    double* mean_level);
/* Divide-and-conquer spanning tree (Sec. 3.3): an octree splits the bodies into
   subgraphs of at most leaf_cap bodies (0: ceil(sqrt(n)); cells split while they hold more,
   down to depth 16; leaves in Morton order); Prim's MST inside each subgraph; the
   meta-graph of the contracted subgraphs weighted by their cheapest connecting edge (cut
   property) and its Prim MST; the union of these edges is ordered by a breadth-first walk
   from the root (the body closest to the COM). Same outputs as orc_prim (order: the walk),
   plus the subgraph of every body and the number of subgraphs (either may be NULL).
   Pinned: equal to Prim's tree for one subgraph and for singleton subgraphs; octree
   invariants; local MSTs; meta edges minimal and forming the meta-graph's MST. */
int orc_dc_mst(int n, const double* r, int leaf_cap, int* parent, int* level, int* order, int* leaf_of,
               int* nleaf);
/* Eq. LCA: 1 if i != j are within n_d tree edges. Pinned. */
int orc_is_near(const int* parent, const int* level, int i, int j, int n_d);
/* MST separation r_j - r_i by walking i -> LCA -> j over edge vectors X (Sec. 3.4). Pinned. */
void orc_near_sep(const int* parent, const int* level, const double* X, int i, int j, double d[3]);
/* Cartesian -> MST edge vectors (Eq. chained on MST edges). Pinned (round trip). */
void orc_to_mst(int n, const int* parent, const double* w, double* W);
/* MST edge vectors -> Cartesian: per-vertex path sum, then COM shift (Sec. 3.5). Pinned. */
void orc_from_mst(int n, const double* m, const int* parent, const double* W, double* w);
/* Eq. 2 with the near/far separation rule (Eq. close-chain generalised, Sec. 3.4):
   accelerations a (n x 3) and force function U. Pinned. */
void orc_forces(int n, const double* m, double G, const int* parent, const int* level, int n_d,
                const double* r, const double* X, double* a, double* U);
/* Aitken-Neville polynomial extrapolation in h^2 to h -> 0 (Sec. 4.2). S is kf x nvar.
   Writes T_{kf,kf} and T_{kf-1,kf-1}. Pinned (polynomial exactness). */
void orc_neville(int kf, const int* nseq, int nvar, const double* S, double* Tkk, double* Tprev);
/* Substep-division assignment to ndiv groups (Sec. 4.2): longest first, to the least-loaded
   group, lowest index on ties. Returns max_i C_i; fills group[k]. Pinned (S_div). */
int orc_div_assign(int kf, int ndiv, int* group);
/* Plain leapfrog (triplet (0,0,1)) + GBS step for x'' = -w^2 x: the same DKD and Neville
   code as the N-body step. out[0]=x, out[1]=p extrapolated. Pinned (order H^(2k+1)). */
void orc_gbs_harmonic(double w, double x0, double p0, double H, int kf, double* out, double* out_prev);

/* Eq. gbs-criterion (readings R6-R8): the error of an attempt of fictitious step H from
   the extrapolants Tkk = T_{kf,kf} and Tprev = T_{kf-1,kf-1} (each 6n+1: X, V as n x 3
   edge vectors stored at the child vertex, then t) and the step-start state X0, V0, A0
   (edge vectors; A0 = a_v - a_parent(v)), t0, T0, B, U0. With delta = H/(2 k_fix):
     eps = max over non-root v of |dX_v| / |X0_v + delta V0_v/(T0+B)| and
           |dV_v| / |V0_v + delta A0_v/U0|, and |dt| / |t0 + delta/(T0+B)|,
   d = Tkk - Tprev, |.| the Euclidean norm of a 3-vector, every denominator floored at
   1e-300; NaN if any ratio is NaN. Pinned on hand-worked cases (each term, the root
   skipped, the floor, NaN). */
double orc_gbs_error(int n, const int* parent, const double* Tkk, const double* Tprev, const double* X0,
                     const double* V0, const double* A0, double t0, double T0, double B, double U0, double H,
                     int k_fix);

/* Systems (state owned by the oracle). */
orc_system* orc_create(int n, const double* m, const double* r, const double* v, const orc_params* p);
void orc_free(orc_system* s);
void orc_get_state(const orc_system* s, double* t, double* r, double* v, double* H, double* B);
void orc_set_H(orc_system* s, double H);
/* One GBS step attempt with fictitious step H from the current state; the state is not
   changed. Writes eps and the extrapolated (r, v, t), plus U0 at the step start. Pinned:
   the error estimate has order 2 k_fix - 1 in H; a step of H then -H returns within eps
   (time symmetry); the norm itself through orc_gbs_error. */
int orc_attempt(orc_system* s, double H, double* eps, double* r_out, double* v_out, double* t_out,
                double* U0_out);
/* One leapfrog division with nsub substeps over H from the current state, without
   extrapolation (Sec. 2.3); the state is not changed. Pinned (Kepler exactness). */
int orc_leapfrog(orc_system* s, int nsub, double H, double* r_out, double* v_out, double* t_out);
/* Overwrite the Cartesian state (keeps B, H). */
void orc_set_state(orc_system* s, double t, const double* r, const double* v);
/* Take accepted GBS steps towards t_end (Sec. 2.3-2.4) until |t - t_end| <= t_tol |t_end|
   or max_steps accepted steps. Pinned: the analytic Kepler solution, energy and momentum
   conservation, the end time, and the controller's fixed point a_GBS^(2k_fix-1) eta; the
   values of a_GBS, the growth clamp, q and t_tol are parity unpinned. */
int orc_integrate(orc_system* s, double t_end, int max_steps, orc_stats* st);
/* Energy diagnostics of the current state: E = T - U (Eq. 1), momentum P, angular momentum L. */
void orc_energy(const orc_system* s, double* E, double* T, double* U, double P[3], double L[3]);
/* Fixed-step run: nsteps GBS steps of fictitious step H from the current state, every
   attempt accepted (the error test and step control of Sec. 2.3-2.4 switched off). */
int orc_fixed_run(orc_system* s, double H, int nsteps);
/* Tangent-linear of the fixed-step run from the initial inputs (m, r, v; before the COM
   shift) along (dm, dr, dv): the final state (r_f, v_f, E_f = T - U) and its directional
   derivatives. Cartesian form of the same LogH leapfrog + extrapolation (equal to the MST
   form in real arithmetic); B = U0 - T0 carries its tangent. Pinned: central finite
   differences of orc_fixed_run, translation invariance, rotation equivariance. */
int orc_fixed_run_tl(int n, const double* m, const double* r, const double* v, const double* dm,
                     const double* dr, const double* dv, const orc_params* p, double H, int nsteps,
                     double* r_f, double* v_f, double* E_f, double* dr_f, double* dv_f, double* dE_f);
/* Threads used by the pair loop (OpenMP over i; results do not depend on it). */
void orc_set_threads(int nthreads);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
