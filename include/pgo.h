/*
 * pgo.h - C ABI of the GB300 Sim(3) essential-graph optimiser.
 *
 * The operation is the pose graph optimisation step of loop correction
 * (FastLoop, Sec. III-B: after loop fusion, pose graph optimisation over the
 * essential graph propagates the loop correction to every keyframe;
 * Sec. IV-F: Levenberg-Marquardt with automatically differentiated
 * Jacobians; Sec. VI: a Levenberg-Marquardt pose optimisation scheme).
 *
 * Problem (readings where the paper is silent are stated once here):
 *   vertices   keyframe poses S_v = (q, t, s) in Sim(3), world -> camera,
 *              x_c = s R(q) x_w + t, stored as 8 doubles
 *              (qx, qy, qz, qw, tx, ty, tz, s), "pose8" below;
 *   edges      (i, j, Z_ij, w_ij, Omega_ij): measured relative transform
 *              Z_ij ~ S_j S_i^-1 (pose8), scalar weight w (default 1) and
 *              7x7 information Omega (default identity);
 *   residual   r_ij = log(Z_ij S_i S_j^-1) in R^7, tangent order
 *              [omega(3), upsilon(3), sigma(1)];
 *   cost       F = sum_ij w_ij r_ij^T Omega_ij r_ij;
 *   gauge      one fixed vertex (the loop keyframe) is held constant;
 *   update     S_v <- exp(delta_v) S_v (left perturbation), quaternion
 *              renormalised;
 *   LM step    (H + lambda I) delta = -b with H = sum w A^T Omega A,
 *              b = sum w A^T Omega r, A = dr/d(delta) (exact Jacobians);
 *              gain ratio rho = (F - F') / (delta^T (lambda delta - b));
 *              accept if rho > 0 (lambda *= max(1/3, 1 - (2 rho - 1)^3),
 *              nu = 2), else lambda *= nu, nu *= 2;
 *              lambda_0 = tau * max diag(H).
 *
 * Conventions:
 *   - Every call is ordered on the graph's CUDA stream (given at creation).
 *     Calls that return data to host memory, or fill a report, synchronise
 *     that stream before returning.
 *   - Pointers flagged by a mem_space argument are host (PGO_MEM_HOST) or
 *     device (PGO_MEM_DEVICE) memory of the current device; the caller owns
 *     them.  The library copies inputs into its own device buffers.
 *   - Errors: every function returns a pgo_status; pgo_last_error() gives a
 *     thread-local message for the last failure on the calling thread.  A
 *     failing call leaves the graph usable unless it returned PGO_ERR_CUDA.
 *   - Edge-indexed outputs use the caller's edge order.
 */
#ifndef PGO_GB300_H
#define PGO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PGO_OK = 0,
  PGO_ERR_INVALID_ARG = 1,   /* bad size, index, self-edge, non-finite or
                                non-positive scale, NULL where required */
  PGO_ERR_OOM = 2,           /* device or host allocation failed */
  PGO_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  PGO_ERR_NUMERICAL = 4,     /* non-finite cost or a non-PD block */
  PGO_ERR_NOT_CONVERGED = 5, /* an iteration cap was reached */
  PGO_ERR_STATE = 6          /* call out of order (e.g. backward before solve) */
} pgo_status;

typedef enum { PGO_FP64 = 0, PGO_MIXED = 1 } pgo_precision;
typedef enum { PGO_MEM_HOST = 0, PGO_MEM_DEVICE = 1 } pgo_mem_space;
typedef enum { PGO_GRAD_TANGENT7 = 0, PGO_GRAD_POSE8 = 1 } pgo_grad_layout;

/* Graph description (Sec. III-B: the essential graph's keyframes and edges).
 * All arrays are in mem_space.  edge_i/edge_j: int32[n_edges], endpoints in
 * [0, n_vertices), i != j.  meas: double[n_edges * 8] pose8 of Z_ij (the
 * quaternion need not be normalised; it is normalised on copy).  weight:
 * double[n_edges] or NULL (all 1).  info: double[n_edges * 49] row-major
 * symmetric positive definite 7x7 matrices, or NULL (identity).  poses:
 * double[n_vertices * 8] initial estimate, or NULL (set later with
 * pgo_graph_set_poses).  stream: a cudaStream_t (NULL = legacy default
 * stream) on which every later call on this graph is ordered. */
typedef struct {
  int32_t n_vertices;
  int32_t n_edges;
  int32_t fixed_vertex;
  int32_t mem_space;
  const int32_t* edge_i;
  const int32_t* edge_j;
  const double* meas;
  const double* weight;
  const double* info;
  const double* poses;
  void* stream;
} pgo_graph_desc;

/* Preconditioner of the PCG linear solve (Sec. IV-F's damped normal
 * equations).  BLOCK_JACOBI: the inverse 7x7 diagonal blocks of H + lambda I.
 * MULTIGRID: one V(1,1) cycle of smoothed-aggregation multigrid whose coarse
 * unknowns are the rigid Sim(3) motions of runs of 4 consecutive vertices
 * (recursively), block-Jacobi smoothing, dense coarsest solve; its sparsity
 * is analysed once per graph on the host at the first solve that uses it.
 * Both are symmetric positive definite, so either gives the same solution
 * to the PCG tolerance; they differ in iteration count.  Every solve entry
 * point honours this choice: pgo_solve, pgo_graph_damped_step,
 * pgo_graph_resolve, pgo_backward and the batched pgo_batch_solve (where the
 * hierarchy has one independent segment per graph). */
typedef enum { PGO_PRECOND_BLOCK_JACOBI = 0, PGO_PRECOND_MULTIGRID = 1 } pgo_preconditioner;

/* Solve options.  pgo_default_options() fills the documented defaults. */
typedef struct {
  int32_t max_iters;      /* LM iterations, rejected ones included (20) */
  int32_t precision;      /* pgo_precision (PGO_FP64) */
  double tau;             /* lambda_0 = tau * max diag(H) (1e-5) */
  double lambda_init;     /* > 0: use as lambda_0 instead (0) */
  double ftol;            /* stop when |F - F'| <= ftol * F after a step,
                             accepted or rejected (1e-14) */
  double gtol;            /* stop when |b|_inf <= gtol (1e-13) */
  double pcg_tol;         /* PCG: |r| <= pcg_tol * |b| (1e-6; in PGO_MIXED the
                             FP64 refinement residual is held to it).  LM
                             needs no exact step: on the 200- to 4,000-keyframe
                             graphs the final cost and the LM iteration count
                             were the same for every value from 1e-10 to
                             1e-3; pgo_graph_damped_step callers that want
                             an exact step pass a smaller value */
  int32_t pcg_max_iters;  /* PCG iteration cap per linear solve (5000) */
  int32_t refine_steps;   /* PGO_MIXED: FP64 iterative-refinement passes (2):
                             the first solves with FP32 PCG to refine_tol;
                             a later pass whose FP64 residual is within 1000x
                             of pcg_tol |b| applies one multigrid cycle to it
                             (block-Jacobi: PCG), a pass further away runs
                             PCG to the tolerance it needs */
  double refine_tol;      /* PGO_MIXED: inner FP32 PCG relative tolerance (1e-5:
                             on the 2,000- and 4,000-keyframe graphs an inner
                             solve to 1e-5 left the same FP64 residual, about
                             7e-6 of |b|, as one to 1e-6, with one iteration
                             fewer; the FP32 recurrence no longer tracks the
                             FP64 residual below that) */
  int32_t polish_iters;   /* undamped Newton steps after LM on the full
                             Hessian (second-order residual terms included),
                             each kept only while it lowers |b|_2 (0; use > 0
                             before pgo_backward); their PCG runs to
                             min(pcg_tol, 1e-10) */
  int32_t schedule;       /* kernel schedule id; -1 = library default */
  int32_t preconditioner; /* pgo_preconditioner (PGO_PRECOND_MULTIGRID) */
  int32_t multigrid_refresh; /* multigrid inside LM: rebuild the coarse levels
                             at every k-th linearisation, refresh only the
                             finest level in between (1 = always rebuild) */
  int32_t linear_solver;  /* pgo_linear_solver (PGO_SOLVER_PCG) */
} pgo_solve_options;

/* Linear solver of the damped step (Sec. IV-F; Fig. 4 compares a direct
 * factorisation with a GPU sparse solver by problem size).  PCG: the
 * preconditioned conjugate gradient method with opt->preconditioner.
 * DIRECT: a block Cholesky factorisation on the GPU -- in keyframe order the
 * normal matrix is block-banded; the free endpoints of edges longer than 20
 * keyframes (loop edges) are ordered last as separators (at most 16), and
 * one thread block factors the band right-looking with its window in shared
 * memory, then the separators' dense block; the mixed-precision solve
 * factors in FP32 once per LM iteration and reuses the factor in every FP64
 * refinement pass.  PGO_ERR_INVALID_ARG if the graph does not fit these
 * limits (pgo_solve, pgo_graph_damped_step, pgo_graph_resolve only; the
 * adjoint, the Newton polish and the batched form use PCG).  AUTO: DIRECT
 * when the graph fits and has at most PGO_DIRECT_CROSSOVER_VERTICES
 * vertices, PCG otherwise.  The crossover is the size below which DIRECT was
 * measured faster on GB300: on figure-8 graphs of 100 to 2,000 keyframes the
 * multigrid PCG was faster at every size (the sequential factorisation pays
 * a few microseconds of latency per keyframe), so it is 0 and AUTO selects
 * PCG. */
typedef enum { PGO_SOLVER_PCG = 0, PGO_SOLVER_DIRECT = 1, PGO_SOLVER_AUTO = 2 } pgo_linear_solver;
#define PGO_DIRECT_CROSSOVER_VERTICES 0

/* Solve report. */
typedef struct {
  double initial_cost;
  double final_cost;
  double final_lambda;
  double grad_inf_norm;   /* |b|_inf at the last linearisation */
  int32_t iterations;     /* LM iterations executed (rejected included) */
  int32_t accepted;
  int32_t pcg_iterations; /* total inner PCG iterations */
  int32_t stop_reason;    /* 0 max_iters, 1 |dF| <= ftol F, 2 gtol, 3 lambda overflow,
                             4 numerical failure */
  int32_t status;         /* pgo_status of the solve */
  float ms_total;         /* device time of the solve (CUDA events) */
} pgo_report;

typedef struct pgo_graph pgo_graph;
typedef struct pgo_batch pgo_batch;

/* Thread-local message describing the last failure on this thread. */
const char* pgo_last_error(void);

/* Library version string. */
const char* pgo_version(void);

/* Fill *opt with the defaults listed in pgo_solve_options. */
pgo_status pgo_default_options(pgo_solve_options* opt);

/* Create a resident device copy of an essential graph (Sec. III-B, IV-E:
 * keep the data on the GPU and allocate once).  Validates the description,
 * sorts edges by endpoint, builds the block-sparse pattern of the normal
 * matrix and allocates every buffer a solve needs.  The host analysis of the
 * multigrid hierarchy starts on a host thread here (pool threads of the
 * library, created on first use) and is uploaded by the first multigrid
 * solve.  *out receives a handle owned by the caller (free with
 * pgo_graph_destroy).  On error *out is NULL.
 * Process-wide resources, kept until exit and reused by later graphs: the
 * analysis worker threads, small pinned host buffers, and one pinned staging
 * buffer for hierarchy uploads as large as the largest hierarchy's index
 * lists and recipes so far (about 10 MB for 2,000 keyframes). */
pgo_status pgo_graph_create(const pgo_graph_desc* desc, pgo_graph** out);

/* Release every resource of a graph (NULL is ignored).  Synchronises the
 * graph's stream first. */
void pgo_graph_destroy(pgo_graph* g);

/* Replace the current vertex estimate: poses double[n_vertices * 8] pose8 in
 * mem_space.  Quaternions are normalised on copy.  Host poses are validated
 * (finite, non-zero quaternion, scale > 0) and the call returns once they are
 * copied; device poses are copied on the graph's stream with no host round
 * trip and no host validation (a non-finite pose makes the next solve report
 * PGO_ERR_NUMERICAL). */
pgo_status pgo_graph_set_poses(pgo_graph* g, const double* poses, int32_t mem_space);

/* Replace the edge measurements (double[n_edges * 8] pose8, caller's edge
 * order) and, if weight is non-NULL, the weights (double[n_edges]); the graph
 * structure is unchanged (Sec. III-B: loop fusion updates the essential
 * graph's constraints).  Host inputs are validated like pgo_graph_create's;
 * device inputs are copied on the graph's stream without host validation. */
pgo_status pgo_graph_set_measurements(pgo_graph* g, const double* meas, const double* weight,
                                      int32_t mem_space);

/* Copy the current vertex estimate to poses (double[n_vertices * 8]). */
pgo_status pgo_graph_get_poses(pgo_graph* g, double* poses, int32_t mem_space);

/* Cost F at the current estimate (Sec. IV-F objective) and, optionally, the
 * per-edge residuals r_ij (double[n_edges * 7], NULL to skip).  *cost is host
 * memory; residuals are in mem_space. */
pgo_status pgo_graph_cost(pgo_graph* g, double* cost, double* residuals, int32_t mem_space);

/* Linearise at the current estimate (Sec. IV-F: exact Jacobians of every
 * edge residual, then the block-sparse normal equations).  Outputs (any may
 * be NULL) in mem_space, all FP64 whatever the precision:
 *   jac     double[n_edges * 2 * 49]: A_i then A_j per edge, row-major 7x7;
 *   h_diag  double[n_vertices * 49]: diagonal blocks sum w A^T Omega A;
 *   h_off   double[n_edges * 49]: the (i, j) block w A_i^T Omega A_j;
 *   b       double[n_vertices * 7]: sum w A^T Omega r.
 * No rows are dropped: the fixed vertex's blocks are reported as computed. */
pgo_status pgo_graph_linearize(pgo_graph* g, int32_t precision, double* jac, double* h_diag,
                               double* h_off, double* b, int32_t mem_space);

/* One damped linear solve at the current estimate (Sec. IV-F linear solver):
 * (H + lambda I) delta = -b by the preconditioned conjugate gradient method
 * with the preconditioner opt->preconditioner names (block-Jacobi or
 * multigrid; opt NULL = defaults), in opt->precision (mixed: FP32 PCG inside
 * FP64 refinement), the fixed vertex's rows and columns removed.
 * delta: double[n_vertices * 7] in mem_space (fixed row = 0).  *pcg_iters
 * (host, nullable) receives the iteration count.  Returns
 * PGO_ERR_NOT_CONVERGED when opt->pcg_max_iters is reached (delta is still
 * written). */
pgo_status pgo_graph_damped_step(pgo_graph* g, const pgo_solve_options* opt, double lambda,
                                 double* delta, int32_t* pcg_iters, int32_t mem_space);

/* Re-solve the damped system at the last linearisation (the one made by
 * pgo_graph_linearize, pgo_graph_damped_step or the last LM iteration of
 * pgo_solve) for a new lambda, without relinearising: this is the LM step
 * after a rejected update (Sec. IV-F linear solver).  delta (nullable,
 * double[n_vertices * 7] in mem_space) and *pcg_iters (nullable, host)
 * are written after synchronising; with both NULL the call only enqueues the
 * work on the graph's stream and returns. */
pgo_status pgo_graph_resolve(pgo_graph* g, const pgo_solve_options* opt, double lambda, double* delta,
                             int32_t* pcg_iters, int32_t mem_space);

/* The preconditioner set-up of one linear solve at the last linearisation
 * (the one made by pgo_graph_linearize, pgo_graph_damped_step or pgo_solve,
 * in the precision opt->precision names), without the solve (Sec. IV-F
 * linear solver; a piece of pgo_graph_resolve for timing and composition):
 * the inverse damped diagonal blocks (H_vv + lambda I)^-1 and, for
 * PGO_PRECOND_MULTIGRID, the numeric multigrid hierarchy (smoothed
 * prolongations, Galerkin coarse operators, coarsest inverse).  Enqueued on
 * the graph's stream; no synchronisation.  PGO_ERR_STATE without a
 * linearisation. */
pgo_status pgo_graph_precondition(pgo_graph* g, const pgo_solve_options* opt, double lambda);

/* Fill *report from the device state of the last pgo_solve (synchronises the
 * graph's stream); use after a pgo_solve called with report == NULL. */
pgo_status pgo_graph_report(pgo_graph* g, pgo_report* report);

/* Shape of the graph's multigrid hierarchy (PGO_PRECOND_MULTIGRID; analysed
 * at the first solve that uses it, or by this call).  *n_levels receives the
 * number of levels including the coarsest (at most 13); for each level k the
 * host arrays (each with room for 13 entries, nullable) receive its nodes,
 * the 7x7 blocks of its operator (level 0: the graph's stored blocks, one
 * per edge plus one per vertex), of its prolongation P and of A P (0 at the
 * coarsest level).  No counterpart in the paper: it sizes the preconditioner
 * for memory planning and for the roofline accounting of the PCG.
 * PGO_ERR_STATE if the graph has no free vertex. */
pgo_status pgo_graph_multigrid_info(pgo_graph* g, int32_t* n_levels, int32_t* nodes, int64_t* a_blocks,
                                    int64_t* p_blocks, int64_t* ap_blocks);

/* Arrays of the multigrid hierarchy (pgo_graph_multigrid_export). */
typedef enum {
  PGO_MG_A_PTR = 0,   /* levels >= 1: Galerkin operator P^T A P, block-CSR row pointers (n + 1, int32) */
  PGO_MG_A_COL = 1,   /*   its block columns, full rows with the diagonal first (int32) */
  PGO_MG_A = 2,       /*   its blocks */
  PGO_MG_P_PTR = 3,   /* levels < L: smoothed prolongation P (n x n_next), row pointers (int32) */
  PGO_MG_P_COL = 4,   /*   its block columns (int32) */
  PGO_MG_P = 5,       /*   its blocks */
  PGO_MG_AP_PTR = 6,  /* levels < L: pattern of A P, row pointers (int32) */
  PGO_MG_AP_COL = 7,  /*   its block columns (int32) */
  PGO_MG_Q = 8,       /* levels < L: Q = (I - D^-1 A / rho) P in the pattern of A P */
  PGO_MG_DINV = 9,    /* every level: D^-1 per node (level 0: (H_vv + lambda I)^-1, zero at the gauge vertex) */
  PGO_MG_T = 10,      /* levels < L: tentative prolongation block per node */
  PGO_MG_AGG = 11,    /* levels < L: next-level node of each node, -1 for the gauge vertex (int32) */
  PGO_MG_RHO = 12,    /* levels < L: the rho(D^-1 A) that P (4 / (3 rho)) and Q (1 / rho) use (1 value) */
  PGO_MG_W = 13       /* level L - 1: dense W = Q C^-1 Q^T, n x n blocks, block (v, u) at v n + u */
} pgo_mg_array;

/* Copies array `which` (pgo_mg_array) of level `level` of the graph's
 * multigrid hierarchy, as left by its last numeric set-up in `precision`
 * (PGO_FP64 or PGO_MIXED, the FP32 set-up), to the host buffer dst of
 * `capacity` bytes.  *count (nullable) receives the array's element count;
 * dst NULL only queries it.  Integer arrays are int32; numeric arrays are
 * float64, a 7x7 block as 49 row-major values.  L is the coarsest level
 * (pgo_graph_multigrid_info's n_levels - 1).  Test and introspection only
 * (no counterpart in the paper): it lets a test check the set-up's products
 * (Sec. IV-F's damped system, preconditioned) against a plain construction.
 * PGO_ERR_STATE if the hierarchy has not been set up in that precision
 * (a multigrid solve, damped step or pgo_graph_precondition does it);
 * PGO_ERR_INVALID_ARG for an array the level does not have or a buffer
 * smaller than the array.  Synchronises the graph's stream. */
pgo_status pgo_graph_multigrid_export(pgo_graph* g, int32_t level, int32_t which, int32_t precision, void* dst,
                                      int64_t capacity, int64_t* count);

/* Run Levenberg-Marquardt from the current estimate (Sec. IV-F, Sec. VI) and
 * keep the result as the new current estimate.  opt NULL = defaults.
 * report (host, nullable) is filled after synchronising.  poses_out
 * (double[n_vertices * 8], nullable) receives the optimised poses in
 * out_mem_space.  The whole solve runs on the device as one CUDA graph;
 * the host issues no per-iteration work. */
pgo_status pgo_solve(pgo_graph* g, const pgo_solve_options* opt, pgo_report* report,
                     double* poses_out, int32_t out_mem_space);

/* Implicit adjoint of the last solve (extends Sec. IV-F's differentiated
 * objective): with b(x*, Z, w) = 0 at the optimum, mu = H_full^-1 dL/dx and
 * dL/dtheta = -mu^T db/dtheta, H_full the full (second-order) Hessian of F/2.
 *   dL_dposes   N x 7 left-tangent gradient (PGO_GRAD_TANGENT7) or N x 8
 *               gradient w.r.t. the pose8 entries (PGO_GRAD_POSE8);
 *               the fixed vertex's row is ignored;
 *   dL_dmeas    E x 7 left-tangent gradient w.r.t. each Z (TANGENT7) or
 *               E x 8 w.r.t. its pose8 entries (POSE8); nullable;
 *   dL_dweight  E; nullable.
 * Needs a solve converged to a stationary point (use polish_iters > 0);
 * returns PGO_ERR_STATE if no solve has run.  The linear solve uses PCG on
 * H_full (tolerance min(opt->pcg_tol, 1e-10), cap opt->pcg_max_iters). */
pgo_status pgo_backward(pgo_graph* g, const pgo_solve_options* opt, const double* dL_dposes,
                        int32_t grad_layout, double* dL_dmeas, double* dL_dweight,
                        int32_t mem_space);

/* Batched form: many independent graphs of uneven size solved together in
 * one persistent device schedule captured in a CUDA graph.  descs: n_graphs
 * descriptions (host structs; their arrays in each desc's mem_space).
 * stream: the batch's stream. */
pgo_status pgo_batch_create(int32_t n_graphs, const pgo_graph_desc* descs, void* stream,
                            pgo_batch** out);
void pgo_batch_destroy(pgo_batch* b);

/* Solve every graph of the batch with LM (same rules as pgo_solve, per-graph
 * lambda, acceptance and stopping), starting from each graph's current
 * estimate.  One persistent kernel launch (a one-node CUDA graph): each
 * thread block solves whole graphs taken from a device work queue, largest
 * first.  opt->schedule < 0 picks the launch schedule (lanes per block row,
 * threads per block) with the autotuner on the first solve of each
 * precision (one timed LM iteration per candidate; the estimate is restored
 * after each trial); a schedule id >= 0 forces one.  reports: host array of
 * n_graphs (nullable; ms_total is the whole batch).  poses_out: host array
 * of n_graphs pointers, each double[n_vertices_k * 8] in out_mem_space
 * (nullable).  With both NULL the call only enqueues the solve. */
pgo_status pgo_batch_solve(pgo_batch* b, const pgo_solve_options* opt, pgo_report* reports,
                           double* const* poses_out, int32_t out_mem_space);

/* The schedule of the last batch solve: lanes per block row in the SpMV,
 * threads per block, resident blocks per SM (graphs solved side by side on
 * one SM), and the autotuner's best trial time in ms (nullable outputs).
 * PGO_ERR_STATE before the first solve. */
pgo_status pgo_batch_schedule(const pgo_batch* b, int32_t* lanes, int32_t* threads, int32_t* blocks_per_sm,
                              float* tune_ms);

/* Stateless cost evaluation (the Sec. IV-F objective) over caller-owned
 * device arrays: n_vertices poses (pose8), n_edges edges (edge_i, edge_j,
 * meas pose8, weight nullable).  *cost_out is a device double written on
 * `stream`.  An edge with an endpoint outside [0, n_vertices) or with
 * i == j is skipped; *bad_edges_out (device int32, nullable) receives the
 * number of skipped edges on the same stream, so a caller that passes it can
 * tell a complete cost from a partial one.  Uses a temporary device
 * workspace of one double per thread block, allocated and freed on the
 * stream (stream-ordered allocator).  Returns PGO_ERR_INVALID_ARG for
 * negative sizes or NULL arrays. */
pgo_status pgo_evaluate_cost(int32_t n_vertices, int32_t n_edges, const int32_t* edge_i,
                             const int32_t* edge_j, const double* meas, const double* weight,
                             const double* poses, double* cost_out, int32_t* bad_edges_out,
                             void* stream);

/* Loop correction before the pose graph optimisation (Sec. III-B, "Loop
 * Correction": the keyframes connected to the keyframe that closed the loop
 * have their poses corrected with the Sim(3) the loop detection estimated,
 * before the optimisation propagates the correction to the whole map).
 * With S_c the pose of keyframe `current` in `poses` and S_c' = *corrected,
 * every keyframe k listed in `connected` keeps its pose relative to c:
 *     S_k' = (S_k S_c^-1) S_c'
 * (list `current` itself to move it to S_c'); every other keyframe is copied.
 * Arguments (device memory of the current device, caller-owned, ordered on
 * `stream`, no synchronisation):
 *   poses      double[n_vertices * 8] pose8, 16-byte aligned;
 *   corrected  double[8] pose8 of S_c', 16-byte aligned;
 *   connected  int32[n_connected] keyframe indices (an index outside
 *              [0, n_vertices) is skipped and counted);
 *   poses_out  double[n_vertices * 8], 16-byte aligned, must not overlap
 *              poses; quaternions written normalised with w >= 0;
 *   bad_out    int32 (nullable): number of skipped indices.
 * PGO_ERR_INVALID_ARG for bad sizes, a current index out of range, NULL or
 * misaligned arrays, or overlapping poses_out. */
pgo_status pgo_propagate_correction(int32_t n_vertices, const double* poses, int32_t current,
                                    const double* corrected, int32_t n_connected, const int32_t* connected,
                                    double* poses_out, int32_t* bad_out, void* stream);

/* Map-point correction (Sec. III-B: the loop correction carried from the
 * keyframes to the map).  A point keeps its position in the camera frame of
 * its reference keyframe r while that keyframe's pose changes from
 * S_before[r] to S_after[r]:
 *     x' = S_after[r]^-1 (S_before[r] x),   S x = s R x + t.
 * Used after pgo_propagate_correction (before = the poses it read, after =
 * its output, the connected keyframes' points listed) and after pgo_solve
 * (before = the initial estimate, after = the optimised poses, every point).
 * Arguments (device memory, caller-owned, ordered on `stream`):
 *   poses_before, poses_after  double[n_vertices * 8] pose8, 16-byte aligned;
 *   points      double[n_points * 3] world coordinates (x, y, z);
 *   ref_kf      int32[n_points]: reference keyframe of each point; r < 0
 *               leaves the point unchanged, r >= n_vertices also leaves it
 *               unchanged and is counted;
 *   points_out  double[n_points * 3]; may be `points` itself (in place);
 *   bad_out     int32 (nullable): number of points with r >= n_vertices.
 * Uses a temporary device table of 128 bytes per keyframe from the
 * stream-ordered allocator.  PGO_ERR_INVALID_ARG for bad sizes or NULL or
 * misaligned pose arrays. */
pgo_status pgo_correct_points(int32_t n_vertices, const double* poses_before, const double* poses_after,
                              int32_t n_points, const double* points, const int32_t* ref_kf,
                              double* points_out, int32_t* bad_out, void* stream);

/* ---- projection search and loop fusion (Sec. IV-D) ----
 * Map points are projected into keyframes with a Sim(3) pose and matched to
 * the keyframes' features by 256-bit (ORB) descriptor distance within a
 * window around the projection: the projection searches PS1 and PS3a-c
 * (correspondences between map points and one or three keyframes) and the
 * loop fusion (duplicate map points between the loop's map points and each
 * connected keyframe's).  Per (keyframe, point) pair, in single precision:
 *   p = s R x + t (pose (q, t, s) taken to float, R = R(q / |q|)), rejected
 *   if p_z <= 0; u = fx p_x / p_z + cx, v = fy p_y / p_z + cy, rejected
 *   outside [min_x, max_x) x [min_y, max_y); d = |x - O| with O = -(R^T t)/s
 *   the camera centre, rejected unless min_dist <= d <= max_dist, and if
 *   (x - O) . n < cos_min d; level = smallest L >= 0 with
 *   max_dist <= d scale^L (at most n_levels - 1); candidates: features with
 *   |u_f - u| < r, |v_f - v| < r (r = th scale^level) and octave in
 *   [level - 1, level] (search: not matched before); the best candidate has
 *   the smallest Hamming distance (ties: lower feature index) and is a match
 *   if its distance is <= th_low.
 * Conflicts: search -- a feature chosen by several points goes to the one
 * with the smallest (distance, point index), the others get no match;
 * fusion -- a feature that holds a map point makes every loop point choosing
 * it fuse with that point; otherwise the smallest (distance, point index)
 * adds its observation and the other points choosing it fuse with that one.
 * The paper names the operations only; these rules follow the ORB-SLAM
 * system it builds on. */
typedef struct pgo_frames pgo_frames;

typedef enum { PGO_MATCH_SEARCH = 0, PGO_MATCH_FUSE = 1 } pgo_match_mode;

/* Keyframe features (Sec. IV-E: kept resident on the device).  feat_ptr:
 * host int32[n_keyframes + 1], keyframe k owns features
 * [feat_ptr[k], feat_ptr[k + 1]) of the arrays below (in mem_space):
 * uv float[F * 2] keypoint (u, v); octave int32[F]; desc uint32[F * 8];
 * map_point int32[F] map point id at each feature, -1 = none (nullable: all
 * -1).  The image bounds define the 64 x 48 feature grid and must equal the
 * match parameters' bounds.  stream: every call on the object is ordered on
 * it. */
typedef struct {
  int32_t n_keyframes;
  int32_t mem_space;
  const int32_t* feat_ptr;
  const float* uv;
  const int32_t* octave;
  const uint32_t* desc;
  const int32_t* map_point;
  float min_x, max_x, min_y, max_y;
  void* stream;
} pgo_frames_desc;

/* Camera and search parameters (pixels; th: search radius at octave 0;
 * th_low: largest accepted Hamming distance; cos_min: smallest cosine of the
 * viewing angle). */
typedef struct {
  float fx, fy, cx, cy;
  float min_x, max_x, min_y, max_y;
  float scale_factor, th, cos_min;
  int32_t n_levels, th_low;
} pgo_match_params;

/* Map points (device memory): xyz float[n * 3] world position; desc
 * uint32[n * 8] (16-byte aligned); min_dist, max_dist float[n] scale
 * invariance range; normal float[n * 3] mean viewing direction (unit);
 * id int32[n] map point ids (fusion; nullable for the search). */
typedef struct {
  int32_t n_points;
  const float* xyz;
  const uint32_t* desc;
  const float* min_dist;
  const float* max_dist;
  const float* normal;
  const int32_t* id;
} pgo_points_desc;

/* Copy keyframe features to the device, bucketed by grid cell.  *out is NULL
 * on error; free with pgo_frames_destroy. */
pgo_status pgo_frames_create(const pgo_frames_desc* desc, pgo_frames** out);
void pgo_frames_destroy(pgo_frames* f);

/* Every (keyframe, point) pair (Sec. IV-D: one thread per map point and
 * keyframe).  poses: device double[n_keyframes * 8] pose8 (16-byte aligned),
 * the pose each keyframe is projected with (the Sim(3) estimate for the
 * search, the corrected pose for fusion).  matched: device uint8[F] in the
 * caller's feature order, nonzero = matched before this search (search only,
 * nullable).  Outputs (device, n_keyframes * n_points, keyframe-major):
 * match int32 feature index within the keyframe or -1; dist int32 Hamming
 * distance of the pair's best candidate (256: none; search losers 256);
 * fuse int32 (fusion only): the map point id the point fuses with, -1 = it
 * adds a new observation or has no match.  A fusion pair whose keyframe
 * already observes the point (a feature holds its id) has no match.  Ordered
 * on the frames' stream; no synchronisation. */
pgo_status pgo_project_match(pgo_frames* f, const pgo_match_params* params, int32_t mode, const double* poses,
                             const uint8_t* matched, const pgo_points_desc* points, int32_t* match,
                             int32_t* dist, int32_t* fuse);

/* pgo_evaluate_cost without any device allocation (no counterpart in the
 * paper: an addition for callers that cannot allocate device memory at call
 * time, such as a real-time loop-closing thread that must not stall on the
 * allocator, or an application that reserves the whole device memory budget
 * at start-up).  Same arguments and result as pgo_evaluate_cost, computed by
 * the same kernel, but its workspace is a fixed 33,024-byte array inside the
 * library's device image, held by every GPU that loads the library until the
 * process exits.  Limits and rules:
 *   - n_edges <= 1,048,576, else PGO_ERR_INVALID_ARG (use pgo_evaluate_cost);
 *   - the first call in each CUDA context, with that context's device
 *     current, looks up the workspace address (cudaGetSymbolAddress) and
 *     caches it with the context's unique id (a new context, e.g. after
 *     cudaDeviceReset, triggers a new look-up): make that first call before
 *     any stream capture;
 *   - every call shares the one workspace and it keeps the last call's
 *     contents (each call clears its counters first); calls that overlap on
 *     the GPU, from several streams or threads, race and must be avoided;
 *   - it calls no cudaMalloc, cudaFree or allocating library routine. */
pgo_status pgo_evaluate_cost_noalloc(int32_t n_vertices, int32_t n_edges, const int32_t* edge_i,
                                     const int32_t* edge_j, const double* meas, const double* weight,
                                     const double* poses, double* cost_out, int32_t* bad_edges_out,
                                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PGO_GB300_H */
