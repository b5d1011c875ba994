// Internal device data structures and kernel launchers of the GB300 Sim(3)
// essential-graph optimiser.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pgo.h"

namespace pgo {

// 32-byte aligned 4-vector of doubles (one 256-bit access).
struct alignas(32) D4 {
  double x, y, z, w;
};

// Padded block strides (elements): 7x7 row-major blocks padded so every block
// starts on a 16-byte boundary for vector loads.
constexpr int BLK64 = 50;   // doubles per FP64 block (400 B)
constexpr int BLK32 = 52;   // floats per FP32 block (208 B)
constexpr int VEC = 8;      // per-vertex vector stride (7 used, 1 zero pad)
constexpr int CONTRIB = 36; // per edge-side: 28 upper-triangular H entries + 7 b + pad

// Reduction tickets (one per reducing kernel family).
enum Ticket {
  T_ASSEMBLE = 0, T_PCG_INIT, T_PCG_SPMV, T_PCG_UPDATE, T_UPDATE, T_COST, T_REFINE,
  T_COST_STATELESS, T_POLISH, T_MISC, T_AMG, T_AMG_ABORT, T_AMG_DONE, T_COUNT
};

// Device-resident solver state (LM + PCG scalars); one per graph.
struct SolverState {
  double F0;        // cost at the start of the solve
  double F;         // cost at the current estimate
  double F_new;     // cost at the candidate
  double lambda, nu;
  double pred;      // predicted decrease delta^T (lambda delta - b)
  double gmax;      // |b|_inf (free vertices)
  double maxdiag;   // max diag(H) (free vertices)
  double bnorm2;    // |b|^2 of the LM right-hand side
  double rz, pq, alpha, beta, rr, bb;   // PCG scalars (current linear solve)
  double ref_rr;    // mixed: FP64 residual norm^2 of the refined solution
  int it, accepted, done, need_lin, stop_reason, status, cur, pcg_total;
  int pcg_iter, pcg_done, pcg_hit_cap, ref_done;
  int polish_it, polish_done;
  unsigned ticket[T_COUNT];
};

// Options as read by the kernels (copied from pgo_solve_options per solve).
struct DevOptions {
  int max_iters, precision, pcg_max_iters, refine_steps, polish_iters;
  double tau, lambda_init, ftol, gtol, pcg_tol, refine_tol;
  double lambda_fixed;   // lambda of a standalone re-solve
  int amg_refresh;       // rebuild the coarse multigrid levels every k-th LM linearisation
  int test_absent_block; // test hook: this block of the PCG launch never arrives (-1: none)
};

// ---- smoothed-aggregation multigrid preconditioner ----
// Level 0 is the damped normal matrix over the vertices; level l + 1 has one
// node per aggregate of AMG_M consecutive level-l nodes, with 7 coarse
// unknowns each (the aggregate's rigid Sim(3) motion), down to at most
// AMG_CMAX nodes, which are solved exactly.
constexpr int AMG_M = 4;
constexpr int AMG_CMAX = 8;
constexpr int AMG_MAXL = 12;

// Inner tolerance from which a refinement pass of the mixed solve takes one
// multigrid cycle instead of CG: the FP32 PCG of the first pass leaves an
// FP64 residual of 5e-6 to 1e-3 of |b| (its own recurrence reaches
// refine_tol, the true residual carries the FP32 rounding of the products;
// the worst at the small damping of the last LM iterations), one cycle
// lowers it about tenfold, and an LM step needs no more (the final cost and
// the LM iteration count were the same for linear tolerances up to 1e-3), so
// a correction pass whose target is within 1000x of its residual is one
// cycle; tighter targets (an exact damped step) keep CG.
constexpr double kOneCycleTol = 1e-3;

constexpr int AMG_POWER_ITS = 12;       // first set-up of a graph
constexpr int AMG_POWER_ITS_WARM = 3;   // later set-ups, from the previous vector

struct AmgLevel {
  int n, n_next;          // nodes at this level and at the next
  int nnz_a, nnz_p, nnz_ap, nnz_next;
  // operator of levels >= 1: block-CSR, full rows, the diagonal block first;
  // a_src[k] >= 0: block k is the transpose of block a_src[k]
  const int* a_ptr;
  const int* a_col;
  const int* a_src;
  double* a64;
  float* a32;
  double* dinv64;         // levels >= 1: inverse diagonal blocks
  float* dinv32;
  double* t64;            // tentative prolongation block per node
  float* t32;
  const int* ref;         // reference vertex of each node
  const int* refc;        // reference vertex of the node's aggregate
  const int* agg;         // next-level node of each node (-1: the fixed vertex)
  // smoothed prolongation P (n x n_next): block-CSR, its row per block, CSC
  const int* p_ptr;
  const int* p_col;
  const int* p_row;
  double* p64;
  float* p32;
  const int* pt_ptr;
  const int* pt_row;
  const int* pt_blk;
  // A P (n x n_next), block-CSR
  const int* ap_ptr;
  const int* ap_col;
  double* ap64;
  float* ap32;
  // single-graph hierarchies: Q = (I - D^-1 A / rho) P in the pattern of A P
  // (the prolongation with the post-smoothing folded in), the row of each
  // block, the P block at the same place (-1: none) and the CSC of the pattern
  const int* ap_row;
  const int* ap_pblk;
  const int* apt_ptr;
  const int* apt_row;
  const int* apt_blk;
  double* q64;
  float* q32;
  // numeric recipes (CSR lists of index pairs per output block)
  const int* r1_ptr;      // per P block: (A ref, node w) terms of A T
  const int2* r1;
  const int* r2_ptr;      // per AP block: (A ref, P block)
  const int2* r2;
  const int* r3_ptr;      // per next-level block (upper half): (P block, AP block)
  const int2* r3;
  // processing order of the output blocks of the P, A P and P^T A P phases:
  // by recipe length, longest first, so that the blocks that run side by side
  // (a warp's four, a block's eight teams) have similar lengths
  const int* ord1;        // P phase, eight lanes per block: sorted in windows of 32 blocks
  const int* ord2;        // A P phase, eight lanes per block: the same
  const int* ord1t;       // P and A P phases with 64-thread teams: sorted over the whole list
  const int* ord2t;
  const int* ord3;        // P^T A P phase: sorted over the whole list
  // V-cycle vectors (n x VEC): restricted residual, pre-smoothed iterate,
  // vs: the smoothing part f = x + w D^-1 (r - A x) of the single-graph cycle,
  // or the residual after pre-smoothing of the batch cycle; the result
  double *vr64, *vx64, *vs64, *vy64;
  float *vr32, *vx32, *vs32, *vy32;
  // power-iteration vector kept from the previous set-up (warm start)
  double* pv64;
  float* pv32;
};

struct AmgDev {
  int L;                  // smoothing levels 0..L-1; level L is the coarsest
  int nL;                 // nodes at the coarsest level
  int nseg;               // independent segments (graphs of a batch; 1 otherwise)
  const int* seg_off;     // (L + 1) x (nseg + 1): first node of each segment per level
  AmgLevel lv[AMG_MAXL + 1];
  double* cinv64;         // dense inverse of the coarsest operator (nL x nL blocks;
  float* cinv32;          // per segment AMG_CMAX^2 blocks when nseg > 1)
  // single-graph hierarchies (dense != 0): level L - 1 takes its coarse
  // correction as one dense product, W = Q C^-1 Q^T (n x n blocks, n the
  // nodes of level L - 1), with H = Q C^-1 (n x nL blocks) on the way
  int dense;
  int pad_;
  double* w64;
  float* w32;
  double* h64;
  float* h32;
  double* rho;            // per segment and level: the rho(D^-1 A) the hierarchy was built with
  double* rho_next;       // single graph, per level: the estimate refined during the last set-up
  double* pw64[2];        // power-iteration vectors
  float* pw32[2];
  int* flag;              // per segment, nonzero: the coarsest factorisation failed
  int* warm;              // per segment [2 s] FP64, [2 s + 1] FP32: a previous
                          // set-up left pv vectors
};

// Device view of one graph.
struct DevGraph {
  int N, E, fixed;
  int pcg_block_entries;  // most incidence entries of one PCG row block (0: unknown)
  const int* ei;          // internal (sorted) edge order
  const int* ej;
  const D4* zq;           // measurement quaternion (x, y, z, w), normalised
  const D4* zt;           // measurement (tx, ty, tz, s)
  const double* w;        // weight per edge
  const double* zqn;      // norm of the caller's measurement quaternion (pose8 gradients)
  const double* L;        // E x 28 lower-triangular factor of Omega, or nullptr
  const int* inc_ptr;     // N + 1: incidence CSR over vertices
  const int* inc_code;    // 2E: edge * 2 + side (0: vertex is i, 1: vertex is j)
  const int* inc_other;   // 2E: the other endpoint
  const int* inc_split;   // N: first entry of the vertex's side-1 (v is j) entries;
                          //    each vertex lists its side-0 entries first
  D4* pq[2];              // pose buffers (current = pq[cur])
  D4* pt[2];
  // normal equations
  double* off64;          // E x BLK64  (i, j) block w A_i^T Omega A_j
  float* off32;           // E x BLK32  (mixed)
  double* diag64;         // N x BLK64  H_vv (undamped)
  float* diag32;          // N x BLK32
  double* b;              // N x VEC
  double* contrib;        // E x 2 x CONTRIB per-edge-side contributions
  double* rcache;         // 2 x E x 12 residual cache of the mixed LM loop (r and T per pose buffer)
  // preconditioner (explicit inverse of the damped diagonal block)
  double* minv64;         // N x BLK64
  float* minv32;          // N x BLK32
  // PCG vectors (FP64 and FP32 sets)
  double *x64, *r64, *z64, *p64[2], *q64;
  float *x32, *r32, *z32, *p32[2], *q32;
  double* dx64;           // mixed: accumulated FP64 solution
  double* res64;          // mixed: FP64 refinement residual
  double* partial;        // reduction partials (max blocks)
  int partial_cap;
  SolverState* st;
  DevOptions* opt;
  const AmgDev* amg;      // multigrid hierarchy (device), or nullptr
};

// ---- batched form (one thread block solves one graph at a time) ----
struct BatchGraphState {
  double F0, F, lambda, gmax;
  int it, accepted, pcg_total, stop_reason, status, cur, pad0, pad1;
};

struct BatchArgs {
  int n_graphs;
  const int* v0;       // first vertex of each graph (global index)
  const int* nv;       // vertices per graph
  const int* e0;       // first edge (internal order)
  const int* ne;       // edges per graph
  const int* fixed;    // global index of each graph's fixed vertex
  const int* order;    // processing order (largest first)
  unsigned* queue;     // work counter (zeroed before the launch)
  BatchGraphState* gst;
  int amg;             // 1: multigrid (g.amg holds one segment per graph), 0: block-Jacobi
};

int batch_schedule_count();
int batch_schedule_mixed(int s);
int batch_schedule_lanes(int s);
int batch_schedule_threads(int s);
int batch_schedule_blocks_per_sm(int s);
cudaError_t launch_batch_lm(const DevGraph& g, const BatchArgs& a, int schedule, cudaStream_t s);
void launch_batch_get_poses(const DevGraph& g, const BatchArgs& a, double* dst, cudaStream_t s);
void launch_batch_reset(const DevGraph& g, const BatchArgs& a, cudaStream_t s);

// ---- launchers (each enqueues on `s`; inside stream capture they become
// graph nodes).  `cond` is a graph conditional handle set by the last block
// of the kernel, or 0 when the kernel is not inside a conditional body. ----
void launch_cost(const DevGraph& g, int mode, cudaStream_t s, unsigned long long lm_cond, int store = 0);
void launch_linearize(const DevGraph& g, int mixed, cudaStream_t s);
void launch_assemble(const DevGraph& g, int mixed, cudaStream_t s);
// Mixed precision: the fused linearisation and assembly (k_lin_assemble);
// cached = 1 when the cost kernel has just stored the residuals of the current
// poses (inside the LM loop), else a residual pass runs first.
void launch_lin_assemble_mixed(const DevGraph& g, int cached, cudaStream_t s);
// mode 1: full-Hessian assembly for the adjoint; mode 2: polish step
// (both skip the LM lambda_0 and gradient-stop logic)
void launch_assemble_mode(const DevGraph& g, int mode, cudaStream_t s);
// with_grad: also the edge gradients (Newton polish); 0: zero gradient slots (adjoint)
void launch_adj_hessian(const DevGraph& g, int with_grad, cudaStream_t s);
void launch_adj_rhs(const DevGraph& g, const double* dL, int layout, cudaStream_t s);
void launch_adj_edges(const DevGraph& g, const int* perm, double* dL_dmeas, double* dL_dw, int layout,
                      cudaStream_t s);
void launch_set_meas(const DevGraph& g, const int* perm, const double* meas8, const double* weight,
                     cudaStream_t s);
// state control: 0 prepare a standalone step at lambda = opt->lambda_fixed
// (done = 0, need_lin = 1), 1 swap the current pose buffer
void launch_state_ctl(const DevGraph& g, int op, cudaStream_t s);
void launch_scale_x(const DevGraph& g, double f, cudaStream_t s);
void launch_precond(const DevGraph& g, int mixed, cudaStream_t s);
// amg: host copy of the hierarchy (nullptr: block-Jacobi preconditioner)
// Most incidence entries of one row block of the PCG launch over N rows.
int pcg_block_entries(int N, const int* inc_ptr);
cudaError_t launch_pcg(const DevGraph& g, int mixed, int from_residual, const AmgDev* amg, cudaStream_t s);
// lm: the set-up of an LM iteration (may keep the coarse levels, see
// DevOptions::amg_refresh); 0: a standalone solve (always complete)
cudaError_t launch_amg_setup(const DevGraph& g, const AmgDev& amg, int mixed, int lm, cudaStream_t s);
// Symbolic multigrid hierarchy of a graph (host analysis + one device
// allocation); returns the host copy of the device descriptor.
struct AmgHost;
// The same in two steps: the host analysis (no CUDA call; may run on another
// host thread) and the device allocation and upload.
struct AmgPlan;
AmgPlan* amg_analyze(int N, int nseg, const int* seg_v0, const int* seg_nv, const int* seg_fixed, const int* inc_ptr,
                     const int* inc_code, const int* inc_other, const char** err);
AmgHost* amg_upload(AmgPlan* P, cudaStream_t s, const char** err);
void amg_plan_free(AmgPlan* P);
long long amg_plan_array(const AmgPlan* P, int level, int what, const int** data);
AmgHost* amg_build(int N, int nseg, const int* seg_v0, const int* seg_nv, const int* seg_fixed, const int* inc_ptr,
                   const int* inc_code, const int* inc_other, cudaStream_t s, const char** err);
void amg_free(AmgHost* h);
const AmgDev* amg_host_desc(const AmgHost* h);
const AmgDev* amg_device_desc(const AmgHost* h);
size_t amg_bytes(const AmgHost* h);
int pcg_partials_needed(int N);
void launch_refine_residual(const DevGraph& g, int first, cudaStream_t s);
void launch_refine_accumulate(const DevGraph& g, cudaStream_t s);
void launch_update(const DevGraph& g, int mixed, cudaStream_t s);
void launch_lm_reset(const DevGraph& g, cudaStream_t s);
void launch_resolve_reset(const DevGraph& g, cudaStream_t s);
int max_partials(int N, int E);
void launch_set_poses(const DevGraph& g, const double* src, int buf, cudaStream_t s);
void launch_get_poses(const DevGraph& g, int buf, double* dst, cudaStream_t s);
void launch_residuals(const DevGraph& g, int buf, const int* perm, double* r_out, double* cost_out,
                      cudaStream_t s);
void launch_scatter(int n, int width, const int* perm, const double* src, int sstride, double* dst,
                    int dstride, cudaStream_t s);
void launch_jacobians_out(const DevGraph& g, int buf, const int* perm, double* out, cudaStream_t s);
int eval_cost_blocks(int E);
void launch_eval_cost_raw(int N, int E, const int* ei, const int* ej, const double* meas, const double* w,
                          const double* poses, double* partial, unsigned* ticket, int* bad,
                          double* cost_out, int* bad_out, cudaStream_t s);
void launch_eval_cost_raw_blocks(int N, int E, const int* ei, const int* ej, const double* meas, const double* w,
                                 const double* poses, double* partial, unsigned* ticket, int* bad,
                                 double* cost_out, int* bad_out, int blocks, cudaStream_t s);
// ---- projection search and loop fusion (matching.cu) ----
constexpr int kGridCols = 64;   // image grid of the feature buckets
constexpr int kGridRows = 48;

// Device view of a frames object: K keyframes' features sorted by grid cell.
struct FramesDev {
  int K, n_features;
  float inv_cw, inv_ch;          // grid cells per pixel (x, y)
  const int* kf_ptr;             // K + 1: first feature of each keyframe (caller order)
  const int* cell_ptr;           // K * cells + 1: first sorted feature of each (keyframe, cell)
  const float2* uv;              // sorted: keypoint position
  const int* oct;                // sorted: octave
  const int* orig;               // sorted: the caller's feature index within its keyframe
  const uint4* desc;             // sorted: 256-bit descriptor (2 x uint4)
  const int* mp;                 // caller order: map point id at each feature (-1: none)
  const int* obs_ptr;            // K + 1
  const int* obs_ids;            // per keyframe, ascending: the map point ids it observes
  float* kf_tab;                 // K x 16: per-call keyframe pose table
  unsigned long long* win;       // n_features: per-call claims (distance, point)
};

struct MatchParams {
  float fx, fy, cx, cy, min_x, max_x, min_y, max_y, scale_factor, th, cos_min;
  int n_levels, th_low;
};

struct PointsDev {
  int n;
  const float* xyz;              // n x 3
  const unsigned* desc;          // n x 8
  const float* min_dist;
  const float* max_dist;
  const float* normal;           // n x 3
  const int* id;                 // n (fusion)
};

cudaError_t launch_project_match(const FramesDev& F, const MatchParams& mp, int mode, const double* poses,
                                 const unsigned char* matched, const PointsDev& pts, int* match, int* dist, int* fuse,
                                 cudaStream_t s);

// ---- direct block Cholesky solve of the damped system (direct.cu) ----
struct DirectDev {
  int nb, ns, w;          // band vertices, separators, bandwidth (blocks)
  int n_targets;          // assembled blocks
  long long n_blocks;     // storage blocks (band nb (w+1), border ns nb, corner ns ns)
  size_t border0, corner0;   // offsets (values) of the border and corner storage
  const int* band_v;      // nb: vertex of each band position
  const int* sep_v;       // ns: vertex of each separator
  const int* r_ptr;       // n_targets + 1: recipe of each assembled block
  const int* r_code;      // edge * 2 + transposed, or -(vertex + 1) for a damped diagonal block
  const int* r_dst;       // n_targets: storage block of each target
  float* s32;             // storage (49 values per block), FP32 and FP64
  double* s64;
};
struct DirectHost;
DirectHost* direct_build(int N, int fixed, const int* inc_ptr, const int* inc_code, const int* inc_other,
                         cudaStream_t s, const char** why);
void direct_free(DirectHost* h);
const DirectDev* direct_desc(const DirectHost* h);
bool direct_fits(const DirectHost* h, int mixed, const char** why);
cudaError_t launch_direct_factor(const DevGraph& g, const DirectDev& D, int mixed, cudaStream_t s);
cudaError_t launch_direct_solve(const DevGraph& g, const DirectDev& D, int mixed, int from_residual, cudaStream_t s);

// Loop-correction steps around the optimisation (correction.cu).
cudaError_t launch_propagate_correction(int n, const double* poses, int current, const double* corrected, int n_conn,
                                        const int* conn, double* out, int* bad, cudaStream_t s);
size_t point_table_bytes(int n);
cudaError_t launch_correct_points(int n, const double* before, const double* after, int P, const double* X,
                                  const int* ref, double* table, double* out, int* bad, cudaStream_t s);
void set_last_error(const char* msg);   // message returned by pgo_last_error()
// test hooks: grid-barrier wait limit of the PCG and set-up kernels (ns, 0 = 2 s)
void set_barrier_limit_pcg(unsigned long long ns);
void set_barrier_limit_amg(unsigned long long ns);

}  // namespace pgo
