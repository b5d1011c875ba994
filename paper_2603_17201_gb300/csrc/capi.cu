// Host runtime and C ABI of the GB300 Sim(3) essential-graph optimiser.
//
// pgo_graph_create validates the description, orders edges by their lower
// endpoint, builds the vertex incidence lists that define the block-sparse
// pattern of the normal matrix and allocates every device buffer once
// (FastLoop keeps its loop-closing data resident on the GPU and allocates
// once, Sec. IV-E).  pgo_solve replays one CUDA graph per (precision,
// refinement passes): a WHILE node runs the LM iterations and a nested WHILE
// node runs the PCG iterations, with every decision taken on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <future>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace pgo;

namespace {

thread_local std::string g_last_error;

pgo_status fail(pgo_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CUDA_TRY(expr)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      if (e_ == cudaErrorMemoryAllocation)                                                     \
        return fail(PGO_ERR_OOM, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return fail(PGO_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                          \
  } while (0)

// Test hook: fail device allocations above this many bytes (0 = off).
size_t g_alloc_limit = 0;
// Test hook of the bounded grid barrier: a PCG block that never arrives
// (-1 = off).
int g_test_absent_block = -1;

// One device arena per graph, sub-allocated with 256-byte alignment.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

template <class T>
size_t arena_bytes(size_t count) {
  return (count * sizeof(T) + 255) & ~size_t(255);
}

bool copy_in(void* dst, const void* src, size_t bytes, int mem_space, cudaStream_t s) {
  if (bytes == 0) return true;
  cudaMemcpyKind kind = mem_space == PGO_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  return cudaMemcpyAsync(dst, src, bytes, kind, s) == cudaSuccess;
}

// Helper that assembles a CUDA graph from captured segments and WHILE nodes.
struct GraphBuilder {
  cudaStream_t cs;
  std::vector<cudaGraphNode_t> tail;
  cudaError_t err = cudaSuccess;

  void capture(cudaGraph_t graph, const std::function<void(cudaStream_t)>& fn) {
    if (err != cudaSuccess) return;
    err = cudaStreamBeginCaptureToGraph(cs, graph, tail.empty() ? nullptr : tail.data(), nullptr, tail.size(),
                                        cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return;
    fn(cs);
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    err = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
    std::vector<cudaGraphNode_t> nt;
    if (err == cudaSuccess) nt.assign(deps, deps + ndeps);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &out);
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess && !nt.empty()) tail = nt;
  }

  // Adds a WHILE node after the current tail; returns its body graph.
  cudaGraph_t add_while(cudaGraph_t graph, cudaGraphConditionalHandle h) {
    if (err != cudaSuccess) return nullptr;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    err = cudaGraphAddNode(&node, graph, tail.empty() ? nullptr : tail.data(), nullptr, tail.size(), &p);
    if (err != cudaSuccess) return nullptr;
    tail.assign(1, node);
    return p.conditional.phGraph_out[0];
  }
};

}  // namespace

namespace pgo {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace pgo

// Small pinned host buffers (a graph's solver-state and options staging),
// recycled across graphs for the life of the process: a cudaMallocHost /
// cudaFreeHost pair per graph costs more than the rest of creating a small
// graph.
static std::mutex g_pinned_mu;
static std::map<size_t, std::vector<void*>> g_pinned_free;

static void* pinned_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto& v = g_pinned_free[bytes];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free[bytes].push_back(p);
}

struct pgo_graph {
  int N = 0, E = 0, fixed = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  Arena arena;
  DevGraph g{};
  int* d_perm = nullptr;          // internal edge -> caller edge
  double* d_scratch = nullptr;    // N * 8 doubles + E * 98 staging for exports
  size_t scratch_doubles = 0;
  double* d_cost = nullptr;
  SolverState* h_state = nullptr; // pinned copy for reports
  DevOptions* h_opt = nullptr;    // pinned staging of options
  std::map<long long, cudaGraphExec_t> execs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool solved = false;
  bool has_info = false;
  bool lin_valid = false;
  // multigrid hierarchy: its host analysis starts on a host thread at
  // creation (it needs only the incidence lists), the upload happens at the
  // first solve that uses it
  AmgHost* amg = nullptr;
  bool amg_failed = false;
  std::future<AmgPlan*> amg_plan;
  const char* amg_plan_err = nullptr;
  // direct block Cholesky structure, analysed at the first solve that asks for it
  DirectHost* direct = nullptr;
  bool direct_failed = false;
  std::string direct_why;
  std::vector<int> h_inc_ptr, h_inc_code, h_inc_other;
};

struct pgo_batch {
  pgo_graph* G = nullptr;          // the graphs concatenated (disjoint vertex and edge ranges)
  int n = 0;
  std::vector<int> nv, ne, v0;
  BatchArgs args{};                // device pointers
  void* meta = nullptr;            // device allocation holding the per-graph arrays
  double* saved_poses = nullptr;   // autotuning: the estimate to restore after each trial
  int schedule = -1;               // tuned schedule per precision and preconditioner
  int tuned[4] = {-1, -1, -1, -1}; // [mixed + 2 * multigrid]
  float tune_ms[4] = {0.f, 0.f, 0.f, 0.f};
  std::map<int, cudaGraphExec_t> execs;
  std::vector<int> fixed;          // gauge vertex of each graph (concatenated index)
  bool amg_failed = false;
  bool schedule_amg = false;       // the last solve used multigrid
};

namespace {

void fill_dev_options(const pgo_solve_options& o, DevOptions* d) {
  d->max_iters = o.max_iters;
  d->precision = o.precision;
  d->pcg_max_iters = o.pcg_max_iters;
  d->refine_steps = o.refine_steps;
  d->polish_iters = o.polish_iters;
  d->tau = o.tau;
  d->lambda_init = o.lambda_init;
  d->ftol = o.ftol;
  d->gtol = o.gtol;
  d->pcg_tol = o.pcg_tol;
  d->refine_tol = o.refine_tol;
  d->lambda_fixed = 0.0;
  d->amg_refresh = o.multigrid_refresh;
  d->test_absent_block = g_test_absent_block;
}

pgo_status check_options(const pgo_solve_options& o) {
  if (o.max_iters < 0 || o.pcg_max_iters < 1 || o.refine_steps < 1 || o.refine_steps > 16)
    return fail(PGO_ERR_INVALID_ARG, "options: max_iters >= 0, pcg_max_iters >= 1, 1 <= refine_steps <= 16");
  if (o.precision != PGO_FP64 && o.precision != PGO_MIXED)
    return fail(PGO_ERR_INVALID_ARG, "options: unknown precision %d", o.precision);
  if (!(o.tau > 0) || !(o.pcg_tol > 0) || !(o.refine_tol > 0) || !(o.ftol >= 0) || !(o.gtol >= -1.0))
    return fail(PGO_ERR_INVALID_ARG, "options: tau, pcg_tol, refine_tol must be > 0");
  if (o.preconditioner != PGO_PRECOND_BLOCK_JACOBI && o.preconditioner != PGO_PRECOND_MULTIGRID)
    return fail(PGO_ERR_INVALID_ARG, "options: unknown preconditioner %d", o.preconditioner);
  if (o.multigrid_refresh < 1) return fail(PGO_ERR_INVALID_ARG, "options: multigrid_refresh must be >= 1");
  if (o.linear_solver != PGO_SOLVER_PCG && o.linear_solver != PGO_SOLVER_DIRECT && o.linear_solver != PGO_SOLVER_AUTO)
    return fail(PGO_ERR_INVALID_ARG, "options: unknown linear_solver %d", o.linear_solver);
  return PGO_OK;
}

// How one damped linear solve runs: the direct factorisation (dd) or PCG with
// the multigrid hierarchy (amg) or block-Jacobi (both nullptr).
struct LinSolve {
  const AmgDev* amg = nullptr;
  const DirectDev* dd = nullptr;
};

// The preconditioner set-up and the PCG launches of one linear solve at the
// current linearisation (amg: multigrid hierarchy, nullptr: block-Jacobi).
void enqueue_pcg(const DevGraph& g, int mixed, const AmgDev* amg, int from_residual, cudaStream_t s,
                 cudaError_t* err) {
  cudaError_t e = launch_pcg(g, mixed, from_residual, amg, s);
  if (e != cudaSuccess && *err == cudaSuccess) *err = e;
}

// The block-Jacobi blocks (H_vv + lambda I)^-1, or the multigrid set-up,
// whose first phase forms the same blocks as its level-0 smoother.
void enqueue_precond(const DevGraph& g, int mixed, const AmgDev* amg, cudaStream_t s, cudaError_t* err, int lm = 0) {
  if (!amg) {
    launch_precond(g, mixed, s);
    return;
  }
  cudaError_t e = launch_amg_setup(g, *amg, mixed, lm, s);
  if (e != cudaSuccess && *err == cudaSuccess) *err = e;
}

// The linear-solve part of one LM iteration.  PCG: the preconditioner
// (block-Jacobi blocks, plus the multigrid hierarchy when enabled), then one
// persistent PCG launch (FP64), or, in mixed precision, FP32 PCG launches
// inside FP64 iterative refinement (refine_steps passes, each skipped on the
// device once the FP64 residual meets pcg_tol).  Direct: the block Cholesky
// factorisation, then the triangular solves (in mixed precision one FP32
// factorisation serves every refinement pass).
void enqueue_linear_solve(const DevGraph& g, int mixed, int refine_steps, LinSolve ls, cudaStream_t s,
                          cudaError_t* err, int lm = 0) {
  auto keep = [&](cudaError_t e) {
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
  };
  if (ls.dd) {
    keep(launch_direct_factor(g, *ls.dd, mixed, s));
    if (!mixed) {
      keep(launch_direct_solve(g, *ls.dd, 0, 0, s));
      return;
    }
    for (int pass = 0; pass < refine_steps; ++pass) {
      launch_refine_residual(g, pass == 0, s);
      keep(launch_direct_solve(g, *ls.dd, 1, 1, s));
      launch_refine_accumulate(g, s);
    }
    return;
  }
  enqueue_precond(g, mixed, ls.amg, s, err, lm);
  if (!mixed) {
    enqueue_pcg(g, 0, ls.amg, 0, s, err);
    return;
  }
  for (int pass = 0; pass < refine_steps; ++pass) {
    launch_refine_residual(g, pass == 0, s);
    enqueue_pcg(g, 1, ls.amg, 1, s, err);
    launch_refine_accumulate(g, s);
  }
}

// Linearisation and assembly at the current poses: FP64 per edge, then the
// per-vertex gather; mixed, the fused kernel (cached: the cost kernel of
// these poses stored their residuals).
void linearize_assemble(const DevGraph& g, int mixed, int cached, cudaStream_t s) {
  if (mixed) {
    launch_lin_assemble_mixed(g, cached, s);
    return;
  }
  launch_linearize(g, 0, s);
  launch_assemble(g, 0, s);
}

// One LM iteration (the body of the WHILE node, or one host-driven step).
// The mixed mode linearises with the fused kernel from the residuals that
// the cost kernel of the same poses stored (the start cost, or the accepted
// candidate's).
void enqueue_lm_body(const DevGraph& g, int mixed, int refine_steps, LinSolve ls, cudaStream_t s,
                     unsigned long long lm_cond, cudaError_t* err) {
  linearize_assemble(g, mixed, 1, s);
  enqueue_linear_solve(g, mixed, refine_steps, ls, s, err, 1);
  launch_update(g, mixed, s);
  launch_cost(g, 1, s, lm_cond, mixed);
}

// The hierarchy (host descriptor) if the options ask for multigrid and the
// graph has one; nullptr selects block-Jacobi.
const AmgDev* amg_for(const pgo_graph* G, int precond) {
  return precond == PGO_PRECOND_MULTIGRID && G->amg ? amg_host_desc(G->amg) : nullptr;
}

// Analyses the multigrid hierarchy of the graph the first time a solve asks
// for it.  A graph without free vertices has nothing to precondition and
// keeps block-Jacobi.
pgo_status ensure_amg(pgo_graph* G, int precond) {
  if (precond != PGO_PRECOND_MULTIGRID || G->amg || G->amg_failed) return PGO_OK;
  if (G->N < 2) {
    G->amg_failed = true;
    return PGO_OK;
  }
  const char* err = nullptr;
  if (G->amg_plan.valid()) {
    AmgPlan* P = G->amg_plan.get();   // waits for the analysis started at creation
    err = G->amg_plan_err;
    if (P) {
      G->amg = amg_upload(P, G->stream, &err);
      amg_plan_free(P);
    }
  } else {
    const int v0 = 0, nv = G->N, fx = G->fixed;
    G->amg = amg_build(G->N, 1, &v0, &nv, &fx, G->h_inc_ptr.data(), G->h_inc_code.data(), G->h_inc_other.data(),
                       G->stream, &err);
  }
  if (!G->amg) return fail(PGO_ERR_OOM, "multigrid set-up: %s", err ? err : "unknown error");
  G->g.amg = amg_device_desc(G->amg);
  return PGO_OK;
}

// The linear solver of a solve: analyses the direct structure (and the
// multigrid hierarchy) the first time they are asked for.  DIRECT on a graph
// that does not fit its limits is an error; AUTO falls back to PCG.
pgo_status choose_solver(pgo_graph* G, const pgo_solve_options& o, LinSolve* ls) {
  *ls = LinSolve{};
  const int mixed = o.precision == PGO_MIXED;
  if (o.linear_solver != PGO_SOLVER_PCG) {
    const bool want = o.linear_solver == PGO_SOLVER_DIRECT || G->N <= PGO_DIRECT_CROSSOVER_VERTICES;
    if (want && !G->direct && !G->direct_failed) {
      const char* why = nullptr;
      if (G->N < 2) {
        G->direct_failed = true;
        G->direct_why = "the graph has no free vertex";
      } else {
        G->direct = direct_build(G->N, G->fixed, G->h_inc_ptr.data(), G->h_inc_code.data(), G->h_inc_other.data(),
                                 G->stream, &why);
        if (!G->direct) {
          G->direct_failed = true;
          G->direct_why = why ? why : "unknown";
        }
      }
    }
    if (want && G->direct) {
      const char* why = nullptr;
      if (direct_fits(G->direct, mixed, &why)) {
        ls->dd = direct_desc(G->direct);
        return PGO_OK;
      }
      if (o.linear_solver == PGO_SOLVER_DIRECT) return fail(PGO_ERR_INVALID_ARG, "direct solver: %s", why);
    } else if (o.linear_solver == PGO_SOLVER_DIRECT) {
      return fail(PGO_ERR_INVALID_ARG, "direct solver: %s", G->direct_why.c_str());
    }
  }
  pgo_status st = ensure_amg(G, o.preconditioner);
  if (st != PGO_OK) return st;
  ls->amg = amg_for(G, o.preconditioner);
  return PGO_OK;
}

pgo_status build_solve_graph(pgo_graph* G, int mixed, int refine_steps, LinSolve ls, cudaGraphExec_t* out) {
  const DevGraph& g = G->g;
  cudaGraph_t graph;
  CUDA_TRY(cudaGraphCreate(&graph, 0));
  GraphBuilder b{G->cap_stream};
  cudaGraphConditionalHandle hl;
  b.err = cudaGraphConditionalHandleCreate(&hl, graph, 0, 0);
  b.capture(graph, [&](cudaStream_t s) {
    launch_lm_reset(g, s);
    launch_cost(g, 0, s, hl, mixed);
  });
  cudaGraph_t body = b.add_while(graph, hl);
  if (body) {
    GraphBuilder lb{G->cap_stream};
    cudaError_t le = cudaSuccess;
    lb.capture(body, [&](cudaStream_t s) { enqueue_lm_body(g, mixed, refine_steps, ls, s, hl, &le); });
    if (lb.err != cudaSuccess) b.err = lb.err;
    if (le != cudaSuccess) b.err = le;
  }
  if (b.err != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(PGO_ERR_CUDA, "building the solve graph: %s", cudaGetErrorString(b.err));
  }
  cudaError_t e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, "instantiating the solve graph: %s", cudaGetErrorString(e));
  return PGO_OK;
}

// A linear solve at a given lambda (pgo_graph_damped_step): linearise, then
// the same linear-solve sequence as one LM iteration.
pgo_status build_step_graph(pgo_graph* G, int mixed, int refine_steps, LinSolve ls, cudaGraphExec_t* out) {
  const DevGraph& g = G->g;
  cudaGraph_t graph;
  CUDA_TRY(cudaGraphCreate(&graph, 0));
  GraphBuilder b{G->cap_stream};
  cudaError_t le = cudaSuccess;
  b.capture(graph, [&](cudaStream_t s) {
    linearize_assemble(g, mixed, 0, s);
    enqueue_linear_solve(g, mixed, refine_steps, ls, s, &le);
  });
  if (le != cudaSuccess) b.err = le;
  if (b.err != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(PGO_ERR_CUDA, "building the step graph: %s", cudaGetErrorString(b.err));
  }
  cudaError_t e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, "instantiating the step graph: %s", cudaGetErrorString(e));
  return PGO_OK;
}

// Host-driven LM loop with plain stream launches (schedule 1): the same
// kernels, for profilers that cannot look inside conditional graph nodes.
pgo_status run_eager(pgo_graph* G, int mixed, int refine_steps, int max_iters, LinSolve ls) {
  const DevGraph& g = G->g;
  cudaStream_t s = G->stream;
  cudaError_t le = cudaSuccess;
  launch_lm_reset(g, s);
  launch_cost(g, 0, s, 0, mixed);
  for (int it = 0; it < max_iters + 1; ++it) {
    CUDA_TRY(cudaMemcpyAsync(G->h_state, g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (G->h_state->done || G->h_state->it >= max_iters) break;
    enqueue_lm_body(g, mixed, refine_steps, ls, s, 0, &le);
    CUDA_TRY(le);
    CUDA_TRY(cudaGetLastError());
  }
  return PGO_OK;
}

// Re-solve at the last linearisation: state reset, then the linear solve.
pgo_status build_resolve_graph(pgo_graph* G, int mixed, int refine_steps, LinSolve ls, cudaGraphExec_t* out) {
  const DevGraph& g = G->g;
  cudaGraph_t graph;
  CUDA_TRY(cudaGraphCreate(&graph, 0));
  GraphBuilder b{G->cap_stream};
  cudaError_t le = cudaSuccess;
  b.capture(graph, [&](cudaStream_t s) {
    launch_resolve_reset(g, s);
    enqueue_linear_solve(g, mixed, refine_steps, ls, s, &le);
  });
  if (le != cudaSuccess) b.err = le;
  if (b.err != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(PGO_ERR_CUDA, "building the re-solve graph: %s", cudaGetErrorString(b.err));
  }
  cudaError_t e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, "instantiating the re-solve graph: %s", cudaGetErrorString(e));
  return PGO_OK;
}

pgo_status get_exec(pgo_graph* G, int kind, int mixed, int refine_steps, LinSolve ls, cudaGraphExec_t* out) {
  const long long key = ((long long)kind << 32) | ((long long)(ls.dd != nullptr) << 25) |
                        ((long long)(ls.amg != nullptr) << 24) | ((long long)mixed << 16) | (mixed ? refine_steps : 0);
  auto it = G->execs.find(key);
  if (it != G->execs.end()) {
    *out = it->second;
    return PGO_OK;
  }
  cudaGraphExec_t ex = nullptr;
  pgo_status st = kind == 0   ? build_solve_graph(G, mixed, refine_steps, ls, &ex)
                  : kind == 1 ? build_step_graph(G, mixed, refine_steps, ls, &ex)
                              : build_resolve_graph(G, mixed, refine_steps, ls, &ex);
  if (st != PGO_OK) return st;
  G->execs[key] = ex;
  *out = ex;
  return PGO_OK;
}

bool finite_pose(const double* p) {
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(p[k])) return false;
  const double n = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + p[3] * p[3];
  return n > 1e-20 && p[7] > 0.0;
}

// Cholesky Omega = L L^T of a symmetric 7x7 (row-major); packed lower output.
bool chol_pack(const double* O, double* Lp) {
  double L[7][7] = {};
  for (int j = 0; j < 7; ++j) {
    double d = O[j * 7 + j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    L[j][j] = std::sqrt(d);
    for (int i = j + 1; i < 7; ++i) {
      double s = O[i * 7 + j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  for (int a = 0; a < 7; ++a)
    for (int c = 0; c <= a; ++c) Lp[a * (a + 1) / 2 + c] = L[a][c];
  return true;
}

template <class T>
bool fetch(std::vector<T>& dst, const T* src, size_t n, int mem_space) {
  dst.resize(n);
  if (n == 0) return true;
  if (mem_space == PGO_MEM_DEVICE) return cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
  std::memcpy(dst.data(), src, n * sizeof(T));
  return true;
}

pgo_status copy_out(void* dst, const void* src_dev, size_t bytes, int mem_space, cudaStream_t s) {
  if (bytes == 0) return PGO_OK;
  cudaMemcpyKind kind = mem_space == PGO_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpyAsync(dst, src_dev, bytes, kind, s));
  if (mem_space != PGO_MEM_DEVICE) CUDA_TRY(cudaStreamSynchronize(s));
  return PGO_OK;
}

}  // namespace

extern "C" {

const char* pgo_last_error(void) { return g_last_error.c_str(); }

const char* pgo_version(void) { return "pgo-gb300 0.1 (sm_103a)"; }

// Test hook (not in the public header): cap device allocations in bytes.
void pgo_test_set_alloc_limit(size_t bytes) { g_alloc_limit = bytes; }

// Test hook (not in the public header): the grid-barrier wait limit of later
// solves (seconds, <= 0 restores the 2 s default) and a block of the PCG
// launch that never arrives at its barriers (-1 = none).  With a block absent
// the other blocks wait out the limit, the solve stops and reports
// PGO_ERR_CUDA: this exercises the bounded wait without any device fault.
void pgo_test_set_barrier(double limit_s, int absent_block) {
  const unsigned long long ns = limit_s > 0.0 ? (unsigned long long)(limit_s * 1e9) : 0ull;
  set_barrier_limit_pcg(ns);
  set_barrier_limit_amg(ns);
  g_test_absent_block = absent_block;
}

pgo_status pgo_default_options(pgo_solve_options* opt) {
  if (!opt) return fail(PGO_ERR_INVALID_ARG, "opt is NULL");
  opt->max_iters = 20;
  opt->precision = PGO_FP64;
  opt->tau = 1e-5;
  opt->lambda_init = 0.0;
  opt->ftol = 1e-14;
  opt->gtol = 1e-13;
  opt->pcg_tol = 1e-6;
  opt->pcg_max_iters = 5000;
  opt->refine_steps = 2;
  opt->refine_tol = 1e-5;
  opt->polish_iters = 0;
  opt->schedule = -1;
  opt->preconditioner = PGO_PRECOND_MULTIGRID;
  opt->multigrid_refresh = 1;
  opt->linear_solver = PGO_SOLVER_PCG;
  return PGO_OK;
}

// The internal edge order, by (min endpoint, max endpoint, caller index), as
// two stable counting sorts (by the max endpoint, then by the min), and the
// incidence lists over it: for each vertex its side-0 entries (vertex is i),
// then its side-1 entries (vertex is j), each group in edge order.  The
// endpoints must be in range.
struct EdgeOrder {
  std::vector<int> perm, sei, sej, inc_ptr, inc_split, inc_code, inc_other;
};

static void order_edges(int N, int E, const int32_t* ei, const int32_t* ej, EdgeOrder& o) {
  std::vector<int>& perm = o.perm;
  perm.resize(E);
  {
    std::vector<int> tmp(E), cnt((size_t)N + 1);
    auto pass = [&](const std::vector<int>& src, std::vector<int>& dst, bool by_min) {
      std::fill(cnt.begin(), cnt.end(), 0);
      auto key = [&](int e) { return by_min ? std::min(ei[e], ej[e]) : std::max(ei[e], ej[e]); };
      for (int k = 0; k < E; ++k) cnt[key(src[k]) + 1]++;
      for (int v = 0; v < N; ++v) cnt[v + 1] += cnt[v];
      for (int k = 0; k < E; ++k) dst[cnt[key(src[k])]++] = src[k];
    };
    std::iota(perm.begin(), perm.end(), 0);
    pass(perm, tmp, false);
    pass(tmp, perm, true);
  }
  std::vector<int>& sei = o.sei;
  std::vector<int>& sej = o.sej;
  sei.resize(E);
  sej.resize(E);
  for (int k = 0; k < E; ++k) {
    sei[k] = ei[perm[k]];
    sej[k] = ej[perm[k]];
  }
  o.inc_ptr.assign(N + 1, 0);
  o.inc_split.resize(N);
  o.inc_code.resize((size_t)2 * E);
  o.inc_other.resize((size_t)2 * E);
  std::vector<int>& inc_ptr = o.inc_ptr;
  std::vector<int> deg0(N, 0);
  for (int k = 0; k < E; ++k) {
    inc_ptr[sei[k] + 1]++;
    inc_ptr[sej[k] + 1]++;
    deg0[sei[k]]++;
  }
  for (int v = 0; v < N; ++v) inc_ptr[v + 1] += inc_ptr[v];
  std::vector<int> fill0(N), fill1(N);
  for (int v = 0; v < N; ++v) {
    fill0[v] = inc_ptr[v];
    o.inc_split[v] = fill1[v] = inc_ptr[v] + deg0[v];
  }
  for (int k = 0; k < E; ++k) {
    const int a = fill0[sei[k]]++;
    o.inc_code[a] = 2 * k;
    o.inc_other[a] = sej[k];
    const int b2 = fill1[sej[k]]++;
    o.inc_code[b2] = 2 * k + 1;
    o.inc_other[b2] = sei[k];
  }
}

static pgo_status graph_create(const pgo_graph_desc* d, pgo_graph** out, bool analyse_early) {
  if (!out) return fail(PGO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(PGO_ERR_INVALID_ARG, "desc is NULL");
  const int N = d->n_vertices, E = d->n_edges;
  if (N < 1) return fail(PGO_ERR_INVALID_ARG, "n_vertices must be >= 1 (got %d)", N);
  if (E < 0) return fail(PGO_ERR_INVALID_ARG, "n_edges must be >= 0 (got %d)", E);
  if (d->fixed_vertex < 0 || d->fixed_vertex >= N)
    return fail(PGO_ERR_INVALID_ARG, "fixed_vertex %d out of range [0, %d)", d->fixed_vertex, N);
  if (d->mem_space != PGO_MEM_HOST && d->mem_space != PGO_MEM_DEVICE)
    return fail(PGO_ERR_INVALID_ARG, "mem_space must be PGO_MEM_HOST or PGO_MEM_DEVICE");
  if (E > 0 && (!d->edge_i || !d->edge_j || !d->meas)) return fail(PGO_ERR_INVALID_ARG, "edge arrays are NULL");
  if ((long long)E * 2 > 0x7fffffffLL) return fail(PGO_ERR_INVALID_ARG, "too many edges");
  const int ms = d->mem_space;
  std::vector<int32_t> ei, ej;
  std::vector<double> meas, w, info, poses;
  if (!fetch(ei, d->edge_i, E, ms) || !fetch(ej, d->edge_j, E, ms) || !fetch(meas, d->meas, (size_t)E * 8, ms))
    return fail(PGO_ERR_CUDA, "reading the edge arrays failed");
  if (d->weight && !fetch(w, d->weight, E, ms)) return fail(PGO_ERR_CUDA, "reading weights failed");
  if (d->info && !fetch(info, d->info, (size_t)E * 49, ms)) return fail(PGO_ERR_CUDA, "reading info failed");
  if (d->poses && !fetch(poses, d->poses, (size_t)N * 8, ms)) return fail(PGO_ERR_CUDA, "reading poses failed");
  // the endpoints first: the edge order, the incidence lists and the
  // multigrid analysis need only them, and the analysis then runs beside the
  // checks of the values below
  for (int e = 0; e < E; ++e) {
    if (ei[e] < 0 || ei[e] >= N || ej[e] < 0 || ej[e] >= N)
      return fail(PGO_ERR_INVALID_ARG, "edge %d: endpoint out of range (%d, %d), n_vertices %d", e, ei[e], ej[e], N);
    if (ei[e] == ej[e]) return fail(PGO_ERR_INVALID_ARG, "edge %d is a self-edge (%d, %d)", e, ei[e], ej[e]);
  }

  EdgeOrder eo;
  order_edges(N, E, ei.data(), ej.data(), eo);
  const std::vector<int>& perm = eo.perm;
  const std::vector<int>& sei = eo.sei;
  const std::vector<int>& sej = eo.sej;
  const std::vector<int>& inc_split = eo.inc_split;

  pgo_graph* G = new pgo_graph();
  G->N = N;
  G->E = E;
  G->h_inc_ptr = std::move(eo.inc_ptr);
  G->h_inc_code = std::move(eo.inc_code);
  G->h_inc_other = std::move(eo.inc_other);
  if (analyse_early && N >= 2) {
    // the multigrid analysis (the default preconditioner) runs beside the
    // allocations and uploads below and whatever the caller does before its
    // first solve; the graph owns the incidence arrays it reads
    const int fx = d->fixed_vertex;
    const int* ip = G->h_inc_ptr.data();
    const int* ic = G->h_inc_code.data();
    const int* io = G->h_inc_other.data();
    const char** perr = &G->amg_plan_err;
    G->amg_plan = std::async(std::launch::async, [=]() {
      const int v0 = 0, nv = N, f = fx;
      return amg_analyze(N, 1, &v0, &nv, &f, ip, ic, io, perr);
    });
  }
  // the values: measurements, weights, poses, information matrices (a
  // rejected input ends the graph, and with it the analysis started above)
  auto reject = [&](pgo_status st) {
    pgo_graph_destroy(G);
    return st;
  };
  for (int e = 0; e < E; ++e) {
    if (!finite_pose(&meas[(size_t)e * 8]))
      return reject(fail(PGO_ERR_INVALID_ARG, "edge %d: measurement not finite, zero quaternion or scale <= 0", e));
    if (d->weight && !(std::isfinite(w[e]) && w[e] >= 0.0))
      return reject(fail(PGO_ERR_INVALID_ARG, "edge %d: weight must be finite and >= 0", e));
  }
  if (d->poses)
    for (int v = 0; v < N; ++v)
      if (!finite_pose(&poses[(size_t)v * 8]))
        return reject(fail(PGO_ERR_INVALID_ARG, "vertex %d: pose not finite, zero quaternion or scale <= 0", v));
  std::vector<double> Lpack;
  if (d->info) {
    Lpack.resize((size_t)E * 28);
    for (int e = 0; e < E; ++e)
      if (!chol_pack(&info[(size_t)e * 49], &Lpack[(size_t)e * 28]))
        return reject(
            fail(PGO_ERR_INVALID_ARG, "edge %d: information matrix is not symmetric positive definite", e));
  }
  std::vector<D4> zq(E), zt(E);
  std::vector<double> sw(E), szqn(E), sL(d->info ? (size_t)E * 28 : 0);
  for (int k = 0; k < E; ++k) {
    const int e = perm[k];
    const double* m = &meas[(size_t)e * 8];
    const double n = std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
    zq[k] = D4{m[0] / n, m[1] / n, m[2] / n, m[3] / n};
    szqn[k] = n;
    zt[k] = D4{m[4], m[5], m[6], m[7]};
    sw[k] = d->weight ? w[e] : 1.0;
    if (d->info) std::memcpy(&sL[(size_t)k * 28], &Lpack[(size_t)e * 28], sizeof(double) * 28);
  }
  G->fixed = d->fixed_vertex;
  G->stream = (cudaStream_t)d->stream;
  G->has_info = d->info != nullptr;
  const size_t Ep = E > 0 ? E : 1;
  const int pcap = std::max(max_partials(N, E), pcg_partials_needed(N));
  G->scratch_doubles = std::max((size_t)N * 8, (size_t)Ep * 98) + std::max((size_t)N * 49, (size_t)Ep * 49);
  size_t total = 0;
  total += 2 * arena_bytes<int>(Ep) + 2 * arena_bytes<D4>(Ep) + 2 * arena_bytes<double>(Ep);
  total += d->info ? arena_bytes<double>(Ep * 28) : 0;
  total += arena_bytes<int>(N + 1) + arena_bytes<int>(N) + 2 * arena_bytes<int>(2 * Ep) + arena_bytes<int>(Ep);
  total += 4 * arena_bytes<D4>(N);
  total += arena_bytes<double>(Ep * BLK64) + arena_bytes<float>(Ep * BLK32);
  total += 2 * arena_bytes<double>((size_t)N * BLK64) + 2 * arena_bytes<float>((size_t)N * BLK32);
  total += arena_bytes<double>((size_t)N * VEC) + arena_bytes<double>(Ep * 2 * CONTRIB);
  total += arena_bytes<double>(Ep * 2 * 12);
  total += 8 * arena_bytes<double>((size_t)N * VEC) + 6 * arena_bytes<float>((size_t)N * VEC);
  total += arena_bytes<double>((size_t)pcap * 4) + arena_bytes<SolverState>(1) + arena_bytes<DevOptions>(1);
  total += arena_bytes<double>(G->scratch_doubles) + arena_bytes<double>(8);
  auto cleanup = [&](pgo_status st) {
    pgo_graph_destroy(G);
    return st;
  };
  if (g_alloc_limit && total > g_alloc_limit)
    return cleanup(fail(PGO_ERR_OOM, "device allocation of %zu bytes exceeds the test limit", total));
  cudaError_t ce = cudaMalloc(&G->arena.base, total);
  if (ce != cudaSuccess) {
    G->arena.base = nullptr;
    cudaGetLastError();
    return cleanup(fail(ce == cudaErrorMemoryAllocation ? PGO_ERR_OOM : PGO_ERR_CUDA,
                        "cudaMalloc(%zu): %s", total, cudaGetErrorString(ce)));
  }
  G->arena.size = total;
  Arena& A = G->arena;
  DevGraph& g = G->g;
  g.N = N;
  g.E = E;
  g.fixed = d->fixed_vertex;
  g.pcg_block_entries = pcg_block_entries(N, G->h_inc_ptr.data());
  int* d_ei = A.take<int>(Ep);
  int* d_ej = A.take<int>(Ep);
  D4* d_zq = A.take<D4>(Ep);
  D4* d_zt = A.take<D4>(Ep);
  double* d_w = A.take<double>(Ep);
  double* d_zqn = A.take<double>(Ep);
  double* d_L = d->info ? A.take<double>(Ep * 28) : nullptr;
  int* d_ptr = A.take<int>(N + 1);
  int* d_split = A.take<int>(N);
  int* d_code = A.take<int>(2 * Ep);
  int* d_other = A.take<int>(2 * Ep);
  G->d_perm = A.take<int>(Ep);
  g.ei = d_ei; g.ej = d_ej; g.zq = d_zq; g.zt = d_zt; g.w = d_w; g.L = d_L; g.zqn = d_zqn;
  g.inc_ptr = d_ptr; g.inc_code = d_code; g.inc_other = d_other; g.inc_split = d_split;
  for (int k = 0; k < 2; ++k) { g.pq[k] = A.take<D4>(N); g.pt[k] = A.take<D4>(N); }
  g.off64 = A.take<double>(Ep * BLK64);
  g.off32 = A.take<float>(Ep * BLK32);
  g.diag64 = A.take<double>((size_t)N * BLK64);
  g.minv64 = A.take<double>((size_t)N * BLK64);
  g.diag32 = A.take<float>((size_t)N * BLK32);
  g.minv32 = A.take<float>((size_t)N * BLK32);
  g.b = A.take<double>((size_t)N * VEC);
  g.contrib = A.take<double>(Ep * 2 * CONTRIB);
  g.rcache = A.take<double>(Ep * 2 * 12);
  g.x64 = A.take<double>((size_t)N * VEC);
  g.r64 = A.take<double>((size_t)N * VEC);
  g.z64 = A.take<double>((size_t)N * VEC);
  g.p64[0] = A.take<double>((size_t)N * VEC);
  g.p64[1] = A.take<double>((size_t)N * VEC);
  g.q64 = A.take<double>((size_t)N * VEC);
  g.dx64 = A.take<double>((size_t)N * VEC);
  g.res64 = A.take<double>((size_t)N * VEC);
  g.x32 = A.take<float>((size_t)N * VEC);
  g.r32 = A.take<float>((size_t)N * VEC);
  g.z32 = A.take<float>((size_t)N * VEC);
  g.p32[0] = A.take<float>((size_t)N * VEC);
  g.p32[1] = A.take<float>((size_t)N * VEC);
  g.q32 = A.take<float>((size_t)N * VEC);
  g.partial = A.take<double>((size_t)pcap * 4);
  g.partial_cap = pcap;
  g.st = A.take<SolverState>(1);
  g.opt = A.take<DevOptions>(1);
  G->d_scratch = A.take<double>(G->scratch_doubles);
  G->d_cost = A.take<double>(8);
  if (A.used > A.size) return cleanup(fail(PGO_ERR_CUDA, "internal arena overflow"));

  cudaStream_t s = G->stream;
  if (cudaStreamCreateWithFlags(&G->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&G->ev0) != cudaSuccess || cudaEventCreate(&G->ev1) != cudaSuccess ||
      !(G->h_state = static_cast<SolverState*>(pinned_get(sizeof(SolverState)))) ||
      !(G->h_opt = static_cast<DevOptions*>(pinned_get(sizeof(DevOptions)))))
    return cleanup(fail(PGO_ERR_CUDA, "creating streams/events/pinned buffers failed"));
  bool ok = true;
  ok &= cudaMemsetAsync(A.base, 0, A.used, s) == cudaSuccess;
  ok &= copy_in(d_ei, sei.data(), sizeof(int) * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_ej, sej.data(), sizeof(int) * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_zq, zq.data(), sizeof(D4) * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_zt, zt.data(), sizeof(D4) * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_w, sw.data(), sizeof(double) * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_zqn, szqn.data(), sizeof(double) * E, PGO_MEM_HOST, s);
  if (d->info) ok &= copy_in(d_L, sL.data(), sizeof(double) * 28 * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_ptr, G->h_inc_ptr.data(), sizeof(int) * (N + 1), PGO_MEM_HOST, s);
  ok &= copy_in(d_split, inc_split.data(), sizeof(int) * N, PGO_MEM_HOST, s);
  ok &= copy_in(d_code, G->h_inc_code.data(), sizeof(int) * 2 * E, PGO_MEM_HOST, s);
  ok &= copy_in(d_other, G->h_inc_other.data(), sizeof(int) * 2 * E, PGO_MEM_HOST, s);
  ok &= copy_in(G->d_perm, perm.data(), sizeof(int) * E, PGO_MEM_HOST, s);
  if (!ok) return cleanup(fail(PGO_ERR_CUDA, "uploading the graph failed"));
  // identity poses by default, then the caller's initial estimate
  {
    std::vector<double> init((size_t)N * 8, 0.0);
    for (int v = 0; v < N; ++v) { init[(size_t)v * 8 + 3] = 1.0; init[(size_t)v * 8 + 7] = 1.0; }
    const double* src = d->poses ? poses.data() : init.data();
    if (!copy_in(G->d_scratch, src, sizeof(double) * 8 * N, PGO_MEM_HOST, s))
      return cleanup(fail(PGO_ERR_CUDA, "uploading poses failed"));
    launch_set_poses(g, G->d_scratch, 0, s);
  }
  pgo_solve_options def;
  pgo_default_options(&def);
  fill_dev_options(def, G->h_opt);
  if (!copy_in(g.opt, G->h_opt, sizeof(DevOptions), PGO_MEM_HOST, s))
    return cleanup(fail(PGO_ERR_CUDA, "uploading options failed"));
  ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cleanup(fail(PGO_ERR_CUDA, "graph upload: %s", cudaGetErrorString(ce)));
  *out = G;
  return PGO_OK;
}

pgo_status pgo_graph_create(const pgo_graph_desc* d, pgo_graph** out) { return graph_create(d, out, true); }

// Test hook (not in the public header; no device needed): the host analysis
// of the multigrid hierarchy for a graph given by its edge list, over the
// edge order and incidence lists graph creation builds, and one integer
// array of one level of the plan (what: 0 the node count of every level,
// 1 aggregates, 2 / 3 the CSR of P's pattern, 4 / 5 of A P's, 6 / 7 of the
// level's operator pattern), or of the graph's edge order (what: 8 the
// caller's index of each internal edge, 9 inc_ptr, 10 inc_split, 11
// inc_code, 12 inc_other; level ignored).  out == NULL: *count receives the
// length; otherwise at most *count values are copied and *count receives the
// length.
pgo_status pgo_test_multigrid_plan(int32_t n_vertices, int32_t n_edges, const int32_t* edge_i,
                                   const int32_t* edge_j, int32_t fixed_vertex, int32_t level, int32_t what,
                                   int32_t* out, int64_t* count) {
  if (!count) return fail(PGO_ERR_INVALID_ARG, "count is NULL");
  const int N = n_vertices, E = n_edges;
  if (N < 2 || E < 0 || (E > 0 && (!edge_i || !edge_j)) || fixed_vertex < 0 || fixed_vertex >= N)
    return fail(PGO_ERR_INVALID_ARG, "bad graph description");
  for (int e = 0; e < E; ++e)
    if (edge_i[e] < 0 || edge_i[e] >= N || edge_j[e] < 0 || edge_j[e] >= N || edge_i[e] == edge_j[e])
      return fail(PGO_ERR_INVALID_ARG, "edge %d: endpoint out of range or a self-edge", e);
  EdgeOrder eo;
  order_edges(N, E, edge_i, edge_j, eo);
  auto give = [&](const std::vector<int>& v) {
    const long long n = std::max<long long>(0, std::min<long long>((long long)v.size(), *count));
    if (out) std::memcpy(out, v.data(), sizeof(int32_t) * (size_t)n);
    *count = (int64_t)v.size();
    return PGO_OK;
  };
  switch (what) {
    case 8: return give(eo.perm);
    case 9: return give(eo.inc_ptr);
    case 10: return give(eo.inc_split);
    case 11: return give(eo.inc_code);
    case 12: return give(eo.inc_other);
    default: break;
  }
  const char* err = nullptr;
  const int v0 = 0, nv = N, fx = fixed_vertex;
  AmgPlan* P = amg_analyze(N, 1, &v0, &nv, &fx, eo.inc_ptr.data(), eo.inc_code.data(), eo.inc_other.data(), &err);
  if (!P) return fail(PGO_ERR_INVALID_ARG, "multigrid analysis: %s", err ? err : "failed");
  const int* data = nullptr;
  const long long n = amg_plan_array(P, level, what, &data);
  pgo_status st = PGO_OK;
  if (n < 0) {
    st = fail(PGO_ERR_INVALID_ARG, "no array %d at level %d", what, level);
  } else {
    if (out) std::memcpy(out, data, sizeof(int32_t) * (size_t)std::max<long long>(0, std::min<long long>(n, *count)));
    *count = n;
  }
  amg_plan_free(P);
  return st;
}

void pgo_graph_destroy(pgo_graph* G) {
  if (!G) return;
  if (G->amg_plan.valid()) amg_plan_free(G->amg_plan.get());
  if (G->stream || G->arena.base) cudaStreamSynchronize(G->stream);
  for (auto& kv : G->execs) cudaGraphExecDestroy(kv.second);
  if (G->cap_stream) cudaStreamDestroy(G->cap_stream);
  if (G->ev0) cudaEventDestroy(G->ev0);
  if (G->ev1) cudaEventDestroy(G->ev1);
  pinned_put(G->h_state, sizeof(SolverState));
  pinned_put(G->h_opt, sizeof(DevOptions));
  if (G->arena.base) cudaFree(G->arena.base);
  amg_free(G->amg);
  direct_free(G->direct);
  delete G;
}

pgo_status pgo_graph_set_poses(pgo_graph* G, const double* poses, int32_t mem_space) {
  if (!G || !poses) return fail(PGO_ERR_INVALID_ARG, "graph or poses is NULL");
  if (mem_space != PGO_MEM_HOST && mem_space != PGO_MEM_DEVICE) return fail(PGO_ERR_INVALID_ARG, "bad mem_space");
  cudaStream_t s = G->stream;
  if (mem_space == PGO_MEM_DEVICE) {
    // device poses are copied on the stream without a host round trip (and
    // without host-side validation; a non-finite pose makes the next solve
    // stop with PGO_ERR_NUMERICAL)
    launch_set_poses(G->g, poses, -1, s);
    CUDA_TRY(cudaGetLastError());
    G->solved = false;
    return PGO_OK;
  }
  for (int v = 0; v < G->N; ++v)
    if (!finite_pose(&poses[(size_t)v * 8]))
      return fail(PGO_ERR_INVALID_ARG, "vertex %d: pose not finite, zero quaternion or scale <= 0", v);
  CUDA_TRY(cudaMemcpyAsync(G->d_scratch, poses, sizeof(double) * 8 * G->N, cudaMemcpyHostToDevice, s));
  launch_set_poses(G->g, G->d_scratch, -1, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));   // the host buffer may be reused on return
  G->solved = false;
  return PGO_OK;
}

static pgo_status current_buf(pgo_graph* G, int* buf) {
  CUDA_TRY(cudaMemcpyAsync(G->h_state, G->g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, G->stream));
  CUDA_TRY(cudaStreamSynchronize(G->stream));
  *buf = G->h_state->cur;
  return PGO_OK;
}

pgo_status pgo_graph_get_poses(pgo_graph* G, double* poses, int32_t mem_space) {
  if (!G || !poses) return fail(PGO_ERR_INVALID_ARG, "graph or poses is NULL");
  int buf = 0;
  pgo_status st = current_buf(G, &buf);
  if (st != PGO_OK) return st;
  launch_get_poses(G->g, buf, G->d_scratch, G->stream);
  CUDA_TRY(cudaGetLastError());
  return copy_out(poses, G->d_scratch, sizeof(double) * 8 * G->N, mem_space, G->stream);
}

pgo_status pgo_graph_cost(pgo_graph* G, double* cost, double* residuals, int32_t mem_space) {
  if (!G || !cost) return fail(PGO_ERR_INVALID_ARG, "graph or cost is NULL");
  int buf = 0;
  pgo_status st = current_buf(G, &buf);
  if (st != PGO_OK) return st;
  double* rdev = nullptr;
  if (residuals) rdev = mem_space == PGO_MEM_DEVICE ? residuals : G->d_scratch;
  launch_residuals(G->g, buf, G->d_perm, rdev, G->d_cost, G->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(cost, G->d_cost, sizeof(double), cudaMemcpyDeviceToHost, G->stream));
  CUDA_TRY(cudaStreamSynchronize(G->stream));
  if (residuals && mem_space != PGO_MEM_DEVICE) return copy_out(residuals, rdev, sizeof(double) * 7 * G->E, mem_space, G->stream);
  return PGO_OK;
}

// Load a state for a standalone linearisation / linear solve at `lambda`.
static pgo_status prepare_standalone(pgo_graph* G, const pgo_solve_options& o, double lambda) {
  int buf = 0;
  pgo_status st = current_buf(G, &buf);
  if (st != PGO_OK) return st;
  SolverState* h = G->h_state;
  std::memset(h, 0, sizeof(SolverState));
  h->cur = buf;
  h->need_lin = 1;
  h->lambda = lambda;
  h->nu = 2.0;
  fill_dev_options(o, G->h_opt);
  G->h_opt->gtol = -1.0;   // never stop on the gradient here
  CUDA_TRY(cudaMemcpyAsync(G->g.st, h, sizeof(SolverState), cudaMemcpyHostToDevice, G->stream));
  CUDA_TRY(cudaMemcpyAsync(G->g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, G->stream));
  return PGO_OK;
}

pgo_status pgo_graph_linearize(pgo_graph* G, int32_t precision, double* jac, double* h_diag, double* h_off,
                               double* b, int32_t mem_space) {
  if (!G) return fail(PGO_ERR_INVALID_ARG, "graph is NULL");
  if (precision != PGO_FP64 && precision != PGO_MIXED) return fail(PGO_ERR_INVALID_ARG, "bad precision");
  pgo_solve_options o;
  pgo_default_options(&o);
  pgo_status st = prepare_standalone(G, o, 1.0);
  if (st != PGO_OK) return st;
  cudaStream_t s = G->stream;
  const DevGraph& g = G->g;
  linearize_assemble(g, precision == PGO_MIXED, 0, s);
  CUDA_TRY(cudaGetLastError());
  G->lin_valid = true;
  const int E = G->E, N = G->N;
  double* tmp = G->d_scratch;
  if (jac) {
    double* dst = mem_space == PGO_MEM_DEVICE ? jac : tmp;
    launch_jacobians_out(g, G->h_state->cur, G->d_perm, dst, s);
    CUDA_TRY(cudaGetLastError());
    if (mem_space != PGO_MEM_DEVICE) { st = copy_out(jac, tmp, sizeof(double) * 98 * E, mem_space, s); if (st) return st; }
  }
  if (h_off) {
    double* dst = mem_space == PGO_MEM_DEVICE ? h_off : tmp;
    launch_scatter(E, 49, G->d_perm, g.off64, BLK64, dst, 49, s);
    CUDA_TRY(cudaGetLastError());
    if (mem_space != PGO_MEM_DEVICE) { st = copy_out(h_off, tmp, sizeof(double) * 49 * E, mem_space, s); if (st) return st; }
  }
  if (h_diag) {
    double* dst = mem_space == PGO_MEM_DEVICE ? h_diag : tmp;
    launch_scatter(N, 49, nullptr, g.diag64, BLK64, dst, 49, s);
    CUDA_TRY(cudaGetLastError());
    if (mem_space != PGO_MEM_DEVICE) { st = copy_out(h_diag, tmp, sizeof(double) * 49 * N, mem_space, s); if (st) return st; }
  }
  if (b) {
    double* dst = mem_space == PGO_MEM_DEVICE ? b : tmp;
    launch_scatter(N, 7, nullptr, g.b, VEC, dst, 7, s);
    CUDA_TRY(cudaGetLastError());
    if (mem_space != PGO_MEM_DEVICE) { st = copy_out(b, tmp, sizeof(double) * 7 * N, mem_space, s); if (st) return st; }
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return PGO_OK;
}

pgo_status pgo_graph_damped_step(pgo_graph* G, const pgo_solve_options* opt, double lambda, double* delta,
                                 int32_t* pcg_iters, int32_t mem_space) {
  if (!G || !delta) return fail(PGO_ERR_INVALID_ARG, "graph or delta is NULL");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(PGO_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  pgo_solve_options o;
  if (opt) o = *opt; else pgo_default_options(&o);
  pgo_status st = check_options(o);
  if (st != PGO_OK) return st;
  const int mixed = o.precision == PGO_MIXED;
  cudaGraphExec_t ex;
  LinSolve ls;
  st = choose_solver(G, o, &ls);
  if (st != PGO_OK) return st;
  st = get_exec(G, 1, mixed, o.refine_steps, ls, &ex);
  if (st != PGO_OK) return st;
  st = prepare_standalone(G, o, lambda);
  if (st != PGO_OK) return st;
  cudaStream_t s = G->stream;
  CUDA_TRY(cudaGraphLaunch(ex, s));
  G->lin_valid = true;
  launch_scatter(G->N, 7, nullptr, mixed ? G->g.dx64 : G->g.x64, VEC, G->d_scratch, 7, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(G->h_state, G->g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  st = copy_out(delta, G->d_scratch, sizeof(double) * 7 * G->N, mem_space, s);
  if (st != PGO_OK) return st;
  if (pcg_iters) *pcg_iters = G->h_state->pcg_total;
  if (G->h_state->pcg_hit_cap) return fail(PGO_ERR_NOT_CONVERGED, "PCG reached pcg_max_iters (%d)", o.pcg_max_iters);
  return PGO_OK;
}

// The Newton polish and the adjoint solve need accurate steps (they drive
// b to zero and differentiate through it): their PCG runs to at most this
// relative residual, whatever the LM's looser pcg_tol.
constexpr double kExactPcgTol = 1e-10;

// Newton steps after LM on the full Hessian (second-order residual terms
// included, the same exact nested-dual Hessian as the adjoint), each kept
// only while it lowers the gradient norm |b|_2.  LM's cost-based stop cannot
// resolve the last digits of the optimum (a tiny change of the measurements
// changes F by less than ftol F), and Gauss-Newton steps need not lower |b|
// on noisy, ill-conditioned graphs; the implicit adjoint needs b(x*) ~ 0.  A
// step that does not lower |b| is halved up to three times before polishing
// stops.  FP64, host-driven: a few steps with a synchronisation each.
static pgo_status run_polish(pgo_graph* G, const pgo_solve_options& o) {
  const DevGraph& g = G->g;
  cudaStream_t s = G->stream;
  fill_dev_options(o, G->h_opt);
  G->h_opt->lambda_fixed = 0.0;
  G->h_opt->pcg_tol = std::min(o.pcg_tol, kExactPcgTol);
  CUDA_TRY(cudaMemcpyAsync(g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  auto linearize_here = [&](double* b2, double* gmax) -> pgo_status {
    launch_state_ctl(g, 0, s);
    launch_adj_hessian(g, 1, s);
    launch_assemble_mode(g, 2, s);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(G->h_state, g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *b2 = G->h_state->bnorm2;
    *gmax = G->h_state->gmax;
    return PGO_OK;
  };
  double b0 = 0.0, g0 = 0.0;
  pgo_status st = linearize_here(&b0, &g0);
  if (st != PGO_OK) return st;
  const AmgDev* amg = amg_for(G, o.preconditioner);
  for (int k = 0; k < o.polish_iters && g0 > o.gtol; ++k) {
    cudaError_t le = cudaSuccess;
    enqueue_precond(g, 0, amg, s, &le);
    enqueue_pcg(g, 0, amg, 0, s, &le);      // delta = -H^-1 b (x64)
    CUDA_TRY(le);
    bool improved = false;
    double b1 = 0.0, g1 = 0.0;
    for (int half = 0; half < 4 && !improved; ++half) {
      if (half > 0) launch_scale_x(g, 0.5, s);
      launch_update(g, 0, s);               // candidate into the other buffer
      launch_state_ctl(g, 1, s);            // make it current
      st = linearize_here(&b1, &g1);
      if (st != PGO_OK) return st;
      improved = b1 < b0;
      if (!improved) launch_state_ctl(g, 1, s);   // back to the previous poses
    }
    if (!improved) {
      st = linearize_here(&b1, &g1);        // restore b and H at the kept poses
      if (st != PGO_OK) return st;
      break;
    }
    b0 = b1;
    g0 = g1;
  }
  // the final cost and gradient go into the report
  launch_residuals(g, -1, G->d_perm, nullptr, &g.st->F, s);
  CUDA_TRY(cudaGetLastError());
  return PGO_OK;
}

pgo_status pgo_graph_resolve(pgo_graph* G, const pgo_solve_options* opt, double lambda, double* delta,
                             int32_t* pcg_iters, int32_t mem_space) {
  if (!G) return fail(PGO_ERR_INVALID_ARG, "graph is NULL");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(PGO_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  pgo_solve_options o;
  if (opt) o = *opt; else pgo_default_options(&o);
  pgo_status st = check_options(o);
  if (st != PGO_OK) return st;
  const int mixed = o.precision == PGO_MIXED;
  cudaGraphExec_t ex;
  LinSolve ls;
  st = choose_solver(G, o, &ls);
  if (st != PGO_OK) return st;
  st = get_exec(G, 2, mixed, o.refine_steps, ls, &ex);
  if (st != PGO_OK) return st;
  cudaStream_t s = G->stream;
  fill_dev_options(o, G->h_opt);
  G->h_opt->lambda_fixed = lambda;
  CUDA_TRY(cudaMemcpyAsync(G->g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaGraphLaunch(ex, s));
  if (!delta && !pcg_iters) return PGO_OK;
  if (delta) {
    launch_scatter(G->N, 7, nullptr, mixed ? G->g.dx64 : G->g.x64, VEC, G->d_scratch, 7, s);
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaMemcpyAsync(G->h_state, G->g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (delta) {
    st = copy_out(delta, G->d_scratch, sizeof(double) * 7 * G->N, mem_space, s);
    if (st != PGO_OK) return st;
  }
  if (pcg_iters) *pcg_iters = G->h_state->pcg_total;
  if (G->h_state->status) return fail((pgo_status)G->h_state->status, "re-solve failed on the device");
  if (G->h_state->pcg_hit_cap) return fail(PGO_ERR_NOT_CONVERGED, "PCG reached pcg_max_iters (%d)", o.pcg_max_iters);
  return PGO_OK;
}

pgo_status pgo_graph_precondition(pgo_graph* G, const pgo_solve_options* opt, double lambda) {
  if (!G) return fail(PGO_ERR_INVALID_ARG, "graph is NULL");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(PGO_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  if (!G->lin_valid) return fail(PGO_ERR_STATE, "no linearisation to precondition (linearise or solve first)");
  pgo_solve_options o;
  if (opt) o = *opt; else pgo_default_options(&o);
  pgo_status st = check_options(o);
  if (st != PGO_OK) return st;
  st = ensure_amg(G, o.preconditioner);
  if (st != PGO_OK) return st;
  cudaStream_t s = G->stream;
  fill_dev_options(o, G->h_opt);
  G->h_opt->lambda_fixed = lambda;
  CUDA_TRY(cudaMemcpyAsync(G->g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  launch_resolve_reset(G->g, s);
  cudaError_t le = cudaSuccess;
  enqueue_precond(G->g, o.precision == PGO_MIXED, amg_for(G, o.preconditioner), s, &le);
  CUDA_TRY(le);
  CUDA_TRY(cudaGetLastError());
  return PGO_OK;
}

static void fill_report(pgo_graph* G, pgo_report* report) {
  const SolverState* h = G->h_state;
  std::memset(report, 0, sizeof(*report));
  report->initial_cost = h->F0;
  report->final_cost = h->F;
  report->final_lambda = h->lambda;
  report->grad_inf_norm = h->gmax;
  report->iterations = h->it;
  report->accepted = h->accepted;
  report->pcg_iterations = h->pcg_total;
  report->stop_reason = h->stop_reason;
  report->status = h->status;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, G->ev0, G->ev1) != cudaSuccess) {
    cudaGetLastError();
    ms = 0.f;
  }
  report->ms_total = ms;
}

pgo_status pgo_graph_multigrid_info(pgo_graph* G, int32_t* n_levels, int32_t* nodes, int64_t* a_blocks,
                                    int64_t* p_blocks, int64_t* ap_blocks) {
  if (!G || !n_levels) return fail(PGO_ERR_INVALID_ARG, "graph or n_levels is NULL");
  pgo_status st = ensure_amg(G, PGO_PRECOND_MULTIGRID);
  if (st != PGO_OK) return st;
  if (!G->amg) return fail(PGO_ERR_STATE, "the graph has no free vertex: no multigrid hierarchy");
  const AmgDev* D = amg_host_desc(G->amg);
  *n_levels = D->L + 1;
  for (int l = 0; l <= D->L; ++l) {
    const AmgLevel& a = D->lv[l];
    if (nodes) nodes[l] = a.n;
    if (a_blocks) a_blocks[l] = l == 0 ? (int64_t)G->E + G->N : a.nnz_a;
    if (p_blocks) p_blocks[l] = l < D->L ? a.nnz_p : 0;
    if (ap_blocks) ap_blocks[l] = l < D->L ? a.nnz_ap : 0;
  }
  return PGO_OK;
}

pgo_status pgo_graph_multigrid_export(pgo_graph* G, int32_t level, int32_t which, int32_t precision, void* dst,
                                      int64_t capacity, int64_t* count) {
  if (!G) return fail(PGO_ERR_INVALID_ARG, "graph is NULL");
  if (precision != PGO_FP64 && precision != PGO_MIXED) return fail(PGO_ERR_INVALID_ARG, "bad precision");
  if (!G->amg) return fail(PGO_ERR_STATE, "no multigrid hierarchy: run a multigrid solve or set-up first");
  const AmgDev* D = amg_host_desc(G->amg);
  if (level < 0 || level > D->L) return fail(PGO_ERR_INVALID_ARG, "level %d out of range [0, %d]", level, D->L);
  const bool f64 = precision == PGO_FP64;
  cudaStream_t s = G->stream;
  int warm = 0;
  CUDA_TRY(cudaMemcpyAsync(&warm, D->warm + (f64 ? 0 : 1), sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (!warm) return fail(PGO_ERR_STATE, "the hierarchy has not been set up in this precision");
  const AmgLevel& a = D->lv[level];
  const bool below = level < D->L;
  const int* ints = nullptr;   // integer array on the device
  const void* blocks = nullptr; // block array on the device (FP64 or FP32, padded)
  const double* dbl = nullptr;  // plain doubles on the device
  int64_t n = 0;                // integers, blocks or doubles
  switch (which) {
    case PGO_MG_A_PTR: if (level >= 1) { ints = a.a_ptr; n = a.n + 1; } break;
    case PGO_MG_A_COL: if (level >= 1) { ints = a.a_col; n = a.nnz_a; } break;
    case PGO_MG_A: if (level >= 1) { blocks = f64 ? (const void*)a.a64 : (const void*)a.a32; n = a.nnz_a; } break;
    case PGO_MG_P_PTR: if (below) { ints = a.p_ptr; n = a.n + 1; } break;
    case PGO_MG_P_COL: if (below) { ints = a.p_col; n = a.nnz_p; } break;
    case PGO_MG_P: if (below) { blocks = f64 ? (const void*)a.p64 : (const void*)a.p32; n = a.nnz_p; } break;
    case PGO_MG_AP_PTR: if (below) { ints = a.ap_ptr; n = a.n + 1; } break;
    case PGO_MG_AP_COL: if (below) { ints = a.ap_col; n = a.nnz_ap; } break;
    case PGO_MG_Q: if (below && D->dense) { blocks = f64 ? (const void*)a.q64 : (const void*)a.q32; n = a.nnz_ap; } break;
    case PGO_MG_DINV:
      if (level == 0) blocks = f64 ? (const void*)G->g.minv64 : (const void*)G->g.minv32;
      else if (below) blocks = f64 ? (const void*)a.dinv64 : (const void*)a.dinv32;
      n = a.n;
      break;
    case PGO_MG_T: if (below) { blocks = f64 ? (const void*)a.t64 : (const void*)a.t32; n = a.n; } break;
    case PGO_MG_AGG: if (below) { ints = a.agg; n = a.n; } break;
    case PGO_MG_RHO: if (below) { dbl = D->rho + level; n = 1; } break;
    case PGO_MG_W:
      if (D->dense && level == D->L - 1) {
        blocks = f64 ? (const void*)D->w64 : (const void*)D->w32;
        n = (int64_t)a.n * a.n;
      }
      break;
    default: return fail(PGO_ERR_INVALID_ARG, "unknown array %d", which);
  }
  if (!ints && !blocks && !dbl) return fail(PGO_ERR_INVALID_ARG, "level %d has no array %d", level, which);
  if (n < 0) return fail(PGO_ERR_INVALID_ARG, "level %d: array %d has a negative size", level, which);
  const int64_t elems = blocks ? n * 49 : n;
  const int64_t esize = ints ? (int64_t)sizeof(int32_t) : (int64_t)sizeof(double);
  if (count) *count = elems;
  if (!dst) return PGO_OK;
  if (capacity < elems * esize) return fail(PGO_ERR_INVALID_ARG, "buffer of %lld bytes, the array needs %lld",
                                            (long long)capacity, (long long)(elems * esize));
  if (elems == 0) return PGO_OK;
  if (ints) {
    CUDA_TRY(cudaMemcpyAsync(dst, ints, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return PGO_OK;
  }
  if (dbl) {
    CUDA_TRY(cudaMemcpyAsync(dst, dbl, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return PGO_OK;
  }
  // padded blocks: copy, then repack to 49 values per block as double
  const size_t stride = f64 ? sizeof(double) * BLK64 : sizeof(float) * BLK32;
  std::vector<char> tmp((size_t)n * stride);
  CUDA_TRY(cudaMemcpyAsync(tmp.data(), blocks, tmp.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  double* out = static_cast<double*>(dst);
  for (int64_t b = 0; b < n; ++b)
    for (int k = 0; k < 49; ++k)
      out[b * 49 + k] = f64 ? reinterpret_cast<const double*>(tmp.data())[b * BLK64 + k]
                            : (double)reinterpret_cast<const float*>(tmp.data())[b * BLK32 + k];
  return PGO_OK;
}

pgo_status pgo_graph_report(pgo_graph* G, pgo_report* report) {
  if (!G || !report) return fail(PGO_ERR_INVALID_ARG, "graph or report is NULL");
  if (!G->solved) return fail(PGO_ERR_STATE, "no solve has run on this graph");
  CUDA_TRY(cudaMemcpyAsync(G->h_state, G->g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, G->stream));
  CUDA_TRY(cudaStreamSynchronize(G->stream));
  fill_report(G, report);
  if (report->status) return fail((pgo_status)report->status, "the solve failed on the device (status %d)", report->status);
  return PGO_OK;
}

pgo_status pgo_solve(pgo_graph* G, const pgo_solve_options* opt, pgo_report* report, double* poses_out,
                     int32_t out_mem_space) {
  if (!G) return fail(PGO_ERR_INVALID_ARG, "graph is NULL");
  pgo_solve_options o;
  if (opt) o = *opt; else pgo_default_options(&o);
  pgo_status st = check_options(o);
  if (st != PGO_OK) return st;
  if (poses_out && out_mem_space != PGO_MEM_HOST && out_mem_space != PGO_MEM_DEVICE)
    return fail(PGO_ERR_INVALID_ARG, "bad out_mem_space");
  const int mixed = o.precision == PGO_MIXED;
  const bool eager = o.schedule == 1;
  cudaGraphExec_t ex = nullptr;
  LinSolve ls;
  st = choose_solver(G, o, &ls);
  if (st != PGO_OK) return st;
  if (!eager) {
    st = get_exec(G, 0, mixed, o.refine_steps, ls, &ex);
    if (st != PGO_OK) return st;
  }
  cudaStream_t s = G->stream;
  fill_dev_options(o, G->h_opt);
  CUDA_TRY(cudaMemcpyAsync(G->g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaEventRecord(G->ev0, s));
  if (eager) {
    st = run_eager(G, mixed, o.refine_steps, o.max_iters, ls);
    if (st != PGO_OK) return st;
  } else {
    CUDA_TRY(cudaGraphLaunch(ex, s));
  }
  if (o.polish_iters > 0) {
    st = run_polish(G, o);
    if (st != PGO_OK) return st;
  }
  CUDA_TRY(cudaEventRecord(G->ev1, s));
  G->solved = true;
  G->lin_valid = true;
  if (poses_out) {
    // the current buffer is only known on the device: gather both and let
    // the device pick (k_get_poses reads st->cur through launch_get_poses)
    CUDA_TRY(cudaMemcpyAsync(G->h_state, G->g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    launch_get_poses(G->g, G->h_state->cur, G->d_scratch, s);
    CUDA_TRY(cudaGetLastError());
    st = copy_out(poses_out, G->d_scratch, sizeof(double) * 8 * G->N, out_mem_space, s);
    if (st != PGO_OK) return st;
  }
  if (report) {
    CUDA_TRY(cudaMemcpyAsync(G->h_state, G->g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    fill_report(G, report);
    if (report->status)
      return fail((pgo_status)report->status, "solve failed on the device (status %d, stop reason %d)",
                  report->status, report->stop_reason);
  }
  return PGO_OK;
}

pgo_status pgo_backward(pgo_graph* G, const pgo_solve_options* opt, const double* dL_dposes, int32_t layout,
                        double* dL_dmeas, double* dL_dweight, int32_t mem_space) {
  if (!G || !dL_dposes) return fail(PGO_ERR_INVALID_ARG, "graph or dL_dposes is NULL");
  if (layout != PGO_GRAD_TANGENT7 && layout != PGO_GRAD_POSE8) return fail(PGO_ERR_INVALID_ARG, "bad grad_layout");
  if (mem_space != PGO_MEM_HOST && mem_space != PGO_MEM_DEVICE) return fail(PGO_ERR_INVALID_ARG, "bad mem_space");
  if (!G->solved) return fail(PGO_ERR_STATE, "pgo_backward needs a completed pgo_solve");
  pgo_solve_options o;
  if (opt) o = *opt; else pgo_default_options(&o);
  pgo_status st = check_options(o);
  if (st != PGO_OK) return st;
  cudaStream_t s = G->stream;
  const DevGraph& g = G->g;
  const int N = G->N, E = G->E;
  const int pw = layout == PGO_GRAD_POSE8 ? 8 : 7;
  // scratch: outputs first (E * pw + E doubles), the input gradient after them
  double* d_out_meas = G->d_scratch;
  double* d_out_w = G->d_scratch + (size_t)E * pw;
  double* d_in = G->d_scratch + std::max((size_t)N * 8, (size_t)(E > 0 ? E : 1) * 98);
  const double* dl = dL_dposes;
  if (mem_space == PGO_MEM_HOST) {
    CUDA_TRY(cudaMemcpyAsync(d_in, dL_dposes, sizeof(double) * pw * N, cudaMemcpyHostToDevice, s));
    dl = d_in;
  }
  fill_dev_options(o, G->h_opt);
  G->h_opt->lambda_fixed = 0.0;
  G->h_opt->pcg_tol = std::min(o.pcg_tol, kExactPcgTol);
  CUDA_TRY(cudaMemcpyAsync(g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  launch_state_ctl(g, 0, s);          // done = 0, lambda = 0, tickets cleared
  launch_adj_hessian(g, 0, s);        // full-Hessian blocks of every edge
  launch_assemble_mode(g, 1, s);      // diagonal blocks
  launch_adj_rhs(g, dl, layout, s);   // b = -dL/dx
  cudaError_t le = cudaSuccess;
  st = ensure_amg(G, o.preconditioner);
  if (st != PGO_OK) return st;
  const AmgDev* amg = amg_for(G, o.preconditioner);
  enqueue_precond(g, 0, amg, s, &le);
  enqueue_pcg(g, 0, amg, 0, s, &le);  // mu = H^-1 dL/dx  (x64)
  CUDA_TRY(le);
  double* om = dL_dmeas ? (mem_space == PGO_MEM_DEVICE ? dL_dmeas : d_out_meas) : nullptr;
  double* ow = dL_dweight ? (mem_space == PGO_MEM_DEVICE ? dL_dweight : d_out_w) : nullptr;
  launch_adj_edges(g, G->d_perm, om, ow, layout, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(G->h_state, g.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  G->lin_valid = false;
  if (mem_space == PGO_MEM_HOST) {
    if (dL_dmeas) { st = copy_out(dL_dmeas, d_out_meas, sizeof(double) * pw * E, mem_space, s); if (st) return st; }
    if (dL_dweight) { st = copy_out(dL_dweight, d_out_w, sizeof(double) * E, mem_space, s); if (st) return st; }
  }
  if (G->h_state->status) return fail((pgo_status)G->h_state->status, "adjoint solve failed on the device");
  if (G->h_state->pcg_hit_cap) return fail(PGO_ERR_NOT_CONVERGED, "adjoint PCG reached pcg_max_iters (%d)", o.pcg_max_iters);
  return PGO_OK;
}

pgo_status pgo_graph_set_measurements(pgo_graph* G, const double* meas, const double* weight, int32_t mem_space) {
  if (!G || !meas) return fail(PGO_ERR_INVALID_ARG, "graph or meas is NULL");
  if (mem_space != PGO_MEM_HOST && mem_space != PGO_MEM_DEVICE) return fail(PGO_ERR_INVALID_ARG, "bad mem_space");
  cudaStream_t s = G->stream;
  const int E = G->E;
  if (E == 0) return PGO_OK;
  const double* dm = meas;
  const double* dw = weight;
  if (mem_space == PGO_MEM_HOST) {
    for (int e = 0; e < E; ++e) {
      if (!finite_pose(&meas[(size_t)e * 8]))
        return fail(PGO_ERR_INVALID_ARG, "edge %d: measurement not finite, zero quaternion or scale <= 0", e);
      if (weight && !(std::isfinite(weight[e]) && weight[e] >= 0.0))
        return fail(PGO_ERR_INVALID_ARG, "edge %d: weight must be finite and >= 0", e);
    }
    double* tm = G->d_scratch;
    double* tw = G->d_scratch + (size_t)E * 8;
    CUDA_TRY(cudaMemcpyAsync(tm, meas, sizeof(double) * 8 * E, cudaMemcpyHostToDevice, s));
    if (weight) CUDA_TRY(cudaMemcpyAsync(tw, weight, sizeof(double) * E, cudaMemcpyHostToDevice, s));
    dm = tm;
    dw = weight ? tw : nullptr;
  }
  launch_set_meas(G->g, G->d_perm, dm, dw, s);
  CUDA_TRY(cudaGetLastError());
  if (mem_space == PGO_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(s));
  G->solved = false;
  G->lin_valid = false;
  return PGO_OK;
}

pgo_status pgo_batch_create(int32_t n_graphs, const pgo_graph_desc* descs, void* stream, pgo_batch** out) {
  if (!out) return fail(PGO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_graphs < 1 || !descs) return fail(PGO_ERR_INVALID_ARG, "need n_graphs >= 1 and a descs array");
  std::vector<int32_t> ei, ej;
  std::vector<double> meas, w, info, poses;
  std::vector<int> nv(n_graphs), ne(n_graphs), v0(n_graphs), e0(n_graphs), fixed(n_graphs);
  bool any_w = false, any_info = false;
  for (int k = 0; k < n_graphs; ++k) {
    any_w |= descs[k].weight != nullptr;
    any_info |= descs[k].info != nullptr;
  }
  long long V = 0, Etot = 0;
  for (int k = 0; k < n_graphs; ++k) {
    const pgo_graph_desc& d = descs[k];
    if (d.n_vertices < 1 || d.n_edges < 0 || d.fixed_vertex < 0 || d.fixed_vertex >= d.n_vertices)
      return fail(PGO_ERR_INVALID_ARG, "graph %d: bad sizes or fixed vertex", k);
    if (d.mem_space != PGO_MEM_HOST && d.mem_space != PGO_MEM_DEVICE)
      return fail(PGO_ERR_INVALID_ARG, "graph %d: bad mem_space", k);
    if (d.n_edges > 0 && (!d.edge_i || !d.edge_j || !d.meas)) return fail(PGO_ERR_INVALID_ARG, "graph %d: NULL edge arrays", k);
    nv[k] = d.n_vertices;
    ne[k] = d.n_edges;
    v0[k] = (int)V;
    e0[k] = (int)Etot;
    fixed[k] = (int)V + d.fixed_vertex;
    std::vector<int32_t> a, b;
    std::vector<double> m, ww, ii, pp;
    if (!fetch(a, d.edge_i, d.n_edges, d.mem_space) || !fetch(b, d.edge_j, d.n_edges, d.mem_space) ||
        !fetch(m, d.meas, (size_t)d.n_edges * 8, d.mem_space))
      return fail(PGO_ERR_CUDA, "graph %d: reading edge arrays failed", k);
    for (int e = 0; e < d.n_edges; ++e) {
      if (a[e] < 0 || a[e] >= d.n_vertices || b[e] < 0 || b[e] >= d.n_vertices)
        return fail(PGO_ERR_INVALID_ARG, "graph %d edge %d: endpoint out of range", k, e);
      ei.push_back(a[e] + (int)V);
      ej.push_back(b[e] + (int)V);
    }
    meas.insert(meas.end(), m.begin(), m.end());
    if (any_w) {
      if (d.weight) {
        if (!fetch(ww, d.weight, d.n_edges, d.mem_space)) return fail(PGO_ERR_CUDA, "reading weights failed");
      } else {
        ww.assign(d.n_edges, 1.0);
      }
      w.insert(w.end(), ww.begin(), ww.end());
    }
    if (any_info) {
      if (d.info) {
        if (!fetch(ii, d.info, (size_t)d.n_edges * 49, d.mem_space)) return fail(PGO_ERR_CUDA, "reading info failed");
      } else {
        ii.assign((size_t)d.n_edges * 49, 0.0);
        for (int e = 0; e < d.n_edges; ++e)
          for (int q = 0; q < 7; ++q) ii[(size_t)e * 49 + q * 8] = 1.0;
      }
      info.insert(info.end(), ii.begin(), ii.end());
    }
    if (d.poses) {
      if (!fetch(pp, d.poses, (size_t)d.n_vertices * 8, d.mem_space)) return fail(PGO_ERR_CUDA, "reading poses failed");
    } else {
      pp.assign((size_t)d.n_vertices * 8, 0.0);
      for (int v = 0; v < d.n_vertices; ++v) { pp[(size_t)v * 8 + 3] = 1.0; pp[(size_t)v * 8 + 7] = 1.0; }
    }
    poses.insert(poses.end(), pp.begin(), pp.end());
    V += d.n_vertices;
    Etot += d.n_edges;
    if (V > 0x3fffffffLL || Etot > 0x3fffffffLL) return fail(PGO_ERR_INVALID_ARG, "batch too large");
  }
  pgo_graph_desc big = {};
  big.n_vertices = (int)V;
  big.n_edges = (int)Etot;
  big.fixed_vertex = fixed[0];
  big.mem_space = PGO_MEM_HOST;
  big.edge_i = ei.data();
  big.edge_j = ej.data();
  big.meas = meas.data();
  big.weight = any_w ? w.data() : nullptr;
  big.info = any_info ? info.data() : nullptr;
  big.poses = poses.data();
  big.stream = stream;
  pgo_graph* G = nullptr;
  pgo_status st = graph_create(&big, &G, false);
  if (st != PGO_OK) return st;
  pgo_batch* B = new pgo_batch();
  B->G = G;
  B->n = n_graphs;
  B->nv = nv;
  B->ne = ne;
  B->v0 = v0;
  B->fixed = fixed;
  // processing order: largest graphs first (longest-processing-time rule)
  std::vector<int> order(n_graphs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)ne[a] + nv[a] > (long long)ne[b] + nv[b];
  });
  const size_t ints = (size_t)n_graphs * 6 + 4;
  const size_t bytes = ints * sizeof(int) + 256 + (size_t)n_graphs * sizeof(BatchGraphState);
  cudaError_t ce = cudaMalloc(&B->meta, bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(&B->saved_poses, sizeof(D4) * 2 * (size_t)V);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    pgo_batch_destroy(B);
    return fail(ce == cudaErrorMemoryAllocation ? PGO_ERR_OOM : PGO_ERR_CUDA, "batch metadata: %s", cudaGetErrorString(ce));
  }
  int* m = reinterpret_cast<int*>(B->meta);
  std::vector<int> hostm(ints, 0);
  for (int k = 0; k < n_graphs; ++k) {
    hostm[k] = v0[k];
    hostm[n_graphs + k] = nv[k];
    hostm[2 * n_graphs + k] = e0[k];
    hostm[3 * n_graphs + k] = ne[k];
    hostm[4 * n_graphs + k] = fixed[k];
    hostm[5 * n_graphs + k] = order[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  BatchArgs& a = B->args;
  a.n_graphs = n_graphs;
  a.v0 = m;
  a.nv = m + n_graphs;
  a.e0 = m + 2 * n_graphs;
  a.ne = m + 3 * n_graphs;
  a.fixed = m + 4 * n_graphs;
  a.order = m + 5 * n_graphs;
  a.queue = reinterpret_cast<unsigned*>(m + 6 * n_graphs);
  a.gst = reinterpret_cast<BatchGraphState*>(reinterpret_cast<char*>(B->meta) + ((ints * sizeof(int) + 255) & ~size_t(255)));
  bool ok = cudaMemcpyAsync(m, hostm.data(), ints * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemsetAsync(a.gst, 0, (size_t)n_graphs * sizeof(BatchGraphState), s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    pgo_batch_destroy(B);
    return fail(PGO_ERR_CUDA, "uploading batch metadata failed");
  }
  *out = B;
  return PGO_OK;
}

void pgo_batch_destroy(pgo_batch* B) {
  if (!B) return;
  for (auto& kv : B->execs) cudaGraphExecDestroy(kv.second);
  if (B->G) pgo_graph_destroy(B->G);   // synchronises the stream
  if (B->meta) cudaFree(B->meta);
  if (B->saved_poses) cudaFree(B->saved_poses);
  delete B;
}

// The multigrid hierarchy of the batch: one segment per graph, so that every
// level stays block-diagonal over the graphs (analysed at the first batch
// solve that asks for it).  False when the batch has no free vertex.
static pgo_status ensure_batch_amg(pgo_batch* B, bool* have) {
  pgo_graph* G = B->G;
  *have = false;
  if (B->amg_failed) return PGO_OK;
  if (!G->amg) {
    int K = 0;
    for (int k = 0; k < B->n; ++k) K += B->nv[k] - 1;
    if (K < 1) {
      B->amg_failed = true;
      return PGO_OK;
    }
    const char* err = nullptr;
    G->amg = amg_build(G->N, B->n, B->v0.data(), B->nv.data(), B->fixed.data(), G->h_inc_ptr.data(),
                       G->h_inc_code.data(), G->h_inc_other.data(), G->stream, &err);
    if (!G->amg) return fail(PGO_ERR_OOM, "batch multigrid set-up: %s", err ? err : "unknown error");
    G->g.amg = amg_device_desc(G->amg);
  }
  *have = true;
  return PGO_OK;
}

static pgo_status batch_exec(pgo_batch* B, int schedule, bool amg, cudaGraphExec_t* out) {
  const int key = schedule * 2 + (amg ? 1 : 0);
  auto it = B->execs.find(key);
  if (it != B->execs.end()) {
    *out = it->second;
    return PGO_OK;
  }
  pgo_graph* G = B->G;
  cudaGraph_t graph;
  CUDA_TRY(cudaGraphCreate(&graph, 0));
  GraphBuilder gb{G->cap_stream};
  cudaError_t le = cudaSuccess;
  BatchArgs args = B->args;
  args.amg = amg ? 1 : 0;
  gb.capture(graph, [&](cudaStream_t s) {
    launch_batch_reset(G->g, args, s);
    cudaMemsetAsync(args.queue, 0, sizeof(unsigned), s);
    le = launch_batch_lm(G->g, args, schedule, s);
  });
  if (le != cudaSuccess) gb.err = le;
  if (gb.err != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(PGO_ERR_CUDA, "building the batch graph: %s", cudaGetErrorString(gb.err));
  }
  cudaGraphExec_t ex;
  cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, "instantiating the batch graph: %s", cudaGetErrorString(e));
  B->execs[key] = ex;
  *out = ex;
  return PGO_OK;
}

// Autotuner: time one LM iteration (PCG capped at 40 iterations) of the
// whole batch for every schedule of the requested precision and keep the
// fastest; the estimate is restored after every trial.
static pgo_status batch_autotune(pgo_batch* B, const pgo_solve_options& o, int mixed, bool amg) {
  pgo_graph* G = B->G;
  cudaStream_t s = G->stream;
  const size_t nbytes = sizeof(D4) * (size_t)G->N;
  launch_batch_reset(G->g, B->args, s);   // current estimate into buffer 0
  char* saved_q = reinterpret_cast<char*>(B->saved_poses);
  char* saved_t = saved_q + nbytes;
  CUDA_TRY(cudaMemcpyAsync(saved_q, G->g.pq[0], nbytes, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(saved_t, G->g.pt[0], nbytes, cudaMemcpyDeviceToDevice, s));
  pgo_solve_options t = o;
  t.max_iters = 1;
  t.pcg_max_iters = std::min(o.pcg_max_iters, 40);
  fill_dev_options(t, G->h_opt);
  CUDA_TRY(cudaMemcpyAsync(G->g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  float best = 1e30f;
  int best_s = -1;
  for (int sc = 0; sc < batch_schedule_count(); ++sc) {
    if (batch_schedule_mixed(sc) != mixed) continue;
    cudaGraphExec_t ex;
    pgo_status st = batch_exec(B, sc, amg, &ex);
    if (st != PGO_OK) return st;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first run warms up
      CUDA_TRY(cudaEventRecord(G->ev0, s));
      CUDA_TRY(cudaGraphLaunch(ex, s));
      CUDA_TRY(cudaEventRecord(G->ev1, s));
      CUDA_TRY(cudaEventSynchronize(G->ev1));
      CUDA_TRY(cudaEventElapsedTime(&ms, G->ev0, G->ev1));
      // restore the estimate
      CUDA_TRY(cudaMemcpyAsync(G->g.pq[0], saved_q, nbytes, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(G->g.pt[0], saved_t, nbytes, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemsetAsync(B->args.gst, 0, (size_t)B->n * sizeof(BatchGraphState), s));
    }
    if (ms < best) {
      best = ms;
      best_s = sc;
    }
  }
  if (best_s < 0) return fail(PGO_ERR_STATE, "no batch schedule for this precision");
  B->tuned[mixed + 2 * amg] = best_s;
  B->tune_ms[mixed + 2 * amg] = best;
  return PGO_OK;
}

pgo_status pgo_batch_solve(pgo_batch* B, const pgo_solve_options* opt, pgo_report* reports, double* const* poses_out,
                           int32_t out_mem_space) {
  if (!B) return fail(PGO_ERR_INVALID_ARG, "batch is NULL");
  pgo_solve_options o;
  if (opt) o = *opt; else pgo_default_options(&o);
  pgo_status st = check_options(o);
  if (st != PGO_OK) return st;
  if (poses_out && out_mem_space != PGO_MEM_HOST && out_mem_space != PGO_MEM_DEVICE)
    return fail(PGO_ERR_INVALID_ARG, "bad out_mem_space");
  pgo_graph* G = B->G;
  cudaStream_t s = G->stream;
  const int mixed = o.precision == PGO_MIXED;
  bool amg = false;
  if (o.preconditioner == PGO_PRECOND_MULTIGRID) {
    st = ensure_batch_amg(B, &amg);
    if (st != PGO_OK) return st;
  }
  const int tk = mixed + 2 * (amg ? 1 : 0);
  int sc = o.schedule;
  if (sc >= 0) {
    if (sc >= batch_schedule_count() || batch_schedule_mixed(sc) != mixed)
      return fail(PGO_ERR_INVALID_ARG, "schedule %d does not exist for this precision", sc);
  } else {
    if (B->tuned[tk] < 0) {
      st = batch_autotune(B, o, mixed, amg);
      if (st != PGO_OK) return st;
    }
    sc = B->tuned[tk];
  }
  B->schedule = sc;
  B->schedule_amg = amg;
  cudaGraphExec_t ex;
  st = batch_exec(B, sc, amg, &ex);
  if (st != PGO_OK) return st;
  fill_dev_options(o, G->h_opt);
  CUDA_TRY(cudaMemcpyAsync(G->g.opt, G->h_opt, sizeof(DevOptions), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaEventRecord(G->ev0, s));
  CUDA_TRY(cudaGraphLaunch(ex, s));
  CUDA_TRY(cudaEventRecord(G->ev1, s));
  if (!reports && !poses_out) return PGO_OK;
  std::vector<BatchGraphState> hs(B->n);
  CUDA_TRY(cudaMemcpyAsync(hs.data(), B->args.gst, sizeof(BatchGraphState) * B->n, cudaMemcpyDeviceToHost, s));
  if (poses_out) {
    launch_batch_get_poses(G->g, B->args, G->d_scratch, s);
    CUDA_TRY(cudaGetLastError());
    cudaMemcpyKind kind = out_mem_space == PGO_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < B->n; ++k)
      if (poses_out[k])
        CUDA_TRY(cudaMemcpyAsync(poses_out[k], G->d_scratch + (size_t)B->v0[k] * 8, sizeof(double) * 8 * B->nv[k], kind, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, G->ev0, G->ev1);
  int bad = 0;
  for (int k = 0; k < B->n; ++k) {
    if (hs[k].status) bad = hs[k].status;
    if (!reports) continue;
    pgo_report& r = reports[k];
    std::memset(&r, 0, sizeof(r));
    r.initial_cost = hs[k].F0;
    r.final_cost = hs[k].F;
    r.final_lambda = hs[k].lambda;
    r.grad_inf_norm = hs[k].gmax;
    r.iterations = hs[k].it;
    r.accepted = hs[k].accepted;
    r.pcg_iterations = hs[k].pcg_total;
    r.stop_reason = hs[k].stop_reason;
    r.status = hs[k].status;
    r.ms_total = ms;
  }
  if (bad) return fail((pgo_status)bad, "a graph of the batch failed on the device (status %d)", bad);
  return PGO_OK;
}

pgo_status pgo_batch_schedule(const pgo_batch* B, int32_t* lanes, int32_t* threads, int32_t* blocks_per_sm,
                              float* tune_ms) {
  if (!B) return fail(PGO_ERR_INVALID_ARG, "batch is NULL");
  if (B->schedule < 0) return fail(PGO_ERR_STATE, "no batch solve has run");
  if (lanes) *lanes = batch_schedule_lanes(B->schedule);
  if (threads) *threads = batch_schedule_threads(B->schedule);
  if (blocks_per_sm) *blocks_per_sm = batch_schedule_blocks_per_sm(B->schedule);
  if (tune_ms) *tune_ms = B->tune_ms[batch_schedule_mixed(B->schedule) + 2 * (B->schedule_amg ? 1 : 0)];
  return PGO_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

pgo_status pgo_propagate_correction(int32_t n_vertices, const double* poses, int32_t current, const double* corrected,
                                    int32_t n_connected, const int32_t* connected, double* poses_out,
                                    int32_t* bad_out, void* stream) {
  if (n_vertices < 1 || n_connected < 0) return fail(PGO_ERR_INVALID_ARG, "need n_vertices >= 1 and n_connected >= 0");
  if (current < 0 || current >= n_vertices)
    return fail(PGO_ERR_INVALID_ARG, "current keyframe %d out of range [0, %d)", current, n_vertices);
  if (!poses || !corrected || !poses_out || (n_connected > 0 && !connected))
    return fail(PGO_ERR_INVALID_ARG, "NULL array");
  if (!aligned16(poses) || !aligned16(corrected) || !aligned16(poses_out))
    return fail(PGO_ERR_INVALID_ARG, "poses, corrected and poses_out must be 16-byte aligned");
  const char* lo = reinterpret_cast<const char*>(poses);
  const char* hi = lo + sizeof(double) * 8 * (size_t)n_vertices;
  const char* o = reinterpret_cast<const char*>(poses_out);
  if (o < hi && o + sizeof(double) * 8 * (size_t)n_vertices > lo)
    return fail(PGO_ERR_INVALID_ARG, "poses_out must not overlap poses");
  CUDA_TRY(launch_propagate_correction(n_vertices, poses, current, corrected, n_connected, connected, poses_out, bad_out,
                                       (cudaStream_t)stream));
  return PGO_OK;
}

pgo_status pgo_correct_points(int32_t n_vertices, const double* poses_before, const double* poses_after,
                              int32_t n_points, const double* points, const int32_t* ref_kf, double* points_out,
                              int32_t* bad_out, void* stream) {
  if (n_vertices < 1 || n_points < 0) return fail(PGO_ERR_INVALID_ARG, "need n_vertices >= 1 and n_points >= 0");
  if (!poses_before || !poses_after || (n_points > 0 && (!points || !ref_kf || !points_out)))
    return fail(PGO_ERR_INVALID_ARG, "NULL array");
  if (!aligned16(poses_before) || !aligned16(poses_after))
    return fail(PGO_ERR_INVALID_ARG, "poses_before and poses_after must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  void* table = nullptr;
  CUDA_TRY(cudaMallocAsync(&table, point_table_bytes(n_vertices), s));
  cudaError_t e = launch_correct_points(n_vertices, poses_before, poses_after, n_points, points, ref_kf,
                                        reinterpret_cast<double*>(table), points_out, bad_out, s);
  cudaError_t e2 = cudaFreeAsync(table, s);
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, "pgo_correct_points: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(PGO_ERR_CUDA, "pgo_correct_points free: %s", cudaGetErrorString(e2));
  return PGO_OK;
}

pgo_status pgo_evaluate_cost(int32_t n_vertices, int32_t n_edges, const int32_t* edge_i, const int32_t* edge_j,
                             const double* meas, const double* weight, const double* poses, double* cost_out,
                             int32_t* bad_edges_out, void* stream) {
  if (n_vertices < 0 || n_edges < 0) return fail(PGO_ERR_INVALID_ARG, "negative size");
  if (!cost_out) return fail(PGO_ERR_INVALID_ARG, "cost_out is NULL");
  if (n_edges > 0 && (!edge_i || !edge_j || !meas || !poses)) return fail(PGO_ERR_INVALID_ARG, "NULL input array");
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = eval_cost_blocks(n_edges);
  // workspace: partials (blocks doubles) + ticket + bad counter
  const size_t bytes = sizeof(double) * blocks + 64;
  void* ws = nullptr;
  CUDA_TRY(cudaMallocAsync(&ws, bytes, s));
  double* partial = reinterpret_cast<double*>(ws);
  unsigned* ticket = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(ws) + sizeof(double) * blocks);
  int* bad = reinterpret_cast<int*>(ticket + 4);
  cudaError_t e = cudaMemsetAsync(ticket, 0, 64, s);
  if (e == cudaSuccess) {
    launch_eval_cost_raw(n_vertices, n_edges, edge_i, edge_j, meas, weight, poses, partial, ticket, bad, cost_out,
                         bad_edges_out, s);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(ws, s);
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, "pgo_evaluate_cost: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(PGO_ERR_CUDA, "pgo_evaluate_cost free: %s", cudaGetErrorString(e2));
  return PGO_OK;
}

}  // extern "C"
