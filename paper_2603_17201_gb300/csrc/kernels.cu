// Edge and vertex kernels of the Levenberg-Marquardt loop (Sec. IV-F):
//   k_linearize     edge residual r = log(Z S_i S_j^-1) and its exact
//                   Jacobians (FP64: forward-mode duals through the log map;
//                   mixed precision: FP32 from the left-Jacobian series),
//                   the off-diagonal block and per-edge-side contributions;
//   k_assemble      deterministic per-vertex gather of the contributions into
//                   the diagonal blocks H_vv and the gradient b_v;
//   k_cost          F = sum w r^T Omega r (FP64) and the LM accept/reject rule;
//   k_update        candidate poses exp(delta) S and the predicted decrease.
#include <cfloat>

#include "phases.cuh"

namespace pgo {

// Linearisation: one thread per edge (MIXED: FP32 Jacobians and H products).
// The LM loop and the standalone entry points linearise the mixed mode with
// the fused k_lin_assemble below; this per-edge form stays for FP64.
template <int MIXED>
__global__ void __launch_bounds__(128) k_linearize(DevGraph g) {
  const SolverState* st = g.st;
  if (st->done || !st->need_lin) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.E) return;
  linearize_edge(g, st->cur, e, MIXED);
}

// End of an assembly pass (every block calls it once, all its threads): the
// last block derives max diag(H), |b|_inf and |b|^2 over the free vertices
// from the blocks' partials, sets lambda_0 on the first linearisation and
// applies the gradient stop test (mode 0); other modes only store the norms.
__device__ void assemble_finish(const DevGraph& g, double mdiag, double mgrad, double b2, int mode, double* sh) {
  SolverState* st = g.st;
  double mx[2] = {mdiag, mgrad};
  double sm[1] = {b2};
  block_max<2>(mx, sh);
  block_sum<1>(sm, sh + 64);
  double part[3] = {mx[0], mx[1], sm[0]};
  if (publish_partials<3>(part, g.partial, &st->ticket[T_ASSEMBLE])) {
    double tot[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
      tot[0] = fmax(tot[0], __ldcg(g.partial + b * 3 + 0));
      tot[1] = fmax(tot[1], __ldcg(g.partial + b * 3 + 1));
      tot[2] += __ldcg(g.partial + b * 3 + 2);
    }
    double m2[2] = {tot[0], tot[1]};
    double s1[1] = {tot[2]};
    block_max<2>(m2, sh);
    block_sum<1>(s1, sh + 64);
    if (threadIdx.x == 0) {
      const DevOptions* o = g.opt;
      st->maxdiag = m2[0];
      st->gmax = m2[1];
      st->bnorm2 = s1[0];
      if (mode != 0) {
        st->need_lin = 0;
        return;
      }
      if (st->lambda < 0.0) st->lambda = (o->lambda_init > 0.0) ? o->lambda_init : o->tau * m2[0];
      st->need_lin = 0;
      if (!(m2[1] > o->gtol)) {
        st->done = 1;
        st->stop_reason = isfinite(m2[1]) ? 2 : 4;
        if (!isfinite(m2[1])) st->status = PGO_ERR_NUMERICAL;
      }
    }
  }
}

// Assembly: 8 lanes per vertex gather the incident edge-side contributions in edge
// order (deterministic), then write H_vv (full symmetric) and b_v.  The last
// block derives max diag(H), |b|_inf and |b|^2 over the free vertices, sets
// lambda_0 on the first linearisation and applies the gradient stop test.
__global__ void __launch_bounds__(256) k_assemble(DevGraph g, int mixed, int mode) {
  SolverState* st = g.st;
  if (mode == 0 && (st->done || !st->need_lin)) return;
  __shared__ double sh[32 * 3];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = tid >> 3, lane = tid & 7;
  double mdiag = 0.0, mgrad = 0.0, b2 = 0.0;
  if (v < g.N) assemble_vertex(g, v, lane, mixed, g.fixed, mdiag, mgrad, b2);
  assemble_finish(g, mdiag, mgrad, b2, mode, sh);
}

// Mixed precision: linearisation and assembly in one pass (Sec. IV-F), a
// warp per vertex.  Lane k of vertex v's warp takes v's incidence entries k,
// k + 32, ...: the edge's FP32 Jacobian on v's side from the cached FP64
// residual, the side's contribution [upper(w A^T A), w A^T r] and, on the i
// side, the off-diagonal block.  The warp's contributions meet in a shared
// memory table and lane u sums entry u over the lanes in lane order: a
// segmented reduction whose segment is the vertex's incident edges, in a
// fixed order (deterministic).  H_vv and b_v are written once; no per-edge
// contribution goes through global memory.
constexpr int kLinWarps = 4;
__global__ void __launch_bounds__(kLinWarps * 32) k_lin_assemble(DevGraph g) {
  SolverState* st = g.st;
  if (st->done || !st->need_lin) return;
  __shared__ float htab[kLinWarps][28 * 33];    // H entry u of lane k at 33 u + k
  __shared__ double btab[kLinWarps][7 * 33];    // b entry a of lane k at 33 a + k
  __shared__ double bpart[kLinWarps][4 * 7];    // b partial sums of 8 lanes
  __shared__ double sh[32 * 3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * kLinWarps + warp;
  float* ht = htab[warp];
  double* bt = btab[warp];
  double mdiag = 0.0, mgrad = 0.0, b2 = 0.0;
  if (v < g.N) {   // whole warps
    const int cur = st->cur;
    const int k0 = __ldg(g.inc_ptr + v), k1 = __ldg(g.inc_ptr + v + 1);
    float hacc = 0.f;    // H entry `lane` (lane < 28)
    double bacc = 0.0;   // b entry `lane` (lane < 7)
    const int bc = lane % 7, bg = lane / 7;   // lanes < 28: b entry bc over lanes 8 bg .. 8 bg + 7
    for (int kb = k0; kb < k1; kb += 32) {
      const int k = kb + lane;
      if (k < k1) {
        lin_entry_mixed(g, cur, __ldg(g.inc_code + k), ht + lane, bt + lane);
      } else {
#pragma unroll
        for (int u = 0; u < 28; ++u) ht[33 * u + lane] = 0.f;
#pragma unroll
        for (int a = 0; a < 7; ++a) bt[33 * a + lane] = 0.0;
      }
      __syncwarp();
      // sums in lane order: H in FP32 (one entry per lane), b in FP64 (four
      // partial sums of 8 lanes, then lanes 0..6 add the four in order)
      if (lane < 28) {
#pragma unroll 8
        for (int q = 0; q < 32; ++q) hacc += ht[33 * lane + q];
        double p = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) p += bt[33 * bc + 8 * bg + q];
        bpart[warp][bg * 7 + bc] = p;
      }
      __syncwarp();
      if (lane < 7) bacc += ((bpart[warp][lane] + bpart[warp][7 + lane]) + bpart[warp][14 + lane]) + bpart[warp][21 + lane];
      __syncwarp();
    }
    const bool free_v = v != g.fixed;
    if (lane < 28) {
      const int ra = c_up_a[lane], rc = c_up_c[lane];
      const double a = (double)hacc;
      g.diag64[(size_t)v * BLK64 + ra * 7 + rc] = a;
      g.diag64[(size_t)v * BLK64 + rc * 7 + ra] = a;
      g.diag32[(size_t)v * BLK32 + ra * 7 + rc] = hacc;
      g.diag32[(size_t)v * BLK32 + rc * 7 + ra] = hacc;
      if (ra == rc && free_v) mdiag = a;
    }
    if (lane < 8) {
      const double bv = lane < 7 ? bacc : 0.0;
      g.b[(size_t)v * VEC + lane] = bv;
      if (lane < 7 && free_v) {
        mgrad = fabs(bv);
        b2 = bv * bv;
      }
    }
  }
  assemble_finish(g, mdiag, mgrad, b2, 0, sh);
}

// Residual cache of the current poses for the fused linearisation outside the
// LM loop (one thread per edge).
__global__ void __launch_bounds__(128) k_residual(DevGraph g) {
  const SolverState* st = g.st;
  if (st->done || !st->need_lin) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < g.E) (void)edge_cost(g, st->cur, e, true);
}

void launch_lin_assemble_mixed(const DevGraph& g, int cached, cudaStream_t s) {
  if (!cached && g.E > 0) k_residual<<<(g.E + 127) / 128, 128, 0, s>>>(g);
  k_lin_assemble<<<(g.N + kLinWarps - 1) / kLinWarps, kLinWarps * 32, 0, s>>>(g);
}

// mode 0: F at the current poses (start of a solve).
// mode 1: F' at the candidate poses, then the LM accept/reject rule.
// store: leave the residual cache of the evaluated poses (mixed LM loop).
__global__ void __launch_bounds__(256) k_cost(DevGraph g, int mode, unsigned long long lm_cond, int store) {
  SolverState* st = g.st;
  if (mode == 1 && st->done) {
    // stopped earlier in this iteration (gradient test): leave the LM loop
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(lm_cond, false);
    return;
  }
  __shared__ double sh[32];
  const int buf = mode == 0 ? st->cur : (st->cur ^ 1);
  double c[1] = {0.0};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.E; e += gridDim.x * blockDim.x)
    c[0] += edge_cost(g, buf, e, store != 0);
  block_sum<1>(c, sh);
  if (!publish_partials<1>(c, g.partial, &st->ticket[T_COST])) return;
  double tot[1];
  gather_partials_sum<1>(g.partial, tot, sh);
  if (threadIdx.x != 0) return;
  const DevOptions* o = g.opt;
  const double Fn = tot[0];
  if (mode == 0) {
    st->F = Fn;
    st->F0 = Fn;
    if (!isfinite(Fn)) {
      st->done = 1;
      st->stop_reason = 4;
      st->status = PGO_ERR_NUMERICAL;
    }
    if (o->max_iters <= 0) st->done = 1;
    set_cond(lm_cond, !st->done);
    return;
  }
  st->F_new = Fn;
  const double F = st->F, pred = st->pred;
  const double rho = (pred > 0.0 && isfinite(Fn)) ? (F - Fn) / pred : -1.0;
  // |F - F'| <= ftol F, accepted or not: no progress is measurable
  const bool flat = isfinite(Fn) && fabs(F - Fn) <= o->ftol * F;
  if (rho > 0.0) {
    st->cur ^= 1;
    double f = 2.0 * rho - 1.0;
    f = 1.0 - f * f * f;
    st->lambda *= fmax(f, 1.0 / 3.0);
    st->nu = 2.0;
    st->need_lin = 1;
    st->accepted += 1;
    st->F = Fn;
    if (flat) {
      st->done = 1;
      st->stop_reason = 1;
    }
  } else {
    st->lambda *= st->nu;
    st->nu *= 2.0;
    if (flat) {
      st->done = 1;
      st->stop_reason = 1;
    } else if (!(st->lambda < 1e32)) {
      st->done = 1;
      st->stop_reason = 3;
    }
  }
  st->it += 1;
  if (st->it >= o->max_iters && !st->done) {
    st->done = 1;
    st->stop_reason = 0;
  }
  set_cond(lm_cond, !st->done && st->it < o->max_iters);
}

// Candidate poses S' = exp(delta) S (delta from x64 or, mixed, dx64) into
// buffer cur^1; the fixed vertex is copied.  The last block stores the
// predicted decrease delta^T (lambda delta - b).
__global__ void __launch_bounds__(256) k_update(DevGraph g, int mixed) {
  SolverState* st = g.st;
  if (st->done) return;
  __shared__ double sh[32];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int cur = st->cur;
  const double lam = st->lambda;
  double pr[1] = {0.0};
  if (v < g.N) pr[0] = update_vertex(g, cur, v, g.fixed, (mixed ? g.dx64 : g.x64) + (size_t)v * VEC, lam);
  block_sum<1>(pr, sh);
  if (!publish_partials<1>(pr, g.partial, &st->ticket[T_UPDATE])) return;
  double tot[1];
  gather_partials_sum<1>(g.partial, tot, sh);
  if (threadIdx.x == 0) st->pred = tot[0];
}

// Fresh LM state for a solve (keeps the current pose buffer).
__global__ void k_lm_reset(DevGraph g) {
  SolverState* st = g.st;
  const int cur = st->cur;
  st->F = 0.0;
  st->F_new = 0.0;
  st->lambda = -1.0;
  st->nu = 2.0;
  st->pred = 0.0;
  st->gmax = 0.0;
  st->maxdiag = 0.0;
  st->it = 0;
  st->accepted = 0;
  st->done = 0;
  st->need_lin = 1;
  st->stop_reason = 0;
  st->status = 0;
  st->pcg_total = 0;
  st->pcg_hit_cap = 0;
  st->ref_done = 0;
  for (int t = 0; t < T_COUNT; ++t) st->ticket[t] = 0u;
  st->cur = cur;
}

// State for a standalone re-solve at opt->lambda_fixed (no linearisation).
__global__ void k_resolve_reset(DevGraph g) {
  SolverState* st = g.st;
  st->done = 0;
  st->need_lin = 0;
  st->ref_done = 0;
  st->status = 0;
  st->pcg_total = 0;
  st->pcg_hit_cap = 0;
  st->lambda = g.opt->lambda_fixed;
  for (int t = 0; t < T_COUNT; ++t) st->ticket[t] = 0u;
}

void launch_resolve_reset(const DevGraph& g, cudaStream_t s) { k_resolve_reset<<<1, 1, 0, s>>>(g); }

// The edge and vertex kernels below are latency chains of FP64 arithmetic
// (log and exp maps) over a few thousand items: small thread blocks spread
// them over every SM instead of a few.
void launch_cost(const DevGraph& g, int mode, cudaStream_t s, unsigned long long lm_cond, int store) {
  int blocks = (g.E + 127) / 128;
  if (blocks > g.partial_cap) blocks = g.partial_cap;
  if (blocks < 1) blocks = 1;
  k_cost<<<blocks, 128, 0, s>>>(g, mode, lm_cond, store);
}

void launch_linearize(const DevGraph& g, int mixed, cudaStream_t s) {
  if (g.E == 0) return;
  if (mixed) k_linearize<1><<<(g.E + 127) / 128, 128, 0, s>>>(g);
  else k_linearize<0><<<(g.E + 127) / 128, 128, 0, s>>>(g);
}

void launch_assemble(const DevGraph& g, int mixed, cudaStream_t s) {
  int blocks = (g.N * 8 + 127) / 128;
  k_assemble<<<blocks, 128, 0, s>>>(g, mixed, 0);
}

void launch_assemble_mode(const DevGraph& g, int mode, cudaStream_t s) {
  int blocks = (g.N * 8 + 127) / 128;
  k_assemble<<<blocks, 128, 0, s>>>(g, 0, mode);
}

// 0: standalone step at opt->lambda_fixed; 1: swap the current pose buffer.
__global__ void k_state_ctl(DevGraph g, int op) {
  SolverState* st = g.st;
  if (op == 0) {
    st->done = 0;
    st->need_lin = 1;
    st->ref_done = 0;
    st->status = 0;
    st->pcg_hit_cap = 0;
    st->lambda = g.opt->lambda_fixed;
    for (int t = 0; t < T_COUNT; ++t) st->ticket[t] = 0u;
  } else {
    st->cur ^= 1;
  }
}

void launch_state_ctl(const DevGraph& g, int op, cudaStream_t s) { k_state_ctl<<<1, 1, 0, s>>>(g, op); }

// x64 *= f (step halving of the Newton polish).
__global__ void k_scale_x(DevGraph g, double f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.N * VEC) g.x64[t] *= f;
}

void launch_scale_x(const DevGraph& g, double f, cudaStream_t s) {
  k_scale_x<<<(g.N * VEC + 255) / 256, 256, 0, s>>>(g, f);
}

void launch_update(const DevGraph& g, int mixed, cudaStream_t s) {
  k_update<<<(g.N + 31) / 32, 32, 0, s>>>(g, mixed);
}

void launch_lm_reset(const DevGraph& g, cudaStream_t s) { k_lm_reset<<<1, 1, 0, s>>>(g); }

int max_partials(int N, int E) {
  int a = (N + 3) / 4;            // warp-per-row kernels (4 rows per block)
  int c = (E + 255) / 256;
  int m = a > c ? a : c;
  return m + 8;
}

}  // namespace pgo
