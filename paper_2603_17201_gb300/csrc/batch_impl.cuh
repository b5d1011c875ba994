// Batched form (device code): many independent essential graphs of uneven size solved by
// one persistent kernel launch, replayed as a one-node CUDA graph.
//
// A thread block solves whole graphs: it takes the next graph from a device
// work queue (largest graphs first), runs the complete Levenberg-Marquardt
// solve of that graph -- linearisation, assembly, block-Jacobi PCG (or the
// mixed-precision FP32 PCG inside FP64 refinement), update, FP64 cost and the
// accept/reject rule of the single-graph solver -- with block-level barriers
// only, writes the graph's report and takes the next graph.  Graphs never
// wait on one another, so the only grid-level coordination is the atomic
// work counter.  The per-edge and per-vertex steps are the same device
// functions as the single-graph kernels.
//
// Schedules (picked by the autotuner in the host runtime): G lanes per block
// row in the SpMV (4, 8 or 16) and NT threads per block (256 or 512).
#pragma once
#include "amg_cta.cuh"
#include "batch_sched.cuh"
#include "phases.cuh"

namespace pgo {

// Block-wide sums / maxima of K doubles; every thread receives the result.
template <int K, bool MAX>
__device__ __forceinline__ void cta_reduce(double (&v)[K], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = MAX ? fmax(v[k], t) : v[k] + t;
    }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = sh[k];
    for (int w = 1; w < nw; ++w) s = MAX ? fmax(s, sh[w * K + k]) : s + sh[w * K + k];
    v[k] = s;
  }
  __syncthreads();
}

template <class V>
struct BBufs;
template <>
struct BBufs<double> {
  static __device__ __forceinline__ const double* off(const DevGraph& g) { return g.off64; }
  static __device__ __forceinline__ const double* diag(const DevGraph& g) { return g.diag64; }
  static __device__ __forceinline__ double* minv(const DevGraph& g) { return g.minv64; }
  static __device__ __forceinline__ double* x(const DevGraph& g) { return g.x64; }
  static __device__ __forceinline__ double* r(const DevGraph& g) { return g.r64; }
  static __device__ __forceinline__ double* z(const DevGraph& g) { return g.z64; }
  static __device__ __forceinline__ double* p(const DevGraph& g) { return g.p64[0]; }
  static __device__ __forceinline__ double* q(const DevGraph& g) { return g.q64; }
  static constexpr int BLK = BLK64;
};
template <>
struct BBufs<float> {
  static __device__ __forceinline__ const float* off(const DevGraph& g) { return g.off32; }
  static __device__ __forceinline__ const float* diag(const DevGraph& g) { return g.diag32; }
  static __device__ __forceinline__ float* minv(const DevGraph& g) { return g.minv32; }
  static __device__ __forceinline__ float* x(const DevGraph& g) { return g.x32; }
  static __device__ __forceinline__ float* r(const DevGraph& g) { return g.r32; }
  static __device__ __forceinline__ float* z(const DevGraph& g) { return g.z32; }
  static __device__ __forceinline__ float* p(const DevGraph& g) { return g.p32[0]; }
  static __device__ __forceinline__ float* q(const DevGraph& g) { return g.q32; }
  static constexpr int BLK = BLK32;
};

// y += B p or B^T p for a row-major 7x7 block (plain loads).
template <class V, bool TR>
__device__ __forceinline__ void bmv7(const V* B, const V (&p)[7], V (&y)[7]) {
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    V row[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) row[c] = B[r * 7 + c];
    if (!TR) {
      V acc = V(0);
#pragma unroll
      for (int c = 0; c < 7; ++c) acc += row[c] * p[c];
      y[r] += acc;
    } else {
#pragma unroll
      for (int c = 0; c < 7; ++c) y[c] += row[c] * p[r];
    }
  }
}

// Block PCG on the rows [v0, v1) of one graph: (H + lambda I) x = rhs with
// rhs = -b (from_res = 0) or the FP64 refinement residual; tolerance tol on
// |r| / |rhs|.  Returns the iteration count.
template <class V, int G>
__device__ int cta_pcg(const DevGraph& g, int v0, int v1, int fixed, double lam, int from_res, double tol,
                       int maxit, double* sh, const AmgDev* A, int sg) {
  constexpr int BLK = BBufs<V>::BLK;
  const V* off = BBufs<V>::off(g);
  const V* diag = BBufs<V>::diag(g);
  const V* minv = BBufs<V>::minv(g);
  V* x = BBufs<V>::x(g);
  V* r = BBufs<V>::r(g);
  V* z = BBufs<V>::z(g);
  V* p = BBufs<V>::p(g);
  V* q = BBufs<V>::q(g);
  const V vl = V(lam);
  // start: x = 0, r = rhs, z = M r, p = z
  double d2[2] = {0.0, 0.0};
  if (A) {
    // multigrid: z = one V-cycle of the graph's segment (q is its scratch)
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      const size_t b = (size_t)v * VEC;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        x[b + k] = V(0);
        r[b + k] = (v == fixed) ? V(0) : V(from_res ? g.res64[b + k] : -g.b[b + k]);
      }
      x[b + 7] = V(0);
      r[b + 7] = V(0);
    }
    __syncthreads();
    cta_vcycle<V, G>(g, *A, sg, fixed, vl, r, q, z);
    if (from_res && tol >= kOneCycleTol) {
      // a correction pass within 1 / kOneCycleTol of its target: one cycle,
      // x = B r, as in the single-graph solver
      for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const size_t b = (size_t)v * VEC;
#pragma unroll
        for (int k = 0; k < 7; ++k) x[b + k] = (v == fixed) ? V(0) : z[b + k];
      }
      __syncthreads();
      return 1;
    }
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      const size_t b = (size_t)v * VEC;
      V lrz = V(0), lrr = V(0);
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const V zv = z[b + k], rv = r[b + k];
        p[b + k] = zv;
        lrz += rv * zv;
        lrr += rv * rv;
      }
      d2[0] += (double)lrz;
      d2[1] += (double)lrr;
    }
  } else
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const size_t b = (size_t)v * VEC;
    V rv[7], zv[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) rv[k] = (v == fixed) ? V(0) : V(from_res ? g.res64[b + k] : -g.b[b + k]);
    const V* M = minv + (size_t)v * BLK;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      V s = V(0);
#pragma unroll
      for (int c = 0; c < 7; ++c) s += M[a * 7 + c] * rv[c];
      zv[a] = s;
    }
    V lrz = V(0), lrr = V(0);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      x[b + k] = V(0);
      r[b + k] = rv[k];
      z[b + k] = zv[k];
      p[b + k] = zv[k];
      lrz += rv[k] * zv[k];
      lrr += rv[k] * rv[k];
    }
    d2[0] += (double)lrz;
    d2[1] += (double)lrr;
  }
  cta_reduce<2, false>(d2, sh);
  double rz = d2[0];
  const double bb = d2[1];
  if (!(bb > 0.0) || !(rz > 0.0)) return 0;
  const double tol2 = tol * tol;
  double rr_best = bb;   // multigrid stall test (see k_pcg)
  int stall = 0;
  const int sl = threadIdx.x & (G - 1);
  const int rows_step = blockDim.x / G;
  const unsigned gm = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (threadIdx.x & (32 - G)));
  int it = 0;
  while (it < maxit) {
    // q = (H + lambda I) p
    double pq[1] = {0.0};
    for (int vb = v0; vb < v1; vb += rows_step) {
      const int v = vb + (int)(threadIdx.x / G);
      const bool has = v < v1;
      V y[7];
#pragma unroll
      for (int a = 0; a < 7; ++a) y[a] = V(0);
      if (has) {
        const int k0 = g.inc_ptr[v], ks = g.inc_split[v], k1 = g.inc_ptr[v + 1];
        for (int k = k0 - 1 + sl; k < ks; k += G) {
          const bool dg = k < k0;
          const int u = dg ? v : g.inc_other[k];
          const V* B = dg ? diag + (size_t)v * BLK : off + (size_t)(g.inc_code[k] >> 1) * BLK;
          V pu[7];
#pragma unroll
          for (int c = 0; c < 7; ++c) pu[c] = p[(size_t)u * VEC + c];
          if (dg) {
#pragma unroll
            for (int a = 0; a < 7; ++a) y[a] += vl * pu[a];
          }
          bmv7<V, false>(B, pu, y);
        }
        for (int k = ks + sl; k < k1; k += G) {
          const int u = g.inc_other[k];
          V pu[7];
#pragma unroll
          for (int c = 0; c < 7; ++c) pu[c] = p[(size_t)u * VEC + c];
          bmv7<V, true>(off + (size_t)(g.inc_code[k] >> 1) * BLK, pu, y);
        }
      }
#pragma unroll
      for (int a = 0; a < 7; ++a)
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) y[a] += __shfl_xor_sync(gm, y[a], o);
      if (has) {
        // after the reduction every lane holds the row's 7 outputs; lane sl
        // stores components sl, sl + G, ... (G may be smaller than 7)
        const size_t b = (size_t)v * VEC;
        const bool live = v != fixed;
#pragma unroll
        for (int a = 0; a < 7; ++a) {
          if (a % G != sl) continue;
          q[b + a] = live ? y[a] : V(0);
          if (live) pq[0] += (double)(p[b + a] * y[a]);
        }
      }
    }
    cta_reduce<1, false>(pq, sh);
    if (!(pq[0] > 0.0)) break;
    const V alpha = V(rz / pq[0]);
    double t2[2] = {0.0, 0.0};
    if (A) {
      for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        if (v == fixed) continue;
        const size_t b = (size_t)v * VEC;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          x[b + k] += alpha * p[b + k];
          r[b + k] = r[b + k] - alpha * q[b + k];
        }
      }
      __syncthreads();
      cta_vcycle<V, G>(g, *A, sg, fixed, vl, r, q, z);
      for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const size_t b = (size_t)v * VEC;
        V lrz = V(0), lrr = V(0);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          lrz += r[b + k] * z[b + k];
          lrr += r[b + k] * r[b + k];
        }
        t2[0] += (double)lrz;
        t2[1] += (double)lrr;
      }
    } else
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      if (v == fixed) continue;
      const size_t b = (size_t)v * VEC;
      V rv[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        x[b + k] += alpha * p[b + k];
        rv[k] = r[b + k] - alpha * q[b + k];
        r[b + k] = rv[k];
      }
      const V* M = minv + (size_t)v * BLK;
      V lrz = V(0), lrr = V(0);
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        V s = V(0);
#pragma unroll
        for (int c = 0; c < 7; ++c) s += M[a * 7 + c] * rv[c];
        z[b + a] = s;
        lrz += rv[a] * s;
        lrr += rv[a] * rv[a];
      }
      t2[0] += (double)lrz;
      t2[1] += (double)lrr;
    }
    cta_reduce<2, false>(t2, sh);
    ++it;
    const double beta = (rz > 0.0) ? t2[0] / rz : 0.0;
    rz = t2[0];
    if (!(t2[1] > tol2 * bb) || !(rz > 0.0) || !isfinite(t2[1])) break;
    if (A) {
      if (t2[1] < 0.81 * rr_best) {
        rr_best = t2[1];
        stall = 0;
      } else if (++stall >= 20) {
        break;
      }
    }
    const V vb2 = V(beta);
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      const size_t b = (size_t)v * VEC;
#pragma unroll
      for (int k = 0; k < 7; ++k) p[b + k] = z[b + k] + vb2 * p[b + k];
    }
    __syncthreads();
  }
  __syncthreads();
  return it;
}

// FP64 refinement residual res = -b - (H + lambda I) dx (first pass: dx = 0,
// res = -b); returns |res|^2 over the free vertices.
static __device__ double cta_refine_residual(const DevGraph& g, int v0, int v1, int fixed, double lam, int first,
                                      double* sh) {
  double rr[1] = {0.0};
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const size_t b = (size_t)v * VEC;
    double y[7] = {0, 0, 0, 0, 0, 0, 0};
    if (!first) {
      double xv[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) xv[k] = g.dx64[b + k];
#pragma unroll
      for (int a = 0; a < 7; ++a) y[a] = lam * xv[a];
      bmv7<double, false>(g.diag64 + (size_t)v * BLK64, xv, y);
      const int k0 = g.inc_ptr[v], ks = g.inc_split[v], k1 = g.inc_ptr[v + 1];
      for (int k = k0; k < k1; ++k) {
        const int u = g.inc_other[k];
        double xu[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) xu[c] = g.dx64[(size_t)u * VEC + c];
        const double* B = g.off64 + (size_t)(g.inc_code[k] >> 1) * BLK64;
        if (k < ks) bmv7<double, false>(B, xu, y);
        else bmv7<double, true>(B, xu, y);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) g.dx64[b + k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const double rv = (v == fixed) ? 0.0 : -g.b[b + k] - y[k];
      g.res64[b + k] = rv;
      rr[0] += rv * rv;
    }
  }
  cta_reduce<1, false>(rr, sh);
  return rr[0];
}

// FP64 cost of the edges [e0, e1) at the poses in `buf`.
static __device__ double cta_cost(const DevGraph& g, int buf, int e0, int e1, double* sh) {
  double c[1] = {0.0};
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) c[0] += edge_cost(g, buf, e);
  cta_reduce<1, false>(c, sh);
  return c[0];
}

// The complete LM solve of one graph by one thread block.
template <int MIXED, int G>
__device__ void solve_graph(const DevGraph& g, const BatchArgs& a, int gi, double* sh, double* dense) {
  const AmgDev* A = a.amg ? g.amg : nullptr;
  const DevOptions* o = g.opt;
  const int v0 = a.v0[gi], v1 = v0 + a.nv[gi];
  const int e0 = a.e0[gi], e1 = e0 + a.ne[gi];
  const int fixed = a.fixed[gi];
  int cur = 0;
  double F = cta_cost(g, cur, e0, e1, sh);
  const double F0 = F;
  double lambda = -1.0, nu = 2.0, gmax = 0.0, bnorm2 = 0.0;
  int it = 0, acc = 0, stop = 0, status = 0, pcg_total = 0;
  bool need_lin = true;
  if (!isfinite(F)) {
    stop = 4;
    status = PGO_ERR_NUMERICAL;
  }
  while (status == 0 && it < o->max_iters) {
    if (need_lin) {
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) linearize_edge(g, cur, e, MIXED);
      __syncthreads();
      double mx[2] = {0.0, 0.0}, sm[1] = {0.0};
      for (int vb = v0; vb < v1; vb += blockDim.x / 8) {
        const int v = vb + (int)(threadIdx.x >> 3);
        if (v < v1) assemble_vertex(g, v, threadIdx.x & 7, MIXED, fixed, mx[0], mx[1], sm[0]);
      }
      cta_reduce<2, true>(mx, sh);
      cta_reduce<1, false>(sm, sh);
      if (lambda < 0.0) lambda = (o->lambda_init > 0.0) ? o->lambda_init : o->tau * mx[0];
      gmax = mx[1];
      bnorm2 = sm[0];
      need_lin = false;
      if (!(gmax > o->gtol)) {
        stop = isfinite(gmax) ? 2 : 4;
        if (!isfinite(gmax)) status = PGO_ERR_NUMERICAL;
        break;
      }
    }
    // preconditioner and damped linear solve
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      if (MIXED) precond_vertex<float>(g, v, fixed, lambda, g.minv32 + (size_t)v * BLK32);
      else precond_vertex<double>(g, v, fixed, lambda, g.minv64 + (size_t)v * BLK64);
    }
    __syncthreads();
    if (A) {
      if (MIXED) cta_amg_setup<float>(g, *A, gi, fixed, lambda, cur, sh, dense);
      else cta_amg_setup<double>(g, *A, gi, fixed, lambda, cur, sh, dense);
    }
    const double* dx;
    if (!MIXED) {
      pcg_total += cta_pcg<double, G>(g, v0, v1, fixed, lambda, 0, o->pcg_tol, o->pcg_max_iters, sh, A, gi);
      dx = g.x64;
    } else {
      for (int pass = 0; pass < o->refine_steps; ++pass) {
        const double rr = cta_refine_residual(g, v0, v1, fixed, lambda, pass == 0, sh);
        if (pass > 0 && !(rr > o->pcg_tol * o->pcg_tol * bnorm2)) break;
        // inner tolerance: only as tight as |res - H dx| <= pcg_tol |b| needs
        double itol = o->refine_tol;
        if (rr > 0.0 && bnorm2 > 0.0) itol = fmax(itol, o->pcg_tol * sqrt(bnorm2 / rr));
        itol = fmin(itol, 0.5);
        pcg_total += cta_pcg<float, G>(g, v0, v1, fixed, lambda, 1, itol, o->pcg_max_iters, sh, A, gi);
        for (int t = v0 * VEC + threadIdx.x; t < v1 * VEC; t += blockDim.x) g.dx64[t] += (double)g.x32[t];
        __syncthreads();
      }
      dx = g.dx64;
    }
    // candidate, predicted decrease, FP64 cost, accept / reject
    double pr[1] = {0.0};
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x)
      pr[0] += update_vertex(g, cur, v, fixed, dx + (size_t)v * VEC, lambda);
    cta_reduce<1, false>(pr, sh);
    const double Fn = cta_cost(g, cur ^ 1, e0, e1, sh);
    const double pred = pr[0];
    const double rho = (pred > 0.0 && isfinite(Fn)) ? (F - Fn) / pred : -1.0;
    const bool flat = isfinite(Fn) && fabs(F - Fn) <= o->ftol * F;
    ++it;
    if (rho > 0.0) {
      cur ^= 1;
      double f = 2.0 * rho - 1.0;
      f = 1.0 - f * f * f;
      lambda *= fmax(f, 1.0 / 3.0);
      nu = 2.0;
      need_lin = true;
      ++acc;
      F = Fn;
      if (flat) {
        stop = 1;
        break;
      }
    } else {
      lambda *= nu;
      nu *= 2.0;
      if (flat) {
        stop = 1;
        break;
      }
      if (!(lambda < 1e32)) {
        stop = 3;
        break;
      }
    }
  }
  if (threadIdx.x == 0) {
    BatchGraphState s;
    s.F0 = F0;
    s.F = F;
    s.lambda = lambda;
    s.gmax = gmax;
    s.it = it;
    s.accepted = acc;
    s.pcg_total = pcg_total;
    s.stop_reason = stop;
    s.status = status;
    s.cur = cur;
    s.pad0 = s.pad1 = 0;
    a.gst[gi] = s;
  }
  __syncthreads();
}

template <int MIXED, int G, int NT, int BPS>
__global__ void __launch_bounds__(NT, BPS) k_batch_lm(DevGraph g, BatchArgs a) {
  __shared__ double sh[(NT / 32) * 2 + 8];
  __shared__ int s_next;
  extern __shared__ double dense[];   // multigrid: the coarsest inverse of the current graph
  for (;;) {
    if (threadIdx.x == 0) s_next = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= a.n_graphs) return;
    solve_graph<MIXED, G>(g, a, a.order[q], sh, dense);
  }
}

// Poses of every graph from its own current buffer into dst (pose8, global

// One launch of the persistent batch kernel for one schedule.  Defined here
// and instantiated explicitly by the batch_part*.cu translation units (a few
// schedules each, so that they compile in parallel).
template <int MIXED, int G, int NT, int BPS>
cudaError_t launch_batch_instance(const DevGraph& g, const BatchArgs& a, int blocks, size_t smem, cudaStream_t s) {
  k_batch_lm<MIXED, G, NT, BPS><<<blocks, NT, smem, s>>>(g, a);
  return cudaGetLastError();
}

}  // namespace pgo
