// Data-movement and evaluation kernels around the solver: pose upload and
// download, edge residuals and cost, Jacobian and normal-equation export in
// the caller's edge order, and the stateless cost evaluation.
#include "edge.cuh"

namespace pgo {

// pose8 (caller layout) -> pose buffer `buf` (buf < 0: the current buffer,
// read on the device), quaternion normalised.
__global__ void k_set_poses(DevGraph g, const double* src, int buf) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.N) return;
  if (buf < 0) buf = g.st->cur;
  Sim3T<double> P;
#pragma unroll
  for (int k = 0; k < 4; ++k) P.q[k] = src[(size_t)v * 8 + k];
#pragma unroll
  for (int k = 0; k < 3; ++k) P.t[k] = src[(size_t)v * 8 + 4 + k];
  P.s = src[(size_t)v * 8 + 7];
  qnormalize(P.q);
  store_pose(g, buf, v, P);
}

__global__ void k_get_poses(DevGraph g, int buf, double* dst) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.N) return;
  Sim3T<double> P = load_pose(g, buf, v);
#pragma unroll
  for (int k = 0; k < 4; ++k) dst[(size_t)v * 8 + k] = P.q[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) dst[(size_t)v * 8 + 4 + k] = P.t[k];
  dst[(size_t)v * 8 + 7] = P.s;
}

// Per-edge residuals (caller order, nullable) and the total cost at the
// poses in `buf`, written to *cost_out.
__global__ void __launch_bounds__(256) k_residuals(DevGraph g, int buf, const int* perm, double* r_out,
                                                   double* cost_out) {
  __shared__ double sh[32];
  if (buf < 0) buf = g.st->cur;
  double c[1] = {0.0};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.E; e += gridDim.x * blockDim.x) {
    const int i = g.ei[e], j = g.ej[e];
    Sim3T<double> Si = load_pose(g, buf, i), Sj = load_pose(g, buf, j), Z = load_meas(g, e);
    Sim3T<double> T = compose(Z, compose(Si, inverse(Sj)));
    qnormalize(T.q);
    double r[7];
    sim3_log(T, r);
    double ce = 0.0;
    if (g.L) {
      const double* L = g.L + (size_t)e * 28;
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) {
        double s = 0.0;
#pragma unroll
        for (int a = cc; a < 7; ++a) s += L[a * (a + 1) / 2 + cc] * r[a];
        ce += s * s;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) ce += r[k] * r[k];
    }
    c[0] += g.w[e] * ce;
    if (r_out) {
      double* o = r_out + (size_t)perm[e] * 7;
#pragma unroll
      for (int k = 0; k < 7; ++k) o[k] = r[k];
    }
  }
  block_sum<1>(c, sh);
  if (!publish_partials<1>(c, g.partial, &g.st->ticket[T_MISC])) return;
  double tot[1];
  gather_partials_sum<1>(g.partial, tot, sh);
  if (threadIdx.x == 0) *cost_out = tot[0];
}

// Repack padded blocks: dst[perm[k]] (stride dstride) <- src[k] (stride sstride).
__global__ void k_scatter(int n, int width, const int* perm, const double* src, int sstride, double* dst,
                          int dstride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * width) return;
  const int k = t / width, c = t % width;
  const int d = perm ? perm[k] : k;
  dst[(size_t)d * dstride + c] = src[(size_t)k * sstride + c];
}

// Stateless cost over caller arrays (pose8 poses and measurements).  Edges
// with an endpoint out of range, or i == j, are skipped and counted in *bad
// (zeroed by the caller); the last block copies the count to *bad_out.
__global__ void __launch_bounds__(256) k_eval_cost_raw(int N, int E, const int* ei, const int* ej,
                                                       const double* meas, const double* w,
                                                       const double* poses, double* partial,
                                                       unsigned* ticket, int* bad, double* cost_out,
                                                       int* bad_out) {
  __shared__ double sh[32];
  double c[1] = {0.0};
  int nbad = 0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int i = ei[e], j = ej[e];
    if (i < 0 || i >= N || j < 0 || j >= N || i == j) {
      ++nbad;
      continue;
    }
    Sim3T<double> Si, Sj, Z;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Si.q[k] = poses[(size_t)i * 8 + k];
      Sj.q[k] = poses[(size_t)j * 8 + k];
      Z.q[k] = meas[(size_t)e * 8 + k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Si.t[k] = poses[(size_t)i * 8 + 4 + k];
      Sj.t[k] = poses[(size_t)j * 8 + 4 + k];
      Z.t[k] = meas[(size_t)e * 8 + 4 + k];
    }
    Si.s = poses[(size_t)i * 8 + 7];
    Sj.s = poses[(size_t)j * 8 + 7];
    Z.s = meas[(size_t)e * 8 + 7];
    qnormalize(Si.q);
    qnormalize(Sj.q);
    qnormalize(Z.q);
    Sim3T<double> T = compose(Z, compose(Si, inverse(Sj)));
    qnormalize(T.q);
    double r[7];
    sim3_log(T, r);
    double ce = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) ce += r[k] * r[k];
    c[0] += (w ? w[e] : 1.0) * ce;
  }
  if (nbad) atomicAdd(bad, nbad);
  block_sum<1>(c, sh);
  if (!publish_partials<1>(c, partial, ticket)) return;
  double tot[1];
  gather_partials_sum<1>(partial, tot, sh);
  if (threadIdx.x == 0) {
    *cost_out = tot[0];
    // every block added its count before publishing its partial
    if (bad_out) *bad_out = atomicAdd(bad, 0);
  }
}

// Exact Jacobians A_i, A_j per edge (caller order, E x 2 x 49) at `buf`.
__global__ void __launch_bounds__(128) k_jacobians_out(DevGraph g, int buf, const int* perm, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.E) return;
  double r[7], Ai[7][7], Aj[7][7];
  edge_jacobians(g, buf, e, r, Ai, Aj);
  double* o = out + (size_t)perm[e] * 98;
#pragma unroll
  for (int a = 0; a < 7; ++a)
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      o[a * 7 + c] = Ai[a][c];
      o[49 + a * 7 + c] = Aj[a][c];
    }
}

// Caller-order measurements (pose8) and weights -> internal edge order.
__global__ void k_set_meas(DevGraph g, const int* perm, const double* meas8, const double* weight) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.E) return;
  const int e = perm[k];
  const double* m = meas8 + (size_t)e * 8;
  const double n = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
  const_cast<D4*>(g.zq)[k] = D4{m[0] / n, m[1] / n, m[2] / n, m[3] / n};
  const_cast<D4*>(g.zt)[k] = D4{m[4], m[5], m[6], m[7]};
  const_cast<double*>(g.zqn)[k] = n;
  if (weight) const_cast<double*>(g.w)[k] = weight[e];
}

void launch_set_meas(const DevGraph& g, const int* perm, const double* meas8, const double* weight, cudaStream_t s) {
  if (g.E == 0) return;
  k_set_meas<<<(g.E + 127) / 128, 128, 0, s>>>(g, perm, meas8, weight);
}

void launch_set_poses(const DevGraph& g, const double* src, int buf, cudaStream_t s) {
  k_set_poses<<<(g.N + 127) / 128, 128, 0, s>>>(g, src, buf);
}
void launch_get_poses(const DevGraph& g, int buf, double* dst, cudaStream_t s) {
  k_get_poses<<<(g.N + 127) / 128, 128, 0, s>>>(g, buf, dst);
}
void launch_residuals(const DevGraph& g, int buf, const int* perm, double* r_out, double* cost_out,
                      cudaStream_t s) {
  int blocks = (g.E + 255) / 256;
  if (blocks > g.partial_cap) blocks = g.partial_cap;
  if (blocks < 1) blocks = 1;
  k_residuals<<<blocks, 256, 0, s>>>(g, buf, perm, r_out, cost_out);
}
void launch_scatter(int n, int width, const int* perm, const double* src, int sstride, double* dst,
                    int dstride, cudaStream_t s) {
  if (n <= 0) return;
  const long long tot = (long long)n * width;
  k_scatter<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, width, perm, src, sstride, dst, dstride);
}
void launch_jacobians_out(const DevGraph& g, int buf, const int* perm, double* out, cudaStream_t s) {
  if (g.E == 0) return;
  k_jacobians_out<<<(g.E + 127) / 128, 128, 0, s>>>(g, buf, perm, out);
}
int eval_cost_blocks(int E) {
  int b = (E + 255) / 256;
  if (b > 1024) b = 1024;
  return b < 1 ? 1 : b;
}
void launch_eval_cost_raw(int N, int E, const int* ei, const int* ej, const double* meas, const double* w,
                          const double* poses, double* partial, unsigned* ticket, int* bad,
                          double* cost_out, int* bad_out, cudaStream_t s) {
  k_eval_cost_raw<<<eval_cost_blocks(E), 256, 0, s>>>(N, E, ei, ej, meas, w, poses, partial, ticket, bad,
                                                      cost_out, bad_out);
}

void launch_eval_cost_raw_blocks(int N, int E, const int* ei, const int* ej, const double* meas, const double* w,
                                 const double* poses, double* partial, unsigned* ticket, int* bad,
                                 double* cost_out, int* bad_out, int blocks, cudaStream_t s) {
  k_eval_cost_raw<<<blocks, 256, 0, s>>>(N, E, ei, ej, meas, w, poses, partial, ticket, bad, cost_out, bad_out);
}

}  // namespace pgo
