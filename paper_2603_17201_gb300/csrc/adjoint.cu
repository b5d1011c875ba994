// Implicit-adjoint gradients of the optimised poses x*(Z, w).
//
// At the optimum the gradient b(x*, Z, w) = sum_e w_e A_e^T Omega_e r_e is
// zero.  Differentiating that identity gives dx*/dtheta = -H^-1 db/dtheta with
// H = db/dx the full (second-order) Hessian of F/2 in left-tangent
// coordinates, so for a loss L(x*):
//     mu = H^-1 dL/dx,        dL/dtheta = -mu^T db/dtheta,
//     db/dw_e = A_e^T Omega_e r_e  (scattered to the edge's two vertices),
//     db/dz_e = d(w_e A_e^T Omega_e r_e)/d(zeta_e),  Z_e <- exp(zeta_e) Z_e.
// This extends the automatically differentiated objective of the paper's
// graph optimisation (Sec. IV-F) by one more order.
//
// Every derivative here is exact forward-mode automatic differentiation: the
// edge gradient g_e = w A^T r is evaluated in nested dual numbers (an outer
// one-direction dual carries d/d(direction); the inner 7-direction dual
// produces the Jacobian A through the log map), one pass per direction.
#include "edge.cuh"

namespace pgo {

using D1 = Dual<double, 1>;

// Rotation matrix of a unit quaternion, generic scalar.
template <class S>
__device__ __forceinline__ void qmat_g(const S* q, S* R) {
  const S x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = addc(scal(y * y + z * z, -2.0), 1.0);
  R[1] = scal(x * y - w * z, 2.0);
  R[2] = scal(x * z + w * y, 2.0);
  R[3] = scal(x * y + w * z, 2.0);
  R[4] = addc(scal(x * x + z * z, -2.0), 1.0);
  R[5] = scal(y * z - w * x, 2.0);
  R[6] = scal(x * z - w * y, 2.0);
  R[7] = scal(y * z + w * x, 2.0);
  R[8] = addc(scal(x * x + y * y, -2.0), 1.0);
}

// A = sign * J * Adj(R, t, s), generic scalar.
template <class S>
__device__ __forceinline__ void jac_adj_g(const S (&J)[7][7], const S* R, const S* t, const S& s, double sign,
                                          S (&A)[7][7]) {
  S tR[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    tR[0 * 3 + c] = t[1] * R[6 + c] - t[2] * R[3 + c];
    tR[1 * 3 + c] = t[2] * R[0 + c] - t[0] * R[6 + c];
    tR[2 * 3 + c] = t[0] * R[3 + c] - t[1] * R[0 + c];
  }
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S v = J[a][0] * R[c] + J[a][3] * tR[c];
#pragma unroll
      for (int k = 1; k < 3; ++k) v = v + J[a][k] * R[k * 3 + c] + J[a][3 + k] * tR[k * 3 + c];
      A[a][c] = scal(v, sign);
      S u = J[a][3] * R[c];
#pragma unroll
      for (int k = 1; k < 3; ++k) u = u + J[a][3 + k] * R[k * 3 + c];
      A[a][3 + c] = scal(s * u, sign);
    }
    A[a][6] = scal(J[a][6] - (J[a][3] * t[0] + J[a][4] * t[1] + J[a][5] * t[2]), sign);
  }
}

// Edge gradient g = w [A_i^T L L^T r ; A_j^T L L^T r] (14 values), generic
// scalar.  With S = D1 the poses / measurement carry one tangent direction
// and the derivative parts of g are one column of the second derivatives.
template <class S>
__device__ __forceinline__ void edge_gradient(const Sim3T<S>& Si, const Sim3T<S>& Sj, const Sim3T<S>& Z, double w,
                                              const double* L, S (&g)[14]) {
  Sim3T<S> T = compose(Z, compose(Si, inverse(Sj)));
  qnormalize(T.q);
  Sim3T<Dual<S, 7>> D = seed_left(T);
  Dual<S, 7> xi[7];
  sim3_log(D, xi);
  S r[7], J[7][7];
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    r[a] = xi[a].v;
#pragma unroll
    for (int k = 0; k < 7; ++k) J[a][k] = xi[a].d[k];
  }
  S RZ[9], RT[9];
  qmat_g(Z.q, RZ);
  qmat_g(T.q, RT);
  S Ai[7][7], Aj[7][7];
  jac_adj_g(J, RZ, Z.t, Z.s, 1.0, Ai);
  jac_adj_g(J, RT, T.t, T.s, -1.0, Aj);
  // Omega r with Omega = L L^T (identity when L is null)
  S Or[7];
  if (L) {
    S u[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      u[c] = lift<S>(0.0);
#pragma unroll
      for (int a = c; a < 7; ++a) u[c] = u[c] + scal(r[a], L[a * (a + 1) / 2 + c]);
    }
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      Or[a] = lift<S>(0.0);
#pragma unroll
      for (int c = 0; c <= a; ++c) Or[a] = Or[a] + scal(u[c], L[a * (a + 1) / 2 + c]);
    }
  } else {
#pragma unroll
    for (int a = 0; a < 7; ++a) Or[a] = r[a];
  }
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    S si = lift<S>(0.0), sj = lift<S>(0.0);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      si = si + Ai[k][a] * Or[k];
      sj = sj + Aj[k][a] * Or[k];
    }
    g[a] = scal(si, w);
    g[7 + a] = scal(sj, w);
  }
}

// A pose as D1 with derivative (I + t G_k) P along generator k (left
// perturbation), or with zero derivative (k < 0).
__device__ __forceinline__ Sim3T<D1> seed_dir(const Sim3T<double>& P, int k) {
  Sim3T<D1> D;
#pragma unroll
  for (int c = 0; c < 4; ++c) D.q[c] = dconst<double, 1>(P.q[c]);
#pragma unroll
  for (int c = 0; c < 3; ++c) D.t[c] = dconst<double, 1>(P.t[c]);
  D.s = dconst<double, 1>(P.s);
  if (k < 0) return D;
  const double* v = P.q;
  const double w = P.q[3];
  const double* t = P.t;
  if (k < 3) {
    // dq = 1/2 (e_k, 0) q, dt = e_k x t
    double e[3] = {0, 0, 0};
    e[k] = 1.0;
    const double ex[3] = {e[1] * v[2] - e[2] * v[1], e[2] * v[0] - e[0] * v[2], e[0] * v[1] - e[1] * v[0]};
#pragma unroll
    for (int c = 0; c < 3; ++c) D.q[c].d[0] = 0.5 * (w * e[c] + ex[c]);
    D.q[3].d[0] = -0.5 * v[k];
    const double et[3] = {e[1] * t[2] - e[2] * t[1], e[2] * t[0] - e[0] * t[2], e[0] * t[1] - e[1] * t[0]};
#pragma unroll
    for (int c = 0; c < 3; ++c) D.t[c].d[0] = et[c];
  } else if (k < 6) {
    D.t[k - 3].d[0] = 1.0;
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) D.t[c].d[0] = t[c];
    D.s.d[0] = P.s;
  }
  return D;
}

// Full-Hessian contributions of one edge: the 14x14 block d g_e / d(x_i, x_j)
// column by column (one nested-dual pass per direction).  Diagonal blocks go
// to the contribution slots (symmetrised upper triangles), the (i, j) block
// symmetrised as (H_ij + H_ji^T) / 2 to off64.  The gradient slots receive the
// edge gradient g_e itself (with_grad: the Newton polish) or zero (adjoint).
__global__ void __launch_bounds__(64) k_adj_hessian(DevGraph g, int with_grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.E) return;
  const int cur = g.st->cur;
  const Sim3T<double> Si = load_pose(g, cur, g.ei[e]), Sj = load_pose(g, cur, g.ej[e]), Z = load_meas(g, e);
  const double w = g.w[e];
  const double* L = g.L ? g.L + (size_t)e * 28 : nullptr;
  double H[14][14];   // H[row][col] = d g_row / d x_col
  double gv[14];      // g_e (the value part, the same in every pass)
  const Sim3T<D1> Zd = seed_dir(Z, -1);
  for (int col = 0; col < 14; ++col) {
    const Sim3T<D1> Pi = seed_dir(Si, col < 7 ? col : -1);
    const Sim3T<D1> Pj = seed_dir(Sj, col >= 7 ? col - 7 : -1);
    D1 gg[14];
    edge_gradient(Pi, Pj, Zd, w, L, gg);
#pragma unroll
    for (int row = 0; row < 14; ++row) H[row][col] = gg[row].d[0];
    if (col == 0)
#pragma unroll
      for (int row = 0; row < 14; ++row) gv[row] = gg[row].v;
  }
  double* ci = g.contrib + (size_t)e * 2 * CONTRIB;
  double* cj = ci + CONTRIB;
  int u = 0;
  for (int a = 0; a < 7; ++a)
    for (int c = a; c < 7; ++c, ++u) {
      ci[u] = 0.5 * (H[a][c] + H[c][a]);
      cj[u] = 0.5 * (H[7 + a][7 + c] + H[7 + c][7 + a]);
    }
  for (int k = 28; k < CONTRIB; ++k) {
    ci[k] = (with_grad && k < 35) ? gv[k - 28] : 0.0;
    cj[k] = (with_grad && k < 35) ? gv[7 + k - 28] : 0.0;
  }
  double* off = g.off64 + (size_t)e * BLK64;
  for (int a = 0; a < 7; ++a)
    for (int c = 0; c < 7; ++c) off[a * 7 + c] = 0.5 * (H[a][7 + c] + H[7 + c][a]);
}

// dL/d(delta) of the fixed-pose layouts: for pose8 input, the chain rule
// through S <- exp(delta) S of (q, t, s):
//   omega_k: 1/2 [w gq_k + (v x gq)_k - gw v_k] + (t x gt)_k
//   upsilon: gt,   sigma: gt . t + gs s
// b_v = -dL/d(delta_v) (the PCG right-hand side is -b), 0 on the fixed vertex.
__global__ void k_adj_rhs(DevGraph g, const double* dL, int layout) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.N) return;
  double gd[7];
  if (layout == PGO_GRAD_POSE8) {
    const Sim3T<double> P = load_pose(g, g.st->cur, v);
    const double* p = dL + (size_t)v * 8;
    const double gq[3] = {p[0], p[1], p[2]}, gw = p[3], gt[3] = {p[4], p[5], p[6]}, gs = p[7];
    const double* q = P.q;
    const double w = q[3];
    const double vxg[3] = {q[1] * gq[2] - q[2] * gq[1], q[2] * gq[0] - q[0] * gq[2], q[0] * gq[1] - q[1] * gq[0]};
    const double* t = P.t;
    const double txg[3] = {t[1] * gt[2] - t[2] * gt[1], t[2] * gt[0] - t[0] * gt[2], t[0] * gt[1] - t[1] * gt[0]};
    for (int k = 0; k < 3; ++k) gd[k] = 0.5 * (w * gq[k] + vxg[k] - gw * q[k]) + txg[k];
    for (int k = 0; k < 3; ++k) gd[3 + k] = gt[k];
    gd[6] = gt[0] * t[0] + gt[1] * t[1] + gt[2] * t[2] + gs * P.s;
  } else {
    for (int k = 0; k < 7; ++k) gd[k] = dL[(size_t)v * 7 + k];
  }
  double* b = g.b + (size_t)v * VEC;
  for (int k = 0; k < 7; ++k) b[k] = (v == g.fixed) ? 0.0 : -gd[k];
  b[7] = 0.0;
}

// Per-edge gradients with mu = x64: dL/dw_e = -mu_e^T (A^T Omega r) and
// dL/dzeta_e = -mu_e^T d g_e / d zeta (7 nested passes), in the caller's
// edge order; for the pose8 layout dL/dzeta is mapped to the measurement's
// (unnormalised) pose8 entries.
__global__ void __launch_bounds__(64) k_adj_edges(DevGraph g, const int* perm, double* dL_dmeas, double* dL_dw,
                                                  int layout) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.E) return;
  const int cur = g.st->cur;
  const int i = g.ei[e], j = g.ej[e];
  const Sim3T<double> Si = load_pose(g, cur, i), Sj = load_pose(g, cur, j), Z = load_meas(g, e);
  const double* L = g.L ? g.L + (size_t)e * 28 : nullptr;
  double mu[14];
  for (int k = 0; k < 7; ++k) {
    mu[k] = g.x64[(size_t)i * VEC + k];
    mu[7 + k] = g.x64[(size_t)j * VEC + k];
  }
  const int ce = perm[e];
  if (dL_dw) {
    double g0[14];
    edge_gradient(Si, Sj, Z, 1.0, L, g0);
    double s = 0.0;
    for (int k = 0; k < 14; ++k) s += mu[k] * g0[k];
    dL_dw[ce] = -s;
  }
  if (!dL_dmeas) return;
  const Sim3T<D1> Pi = seed_dir(Si, -1), Pj = seed_dir(Sj, -1);
  double gz[7];
  for (int k = 0; k < 7; ++k) {
    const Sim3T<D1> Zd = seed_dir(Z, k);
    D1 gg[14];
    edge_gradient(Pi, Pj, Zd, g.w[e], L, gg);
    double s = 0.0;
    for (int m = 0; m < 14; ++m) s += mu[m] * gg[m].d[0];
    gz[k] = -s;
  }
  if (layout != PGO_GRAD_POSE8) {
    for (int k = 0; k < 7; ++k) dL_dmeas[(size_t)ce * 7 + k] = gz[k];
    return;
  }
  // pose8 layout: Z(p) with q = p_q / |p_q|; dzeta = M dp, dL/dp = M^T dL/dzeta:
  //   h = g_omega - t x g_upsilon; dL/dt = g_upsilon; dL/ds = (g_sigma - g_upsilon . t) / s
  //   dL/dq_v = 2 (w h + h x v), dL/dq_w = -2 h . v, then projected through the
  //   normalisation: dL/dp_q = (I - q q^T) dL/dq / |p_q|
  const double pn = g.zqn[e];
  const double* q = Z.q;
  const double* t = Z.t;
  const double gu[3] = {gz[3], gz[4], gz[5]};
  const double txgu[3] = {t[1] * gu[2] - t[2] * gu[1], t[2] * gu[0] - t[0] * gu[2], t[0] * gu[1] - t[1] * gu[0]};
  const double h[3] = {gz[0] - txgu[0], gz[1] - txgu[1], gz[2] - txgu[2]};
  const double hxv[3] = {h[1] * q[2] - h[2] * q[1], h[2] * q[0] - h[0] * q[2], h[0] * q[1] - h[1] * q[0]};
  double gq[4];
  for (int k = 0; k < 3; ++k) gq[k] = 2.0 * (q[3] * h[k] + hxv[k]);
  gq[3] = -2.0 * (h[0] * q[0] + h[1] * q[1] + h[2] * q[2]);
  const double qg = gq[0] * q[0] + gq[1] * q[1] + gq[2] * q[2] + gq[3] * q[3];
  double* o = dL_dmeas + (size_t)ce * 8;
  for (int k = 0; k < 4; ++k) o[k] = (gq[k] - qg * q[k]) / pn;
  for (int k = 0; k < 3; ++k) o[4 + k] = gu[k];
  o[7] = (gz[6] - (gu[0] * t[0] + gu[1] * t[1] + gu[2] * t[2])) / Z.s;
}

void launch_adj_hessian(const DevGraph& g, int with_grad, cudaStream_t s) {
  if (g.E == 0) return;
  k_adj_hessian<<<(g.E + 63) / 64, 64, 0, s>>>(g, with_grad);
}
void launch_adj_rhs(const DevGraph& g, const double* dL, int layout, cudaStream_t s) {
  k_adj_rhs<<<(g.N + 127) / 128, 128, 0, s>>>(g, dL, layout);
}
void launch_adj_edges(const DevGraph& g, const int* perm, double* dL_dmeas, double* dL_dw, int layout,
                      cudaStream_t s) {
  if (g.E == 0) return;
  k_adj_edges<<<(g.E + 63) / 64, 64, 0, s>>>(g, perm, dL_dmeas, dL_dw, layout);
}

}  // namespace pgo
