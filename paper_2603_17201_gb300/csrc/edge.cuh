// Per-edge residual and exact Jacobians shared by the linearisation, the
// Jacobian export and the adjoint kernels.
#pragma once
#include "common.cuh"

namespace pgo {

// A = sign * J * Adj(R, t, s), Adj = [[R, 0, 0], [t^ R, s R, -t], [0, 0, 1]]
__device__ __forceinline__ void jac_times_adj(const double (&J)[7][7], const double* R, const double* t,
                                              double s, double sign, double (&A)[7][7]) {
  // t^ R
  double tR[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    tR[0 * 3 + c] = -t[2] * R[3 + c] + t[1] * R[6 + c];
    tR[1 * 3 + c] = t[2] * R[0 + c] - t[0] * R[6 + c];
    tR[2 * 3 + c] = -t[1] * R[0 + c] + t[0] * R[3 + c];
  }
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) v += J[a][k] * R[k * 3 + c] + J[a][3 + k] * tR[k * 3 + c];
      A[a][c] = sign * v;
      double u = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) u += J[a][3 + k] * R[k * 3 + c];
      A[a][3 + c] = sign * s * u;
    }
    double v6 = J[a][6] - (J[a][3] * t[0] + J[a][4] * t[1] + J[a][5] * t[2]);
    A[a][6] = sign * v6;
  }
}

// Whitening with Omega = L L^T (L packed lower-triangular, row-major):
// r <- L^T r, A <- L^T A.
__device__ __forceinline__ void whiten(const double* L, double (&r)[7], double (&Ai)[7][7], double (&Aj)[7][7]) {
  double l[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) l[k] = L[k];
  // (L^T v)[c] = sum_{a >= c} L[a][c] v[a];  L[a][c] at a*(a+1)/2 + c
  double rr[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    double s = 0.0;
#pragma unroll
    for (int a = c; a < 7; ++a) s += l[a * (a + 1) / 2 + c] * r[a];
    rr[c] = s;
  }
#pragma unroll
  for (int c = 0; c < 7; ++c) r[c] = rr[c];
#pragma unroll
  for (int col = 0; col < 7; ++col) {
    double ti[7], tj[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double si = 0.0, sj = 0.0;
#pragma unroll
      for (int a = c; a < 7; ++a) {
        si += l[a * (a + 1) / 2 + c] * Ai[a][col];
        sj += l[a * (a + 1) / 2 + c] * Aj[a][col];
      }
      ti[c] = si;
      tj[c] = sj;
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) { Ai[c][col] = ti[c]; Aj[c][col] = tj[c]; }
  }
}

// Residual, exact Jacobians (left perturbations of S_i and S_j) of one edge.
// Returns false if the pose data is non-finite.
__device__ __forceinline__ void edge_jacobians(const DevGraph& g, int cur, int e, double (&r)[7],
                                               double (&Ai)[7][7], double (&Aj)[7][7]) {
  const int i = g.ei[e], j = g.ej[e];
  Sim3T<double> Si = load_pose(g, cur, i), Sj = load_pose(g, cur, j), Z = load_meas(g, e);
  Sim3T<double> T = compose(Z, compose(Si, inverse(Sj)));
  qnormalize(T.q);
  // d log(exp(eps) T) / d eps = J_l^-1(r), one column per generator
  Sim3T<Dual<double, 7>> D = seed_left(T);
  Dual<double, 7> xi[7];
  sim3_log(D, xi);
  double J[7][7];
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    r[a] = xi[a].v;
#pragma unroll
    for (int k = 0; k < 7; ++k) J[a][k] = xi[a].d[k];
  }
  // r(exp(d_i) S_i, S_j) = log(exp(Adj(Z) d_i) T)  ->  A_i = J_l^-1 Adj(Z)
  // r(S_i, exp(d_j) S_j) = log(T exp(-d_j))        ->  A_j = -J_l^-1 Adj(T)
  double RZ[9], RT[9];
  qmat(Z.q, RZ);
  qmat(T.q, RT);
  jac_times_adj(J, RZ, Z.t, Z.s, 1.0, Ai);
  jac_times_adj(J, RT, T.t, T.s, -1.0, Aj);
  if (g.L) whiten(g.L + (size_t)e * 28, r, Ai, Aj);
}

}  // namespace pgo
