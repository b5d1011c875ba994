// Per-edge residual and exact Jacobians shared by the linearisation, the
// Jacobian export and the adjoint kernels.
#pragma once
#include "common.cuh"

namespace pgo {

// A = sign * J * Adj(R, t, s), Adj = [[R, 0, 0], [t^ R, s R, -t], [0, 0, 1]]
template <class T>
__device__ __forceinline__ void jac_times_adj(const T (&J)[7][7], const T* R, const T* t, T s, T sign,
                                              T (&A)[7][7]) {
  // t^ R
  T tR[9];
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
      T v = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) v += J[a][k] * R[k * 3 + c] + J[a][3 + k] * tR[k * 3 + c];
      A[a][c] = sign * v;
      T u = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) u += J[a][3 + k] * R[k * 3 + c];
      A[a][3 + c] = sign * s * u;
    }
    T v6 = J[a][6] - (J[a][3] * t[0] + J[a][4] * t[1] + J[a][5] * t[2]);
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
  jac_times_adj<double>(J, RZ, Z.t, Z.s, 1.0, Ai);
  jac_times_adj<double>(J, RT, T.t, T.s, -1.0, Aj);
  if (g.L) whiten(g.L + (size_t)e * 28, r, Ai, Aj);
}

// ---- mixed precision: FP64 residual, FP32 Jacobians ----------------------
// J_l^-1(xi) in FP32: the left Jacobian J_l = sum_n ad^n / (n+1)! (an entire
// series, Horner form with as many terms as |ad| needs for FP32), inverted by
// Gauss-Jordan with partial pivoting.
__device__ __forceinline__ void left_jacobian_inv_f32(const double* xi, float (&Ji)[7][7]) {
  float ad[7][7];
#pragma unroll
  for (int i = 0; i < 7; ++i)
#pragma unroll
    for (int j = 0; j < 7; ++j) ad[i][j] = 0.f;
  const float w0 = (float)xi[0], w1 = (float)xi[1], w2 = (float)xi[2];
  const float u0 = (float)xi[3], u1 = (float)xi[4], u2 = (float)xi[5], sg = (float)xi[6];
  // ad(xi) = [[w^, 0, 0], [u^, w^ + sigma I, -u], [0, 0, 0]]
  const float wh[3][3] = {{0.f, -w2, w1}, {w2, 0.f, -w0}, {-w1, w0, 0.f}};
  const float uh[3][3] = {{0.f, -u2, u1}, {u2, 0.f, -u0}, {-u1, u0, 0.f}};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ad[i][j] = wh[i][j];
      ad[3 + i][j] = uh[i][j];
      ad[3 + i][3 + j] = wh[i][j] + (i == j ? sg : 0.f);
    }
  ad[3][6] = -u0;
  ad[4][6] = -u1;
  ad[5][6] = -u2;
  // terms: |ad|^n / (n+1)! below 1e-9 (|ad| by its largest row sum)
  float nrm = 0.f;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    float rs = 0.f;
#pragma unroll
    for (int j = 0; j < 7; ++j) rs += fabsf(ad[i][j]);
    nrm = fmaxf(nrm, rs);
  }
  int N = 1;
  {
    double term = nrm / 2.0;   // |ad|^n / (n+1)! for n = 1
    while (term > 1e-9 && N < 40) {
      ++N;
      term *= nrm * c_rcp[N];   // 1 / (N + 1)
    }
  }
  // Horner: J = I + ad/2 (I + ad/3 (I + ... (I + ad/(N+1))))
  float M[7][7];
#pragma unroll
  for (int i = 0; i < 7; ++i)
#pragma unroll
    for (int j = 0; j < 7; ++j) M[i][j] = i == j ? 1.f : 0.f;
  for (int n = N; n >= 1; --n) {
    const float f = 1.f / (float)(n + 1);
    float P[7][7];
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 7; ++k) acc += ad[i][k] * M[k][j];
        P[i][j] = (i == j ? 1.f : 0.f) + f * acc;
      }
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int j = 0; j < 7; ++j) M[i][j] = P[i][j];
  }
  // inverse by Gauss-Jordan on [M | I] without pivoting: J_l is block
  // lower-triangular in [omega, upsilon, sigma] ([[J_w, 0, 0], [X, Y, z],
  // [0, 0, 1]]), so the pivots are those of the SO(3) block J_w and of Y,
  // whose eigenvalues (e^l - 1)/l (l = +-i theta, sigma +- i theta, sigma)
  // stay away from zero for |theta| < 2 pi
#pragma unroll
  for (int i = 0; i < 7; ++i)
#pragma unroll
    for (int j = 0; j < 7; ++j) Ji[i][j] = i == j ? 1.f : 0.f;
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const float ip = 1.f / M[c][c];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      M[c][j] *= ip;
      Ji[c][j] *= ip;
    }
#pragma unroll
    for (int r2 = 0; r2 < 7; ++r2) {
      if (r2 == c) continue;
      const float f = M[r2][c];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        M[r2][j] -= f * M[c][j];
        Ji[r2][j] -= f * Ji[c][j];
      }
    }
  }
}

// Residual in FP64 (plain log map) and the Jacobians in FP32.
__device__ __forceinline__ void edge_jacobians_mixed(const DevGraph& g, int cur, int e, double (&r)[7],
                                                     float (&Ai)[7][7], float (&Aj)[7][7]) {
  const int i = g.ei[e], j = g.ej[e];
  Sim3T<double> Si = load_pose(g, cur, i), Sj = load_pose(g, cur, j), Z = load_meas(g, e);
  Sim3T<double> T = compose(Z, compose(Si, inverse(Sj)));
  qnormalize(T.q);
  sim3_log(T, r);
  float J[7][7];
  left_jacobian_inv_f32(r, J);
  double RZd[9], RTd[9];
  qmat(Z.q, RZd);
  qmat(T.q, RTd);
  float RZ[9], RT[9], tZ[3], tT[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    RZ[k] = (float)RZd[k];
    RT[k] = (float)RTd[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tZ[k] = (float)Z.t[k];
    tT[k] = (float)T.t[k];
  }
  jac_times_adj<float>(J, RZ, tZ, (float)Z.s, 1.f, Ai);
  jac_times_adj<float>(J, RT, tT, (float)T.s, -1.f, Aj);
  if (g.L) {
    // whitening: r in FP64, the Jacobians in FP32
    const double* L = g.L + (size_t)e * 28;
    double rr[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double s2 = 0.0;
#pragma unroll
      for (int a = c; a < 7; ++a) s2 += L[a * (a + 1) / 2 + c] * r[a];
      rr[c] = s2;
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) r[c] = rr[c];
    for (int col = 0; col < 7; ++col) {
      float ti[7], tj[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        float si = 0.f, sj = 0.f;
#pragma unroll
        for (int a = c; a < 7; ++a) {
          const float l = (float)L[a * (a + 1) / 2 + c];
          si += l * Ai[a][col];
          sj += l * Aj[a][col];
        }
        ti[c] = si;
        tj[c] = sj;
      }
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        Ai[c][col] = ti[c];
        Aj[c][col] = tj[c];
      }
    }
  }
}

}  // namespace pgo
