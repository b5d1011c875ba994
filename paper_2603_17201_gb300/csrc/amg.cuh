// Precision accessors of the multigrid hierarchy (shared by the setup and
// the V-cycle inside the PCG kernel).
#pragma once
#include "phases.cuh"

namespace pgo {

template <class V>
struct AV;
template <>
struct AV<double> {
  static constexpr int BLK = BLK64;
  static __device__ __forceinline__ const double* off(const DevGraph& g) { return g.off64; }
  static __device__ __forceinline__ const double* diag(const DevGraph& g) { return g.diag64; }
  static __device__ __forceinline__ const double* minv(const DevGraph& g) { return g.minv64; }
  static __device__ __forceinline__ double* a(const AmgLevel& L) { return L.a64; }
  static __device__ __forceinline__ double* dinv(const AmgLevel& L) { return L.dinv64; }
  static __device__ __forceinline__ double* t(const AmgLevel& L) { return L.t64; }
  static __device__ __forceinline__ double* p(const AmgLevel& L) { return L.p64; }
  static __device__ __forceinline__ double* ap(const AmgLevel& L) { return L.ap64; }
  static __device__ __forceinline__ double* q(const AmgLevel& L) { return L.q64; }
  static __device__ __forceinline__ double* w(const AmgDev& A) { return A.w64; }
  static __device__ __forceinline__ double* h(const AmgDev& A) { return A.h64; }
  static __device__ __forceinline__ double* cinv(const AmgDev& A) { return A.cinv64; }
  static __device__ __forceinline__ double* pw(const AmgDev& A, int k) { return A.pw64[k]; }
  static __device__ __forceinline__ double* vr(const AmgLevel& L) { return L.vr64; }
  static __device__ __forceinline__ double* vx(const AmgLevel& L) { return L.vx64; }
  static __device__ __forceinline__ double* vs(const AmgLevel& L) { return L.vs64; }
  static __device__ __forceinline__ double* vy(const AmgLevel& L) { return L.vy64; }
  static __device__ __forceinline__ double* pv(const AmgLevel& L) { return L.pv64; }
};
template <>
struct AV<float> {
  static constexpr int BLK = BLK32;
  static __device__ __forceinline__ const float* off(const DevGraph& g) { return g.off32; }
  static __device__ __forceinline__ const float* diag(const DevGraph& g) { return g.diag32; }
  static __device__ __forceinline__ const float* minv(const DevGraph& g) { return g.minv32; }
  static __device__ __forceinline__ float* a(const AmgLevel& L) { return L.a32; }
  static __device__ __forceinline__ float* dinv(const AmgLevel& L) { return L.dinv32; }
  static __device__ __forceinline__ float* t(const AmgLevel& L) { return L.t32; }
  static __device__ __forceinline__ float* p(const AmgLevel& L) { return L.p32; }
  static __device__ __forceinline__ float* ap(const AmgLevel& L) { return L.ap32; }
  static __device__ __forceinline__ float* q(const AmgLevel& L) { return L.q32; }
  static __device__ __forceinline__ float* w(const AmgDev& A) { return A.w32; }
  static __device__ __forceinline__ float* h(const AmgDev& A) { return A.h32; }
  static __device__ __forceinline__ float* cinv(const AmgDev& A) { return A.cinv32; }
  static __device__ __forceinline__ float* pw(const AmgDev& A, int k) { return A.pw32[k]; }
  static __device__ __forceinline__ float* vr(const AmgLevel& L) { return L.vr32; }
  static __device__ __forceinline__ float* vx(const AmgLevel& L) { return L.vx32; }
  static __device__ __forceinline__ float* vs(const AmgLevel& L) { return L.vs32; }
  static __device__ __forceinline__ float* vy(const AmgLevel& L) { return L.vy32; }
  static __device__ __forceinline__ float* pv(const AmgLevel& L) { return L.pv32; }
};

// A padded 7x7 block (16-byte aligned) into registers with vector loads:
// through the non-coherent cache (NC, data of an earlier launch) or from L2
// (data written by this launch).
template <bool NC>
__device__ __forceinline__ void ld_block(const float* src, float (&B)[49]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 v = NC ? __ldg(s4 + k) : __ldcg(s4 + k);
    B[4 * k] = v.x;
    B[4 * k + 1] = v.y;
    B[4 * k + 2] = v.z;
    B[4 * k + 3] = v.w;
  }
  B[48] = NC ? __ldg(src + 48) : __ldcg(src + 48);
}
template <bool NC>
__device__ __forceinline__ void ld_block(const double* src, double (&B)[49]) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const double2 v = NC ? __ldg(s2 + k) : __ldcg(s2 + k);
    B[2 * k] = v.x;
    B[2 * k + 1] = v.y;
  }
  B[48] = NC ? __ldg(src + 48) : __ldcg(src + 48);
}

// sum over the recipe entries e of (A_e X_e)[i][j].  A_e: level-0 block
// reference (L0: diagonal + lambda, or an off-diagonal block, maybe
// transposed) or a block of this level's operator; X_e = X + rec[e].y * BLK.
// NC: the level-0 blocks come from an earlier launch and may be read through
// the non-coherent cache; everything else is read from L2.  Entries go four
// at a time so that their loads overlap.
template <class V, bool L0, bool NC = true>
__device__ __forceinline__ V recipe_ax(const DevGraph& g, const V* Alev, V lam, const int2* rec, int e0, int e1,
                                       const V* X, int i, int j) {
  constexpr int BLK = AV<V>::BLK;
  V acc = V(0);
  auto arow = [&](int a, V (&r)[7]) {
    if (L0) {
      const V* p;
      bool tr = false;
      V add = V(0);
      if (a < 0) {
        p = AV<V>::diag(g) + (size_t)(-a - 1) * BLK;
        add = lam;
      } else {
        p = AV<V>::off(g) + (size_t)(a >> 1) * BLK;
        tr = (a & 1) != 0;
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const V* q = p + (tr ? k * 7 + i : i * 7 + k);
        r[k] = (NC ? __ldg(q) : __ldcg(q)) + (k == i ? add : V(0));
      }
    } else {
      const V* p = Alev + (size_t)a * BLK + i * 7;
#pragma unroll
      for (int k = 0; k < 7; ++k) r[k] = __ldcg(p + k);
    }
  };
  int e = e0;
  for (; e + 4 <= e1; e += 4) {
    int2 t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = __ldg(rec + e + q);
    V ar[4][7], xc[4][7];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      arow(t[q].x, ar[q]);
      const V* xp = X + (size_t)t[q].y * BLK + j;
#pragma unroll
      for (int k = 0; k < 7; ++k) xc[q][k] = __ldcg(xp + k * 7);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < 7; ++k) acc += ar[q][k] * xc[q][k];
  }
  for (; e < e1; ++e) {
    const int2 t = __ldg(rec + e);
    V ar[7];
    arow(t.x, ar);
    const V* xp = X + (size_t)t.y * BLK + j;
#pragma unroll
    for (int k = 0; k < 7; ++k) acc += ar[k] * __ldcg(xp + k * 7);
  }
  return acc;
}

// sum over the entries e of (P_e^T Q_e)[i][j], both written by this launch.
template <class V>
__device__ __forceinline__ V recipe_ptq(const int2* rec, int e0, int e1, const V* P, const V* Q, int i, int j) {
  constexpr int BLK = AV<V>::BLK;
  V acc = V(0);
  int e = e0;
  for (; e + 4 <= e1; e += 4) {
    int2 t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = __ldg(rec + e + q);
    V pc[4][7], qc[4][7];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const V* pp = P + (size_t)t[q].x * BLK + i;
      const V* qp = Q + (size_t)t[q].y * BLK + j;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        pc[q][k] = __ldcg(pp + k * 7);
        qc[q][k] = __ldcg(qp + k * 7);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < 7; ++k) acc += pc[q][k] * qc[q][k];
  }
  for (; e < e1; ++e) {
    const int2 t = __ldg(rec + e);
    const V* pp = P + (size_t)t.x * BLK + i;
    const V* qp = Q + (size_t)t.y * BLK + j;
#pragma unroll
    for (int k = 0; k < 7; ++k) acc += __ldcg(pp + k * 7) * __ldcg(qp + k * 7);
  }
  return acc;
}

// Adj(S) in [omega, upsilon, sigma] order: [[R, 0, 0], [t^ R, s R, -t], [0, 0, 1]].
__device__ __forceinline__ void adj7(const Sim3T<double>& S, double (&A)[7][7]) {
  double R[9];
  qmat(S.q, R);
  const double* t = S.t;
#pragma unroll
  for (int i = 0; i < 7; ++i)
#pragma unroll
    for (int j = 0; j < 7; ++j) A[i][j] = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    A[0][c] = R[c];
    A[1][c] = R[3 + c];
    A[2][c] = R[6 + c];
    A[3][c] = -t[2] * R[3 + c] + t[1] * R[6 + c];
    A[4][c] = t[2] * R[0 + c] - t[0] * R[6 + c];
    A[5][c] = -t[1] * R[0 + c] + t[0] * R[3 + c];
    A[3][3 + c] = S.s * R[c];
    A[4][3 + c] = S.s * R[3 + c];
    A[5][3 + c] = S.s * R[6 + c];
  }
  A[3][6] = -t[0];
  A[4][6] = -t[1];
  A[5][6] = -t[2];
  A[6][6] = 1.0;
}

// Inverse of the SPD 7x7 block `src` into `dst` by a team of 64 threads of a
// block (thread t < 49 owns entry (t / 7, t % 7)): Gauss-Jordan without
// pivoting in the team's shared scratch M (50 doubles; M[49] flags a
// non-positive pivot), then the symmetrised result.  Every thread of the
// block must call it together (it synchronises the block: the caller's loop
// needs a block-uniform trip count); `has` false skips the team's arithmetic.
// A non-positive pivot falls back to the inverse of the diagonal.
template <class V, bool CG>
__device__ __forceinline__ void inv7_spd_team(const V* src, V* dst, bool has, double* M, int t) {
  // M: 51 doubles of shared scratch (the block, a bad-pivot flag, the reciprocal)
  const int i = t / 7, j = t - 7 * (t / 7);
  const bool on = has && t < 49;
  if (on) M[t] = (double)(CG ? __ldcg(src + t) : src[t]);
  if (t == 0) M[49] = 0.0;
  __syncthreads();
  for (int k = 0; k < 7; ++k) {
    double mkj = 0.0, fik = 0.0;
    if (on) {
      mkj = M[k * 7 + j];
      fik = M[i * 7 + k];
    }
    // the pivot's reciprocal once per team (an FP64 division per lane would
    // cost more than the whole elimination at the FP64 rate)
    if (has && t == 0) {
      const double p = M[k * 7 + k];
      if (!(p > 0.0)) M[49] = 1.0;
      M[50] = 1.0 / p;
    }
    __syncthreads();
    if (on) {
      const double ip = M[50];
      if (i == k) M[t] = (j == k) ? ip : mkj * ip;
      else M[t] = (j == k) ? -fik * ip : M[t] - fik * mkj * ip;
    }
    __syncthreads();
  }
  if (on) {
    double v = 0.5 * (M[t] + M[j * 7 + i]);
    if (M[49] != 0.0) {
      const double d = (double)(CG ? __ldcg(src + i * 8) : src[i * 8]);
      v = (i == j && d > 0.0) ? 1.0 / d : 0.0;
    }
    dst[t] = V(v);
  }
  __syncthreads();
}

}  // namespace pgo
