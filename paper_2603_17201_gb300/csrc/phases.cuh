// Per-edge and per-vertex steps of one LM iteration, shared by the
// single-graph kernels (one graph over the whole GPU) and the batched
// persistent kernel (one graph per thread block).
#pragma once
#include "edge.cuh"

namespace pgo {

// Residual cache of the mixed-precision LM loop: per pose buffer and edge,
// the FP64 residual r = log(T) (7 doubles and a pad) and T = Z S_i S_j^-1
// as 8 floats (q, then t and s).  The cost kernel writes the entry of the
// poses it evaluates; the fused linearisation of the same poses reads it
// instead of evaluating the log map again.
constexpr int RC_STRIDE = 12;   // doubles per edge (96 bytes)
__device__ __forceinline__ double* rcache_at(const DevGraph& g, int buf, int e) {
  return g.rcache + ((size_t)buf * g.E + e) * RC_STRIDE;
}

__device__ __forceinline__ void rcache_store(double* c, const double (&r)[7], const Sim3T<double>& T) {
  double2* c2 = reinterpret_cast<double2*>(c);
  c2[0] = make_double2(r[0], r[1]);
  c2[1] = make_double2(r[2], r[3]);
  c2[2] = make_double2(r[4], r[5]);
  c2[3] = make_double2(r[6], 0.0);
  float4* c4 = reinterpret_cast<float4*>(c + 8);
  c4[0] = make_float4((float)T.q[0], (float)T.q[1], (float)T.q[2], (float)T.q[3]);
  c4[1] = make_float4((float)T.t[0], (float)T.t[1], (float)T.t[2], (float)T.s);
}


// packed upper-triangular index (a <= c) of a symmetric 7x7 block
__device__ __forceinline__ int upk(int a, int c) { return a * 7 - (a * (a - 1)) / 2 + (c - a); }

static __device__ __constant__ unsigned char c_up_a[28] = {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 5, 5, 6};
static __device__ __constant__ unsigned char c_up_c[28] = {0, 1, 2, 3, 4, 5, 6, 1, 2, 3, 4, 5, 6, 2, 3, 4, 5, 6, 3, 4, 5, 6, 4, 5, 6, 5, 6, 6};

// Linearisation of one edge: residual and exact Jacobians (poses in buffer `cur`), the
// off-diagonal (i, j) block w A_i^T A_j (FP64, and FP32 in mixed mode) and
// the two edge-side contributions [upper(w A^T A), w A^T r].
// Mixed precision: FP64 residual, FP32 Jacobians and H products (the
// off-diagonal block also kept promoted in FP64 for the refinement residual),
// the gradient sum A^T r in FP64 from the FP32 Jacobians.
__device__ __forceinline__ void linearize_edge_mixed(const DevGraph& g, int cur, int e) {
  double r[7];
  float Ai[7][7], Aj[7][7];
  edge_jacobians_mixed(g, cur, e, r, Ai, Aj);
  const float w = (float)g.w[e];
  double* off = g.off64 + (size_t)e * BLK64;
  float* off32 = g.off32 + (size_t)e * BLK32;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 7; ++k) s += Ai[k][a] * Aj[k][c];
      s *= w;
      off32[a * 7 + c] = s;
      off[a * 7 + c] = (double)s;
    }
  }
  const double wd = g.w[e];
  double* ci = g.contrib + (size_t)e * 2 * CONTRIB;
  double* cj = ci + CONTRIB;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = a; c < 7; ++c) {
      float si = 0.f, sj = 0.f;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        si += Ai[k][a] * Ai[k][c];
        sj += Aj[k][a] * Aj[k][c];
      }
      ci[upk(a, c)] = (double)(w * si);
      cj[upk(a, c)] = (double)(w * sj);
    }
    double gi = 0.0, gj = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      gi += (double)Ai[k][a] * r[k];
      gj += (double)Aj[k][a] * r[k];
    }
    ci[28 + a] = wd * gi;
    cj[28 + a] = wd * gj;
  }
}

__device__ __forceinline__ void linearize_edge(const DevGraph& g, int cur, int e, int mixed) {
  if (mixed) {
    linearize_edge_mixed(g, cur, e);
    return;
  }
  double r[7], Ai[7][7], Aj[7][7];
  edge_jacobians(g, cur, e, r, Ai, Aj);
  const double w = g.w[e];
  double* off = g.off64 + (size_t)e * BLK64;
  float* off32 = mixed ? g.off32 + (size_t)e * BLK32 : nullptr;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 7; ++k) s += Ai[k][a] * Aj[k][c];
      s *= w;
      off[a * 7 + c] = s;
      if (mixed) off32[a * 7 + c] = (float)s;
    }
  }
  double* ci = g.contrib + (size_t)e * 2 * CONTRIB;
  double* cj = ci + CONTRIB;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = a; c < 7; ++c) {
      double si = 0.0, sj = 0.0;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        si += Ai[k][a] * Ai[k][c];
        sj += Aj[k][a] * Aj[k][c];
      }
      ci[upk(a, c)] = w * si;
      cj[upk(a, c)] = w * sj;
    }
    double gi = 0.0, gj = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      gi += Ai[k][a] * r[k];
      gj += Aj[k][a] * r[k];
    }
    ci[28 + a] = w * gi;
    cj[28 + a] = w * gj;
  }
}

// ---- mixed precision: fused linearisation and assembly --------------------
// A <- L^T A in FP32 (L the packed lower-triangular factor of Omega).
__device__ __forceinline__ void whiten_f32(const double* L, float (&A)[7][7]) {
  float l[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) l[k] = (float)__ldg(L + k);
#pragma unroll
  for (int col = 0; col < 7; ++col) {
    float t[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int a = c; a < 7; ++a) acc += l[a * (a + 1) / 2 + c] * A[a][col];
      t[c] = acc;
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) A[c][col] = t[c];
  }
}

// One side's contribution: upper(w A^T A) into hcol (entry u at hcol[33 u])
// and w A^T r into bcol (entry a at bcol[33 a]), both from FP32 products;
// the sums over the vertex's edges run in FP32 for H and in FP64 for b.
__device__ __forceinline__ void side_contribution(const float (&A)[7][7], const float (&r)[7], float w,
                                                  float* hcol, double* bcol) {
#pragma unroll
  for (int a = 0; a < 7; ++a) {
#pragma unroll
    for (int c = a; c < 7; ++c) {
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < 7; ++k) sacc += A[k][a] * A[k][c];
      hcol[33 * upk(a, c)] = w * sacc;
    }
    float gacc = 0.f;
#pragma unroll
    for (int k = 0; k < 7; ++k) gacc += A[k][a] * r[k];
    bcol[33 * a] = (double)(w * gacc);
  }
}

// Incidence entry `code` (edge code >> 1 seen from side code & 1; side 0:
// the vertex is i) of the fused mixed linearisation at pose buffer `cur`:
// the side's FP32 Jacobian from the cached FP64 residual (A_i = J_l^-1(r)
// Adj(Z), A_j = -J_l^-1(r) Adj(T), the exact Jacobians of the log residual
// for left perturbations), its contribution into the reduction table, and on
// the i side the off-diagonal block w A_i^T Omega A_j (FP32, and promoted to
// FP64 for the refinement residual).
__device__ __forceinline__ void lin_entry_mixed(const DevGraph& g, int cur, int code, float* hcol, double* bcol) {
  const int e = code >> 1;
  const bool iside = (code & 1) == 0;
  const double* c = rcache_at(g, cur, e);
  double r[7];
  {
    const double2* c2 = reinterpret_cast<const double2*>(c);
    const double2 a0 = c2[0], a1 = c2[1], a2 = c2[2], a3 = c2[3];
    r[0] = a0.x; r[1] = a0.y; r[2] = a1.x; r[3] = a1.y; r[4] = a2.x; r[5] = a2.y; r[6] = a3.x;
  }
  const float4 tq = reinterpret_cast<const float4*>(c + 8)[0];
  const float4 tts = reinterpret_cast<const float4*>(c + 8)[1];
  float J[7][7];
  left_jacobian_inv_f32(r, J);
  float rf[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) rf[k] = (float)r[k];
  const double* L = g.L ? g.L + (size_t)e * 28 : nullptr;
  if (L) {   // whitened residual L^T r
    float rr[7];
#pragma unroll
    for (int cc = 0; cc < 7; ++cc) {
      float s2 = 0.f;
#pragma unroll
      for (int a = cc; a < 7; ++a) s2 += (float)__ldg(L + a * (a + 1) / 2 + cc) * rf[a];
      rr[cc] = s2;
    }
#pragma unroll
    for (int cc = 0; cc < 7; ++cc) rf[cc] = rr[cc];
  }
  const float w = (float)g.w[e];
  float A[7][7];   // this side's Jacobian
  {
    const float q[4] = {tq.x, tq.y, tq.z, tq.w};
    float R[9];
    qmat(q, R);
    const float t[3] = {tts.x, tts.y, tts.z};
    jac_times_adj<float>(J, R, t, tts.w, -1.f, A);   // A_j
  }
  if (L) whiten_f32(L, A);
  if (iside) {
    float Ai[7][7];
    {
      const D4 zq = g.zq[e], zt = g.zt[e];
      const float q[4] = {(float)zq.x, (float)zq.y, (float)zq.z, (float)zq.w};
      float R[9];
      qmat(q, R);
      const float t[3] = {(float)zt.x, (float)zt.y, (float)zt.z};
      jac_times_adj<float>(J, R, t, (float)zt.w, 1.f, Ai);
    }
    if (L) whiten_f32(L, Ai);
    double* off = g.off64 + (size_t)e * BLK64;
    float* off32 = g.off32 + (size_t)e * BLK32;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) {
        float sacc = 0.f;
#pragma unroll
        for (int k = 0; k < 7; ++k) sacc += Ai[k][a] * A[k][cc];
        sacc *= w;
        off32[a * 7 + cc] = sacc;
        off[a * 7 + cc] = (double)sacc;
      }
    }
#pragma unroll
    for (int a = 0; a < 7; ++a)
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) A[a][cc] = Ai[a][cc];
  }
  side_contribution(A, rf, w, hcol, bcol);
}

// Assembly for one vertex, lane `lane` of 8: gather the incident contributions in
// incidence order (deterministic), write H_vv (full symmetric) and b_v, and
// fold max diag, |b|_inf and |b|^2 (free vertices only) into the arguments.
__device__ __forceinline__ void assemble_vertex(const DevGraph& g, int v, int lane, int mixed, int fixed,
                                                double& mdiag, double& mgrad, double& b2) {
  double acc[5] = {0, 0, 0, 0, 0};
  const int k0 = g.inc_ptr[v], k1 = g.inc_ptr[v + 1];
  for (int k = k0; k < k1; ++k) {
    const int code = g.inc_code[k];
    const double* src = g.contrib + (size_t)(code >> 1) * 2 * CONTRIB + (code & 1) * CONTRIB;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const int u = lane + 8 * m;
      if (u < CONTRIB) acc[m] += src[u];
    }
  }
  const bool free_v = (v != fixed);
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const int u = lane + 8 * m;
    if (u < 28) {
      const int a = c_up_a[u], c = c_up_c[u];
      g.diag64[(size_t)v * BLK64 + a * 7 + c] = acc[m];
      g.diag64[(size_t)v * BLK64 + c * 7 + a] = acc[m];
      if (mixed) {
        g.diag32[(size_t)v * BLK32 + a * 7 + c] = (float)acc[m];
        g.diag32[(size_t)v * BLK32 + c * 7 + a] = (float)acc[m];
      }
      if (a == c && free_v) mdiag = fmax(mdiag, acc[m]);
    } else if (u < 35) {
      g.b[(size_t)v * VEC + (u - 28)] = acc[m];
      if (free_v) {
        mgrad = fmax(mgrad, fabs(acc[m]));
        b2 += acc[m] * acc[m];
      }
    } else if (u == 35) {
      g.b[(size_t)v * VEC + 7] = 0.0;
    }
  }
}

// Cost of one edge at the poses in buffer `buf` (FP64); with `store`, also
// its residual cache entry.
__device__ __forceinline__ double edge_cost(const DevGraph& g, int buf, int e, bool store = false) {
  const int i = g.ei[e], j = g.ej[e];
  Sim3T<double> Si = load_pose(g, buf, i), Sj = load_pose(g, buf, j), Z = load_meas(g, e);
  Sim3T<double> T = compose(Z, compose(Si, inverse(Sj)));
  qnormalize(T.q);
  double r[7];
  sim3_log(T, r);
  if (store) rcache_store(rcache_at(g, buf, e), r, T);
  double c = 0.0;
  if (g.L) {
    const double* L = g.L + (size_t)e * 28;
#pragma unroll
    for (int cc = 0; cc < 7; ++cc) {
      double s = 0.0;
#pragma unroll
      for (int a = cc; a < 7; ++a) s += L[a * (a + 1) / 2 + cc] * r[a];
      c += s * s;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 7; ++k) c += r[k] * r[k];
  }
  return g.w[e] * c;
}

// Candidate pose of one vertex: exp(delta_v) S_v into buffer cur^1 (the fixed
// vertex is copied); returns this vertex's term of delta^T (lambda delta - b).
__device__ __forceinline__ double update_vertex(const DevGraph& g, int cur, int v, int fixed, const double* dxv,
                                                double lam) {
  Sim3T<double> S = load_pose(g, cur, v);
  if (v == fixed) {
    store_pose(g, cur ^ 1, v, S);
    return 0.0;
  }
  double d[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) d[k] = dxv[k];
  Sim3T<double> E = sim3_exp(d);
  Sim3T<double> P = compose(E, S);
  qnormalize(P.q);
  store_pose(g, cur ^ 1, v, P);
  const double* bv = g.b + (size_t)v * VEC;
  double pr = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) pr += d[k] * (lam * d[k] - bv[k]);
  return pr;
}

// Block-Jacobi preconditioner for one vertex: M = (H_vv + lambda I)^-1 by a 7x7 Cholesky in FP64,
// stored as V (the inverse of the damped diagonal if the block is not
// positive definite); M = 0 on the fixed vertex (its unknowns stay zero).
template <class V>
__device__ __forceinline__ void precond_vertex(const DevGraph& g, int v, int fixed, double lam, V* M) {
  if (v == fixed) {
#pragma unroll
    for (int k = 0; k < 49; ++k) M[k] = V(0);
    return;
  }
  double A[7][7];
  const double* D = g.diag64 + (size_t)v * BLK64;
#pragma unroll
  for (int a = 0; a < 7; ++a)
#pragma unroll
    for (int c = 0; c < 7; ++c) A[a][c] = D[a * 7 + c] + (a == c ? lam : 0.0);
  // Cholesky A = L L^T with the reciprocals of the pivots (7 divisions: on
  // GB300 an FP64 divide costs many FP64 issue slots)
  bool ok = true;
  double rd[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    double d = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    ok = ok && (d > 0.0);
    d = sqrt(fmax(d, 1e-300));
    A[j][j] = d;
    rd[j] = 1.0 / d;
#pragma unroll
    for (int i = j + 1; i < 7; ++i) {
      double s = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
      A[i][j] = s * rd[j];
    }
  }
  if (!ok) {
#pragma unroll
    for (int a = 0; a < 7; ++a)
#pragma unroll
      for (int c = 0; c < 7; ++c) M[a * 7 + c] = (a == c) ? V(1.0 / fmax(D[a * 8] + lam, 1e-300)) : V(0);
    return;
  }
  // Li = L^-1 (lower triangular), then M = Li^T Li (symmetric: upper half)
  double Li[7][7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      if (a < c) {
        Li[a][c] = 0.0;
        continue;
      }
      double s = (a == c) ? 1.0 : 0.0;
#pragma unroll
      for (int k = c; k < a; ++k) s -= A[a][k] * Li[k][c];
      Li[a][c] = s * rd[a];
    }
  }
#pragma unroll
  for (int a = 0; a < 7; ++a)
#pragma unroll
    for (int c = a; c < 7; ++c) {
      double s = 0.0;
#pragma unroll
      for (int k = c; k < 7; ++k) s += Li[k][a] * Li[k][c];
      M[a * 7 + c] = V(s);
      M[c * 7 + a] = V(s);
    }
}

}  // namespace pgo
