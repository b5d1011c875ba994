// Multigrid inside one thread block, for the batched form: the numeric
// set-up and the V(1,1) cycle of one segment of the hierarchy (one graph of
// the batch) with block barriers only.  The mathematics is that of
// k_amg_setup and of the V-cycle of k_pcg (smoothed aggregation with rigid
// Sim(3) coarse modes, Galerkin coarse operators, dense coarsest solve; see
// amg.cu); only the distribution of the work differs: every loop runs over
// the segment's own nodes and blocks, by the threads of one block.
//
// Every array the block reads here was written by the same block earlier in
// the same launch (the batch kernel assembles H itself), so block data is
// read with coherent loads, never through the non-coherent cache.
#pragma once
#include "amg.cuh"

namespace pgo {

__device__ __forceinline__ int seg_node(const AmgDev& A, int l, int k) {
  return __ldg(A.seg_off + l * (A.nseg + 1) + k);
}

// Block sum of one double (deterministic: fixed shuffle tree, fixed warp
// order); every thread receives it.
__device__ __forceinline__ double cta_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += sh[w];
  __syncthreads();
  return s;
}

// y = D^-1 A (sc x) for the rows [n0, n1) of level l, one warp per row;
// returns the thread's part of |y|^2.
template <class V>
__device__ double cta_power_step(const DevGraph& g, const AmgLevel& Lv, int l, int n0, int n1, int fixed, V lam,
                                 const V* x, V sc, V* y) {
  constexpr int BLK = AV<V>::BLK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double nrm = 0.0;
  for (int u = n0 + warp; u < n1; u += nw) {
    const bool live = !(l == 0 && u == fixed);
    V acc[7];
#pragma unroll
    for (int a = 0; a < 7; ++a) acc[a] = V(0);
    if (live) {
      if (l == 0) {
        const int k0 = __ldg(g.inc_ptr + u), ks = __ldg(g.inc_split + u), k1 = __ldg(g.inc_ptr + u + 1);
        for (int k = k0 - 1 + lane; k < k1; k += 32) {
          int w = u;
          const V* B;
          if (k < k0) {
            B = AV<V>::diag(g) + (size_t)u * BLK;
          } else {
            w = __ldg(g.inc_other + k);
            B = AV<V>::off(g) + (size_t)(__ldg(g.inc_code + k) >> 1) * BLK;
          }
          V xv[7];
#pragma unroll
          for (int c = 0; c < 7; ++c) xv[c] = sc * __ldcg(x + (size_t)w * VEC + c);
          const bool tr = k >= ks;
#pragma unroll
          for (int a = 0; a < 7; ++a) {
            V t = (k < k0) ? lam * xv[a] : V(0);
#pragma unroll
            for (int c = 0; c < 7; ++c) t += __ldcg(B + (tr ? c * 7 + a : a * 7 + c)) * xv[c];
            acc[a] += t;
          }
        }
      } else {
        const V* Ab = AV<V>::a(Lv);
        const int k1 = __ldg(Lv.a_ptr + u + 1);
        for (int k = __ldg(Lv.a_ptr + u) + lane; k < k1; k += 32) {
          const int w = __ldg(Lv.a_col + k);
          V xv[7];
#pragma unroll
          for (int c = 0; c < 7; ++c) xv[c] = sc * __ldcg(x + (size_t)w * VEC + c);
          const V* B = Ab + (size_t)k * BLK;
#pragma unroll
          for (int a = 0; a < 7; ++a) {
            V t = V(0);
#pragma unroll
            for (int c = 0; c < 7; ++c) t += __ldcg(B + a * 7 + c) * xv[c];
            acc[a] += t;
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 7; ++a)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (lane < 8) {
      V yv = V(0);
      if (lane < 7 && live) {
        const V* M = l == 0 ? AV<V>::minv(g) + (size_t)u * BLK : AV<V>::dinv(Lv) + (size_t)u * BLK;
#pragma unroll
        for (int c = 0; c < 7; ++c) yv += __ldcg(M + lane * 7 + c) * acc[c];
      }
      y[(size_t)u * VEC + lane] = yv;
      nrm += (double)yv * (double)yv;
    }
  }
  return nrm;
}

// Dense coarsest inverse of segment sg (Gauss-Jordan on the SPD matrix in
// shared memory `dense`, (7 n)^2 + 7 n doubles); writes the symmetrised
// inverse blocks, or zeros (coarse correction off) if a pivot is not positive.
template <class V>
__device__ void cta_coarsest_inverse(const AmgDev& A, int sg, double* dense) {
  constexpr int BLK = AV<V>::BLK;
  const AmgLevel& Lc = A.lv[A.L];
  const int c0 = seg_node(A, A.L, sg), nL = seg_node(A, A.L, sg + 1) - c0, n7 = 7 * nL;
  const V* Ab = AV<V>::a(Lc);
  V* Ci = AV<V>::cinv(A) + (size_t)(A.nseg > 1 ? sg * AMG_CMAX * AMG_CMAX : 0) * BLK;
  for (int t = threadIdx.x; t < n7 * n7; t += blockDim.x) dense[t] = 0.0;
  __syncthreads();
  for (int c = 0; c < nL; ++c)
    for (int k = __ldg(Lc.a_ptr + c0 + c); k < __ldg(Lc.a_ptr + c0 + c + 1); ++k) {
      const int d = __ldg(Lc.a_col + k) - c0;
      for (int ij = threadIdx.x; ij < 49; ij += blockDim.x) {
        const int i = ij / 7, j = ij - 7 * (ij / 7);
        dense[(7 * c + i) * n7 + 7 * d + j] = (double)__ldcg(Ab + (size_t)k * BLK + ij);
      }
    }
  __syncthreads();
  bool ok = true;
  double* colk = dense + (size_t)n7 * n7;
  for (int k = 0; k < n7; ++k) {
    const double piv = dense[k * n7 + k];
    if (!(piv > 0.0) || !isfinite(piv)) {   // uniform: every thread reads the same pivot
      ok = false;
      break;
    }
    const double ip = 1.0 / piv;
    for (int i = threadIdx.x; i < n7; i += blockDim.x) colk[i] = dense[i * n7 + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n7; j += blockDim.x) dense[k * n7 + j] = (j == k) ? ip : dense[k * n7 + j] * ip;
    __syncthreads();
    for (int t = threadIdx.x; t < n7 * n7; t += blockDim.x) {
      const int i = t / n7, j = t - n7 * i;
      if (i == k) continue;
      const double fik = colk[i];
      dense[t] = (j == k) ? -fik * ip : dense[t] - fik * dense[k * n7 + j];
    }
    __syncthreads();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nL * nL * 49; t += blockDim.x) {
    const int cd = t / 49, ij = t - 49 * cd;
    const int c = cd / nL, d = cd - nL * c;
    const int i = ij / 7, j = ij - 7 * (ij / 7);
    const int R = 7 * c + i, C = 7 * d + j;
    Ci[(size_t)cd * BLK + ij] = ok ? V(0.5 * (dense[R * n7 + C] + dense[C * n7 + R])) : V(0);
  }
  __syncthreads();
}

// Numeric set-up of segment sg at the current linearisation (H, lambda, the
// poses in buffer `cur`); D0^-1 (the graph's block-Jacobi blocks) must be
// current.  `dense`: shared memory for the coarsest inverse.
template <class V>
__device__ void cta_amg_setup(const DevGraph& g, const AmgDev& A, int sg, int fixed, double lam_d, int cur, double* sh,
                              double* dense) {
  constexpr int BLK = AV<V>::BLK;
  __shared__ V sacc[8][49];
  __shared__ double smat[8][52];   // D^-1 teams (51 doubles each)
  const V lam = V(lam_d);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int L = A.L;
  const int prec = sizeof(V) == sizeof(double) ? 0 : 1;
  const bool warm = __ldcg(A.warm + 2 * sg + prec) != 0;
  double* rho_s = A.rho + (size_t)sg * (AMG_MAXL + 1);
  const int slot = tid >> 6, t64 = tid & 63, nslots = nt >> 6;
  const int ti = t64 / 7, tj = t64 - 7 * (t64 / 7);
  const bool lane_on = t64 < 49;
  // tentative prolongation blocks of every level
  for (int l = 0; l < L; ++l) {
    const AmgLevel& Lv = A.lv[l];
    const int n1 = seg_node(A, l, sg + 1);
    for (int u = seg_node(A, l, sg) + tid; u < n1; u += nt) {
      if (__ldg(Lv.agg + u) < 0) continue;
      const Sim3T<double> Sr = load_pose(g, cur, __ldg(Lv.ref + u));
      const Sim3T<double> Sc = load_pose(g, cur, __ldg(Lv.refc + u));
      double T[7][7];
      adj7(compose(Sr, inverse(Sc)), T);
      V* out = AV<V>::t(Lv) + (size_t)u * BLK;
#pragma unroll
      for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int j = 0; j < 7; ++j) out[i * 7 + j] = V(T[i][j]);
    }
  }
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    const AmgLevel& Lv = A.lv[l];
    const AmgLevel& Ln = A.lv[l + 1];
    const int n0 = seg_node(A, l, sg), n1 = seg_node(A, l, sg + 1);
    const int c0 = seg_node(A, l + 1, sg), c1 = seg_node(A, l + 1, sg + 1);
    // ---- rho(D^-1 A) by power iteration (warm-started) ----
    double rho;
    {
      V* x0 = AV<V>::pw(A, 0);
      V* pv = AV<V>::pv(Lv);
      const double rho_prev = rho_s[l];
      double nrm = 0.0;
      for (int t = n0 * VEC + tid; t < n1 * VEC; t += nt) {
        const int u = t / VEC, k = t - u * VEC;
        const bool on = k < 7 && !(l == 0 && u == fixed);
        double v = 0.0;
        if (on) v = warm ? (double)__ldcg(pv + t) : 1.0 + 0.5 * sin(0.7 * (double)(7 * (u - n0) + k));
        x0[t] = V(v);
        nrm += v * v;
      }
      double nx = sqrt(cta_sum(nrm, sh));
      if (!(nx > 0.0) || !isfinite(nx)) nx = 0.0;
      const int its = warm ? AMG_POWER_ITS_WARM : AMG_POWER_ITS;
      for (int it = 0; it < its; ++it) {
        const V sc = V(nx > 0.0 ? 1.0 / nx : 0.0);
        const double ny2 = cta_power_step<V>(g, Lv, l, n0, n1, fixed, lam, AV<V>::pw(A, it & 1), sc,
                                             AV<V>::pw(A, (it + 1) & 1));
        nx = sqrt(cta_sum(ny2, sh));
      }
      rho = nx > 1e-30 ? nx : 1.0;
      if (warm && rho_prev > rho && isfinite(rho_prev)) rho = rho_prev;
      if (tid == 0) rho_s[l] = rho;
      const V* yl = AV<V>::pw(A, its & 1);
      for (int t = n0 * VEC + tid; t < n1 * VEC; t += nt) pv[t] = __ldcg(yl + t);
    }
    // ---- P = T_agg - 4/(3 rho) D^-1 (A T) ----
    {
      const V f = V(4.0 / (3.0 * rho));
      const V* Tb = AV<V>::t(Lv);
      V* Pb = AV<V>::p(Lv);
      const int b1 = __ldg(Lv.p_ptr + n1);
      for (int b0 = __ldg(Lv.p_ptr + n0); b0 < b1; b0 += nslots) {
        const int b = b0 + slot;
        const bool has = b < b1;
        int u = 0, c = 0;
        if (has && lane_on) {
          u = __ldg(Lv.p_row + b);
          c = __ldg(Lv.p_col + b);
          const int e0 = __ldg(Lv.r1_ptr + b), e1 = __ldg(Lv.r1_ptr + b + 1);
          sacc[slot][t64] = l == 0 ? recipe_ax<V, true, false>(g, nullptr, lam, Lv.r1, e0, e1, Tb, ti, tj)
                                   : recipe_ax<V, false, false>(g, AV<V>::a(Lv), lam, Lv.r1, e0, e1, Tb, ti, tj);
        }
        __syncthreads();
        if (has && lane_on) {
          const V* M = (l == 0 ? AV<V>::minv(g) : AV<V>::dinv(Lv)) + (size_t)u * BLK;
          V s = V(0);
#pragma unroll
          for (int k = 0; k < 7; ++k) s += __ldcg(M + ti * 7 + k) * sacc[slot][k * 7 + tj];
          const V tv = (c == __ldg(Lv.agg + u)) ? __ldcg(Tb + (size_t)u * BLK + ti * 7 + tj) : V(0);
          Pb[(size_t)b * BLK + ti * 7 + tj] = tv - f * s;
        }
        __syncthreads();
      }
    }
    // ---- AP = A P ----
    {
      const V* Pb = AV<V>::p(Lv);
      V* APb = AV<V>::ap(Lv);
      const int b1 = __ldg(Lv.ap_ptr + n1);
      if (lane_on)
        for (int b = __ldg(Lv.ap_ptr + n0) + slot; b < b1; b += nslots) {
          const int e0 = __ldg(Lv.r2_ptr + b), e1 = __ldg(Lv.r2_ptr + b + 1);
          APb[(size_t)b * BLK + ti * 7 + tj] =
              l == 0 ? recipe_ax<V, true, false>(g, nullptr, lam, Lv.r2, e0, e1, Pb, ti, tj)
                     : recipe_ax<V, false, false>(g, AV<V>::a(Lv), lam, Lv.r2, e0, e1, Pb, ti, tj);
        }
      __syncthreads();
    }
    // ---- A_next = P^T (A P), upper blocks; then the mirrored lower blocks ----
    {
      const V* Pb = AV<V>::p(Lv);
      const V* APb = AV<V>::ap(Lv);
      V* An = AV<V>::a(Ln);
      const int k0 = __ldg(Ln.a_ptr + c0), k1 = __ldg(Ln.a_ptr + c1);
      if (lane_on)
        for (int b = k0 + slot; b < k1; b += nslots) {
          const int e0 = __ldg(Lv.r3_ptr + b), e1 = __ldg(Lv.r3_ptr + b + 1);
          if (e0 == e1) continue;
          An[(size_t)b * BLK + ti * 7 + tj] = recipe_ptq<V>(Lv.r3, e0, e1, Pb, APb, ti, tj);
        }
      __syncthreads();
      for (int t = k0 * 49 + tid; t < k1 * 49; t += nt) {
        const int b = t / 49, ij = t - 49 * b;
        const int src = __ldg(Ln.a_src + b);
        if (src < 0) continue;
        const int i = ij / 7, j = ij - 7 * (ij / 7);
        An[(size_t)b * BLK + i * 7 + j] = __ldcg(An + (size_t)src * BLK + j * 7 + i);
      }
      __syncthreads();
    }
    if (l + 1 < L) {
      // the next level's D^-1: one 64-thread team per node
      const V* An = AV<V>::a(Ln);
      for (int cb = c0; cb < c1; cb += nslots) {
        const int c = cb + slot;
        const bool has = c < c1;
        inv7_spd_team<V, true>(An + (size_t)(has ? __ldg(Ln.a_ptr + c) : 0) * BLK,
                               AV<V>::dinv(Ln) + (size_t)(has ? c : 0) * BLK, has, smat[slot], t64);
      }
    }
  }
  cta_coarsest_inverse<V>(A, sg, dense);
  if (tid == 0) A.warm[2 * sg + prec] = 1;
  __syncthreads();
}

// y[k] for a lane-dependent k without dynamic register indexing.
template <class V>
__device__ __forceinline__ V cta_pick7(const V (&y)[7], int k) {
  V r = y[0];
#pragma unroll
  for (int i = 1; i < 7; ++i)
    if (k == i) r = y[i];
  return r;
}

// Group sum over the G lanes of a row; every lane receives the 7 sums.
template <class V, int G>
__device__ __forceinline__ void cta_group7(V (&y)[7], unsigned gm) {
#pragma unroll
  for (int a = 0; a < 7; ++a)
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) y[a] += __shfl_xor_sync(gm, y[a], o);
}

// y += B x (TR = false) or B^T x for a row-major 7x7 block.
template <class V, bool TR>
__device__ __forceinline__ void cta_bmv(const V* B, const V (&x)[7], V (&y)[7]) {
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    V row[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) row[c] = B[r * 7 + c];
    if (!TR) {
      V acc = V(0);
#pragma unroll
      for (int c = 0; c < 7; ++c) acc += row[c] * x[c];
      y[r] += acc;
    } else {
#pragma unroll
      for (int c = 0; c < 7; ++c) y[c] += row[c] * x[r];
    }
  }
}

template <class V>
__device__ __forceinline__ void ld7(const V* p, V (&x)[7]) {
#pragma unroll
  for (int c = 0; c < 7; ++c) x[c] = p[c];
}

// z = M r: one V(1,1) cycle of segment sg over its rows (G lanes per row in
// the block-sparse products).  r0: the residual (rows of the graph), s0 and
// x0 scratch vectors of the vertex level, z the output.
template <class V, int G>
__device__ void cta_vcycle(const DevGraph& g, const AmgDev& A, int sg, int fixed, V lam, const V* r0, V* s0, V* z) {
  constexpr int BLK = AV<V>::BLK;
  const int L = A.L;
  const double* rho_s = A.rho + (size_t)sg * (AMG_MAXL + 1);
  const int sl = threadIdx.x & (G - 1), rslot = threadIdx.x / G, nrs = blockDim.x / G;
  const unsigned gm = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (threadIdx.x & (32 - G)));
  V* x0 = AV<V>::vx(A.lv[0]);
  const int v0 = seg_node(A, 0, sg), v1 = seg_node(A, 0, sg + 1);
  // level-0 pre-smoothing
  {
    const V w0 = V(1.0 / rho_s[0]);
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      const size_t b = (size_t)v * VEC;
      V rv[7];
      ld7(r0 + b, rv);
      const V* M = AV<V>::minv(g) + (size_t)v * BLK;
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        V s = V(0);
#pragma unroll
        for (int c = 0; c < 7; ++c) s += M[a * 7 + c] * rv[c];
        x0[b + a] = v == fixed ? V(0) : w0 * s;
      }
      x0[b + 7] = V(0);
    }
    __syncthreads();
  }
  for (int l = 0; l < L; ++l) {
    const AmgLevel& Lv = A.lv[l];
    const AmgLevel& Ln = A.lv[l + 1];
    const int n0 = seg_node(A, l, sg), n1 = seg_node(A, l, sg + 1);
    // ---- s_l = r_l - A_l x_l ----
    {
      const V* xl = l == 0 ? x0 : AV<V>::vx(Lv);
      const V* rl = l == 0 ? r0 : AV<V>::vr(Lv);
      V* sv = l == 0 ? s0 : AV<V>::vs(Lv);
      for (int vb = n0; vb < n1; vb += nrs) {
        const int v = vb + rslot;
        const bool has = v < n1;
        V y[7];
#pragma unroll
        for (int a = 0; a < 7; ++a) y[a] = V(0);
        if (has) {
          if (l == 0) {
            const int k0 = g.inc_ptr[v], ks = g.inc_split[v], k1 = g.inc_ptr[v + 1];
            for (int k = k0 - 1 + sl; k < k1; k += G) {
              const bool dg = k < k0;
              const int u = dg ? v : g.inc_other[k];
              const V* B = dg ? AV<V>::diag(g) + (size_t)v * BLK : AV<V>::off(g) + (size_t)(g.inc_code[k] >> 1) * BLK;
              V xu[7];
              ld7(xl + (size_t)u * VEC, xu);
              if (dg) {
#pragma unroll
                for (int a = 0; a < 7; ++a) y[a] += lam * xu[a];
              }
              if (k < ks) cta_bmv<V, false>(B, xu, y);
              else cta_bmv<V, true>(B, xu, y);
            }
          } else {
            const V* Ab = AV<V>::a(Lv);
            for (int k = __ldg(Lv.a_ptr + v) + sl; k < __ldg(Lv.a_ptr + v + 1); k += G) {
              V xu[7];
              ld7(xl + (size_t)__ldg(Lv.a_col + k) * VEC, xu);
              cta_bmv<V, false>(Ab + (size_t)k * BLK, xu, y);
            }
          }
        }
        cta_group7<V, G>(y, gm);
        if (has)
          for (int a = sl; a < 8; a += G)
            sv[(size_t)v * VEC + a] = (a == 7 || (l == 0 && v == fixed)) ? V(0) : rl[(size_t)v * VEC + a] - cta_pick7(y, a);
      }
      __syncthreads();
    }
    // ---- r_{l+1} = P^T s_l and the next level's pre-smoothing ----
    {
      const V* sv = l == 0 ? s0 : AV<V>::vs(Lv);
      const V* Pb = AV<V>::p(Lv);
      V* rn = AV<V>::vr(Ln);
      V* xn = AV<V>::vx(Ln);
      const bool smooth = l + 1 < L;
      const V wn = smooth ? V(1.0 / rho_s[l + 1]) : V(0);
      const int c0 = seg_node(A, l + 1, sg), c1 = seg_node(A, l + 1, sg + 1);
      for (int cb = c0; cb < c1; cb += nrs) {
        const int c = cb + rslot;
        const bool has = c < c1;
        V y[7];
#pragma unroll
        for (int a = 0; a < 7; ++a) y[a] = V(0);
        if (has)
          for (int t = __ldg(Lv.pt_ptr + c) + sl; t < __ldg(Lv.pt_ptr + c + 1); t += G) {
            V su[7];
            ld7(sv + (size_t)__ldg(Lv.pt_row + t) * VEC, su);
            cta_bmv<V, true>(Pb + (size_t)__ldg(Lv.pt_blk + t) * BLK, su, y);
          }
        cta_group7<V, G>(y, gm);
        if (has)
          for (int a = sl; a < 8; a += G) {
            if (a == 7) {
              rn[(size_t)c * VEC + 7] = V(0);
              if (smooth) xn[(size_t)c * VEC + 7] = V(0);
              continue;
            }
            rn[(size_t)c * VEC + a] = cta_pick7(y, a);
            if (smooth) {
              const V* M = AV<V>::dinv(Ln) + (size_t)c * BLK;
              V s = V(0);
#pragma unroll
              for (int k = 0; k < 7; ++k) s += M[a * 7 + k] * y[k];
              xn[(size_t)c * VEC + a] = wn * s;
            }
          }
      }
      __syncthreads();
    }
  }
  // ---- coarsest: y_L = C^-1 r_L ----
  {
    const AmgLevel& Lc = A.lv[L];
    const int c0 = seg_node(A, L, sg), nL = seg_node(A, L, sg + 1) - c0;
    const V* Ci = AV<V>::cinv(A) + (size_t)(A.nseg > 1 ? sg * AMG_CMAX * AMG_CMAX : 0) * BLK;
    const V* rc = AV<V>::vr(Lc);
    V* yc = AV<V>::vy(Lc);
    for (int t = threadIdx.x; t < nL * 8; t += blockDim.x) {
      const int c = t >> 3, a = t & 7;
      V s = V(0);
      if (a < 7)
        for (int d = 0; d < nL; ++d) {
          const V* B = Ci + (size_t)(c * nL + d) * BLK + a * 7;
          const V* rv = rc + (size_t)(c0 + d) * VEC;
#pragma unroll
          for (int k = 0; k < 7; ++k) s += B[k] * rv[k];
        }
      yc[(size_t)(c0 + c) * VEC + a] = s;
    }
    __syncthreads();
  }
  // ---- way up: y_l = x_l + P y + w D^-1 (s_l - (A P) y) ----
  for (int l = L - 1; l >= 0; --l) {
    const AmgLevel& Lv = A.lv[l];
    const AmgLevel& Ln = A.lv[l + 1];
    const int n0 = seg_node(A, l, sg), n1 = seg_node(A, l, sg + 1);
    const V* yn = AV<V>::vy(Ln);
    const V* Pb = AV<V>::p(Lv);
    const V* APb = AV<V>::ap(Lv);
    const V* xl = l == 0 ? x0 : AV<V>::vx(Lv);
    const V* sv = l == 0 ? s0 : AV<V>::vs(Lv);
    V* out = l == 0 ? z : AV<V>::vy(Lv);
    const V wl = V(1.0 / rho_s[l]);
    for (int vb = n0; vb < n1; vb += nrs) {
      const int v = vb + rslot;
      const bool has = v < n1;
      V px[7], ax[7];
#pragma unroll
      for (int a = 0; a < 7; ++a) px[a] = ax[a] = V(0);
      if (has) {
        for (int k = __ldg(Lv.p_ptr + v) + sl; k < __ldg(Lv.p_ptr + v + 1); k += G) {
          V yu[7];
          ld7(yn + (size_t)__ldg(Lv.p_col + k) * VEC, yu);
          cta_bmv<V, false>(Pb + (size_t)k * BLK, yu, px);
        }
        for (int k = __ldg(Lv.ap_ptr + v) + sl; k < __ldg(Lv.ap_ptr + v + 1); k += G) {
          V yu[7];
          ld7(yn + (size_t)__ldg(Lv.ap_col + k) * VEC, yu);
          cta_bmv<V, false>(APb + (size_t)k * BLK, yu, ax);
        }
      }
      cta_group7<V, G>(px, gm);
      cta_group7<V, G>(ax, gm);
      if (has) {
        const size_t b = (size_t)v * VEC;
        const bool live = !(l == 0 && v == fixed);
        V d7[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) d7[c] = sv[b + c] - ax[c];
        const V* M = (l == 0 ? AV<V>::minv(g) : AV<V>::dinv(Lv)) + (size_t)v * BLK;
        for (int a = sl; a < 8; a += G) {
          if (a == 7) {
            out[b + 7] = V(0);
            continue;
          }
          V s = V(0);
#pragma unroll
          for (int k = 0; k < 7; ++k) s += M[a * 7 + k] * d7[k];
          out[b + a] = live ? xl[b + a] + cta_pick7(px, a) + wl * s : V(0);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace pgo
