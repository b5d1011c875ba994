// Damped linear solve (H + lambda I) delta = rhs by preconditioned conjugate
// gradients over the block-sparse normal matrix, with the block-Jacobi
// preconditioner or one V(1,1) cycle of the multigrid hierarchy of amg.cu.
// (The paper's Sec. IV-F keeps an exact LDL^T on the CPU; here the solve
// stays on the GPU, with no host round trip per iteration.)
//
// k_pcg is a persistent cooperative kernel: one launch runs every PCG
// iteration of one linear solve.  One block per SM owns a contiguous range of
// block rows and stages their diagonal, preconditioner and off-diagonal
// blocks in shared memory once per launch.  In the products, G lanes serve a
// block row: each lane takes whole 7x7 blocks of the row, then the G lanes
// sum their partial 7-vectors by shuffles (on GB300 an FP64 warp instruction
// holds the SM sub-partition's FP64 pipe for ~64 cycles whatever the number
// of active lanes, so lanes are kept busy with whole blocks).  Each stored
// off-diagonal block (i, j) serves row i as H_ij and row j as H_ij^T; each
// vertex lists its side-0 entries first, so the two products never diverge
// within a warp; p = z + beta p_prev is formed on the fly.
// Per iteration: SpMV + local p.q -> grid barrier -> alpha, x/r update and
// the preconditioner (block-Jacobi: z = M r locally; multigrid: the cycle's
// phases, each behind a grid barrier) + local r.z, r.r -> grid barrier ->
// beta and the stopping test.  Every block reduces the per-block partials
// itself in the same fixed order, so all blocks take identical decisions and
// the result is deterministic.
//
// The grid barrier is a monotone arrival counter (release add, acquire poll)
// with a bounded spin: on timeout the kernel records PGO_ERR_CUDA in the
// state and every block returns.
#include "amg.cuh"
#include "gridsync.cuh"
#include "phases.cuh"

namespace pgo {

template <class V>
struct Bufs;

template <>
struct Bufs<double> {
  static __device__ __forceinline__ const double* off(const DevGraph& g) { return g.off64; }
  static __device__ __forceinline__ const double* diag(const DevGraph& g) { return g.diag64; }
  static __device__ __forceinline__ double* minv(const DevGraph& g) { return g.minv64; }
  static __device__ __forceinline__ double* x(const DevGraph& g) { return g.x64; }
  static __device__ __forceinline__ double* r(const DevGraph& g) { return g.r64; }
  static __device__ __forceinline__ double* z(const DevGraph& g) { return g.z64; }
  static __device__ __forceinline__ double* p(const DevGraph& g, int k) { return g.p64[k]; }
  static __device__ __forceinline__ double* q(const DevGraph& g) { return g.q64; }
  static constexpr int BLK = BLK64;
};
template <>
struct Bufs<float> {
  static __device__ __forceinline__ const float* off(const DevGraph& g) { return g.off32; }
  static __device__ __forceinline__ const float* diag(const DevGraph& g) { return g.diag32; }
  static __device__ __forceinline__ float* minv(const DevGraph& g) { return g.minv32; }
  static __device__ __forceinline__ float* x(const DevGraph& g) { return g.x32; }
  static __device__ __forceinline__ float* r(const DevGraph& g) { return g.r32; }
  static __device__ __forceinline__ float* z(const DevGraph& g) { return g.z32; }
  static __device__ __forceinline__ float* p(const DevGraph& g, int k) { return g.p32[k]; }
  static __device__ __forceinline__ float* q(const DevGraph& g) { return g.q32; }
  static constexpr int BLK = BLK32;
};

// ---- block-Jacobi preconditioner M_v = (H_vv + lambda I)^-1 ----------
template <class V>
__global__ void __launch_bounds__(32) k_precond(DevGraph g) {
  const SolverState* st = g.st;
  if (st->done) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.N) return;
  precond_vertex<V>(g, v, g.fixed, st->lambda, Bufs<V>::minv(g) + (size_t)v * Bufs<V>::BLK);
}

// 7x7 block (first 49 entries of a 16-byte aligned padded block), read-only.
__device__ __forceinline__ void load_block(const double* src, double (&B)[49]) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const double2 v = __ldg(s2 + k);
    B[2 * k] = v.x;
    B[2 * k + 1] = v.y;
  }
  B[48] = __ldg(src + 48);
}
__device__ __forceinline__ void load_block(const float* src, float (&B)[49]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 v = __ldg(s4 + k);
    B[4 * k] = v.x;
    B[4 * k + 1] = v.y;
    B[4 * k + 2] = v.z;
    B[4 * k + 3] = v.w;
  }
  B[48] = __ldg(src + 48);
}

// p_u = z_u + beta p_prev_u (vectors written by other blocks: L2 loads).
__device__ __forceinline__ void load_p(const double* z, const double* pp, size_t base, double beta, double (&p)[8]) {
  const double2* z2 = reinterpret_cast<const double2*>(z + base);
  const double2* p2 = reinterpret_cast<const double2*>(pp + base);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldcg(z2 + k), b = __ldcg(p2 + k);
    p[2 * k] = a.x + beta * b.x;
    p[2 * k + 1] = a.y + beta * b.y;
  }
}
__device__ __forceinline__ void load_p(const float* z, const float* pp, size_t base, float beta, float (&p)[8]) {
  const float4* z4 = reinterpret_cast<const float4*>(z + base);
  const float4* p4 = reinterpret_cast<const float4*>(pp + base);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float4 a = __ldcg(z4 + k), b = __ldcg(p4 + k);
    p[4 * k] = a.x + beta * b.x;
    p[4 * k + 1] = a.y + beta * b.y;
    p[4 * k + 2] = a.z + beta * b.z;
    p[4 * k + 3] = a.w + beta * b.w;
  }
}

template <class S>
struct PcgShared {
  S red[32 * 2];
  S tot[2];
};

// Sum of per-block partials (K values each) in fixed order, by every block
// (warp 0 reduces, the block reads the result from shared memory).
template <class S, int K>
__device__ __forceinline__ void reduce_partials(const S* partial, S (&out)[K], S* sh) {
  if (threadIdx.x < 32) {
    S acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = S(0);
    for (int b = threadIdx.x; b < gridDim.x; b += 32) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += __ldcg(partial + b * K + k);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; ++k) sh[k] = acc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = sh[k];
  __syncthreads();
}

// Block sum of per-thread values (K each); thread 0 writes the block partial.
template <class S, int K>
__device__ __forceinline__ void write_partial(S (&v)[K], S* partial, S* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      S s = S(0);
      for (int w = 0; w < nw; ++w) s += sh[w * K + k];
      partial[blockIdx.x * K + k] = s;
    }
  }
  __syncthreads();
}

struct PcgArgs {
  int from_residual;   // 0: rhs = -b; 1: rhs = res64 (refinement)
  int inner;           // tolerance: 0 -> pcg_tol, 1 -> refine_tol
  int rows_per_block;  // contiguous block-row range per block
  int cap_entries;     // off-diagonal blocks staged in shared memory per block
  int amg;             // 1: multigrid V-cycle preconditioner, 0: block-Jacobi
};

// Plain (generic-address) 7x7 block loads: the block may sit in shared or
// global memory; it is read-only for the whole kernel.
__device__ __forceinline__ void load_block_any(const double* src, double (&B)[49]) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const double2 v = s2[k];
    B[2 * k] = v.x;
    B[2 * k + 1] = v.y;
  }
  B[48] = src[48];
}
__device__ __forceinline__ void load_block_any(const float* src, float (&B)[49]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 v = s4[k];
    B[4 * k] = v.x;
    B[4 * k + 1] = v.y;
    B[4 * k + 2] = v.z;
    B[4 * k + 3] = v.w;
  }
  B[48] = src[48];
}

// y += B p (TR = false) or y += B^T p (TR = true), row-major 7x7 block.
template <bool TR>
__device__ __forceinline__ void bmv(const double* Bp, const double (&p)[8], double (&y)[7]) {
  // FP64: one block row at a time keeps register pressure low
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    double row[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) row[c] = Bp[r * 7 + c];
    if (!TR) {
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 7; ++c) acc += row[c] * p[c];
      y[r] += acc;
    } else {
#pragma unroll
      for (int c = 0; c < 7; ++c) y[c] += row[c] * p[r];
    }
  }
}
template <bool TR>
__device__ __forceinline__ void bmv(const float* Bp, const float (&p)[8], float (&y)[7]) {
  float B[49];
  load_block_any(Bp, B);
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 7; ++c) acc += (TR ? B[c * 7 + a] : B[a * 7 + c]) * p[c];
    y[a] += acc;
  }
}

// Copy n 16-byte chunks of padded blocks into shared memory.
template <class V>
__device__ __forceinline__ void stage_blocks(V* dst, const V* src_base, const int* codes, int nblk,
                                             bool by_code) {
  constexpr int CH = Bufs<V>::BLK * (int)sizeof(V) / 16;   // 16-byte chunks per block
  for (int t = threadIdx.x; t < nblk * CH; t += blockDim.x) {
    const int l = t / CH, c = t - l * CH;
    const size_t srcb = by_code ? (size_t)(codes[l] >> 1) : (size_t)l;
    const float4 v = __ldg(reinterpret_cast<const float4*>(src_base + srcb * Bufs<V>::BLK) + c);
    reinterpret_cast<float4*>(dst + (size_t)l * Bufs<V>::BLK)[c] = v;
  }
}

// ---- multigrid V-cycle (inside the persistent PCG kernel) -----------------
// Level-0 context: the block's rows and its staged operator.
template <class V>
struct L0Ctx {
  const V* s_diag;
  const V* s_minv;
  const V* s_off;
  const int* s_code;
  const int* s_other;
  const V* off;
  int nst, e0, row0, row1;
  V lam;
};

// 8-vector from L2 (vectors written by other blocks of this launch).
__device__ __forceinline__ void ld8(const double* p, double (&x)[8]) {
  const double2* p2 = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldcg(p2 + k);
    x[2 * k] = a.x;
    x[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void ld8(const float* p, float (&x)[8]) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float4 a = __ldcg(p4 + k);
    x[4 * k] = a.x;
    x[4 * k + 1] = a.y;
    x[4 * k + 2] = a.z;
    x[4 * k + 3] = a.w;
  }
}

template <class V, int G>
__device__ __forceinline__ void group_reduce7(V (&y)[7], unsigned gmG) {
#pragma unroll
  for (int a2 = 0; a2 < 7; ++a2)
#pragma unroll
    for (int o2 = G / 2; o2 > 0; o2 >>= 1) y[a2] += __shfl_xor_sync(gmG, y[a2], o2);
}

// y = (H + lambda I) x for level-0 row v over the row's G lanes; ld(u, xu)
// loads the 8-vector of vertex u.  With a warp per row (G = 32) each lane
// takes one entry of the whole row in one pass, the transposed side by a
// register select.  With fewer lanes the lanes take the row's side-0
// entries (the diagonal first), then its side-1 entries (stored transposed):
// two loops, so that the lanes of a warp never diverge between the two
// products (walking both sides in lockstep measured slower: its register
// pressure spills).  An absent row (has == false) has no entries.  After the
// call every lane of the group holds the row's 7 outputs.
template <class V, int G, class LD>
__device__ __forceinline__ void row_prod0(const DevGraph& g, const L0Ctx<V>& c, int v, bool has, int sl,
                                          unsigned gmG, LD ld, V (&y)[7]) {
  constexpr int BLK = AV<V>::BLK;
  const int k0 = has ? __ldg(g.inc_ptr + v) : 0, k1 = has ? __ldg(g.inc_ptr + v + 1) : -1;
  const int ks = has ? __ldg(g.inc_split + v) : -1;
#pragma unroll
  for (int a2 = 0; a2 < 7; ++a2) y[a2] = V(0);
  auto entry = [&](int k, int& u, const V*& Bp) {
    const int l = k - c.e0;
    if (l < c.nst) {
      u = c.s_other[l];
      Bp = c.s_off + (size_t)l * BLK;
    } else {
      u = __ldg(g.inc_other + k);
      Bp = c.off + (size_t)(__ldg(g.inc_code + k) >> 1) * BLK;
    }
  };
  const V* Bd = c.s_diag + (size_t)(has ? v - c.row0 : 0) * BLK;
  if (G >= 32) {
    // a warp per row: one pass over all of the row's entries, each lane one
    // entry, the transposed side by a register select (one round trip to L2
    // for a row of up to 32 entries)
    for (int k = k0 - 1 + sl; k < k1; k += G) {
      int u = v;
      const V* Bp = Bd;
      if (k >= k0) entry(k, u, Bp);
      V xa[8];
      ld(u, xa);
      V B[49];
      load_block_any(Bp, B);
      const bool tr = k >= ks;
#pragma unroll
      for (int a2 = 0; a2 < 7; ++a2) {
        V acc = k < k0 ? c.lam * xa[a2] : V(0);
#pragma unroll
        for (int c2 = 0; c2 < 7; ++c2) acc += (tr ? B[c2 * 7 + a2] : B[a2 * 7 + c2]) * xa[c2];
        y[a2] += acc;
      }
    }
    group_reduce7<V, G>(y, gmG);
    return;
  }
  for (int k = k0 - 1 + sl; k < ks; k += G) {
    int u = v;
    const V* Bp = Bd;
    if (k >= k0) entry(k, u, Bp);
    V xa[8];
    ld(u, xa);
    if (k < k0) {
#pragma unroll
      for (int a2 = 0; a2 < 7; ++a2) y[a2] += c.lam * xa[a2];
    }
    bmv<false>(Bp, xa, y);
  }
  for (int k = ks + sl; k < k1; k += G) {
    int u;
    const V* Bp;
    entry(k, u, Bp);
    V xb[8];
    ld(u, xb);
    bmv<true>(Bp, xb, y);
  }
  group_reduce7<V, G>(y, gmG);
}

// y[k] for a lane-dependent k without dynamic register indexing.
template <class V>
__device__ __forceinline__ V pick7(const V (&y)[7], int k) {
  V r = y[0];
#pragma unroll
  for (int i = 1; i < 7; ++i)
    if (k == i) r = y[i];
  return r;
}

// out[a] = sum_c M[a][c] v[c] for the components a this lane stores.
template <class V>
__device__ __forceinline__ V dmul_row(const V* M, int a, const V (&v)[7]) {
  V acc = V(0);
#pragma unroll
  for (int c = 0; c < 7; ++c) acc += M[a * 7 + c] * v[c];
  return acc;
}

// Rows [r0, r1) of a coarse level, one warp per row (coarse rows have tens
// of entries and few rows per block: a full warp keeps the latency of each
// phase to about one entry per lane).
constexpr int GC = 32;

// The V(1,1) cycle after the caller has stored the level-0 pre-smoothed
// iterate x0 = w0 D0^-1 r for its rows.  With the smoothing weight w_l and
// Q_l = (I - w_l D_l^-1 A_l) P_l (the prolongation with the post-smoothing
// folded in; its transpose is the restriction with the pre-smoothing), the
// cycle on level l is
//   x_l = w_l D_l^-1 r_l,  f_l = x_l + w_l D_l^-1 (r_l - A_l x_l),
//   r_{l+1} = Q_l^T r_l,   z_l = f_l + Q_l z_{l+1},
// and on level d = L - 1, next to the coarsest, z_d = f_d + W r_d with the
// dense W = Q_d C^-1 Q_d^T of the set-up.  This is the cycle of pre-smoothing,
// residual, restriction, coarse solve, prolongation and post-smoothing
// written as one linear map per level: f_l and r_{l+1} both depend on r_l
// alone, so each level costs one grid barrier on the way down and one on the
// way up.  Writes z for the block's rows and adds r.z to rz_loc.  Returns
// false on a barrier timeout.
template <class V, class S, int G>
__device__ bool vcycle_rest(const DevGraph& g, const AmgDev& A, const L0Ctx<V>& c0, const V* r0v, V* s0, V* z,
                            S& rz_loc, unsigned* counter, int* abort_flag, unsigned& target) {
  constexpr int BLK = AV<V>::BLK;
  const int sl = threadIdx.x & (G - 1);
  const int sslot = threadIdx.x / G;
  const int nsslots = blockDim.x / G;
  const unsigned gmG = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (threadIdx.x & (32 - G)));
  const int cl = threadIdx.x & 31;          // coarse levels: lane in the row's warp
  const int cslot = threadIdx.x >> 5;
  const int ncslots = blockDim.x >> 5;
  const unsigned full = 0xffffffffu;
  const int d = A.L - 1;
  auto range = [&](int n, int& r0, int& r1) {
    const int rpb = (n + gridDim.x - 1) / gridDim.x;
    r0 = min((int)blockIdx.x * rpb, n);
    r1 = min(r0 + rpb, n);
  };
  // level-0 rows of the block: f_0 (kept in s0 for the way up) or, when level
  // 0 is the dense level, z itself
  auto level0 = [&](bool dense) {
    const AmgLevel& L0 = A.lv[0];
    const V* x0 = AV<V>::vx(L0);
    const V w0 = V(1.0 / A.rho[0]);
    const V* Wb = AV<V>::w(A);
    const int nd = L0.n;
    for (int v0 = c0.row0; v0 < c0.row1; v0 += nsslots) {
      const int v = v0 + sslot;
      const bool has = v < c0.row1;
      const size_t base = (size_t)(has ? v : c0.row0) * VEC;
      V rv[8], xv[8];   // the row's own vectors, in flight with the products
      ld8(r0v + base, rv);
      ld8(x0 + base, xv);
      V y[7], wr[7];
      row_prod0<V, G>(g, c0, v, has, sl, gmG, [&](int u, V (&xu)[8]) { ld8(x0 + (size_t)u * VEC, xu); }, y);
#pragma unroll
      for (int a2 = 0; a2 < 7; ++a2) wr[a2] = V(0);
      if (dense && has) {
        for (int u = sl; u < nd; u += G) {
          V pu[8];
          ld8(r0v + (size_t)u * VEC, pu);
          bmv<false>(Wb + ((size_t)v * nd + u) * BLK, pu, wr);
        }
      }
      if (dense) group_reduce7<V, G>(wr, gmG);
      if (has) {
        V d7[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) d7[c] = rv[c] - y[c];
        const V* M = c0.s_minv + (size_t)(v - c0.row0) * BLK;
        const bool live = v != g.fixed;
        V* out = dense ? z : s0;
#pragma unroll
        for (int a2 = 0; a2 < 8; ++a2) {
          if (a2 % G != sl) continue;
          if (a2 == 7) {
            out[base + 7] = V(0);
            continue;
          }
          const V o = live ? xv[a2] + w0 * dmul_row(M, a2, d7) + wr[a2] : V(0);
          out[base + a2] = o;
          if (dense) rz_loc += S(o) * S(rv[a2]);
        }
      }
    }
  };
  // rows of level l >= 1: f_l = x_l + w_l D_l^-1 (r_l - A_l x_l) (+ W r_l on the dense level)
  auto level_f = [&](int l, bool dense, V* out) {
    const AmgLevel& Lv = A.lv[l];
    const V* Ab = AV<V>::a(Lv);
    const V* xl = AV<V>::vx(Lv);
    const V* rl = AV<V>::vr(Lv);
    const V* Dl = AV<V>::dinv(Lv);
    const V* Wb = AV<V>::w(A);
    const V wl = V(1.0 / A.rho[l]);
    const int nd = Lv.n;
    int r0, r1;
    range(Lv.n, r0, r1);
    for (int v0 = r0; v0 < r1; v0 += ncslots) {
      const int v = v0 + cslot;
      const bool has = v < r1;
      const int k0 = has ? __ldg(Lv.a_ptr + v) : 0, k1 = has ? __ldg(Lv.a_ptr + v + 1) : 0;
      const int w1 = dense && has ? nd : 0;
      const size_t base = (size_t)(has ? v : 0) * VEC;
      // the row's own vectors and D^-1 row, in flight with the products
      V rv[8], drow[7];
      ld8(rl + base, rv);
      const V xo = cl < 7 ? __ldcg(xl + base + cl) : V(0);
#pragma unroll
      for (int c = 0; c < 7; ++c) drow[c] = cl < 7 ? Dl[(size_t)(has ? v : 0) * BLK + cl * 7 + c] : V(0);
      V y[7], wr[7];
#pragma unroll
      for (int a2 = 0; a2 < 7; ++a2) y[a2] = wr[a2] = V(0);
      // the A row and (on the dense level) the W row in lockstep
      for (int k = k0 + cl, u = cl; k < k1 || u < w1; k += GC, u += GC) {
        const bool ha = k < k1, hw = u < w1;
        V pa[8], pw[8];
        if (ha) ld8(xl + (size_t)__ldg(Lv.a_col + k) * VEC, pa);
        if (hw) ld8(rl + (size_t)u * VEC, pw);
        if (ha) bmv<false>(Ab + (size_t)k * BLK, pa, y);
        if (hw) bmv<false>(Wb + ((size_t)v * nd + u) * BLK, pw, wr);
      }
      group_reduce7<V, GC>(y, full);
      if (dense) group_reduce7<V, GC>(wr, full);
      if (has && cl < 8) {
        if (cl == 7) {
          out[base + 7] = V(0);
        } else {
          V acc = V(0);
#pragma unroll
          for (int c = 0; c < 7; ++c) acc += drow[c] * (rv[c] - y[c]);
          out[base + cl] = xo + wl * acc + pick7(wr, cl);
        }
      }
    }
  };
  // ---- way down: f_l and r_{l+1} = Q_l^T r_l, x_{l+1} = w D^-1 r_{l+1} ----
  for (int l = 0; l < d; ++l) {
    const AmgLevel& Lv = A.lv[l];
    const AmgLevel& Ln = A.lv[l + 1];
    if (!grid_sync(counter, abort_flag, target)) return false;
    if (l == 0) level0(false);
    else level_f(l, false, AV<V>::vs(Lv));
    const V* rl = l == 0 ? r0v : AV<V>::vr(Lv);
    const V* Qb = AV<V>::q(Lv);
    V* rn = AV<V>::vr(Ln);
    V* xn = AV<V>::vx(Ln);
    const V wn = V(1.0 / A.rho[l + 1]);
    const V* Dn = AV<V>::dinv(Ln);
    int r0, r1;
    range(Ln.n, r0, r1);
    for (int ci = r0; ci < r1; ci += ncslots) {
      const int c = ci + cslot;
      const bool has = c < r1;
      const int t0 = has ? __ldg(Lv.apt_ptr + c) : 0, t1 = has ? __ldg(Lv.apt_ptr + c + 1) : 0;
      V drow[7];   // D^-1 row of the coarse node, in flight with the products
#pragma unroll
      for (int k = 0; k < 7; ++k) drow[k] = cl < 7 ? Dn[(size_t)(has ? c : 0) * BLK + cl * 7 + k] : V(0);
      V y[7];
#pragma unroll
      for (int a2 = 0; a2 < 7; ++a2) y[a2] = V(0);
      // two entries per lane and step, both loads issued first
      for (int t = t0 + cl; t < t1; t += 2 * GC) {
        const int t2 = t + GC;
        const bool h2 = t2 < t1;
        V pa[8], pb[8];
        ld8(rl + (size_t)__ldg(Lv.apt_row + t) * VEC, pa);
        if (h2) ld8(rl + (size_t)__ldg(Lv.apt_row + t2) * VEC, pb);
        bmv<true>(Qb + (size_t)__ldg(Lv.apt_blk + t) * BLK, pa, y);
        if (h2) bmv<true>(Qb + (size_t)__ldg(Lv.apt_blk + t2) * BLK, pb, y);
      }
      group_reduce7<V, GC>(y, full);
      if (has && cl < 8) {
        const size_t base = (size_t)c * VEC;
        if (cl == 7) {
          rn[base + 7] = V(0);
          xn[base + 7] = V(0);
        } else {
          V acc = V(0);
#pragma unroll
          for (int k = 0; k < 7; ++k) acc += drow[k] * y[k];
          rn[base + cl] = pick7(y, cl);
          xn[base + cl] = wn * acc;
        }
      }
    }
  }
  // ---- level d: f_d + W r_d ----
  if (!grid_sync(counter, abort_flag, target)) return false;
  if (d == 0) {
    level0(true);
    return true;
  }
  level_f(d, true, AV<V>::vy(A.lv[d]));
  // ---- way up: z_l = f_l + Q_l z_{l+1} ----
  for (int l = d - 1; l >= 0; --l) {
    const AmgLevel& Lv = A.lv[l];
    const AmgLevel& Ln = A.lv[l + 1];
    if (!grid_sync(counter, abort_flag, target)) return false;
    const V* yn = AV<V>::vy(Ln);
    const V* Qb = AV<V>::q(Lv);
    if (l == 0) {
      for (int v0 = c0.row0; v0 < c0.row1; v0 += nsslots) {
        const int v = v0 + sslot;
        const bool has = v < c0.row1;
        int k0 = 0, k1 = 0;
        if (has) {
          k0 = __ldg(Lv.ap_ptr + v);
          k1 = __ldg(Lv.ap_ptr + v + 1);
        }
        // lane sl stores component sl (G >= 8): its f and r, in flight with the products
        const size_t base = (size_t)(has ? v : c0.row0) * VEC;
        const V fo = sl < 7 ? __ldcg(s0 + base + sl) : V(0);
        const V ro = sl < 7 ? __ldcg(r0v + base + sl) : V(0);
        V qy[7];
#pragma unroll
        for (int a2 = 0; a2 < 7; ++a2) qy[a2] = V(0);
        for (int k = k0 + sl; k < k1; k += G) {
          V pu[8];
          ld8(yn + (size_t)__ldg(Lv.ap_col + k) * VEC, pu);
          bmv<false>(Qb + (size_t)k * BLK, pu, qy);
        }
        group_reduce7<V, G>(qy, gmG);
        if (has && sl < 8) {
          if (sl == 7) {
            z[base + 7] = V(0);
          } else {
            const V o = v != g.fixed ? fo + pick7(qy, sl) : V(0);
            z[base + sl] = o;
            rz_loc += S(o) * S(ro);
          }
        }
      }
    } else {
      int r0, r1;
      range(Lv.n, r0, r1);
      const V* fl = AV<V>::vs(Lv);
      V* out = AV<V>::vy(Lv);
      for (int v0 = r0; v0 < r1; v0 += ncslots) {
        const int v = v0 + cslot;
        const bool has = v < r1;
        int k0 = 0, k1 = 0;
        if (has) {
          k0 = __ldg(Lv.ap_ptr + v);
          k1 = __ldg(Lv.ap_ptr + v + 1);
        }
        const size_t base = (size_t)(has ? v : 0) * VEC;
        const V fo = cl < 7 ? __ldcg(fl + base + cl) : V(0);   // in flight with the products
        V qy[7];
#pragma unroll
        for (int a2 = 0; a2 < 7; ++a2) qy[a2] = V(0);
        for (int k = k0 + cl; k < k1; k += GC) {
          V pu[8];
          ld8(yn + (size_t)__ldg(Lv.ap_col + k) * VEC, pu);
          bmv<false>(Qb + (size_t)k * BLK, pu, qy);
        }
        group_reduce7<V, GC>(qy, full);
        if (has && cl < 8) out[base + cl] = cl == 7 ? V(0) : fo + pick7(qy, cl);
      }
    }
  }
  return true;
}

// One PCG solve.  V: storage and arithmetic type of blocks and vectors;
// S: type of the dot products and scalars (double for the FP64 solve, float
// for the inner solve of the mixed mode); G: lanes per block row in the SpMV
// (each lane takes whole 7x7 blocks of the row, then the G lanes reduce).
//
// Shared memory (dynamic): the block's diagonal blocks and preconditioner
// blocks, then its first cap_entries off-diagonal blocks (in incidence
// order) with their neighbour indices, staged once at launch so that each
// iteration reads the operator from shared memory; entries beyond the
// capacity are read from global memory.
template <class V, class S, int G>
__global__ void __launch_bounds__(sizeof(V) == 8 ? 256 : 512) k_pcg(DevGraph g, PcgArgs a) {
  SolverState* st = g.st;
  if (st->done || (a.from_residual && st->ref_done)) return;
  __shared__ PcgShared<S> sh;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BLK = Bufs<V>::BLK;
  const DevOptions* o = g.opt;
  unsigned* counter = &st->ticket[T_PCG_SPMV];
  int* abort_flag = reinterpret_cast<int*>(&st->ticket[T_PCG_UPDATE]);
  S* partial = reinterpret_cast<S*>(g.partial);
  unsigned target = 0;
  // test hook: this block never arrives, so the others reach the wait limit
  if ((int)blockIdx.x == o->test_absent_block) return;

  const int sl = threadIdx.x & (G - 1);        // SpMV: lane within the row's group of G
  const int sslot = threadIdx.x / G;
  const int nsslots = blockDim.x / G;
  const int lane8 = threadIdx.x & 7;           // update: component owned by this lane (7 = idle)
  const int slot = threadIdx.x >> 3;           // row slot within the block
  const int nslots = blockDim.x >> 3;
  const int row0 = blockIdx.x * a.rows_per_block;
  const int row1 = min(row0 + a.rows_per_block, g.N);
  const int nrows = row1 - row0;
  const bool act = lane8 < 7;
  const int c7 = act ? lane8 : 0;
  const unsigned gm8 = 0xffu << (threadIdx.x & 24);   // the 8 lanes of a row (update)
  const unsigned gmG = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (threadIdx.x & (32 - G)));

  const V* off = Bufs<V>::off(g);
  V* x = Bufs<V>::x(g);
  V* r = Bufs<V>::r(g);
  V* z = Bufs<V>::z(g);
  V* q = Bufs<V>::q(g);
  const V lam = V(st->lambda);
  // inner solve of the mixed refinement: relative to its own right-hand side
  // (the FP64 residual res), only as tight as the outer target needs,
  // |res - H dx| <= pcg_tol |b|, and never looser than refine_tol demands
  double tol = o->pcg_tol;
  if (a.inner) {
    tol = o->refine_tol;
    if (a.from_residual && st->ref_rr > 0.0 && st->bnorm2 > 0.0)
      tol = fmax(tol, o->pcg_tol * sqrt(st->bnorm2 / st->ref_rr));
    tol = fmin(tol, 0.5);
  }
  const int maxit = o->pcg_max_iters;

  // ---- stage the block's operator in shared memory ----
  V* s_diag = reinterpret_cast<V*>(smem_raw);
  V* s_minv = s_diag + (size_t)a.rows_per_block * BLK;
  V* s_off = s_minv + (size_t)a.rows_per_block * BLK;
  int* s_code = reinterpret_cast<int*>(s_off + (size_t)a.cap_entries * BLK);
  int* s_other = s_code + a.cap_entries;
  const int e0 = __ldg(g.inc_ptr + row0);
  const int nst = min(__ldg(g.inc_ptr + row1) - e0, a.cap_entries);
  for (int l = threadIdx.x; l < nst; l += blockDim.x) {
    s_code[l] = __ldg(g.inc_code + e0 + l);
    s_other[l] = __ldg(g.inc_other + e0 + l);
  }
  stage_blocks<V>(s_diag, Bufs<V>::diag(g) + (size_t)row0 * BLK, nullptr, nrows, false);
  stage_blocks<V>(s_minv, Bufs<V>::minv(g) + (size_t)row0 * BLK, nullptr, nrows, false);
  __syncthreads();
  stage_blocks<V>(s_off, off, s_code, nst, true);
  __syncthreads();

  L0Ctx<V> c0;
  c0.s_diag = s_diag;
  c0.s_minv = s_minv;
  c0.s_off = s_off;
  c0.s_code = s_code;
  c0.s_other = s_other;
  c0.off = off;
  c0.nst = nst;
  c0.e0 = e0;
  c0.row0 = row0;
  c0.row1 = row1;
  c0.lam = lam;
  // multigrid: the level-0 pre-smoothed iterate goes to x0, z is the V-cycle
  // result; block-Jacobi: z = M r directly
  __shared__ AmgDev sA;   // the hierarchy descriptor, cached in shared memory
  if (a.amg) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(g.amg);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sA);
    for (int t = threadIdx.x; t < (int)(sizeof(AmgDev) / 8); t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  V* x0 = a.amg ? AV<V>::vx(sA.lv[0]) : nullptr;
  const V w0 = a.amg ? V(1.0 / sA.rho[0]) : V(1);

  // ---- start: x = 0, r = rhs, z = M r, p_prev = 0 ----
  S loc[2] = {S(0), S(0)};
  // (loops over rows advance in whole-block steps so every lane of a warp
  // runs the same trip count)
  for (int v0 = row0; v0 < row1; v0 += nslots) {
    const int v = v0 + slot;
    const bool has = v < row1;
    const size_t base = (size_t)(has ? v : row0) * VEC;
    V rv = V(0);
    if (has && act && v != g.fixed) {
      const double src = a.from_residual ? g.res64[base + c7] : -g.b[base + c7];
      rv = V(src);
    }
    V zv = V(0);
    const V* M = s_minv + (size_t)((has ? v : row0) - row0) * BLK;
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      const V rc = __shfl_sync(gm8, rv, (threadIdx.x & ~7) + c);
      zv += M[c7 * 7 + c] * rc;
    }
    if (!act || !has) zv = V(0);
    if (has) {
      x[base + lane8] = V(0);
      r[base + lane8] = rv;
      if (a.amg) x0[base + lane8] = w0 * zv;
      else z[base + lane8] = zv;
      Bufs<V>::p(g, 1)[base + lane8] = V(0);
      Bufs<V>::p(g, 0)[base + lane8] = V(0);
    }
    if (!a.amg) loc[0] += S(rv) * S(zv);
    loc[1] += S(rv) * S(rv);
  }
  if (a.amg && !vcycle_rest<V, S, G>(g, sA, c0, r, q, z, loc[0], counter, abort_flag, target)) goto timeout;
  if (a.amg && a.from_residual && tol >= kOneCycleTol) {
    // a correction pass of the mixed refinement whose FP64 residual is within
    // 1 / kOneCycleTol of the target: one multigrid cycle, x = B r (a
    // preconditioned Richardson step), instead of CG, whose first iteration
    // alone applies the cycle twice
    __syncthreads();
    for (int v0 = row0; v0 < row1; v0 += nslots) {
      const int v = v0 + slot;
      if (v < row1 && act) x[(size_t)v * VEC + c7] = __ldcg(z + (size_t)v * VEC + c7);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->pcg_total += 1;
      st->pcg_iter = 1;
    }
    goto finish;
  }
  write_partial<S, 2>(loc, partial, sh.red);
  if (!grid_sync(counter, abort_flag, target)) goto timeout;
  S rz, bb;
  {
    S t[2];
    reduce_partials<S, 2>(partial, t, sh.red);
    rz = t[0];
    bb = t[1];
  }
  {
    S beta = S(0);
    int it = 0;
    bool done = !(bb > S(0)) || !(rz > S(0));
    const S tol2 = S(tol * tol);
    // multigrid: stop once |r| has not dropped by 10% for 20 iterations (an
    // FP32 solve at a tiny lambda reaches its rounding floor above the
    // tolerance; the FP64 refinement and the LM gain ratio handle the rest)
    S rr_best = bb;
    int stall = 0;
    while (!done) {
      // ---- SpMV: q = (H + lambda I) p, p = z + beta p_prev ----
      const V* pprev = Bufs<V>::p(g, (it + 1) & 1);
      V* pcur = Bufs<V>::p(g, it & 1);
      const V vb = V(beta);
      S pq = S(0);
      for (int v0 = row0; v0 < row1; v0 += nsslots) {
        const int v = v0 + sslot;
        const bool has = v < row1;
        const size_t base = (size_t)(has ? v : row0) * VEC;
        // lane sl stores component sl (G >= 8): its z and p_prev, in flight
        // with the row product
        const V zo = sl < 7 ? __ldcg(z + base + sl) : V(0);
        const V po = sl < 7 ? __ldcg(pprev + base + sl) : V(0);
        V y[7];
        row_prod0<V, G>(g, c0, v, has, sl, gmG,
                        [&](int u, V (&pu)[8]) { load_p(z, pprev, (size_t)u * VEC, vb, pu); }, y);
        if (has && sl < 8) {
          if (sl == 7) {
            q[base + 7] = V(0);
            pcur[base + 7] = V(0);
          } else {
            const bool live = v != g.fixed;
            const V pv = zo + vb * po;
            const V yo = pick7(y, sl);
            q[base + sl] = live ? yo : V(0);
            pcur[base + sl] = pv;
            if (live) pq += S(pv) * S(yo);
          }
        }
      }
      {
        S l1[1] = {pq};
        write_partial<S, 1>(l1, partial + 2 * gridDim.x, sh.red);
      }
      if (!grid_sync(counter, abort_flag, target)) goto timeout;
      S alpha;
      {
        S t[1];
        reduce_partials<S, 1>(partial + 2 * gridDim.x, t, sh.red);
        if (!(t[0] > S(0))) break;   // breakdown: keep the current x
        alpha = rz / t[0];
      }
      // ---- update: x += alpha p, r -= alpha q, z = M r ----
      const V va = V(alpha);
      S l2[2] = {S(0), S(0)};
      for (int v0 = row0; v0 < row1; v0 += nslots) {
        const int v = v0 + slot;
        const bool has = v < row1;
        const size_t base = (size_t)(has ? v : row0) * VEC;
        V rv = V(0);
        if (has && act && v != g.fixed) {
          x[base + c7] += va * pcur[base + c7];
          rv = r[base + c7] - va * q[base + c7];
          r[base + c7] = rv;
        }
        V zv = V(0);
        const V* M = s_minv + (size_t)((has ? v : row0) - row0) * BLK;
#pragma unroll
        for (int c = 0; c < 7; ++c) {
          const V rc = __shfl_sync(gm8, rv, (threadIdx.x & ~7) + c);
          zv += M[c7 * 7 + c] * rc;
        }
        if (has && act) {
          if (a.amg) {
            x0[base + c7] = w0 * zv;
          } else {
            z[base + c7] = zv;
            l2[0] += S(rv) * S(zv);
          }
          l2[1] += S(rv) * S(rv);
        }
      }
      if (a.amg && !vcycle_rest<V, S, G>(g, sA, c0, r, q, z, l2[0], counter, abort_flag, target)) goto timeout;
      write_partial<S, 2>(l2, partial + 3 * gridDim.x, sh.red);
      if (!grid_sync(counter, abort_flag, target)) goto timeout;
      S t2[2];
      reduce_partials<S, 2>(partial + 3 * gridDim.x, t2, sh.red);
      beta = (rz > S(0)) ? t2[0] / rz : S(0);
      rz = t2[0];
      ++it;
      done = !(t2[1] > tol2 * bb) || !(rz > S(0)) || !isfinite((double)t2[1]);
      if (a.amg && !done) {
        if (t2[1] < S(0.81) * rr_best) {
          rr_best = t2[1];
          stall = 0;
        } else if (++stall >= 20) {
          done = true;
        }
      }
      if (!done && it >= maxit) {
        done = true;
        if (blockIdx.x == 0 && threadIdx.x == 0) st->pcg_hit_cap = 1;
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->pcg_total += it;
      st->pcg_iter = it;
    }
  }
finish:
  // leave the counter at zero for the next launch: the last block to get here
  // resets it (all blocks have passed their last barrier).
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&st->ticket[T_PCG_INIT], 1u);
    if (t == gridDim.x - 1) {
      st->ticket[T_PCG_INIT] = 0u;
      st->ticket[T_PCG_SPMV] = 0u;
      __threadfence();
    }
  }
  return;
timeout:
  // a barrier wait ran out: stop the solve (later kernels of this LM
  // iteration see done and return) and report a device failure
  // (every block that gave up writes the same values: block 0 may be the absent one)
  if (threadIdx.x == 0) {
    st->status = PGO_ERR_CUDA;
    st->stop_reason = 4;
    st->done = 1;
  }
  return;
}

// ---- mixed precision: FP64 refinement ------------------------------------
// res = -b - (H + lambda I) dx in FP64 with the FP64 blocks (8 lanes per row,
// lane a owns component a); the first pass starts from dx = 0.  The last
// block stores |res|^2 and the outer stopping test |res| <= pcg_tol |b|.
__global__ void __launch_bounds__(256) k_refine_residual(DevGraph g, int first) {
  SolverState* st = g.st;
  if (st->done || (!first && st->ref_done)) return;
  __shared__ double sh[32];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = tid >> 3, lane8 = tid & 7;
  const bool act = lane8 < 7;
  const int c7 = act ? lane8 : 0;
  const unsigned gm8 = 0xffu << (threadIdx.x & 24);   // the 8 lanes of this row
  const double lam = st->lambda;
  double part[1] = {0.0};
  if (v < g.N) {
    const size_t base = (size_t)v * VEC;
    double y = 0.0;
    if (!first) {
      // lane j of the row's 8 takes whole blocks j, j + 8, ... of the row
      // (the damped diagonal block first), then the 8 lanes reduce: 4 blocks
      // in sequence per lane instead of the row's 30
      const int k0 = g.inc_ptr[v], ks = g.inc_split[v], k1 = g.inc_ptr[v + 1];
      double yv[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int k = k0 - 1 + lane8; k < k1; k += 8) {
        int u = v;
        const double* B;
        bool tr = false;
        if (k < k0) {
          B = g.diag64 + (size_t)v * BLK64;
        } else {
          const int code = __ldg(g.inc_code + k);
          u = __ldg(g.inc_other + k);
          B = g.off64 + (size_t)(code >> 1) * BLK64;
          tr = k >= ks;   // side 1: H_uv^T
        }
        double xu[8];
        const double2* x2 = reinterpret_cast<const double2*>(g.dx64 + (size_t)u * VEC);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double2 t2 = __ldcg(x2 + c);
          xu[2 * c] = t2.x;
          xu[2 * c + 1] = t2.y;
        }
        double Bv[49];
        load_block(B, Bv);
#pragma unroll
        for (int a = 0; a < 7; ++a) {
          double t = (k < k0) ? lam * xu[a] : 0.0;
#pragma unroll
          for (int c = 0; c < 7; ++c) t += (tr ? Bv[c * 7 + a] : Bv[a * 7 + c]) * xu[c];
          yv[a] += t;
        }
      }
#pragma unroll
      for (int a = 0; a < 7; ++a) {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) yv[a] += __shfl_xor_sync(gm8, yv[a], o);
      }
      y = yv[0];
#pragma unroll
      for (int a = 1; a < 7; ++a)
        if (c7 == a) y = yv[a];
    } else if (act) {
      g.dx64[base + c7] = 0.0;
    }
    if (!act) {
      g.res64[base + 7] = 0.0;
      if (first) g.dx64[base + 7] = 0.0;
    } else {
      const double rv = (v == g.fixed) ? 0.0 : -g.b[base + c7] - y;
      g.res64[base + c7] = rv;
      part[0] = rv * rv;
    }
  }
  block_sum<1>(part, sh);
  if (!publish_partials<1>(part, g.partial, &st->ticket[T_REFINE])) return;
  double tot[1];
  gather_partials_sum<1>(g.partial, tot, sh);
  if (threadIdx.x == 0) {
    st->ref_rr = tot[0];
    const double tol = g.opt->pcg_tol;
    st->ref_done = !(tot[0] > tol * tol * st->bnorm2);
  }
}

// dx64 += x32 (after an inner FP32 solve).
__global__ void __launch_bounds__(256) k_refine_accumulate(DevGraph g) {
  const SolverState* st = g.st;
  if (st->done || st->ref_done) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N * VEC) return;
  g.dx64[t] += (double)g.x32[t];
}

// ---- launch configuration ---------------------------------------------------
// FP32 lanes per block row when a block's rows do not fit in 512 threads
// with a warp each.
#ifndef PCG_G32
#define PCG_G32 16
#endif
static int g_num_sms = 0;

static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

static int pcg_rows_per_block(int N) {
  const int rpb = (N + num_sms() - 1) / num_sms();
  return rpb < 1 ? 1 : rpb;
}

int pcg_block_entries(int N, const int* inc_ptr) {
  const int rpb = pcg_rows_per_block(N);
  int most = 0;
  for (int r0 = 0; r0 < N; r0 += rpb) {
    const int r1 = r0 + rpb < N ? r0 + rpb : N;
    most = inc_ptr[r1] - inc_ptr[r0] > most ? inc_ptr[r1] - inc_ptr[r0] : most;
  }
  return most;
}

static size_t g_smem_optin = 0;

template <class V, class S, int G>
static cudaError_t launch_pcg_kernel(const DevGraph& g, PcgArgs a, cudaStream_t s) {
  if (g_smem_optin == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g_smem_optin = v > 0 ? (size_t)v : 48 * 1024;
  }
  // one block per SM, rows split evenly; max(8, G) lanes per row, at most
  // the kernel's launch bound (FP64: 256 threads, for its registers; FP32: 512)
  const int lanes = G > 8 ? G : 8;
  const int rows_per_block = pcg_rows_per_block(g.N);
  const int blocks = (g.N + rows_per_block - 1) / rows_per_block;
  int threads = rows_per_block * lanes;
  threads = ((threads + 31) / 32) * 32;
  const int tmax = sizeof(V) == 8 ? 256 : 512;
  if (threads > tmax) threads = tmax;
  if (threads < 32) threads = 32;
  a.rows_per_block = rows_per_block;
  // shared memory: diag + preconditioner blocks of the rows, then as many
  // off-diagonal blocks (and their indices) as fit
  const size_t blk_bytes = (size_t)Bufs<V>::BLK * sizeof(V);
  const size_t budget = g_smem_optin - 8192;   // static shared memory (incl. the hierarchy descriptor) and slack
  const size_t fixed_bytes = 2 * (size_t)rows_per_block * blk_bytes;
  size_t cap = 0;
  if (budget > fixed_bytes) cap = (budget - fixed_bytes) / (blk_bytes + 2 * sizeof(int));
  // no more than the fullest row block stages: the rest of the SM's 256 KB
  // stays L1 cache for the multigrid levels' blocks and indices
  size_t max_entries = (size_t)2 * (size_t)(g.E > 0 ? g.E : 1);
  if (g.pcg_block_entries > 0 && (size_t)g.pcg_block_entries < max_entries) max_entries = (size_t)g.pcg_block_entries;
  if (cap > max_entries) cap = max_entries;
  a.cap_entries = (int)cap;
  const size_t smem = fixed_bytes + cap * (blk_bytes + 2 * sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(k_pcg<V, S, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pcg<V, S, G>, g, a);
}

// Partial slots (of 4 doubles) the persistent solve needs: 5 values per block.
int pcg_partials_needed(int) { return 2 * num_sms() + 8; }

void launch_precond(const DevGraph& g, int mixed, cudaStream_t s) {
  const int nb = (g.N + 31) / 32;
  if (mixed) k_precond<float><<<nb, 32, 0, s>>>(g);
  else k_precond<double><<<nb, 32, 0, s>>>(g);
}

cudaError_t launch_pcg(const DevGraph& g, int mixed, int from_residual, const AmgDev* amg, cudaStream_t s) {
  PcgArgs a;
  a.from_residual = from_residual;
  a.inner = mixed;
  a.rows_per_block = 1;
  a.cap_entries = 0;
  a.amg = amg != nullptr && g.amg != nullptr;
  // FP32: a warp per row (one pass over a row's entries) while a block's rows
  // fit in 512 threads, else 16 lanes per row
  if (mixed && pcg_rows_per_block(g.N) * 32 <= 512) return launch_pcg_kernel<float, float, 32>(g, a, s);
  if (mixed) return launch_pcg_kernel<float, float, PCG_G32>(g, a, s);
  return launch_pcg_kernel<double, double, 8>(g, a, s);
}

void launch_refine_residual(const DevGraph& g, int first, cudaStream_t s) {
  k_refine_residual<<<(g.N * 8 + 127) / 128, 128, 0, s>>>(g, first);
}

void launch_refine_accumulate(const DevGraph& g, cudaStream_t s) {
  k_refine_accumulate<<<(g.N * VEC + 255) / 256, 256, 0, s>>>(g);
}

// Test hook: the grid-barrier wait limit of this file's kernels (0: 2 s).
void set_barrier_limit_pcg(unsigned long long ns) {
  cudaMemcpyToSymbol(g_barrier_limit_ns, &ns, sizeof(ns));
  cudaGetLastError();
}

}  // namespace pgo
