// Direct solve of the damped normal equations (H + lambda I) delta = rhs by
// a block Cholesky factorisation on the GPU (the exact linear solve of
// Sec. IV-F, which the paper runs as an LDL^T on the CPU after finding the
// GPU sparse direct solver slower on small graphs, Fig. 4).
//
// Structure.  In keyframe order the essential graph's normal matrix is
// block-banded: spanning-tree and covisibility edges join keyframes a few
// frames apart.  Only loop edges reach far.  The host analysis (once per
// graph) makes the free endpoints of every edge longer than the band cap
// separators and orders them last, so that the matrix is
//     [ B  C^T ]      B: block-banded (bandwidth w blocks) over the other
//     [ C  D   ]      free vertices, C: the separators' rows, D: their block.
// Its Cholesky factor keeps the shape [L_B 0; L_C L_D] with L_B banded and
// L_C dense (the separators' rows fill in from their first coupling on).
//
// Kernels (each one thread block, sequential over the band, all of its work
// in shared memory; 7x7 blocks of 49 values):
//   k_direct_assemble  the blocks of B, C and D from the linearised blocks
//                      (lambda on the diagonal), per target a recipe of
//                      contributing blocks (transposed where the edge runs
//                      the other way);
//   k_direct_factor    right-looking over the band: per column k the 7x7
//                      Cholesky of the pivot, the panel L_ik = A_ik L_kk^-T of
//                      the next w band rows and of every separator row, and
//                      the rank-7 update of the window, the separator rows'
//                      window and D; a window of w + 1 band rows and the
//                      separator rows' w + 1 columns stay in shared memory as
//                      ring buffers; then the dense Cholesky of D;
//   k_direct_solve     forward and backward substitution with the factor.
// The mixed-precision solve factors once per LM iteration in FP32 and reuses
// the factor for every FP64 refinement pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "common.cuh"

namespace pgo {

struct DirectHost {
  DirectDev dev{};
  DirectDev host_view{};
  char* mem = nullptr;
  size_t blocks = 0;
};

namespace {

constexpr int kBandCap = 20;      // longest edge kept in the band (blocks)
constexpr int kMaxSep = 16;       // separators

template <class V> struct DV;
template <> struct DV<double> {
  static __device__ __forceinline__ double* store(const DirectDev& D) { return D.s64; }
  static __device__ __forceinline__ const double* off(const DevGraph& g) { return g.off64; }
  static __device__ __forceinline__ const double* diag(const DevGraph& g) { return g.diag64; }
  static __device__ __forceinline__ double* x(const DevGraph& g) { return g.x64; }
  static constexpr int BLK = BLK64;
};
template <> struct DV<float> {
  static __device__ __forceinline__ float* store(const DirectDev& D) { return D.s32; }
  static __device__ __forceinline__ const float* off(const DevGraph& g) { return g.off32; }
  static __device__ __forceinline__ const float* diag(const DevGraph& g) { return g.diag32; }
  static __device__ __forceinline__ float* x(const DevGraph& g) { return g.x32; }
  static constexpr int BLK = BLK32;
};

// ---- assembly: one thread per (target block, entry) --------------------------
template <class V>
__global__ void __launch_bounds__(256) k_direct_assemble(DevGraph g, DirectDev D) {
  const SolverState* st = g.st;
  if (st->done) return;
  constexpr int BLK = DV<V>::BLK;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)D.n_targets * 49) return;
  const int tg = (int)(t / 49), e = (int)(t - (long long)tg * 49);
  const int a = e / 7, c = e - 7 * (e / 7);
  const V* off = DV<V>::off(g);
  const V* diag = DV<V>::diag(g);
  V s = V(0);
  const int k0 = __ldg(D.r_ptr + tg), k1 = __ldg(D.r_ptr + tg + 1);
  for (int k = k0; k < k1; ++k) {
    const int code = __ldg(D.r_code + k);
    if (code < 0) {   // the diagonal block of vertex -code - 1, damped
      s += diag[(size_t)(-code - 1) * BLK + a * 7 + c];
      if (a == c) s += V(st->lambda);
    } else {
      const V* B = off + (size_t)(code >> 1) * BLK;
      s += (code & 1) ? B[c * 7 + a] : B[a * 7 + c];
    }
  }
  DV<V>::store(D)[(size_t)__ldg(D.r_dst + tg) * 49 + e] = s;
}

// ---- factorisation -------------------------------------------------------------
// Y = X Linv^T for 7x7 blocks, one output entry (r, c) per call: sum_k X[r][k] Linv[c][k]
template <class V>
__device__ __forceinline__ V panel_entry(const V* X, const V* Li, int r, int c) {
  V s = V(0);
#pragma unroll
  for (int k = 0; k < 7; ++k) s += X[r * 7 + k] * Li[c * 7 + k];
  return s;
}

constexpr int kFactorThreads = 256;

template <class V>
__global__ void __launch_bounds__(kFactorThreads, 1) k_direct_factor(DevGraph g, DirectDev D) {
  SolverState* st = g.st;
  if (st->done) return;
  const int nb = D.nb, w = D.w, ns = D.ns, W1 = D.w + 1;
  V* S = DV<V>::store(D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* win = reinterpret_cast<V*>(smem_raw);              // band ring: W1 rows x W1 blocks (offset o = row - col)
  V* bwin = win + (size_t)W1 * W1 * 49;                 // separator ring: ns rows x W1 columns (column c at c % W1)
  V* corner = bwin + (size_t)ns * W1 * 49;              // ns x ns blocks (lower)
  __shared__ int s_fail;
  __shared__ V s_rdiag[7];   // 1 / L_kk[a][a] of the current pivot
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  if (tid == 0) s_fail = 0;
  // initial window: band rows 0..w (their blocks with col >= 0), separator columns 0..w, D
  for (int r = 0; r < min(W1, nb); ++r)
    for (int t = tid; t < W1 * 49; t += nt) {
      const int o = t / 49;
      win[((size_t)(r % W1) * W1 + o) * 49 + t % 49] = (o <= r) ? S[((size_t)r * W1 + o) * 49 + t % 49] : V(0);
    }
  for (int t = tid; t < ns * W1 * 49; t += nt) {
    const int s = t / (W1 * 49), rem = t - s * W1 * 49, c = rem / 49;
    bwin[t] = c < nb ? S[D.border0 + ((size_t)s * nb + c) * 49 + rem % 49] : V(0);
  }
  for (int t = tid; t < ns * ns * 49; t += nt) corner[t] = S[D.corner0 + t];
  __syncthreads();
  // each thread's share of the row (and separator column) entering the window
  const int pre_n = (W1 + ns) * 49;
  constexpr int kPre = 8;   // (W1 + ns) * 49 <= 8 * 256 for the size limits
  for (int k = 0; k < nb; ++k) {
    V* Akk = win + ((size_t)(k % W1) * W1 + 0) * 49;
    const int rn = k + W1;   // enters the window in the slot of row k
    // prefetch row rn and separator column rn (consumed after the update)
    V pre[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int t = tid + u * nt;
      pre[u] = V(0);
      if (rn < nb && t < pre_n) {
        if (t < W1 * 49) pre[u] = S[((size_t)rn * W1 + t / 49) * 49 + t % 49];
        else {
          const int q = t - W1 * 49;
          pre[u] = S[D.border0 + ((size_t)(q / 49) * nb + rn) * 49 + q % 49];
        }
      }
    }
    // 1. Cholesky of the pivot block on warp 0: lane i < 7 holds row i in registers
    if (tid < 32) {
      V a[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) a[c] = lane < 7 ? Akk[lane * 7 + c] : V(0);
      bool ok = true;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        V d = __shfl_sync(0xffffffffu, a[j], j);
        const V a0 = __shfl_sync(0xffffffffu, Akk[j * 7 + j], 0);
        // single precision at a large condition number: a pivot lost to
        // rounding is regularised (the FP64 refinement and the LM gain ratio
        // absorb the error); in FP64 it is a numerical failure
        if (!(d > V(0))) {
          if (sizeof(V) == 8) ok = false;
          d = fabs(a0) * V(1e-6) + V(1e-30);
        }
        const V ljj = sqrt(d);
        if (lane == j) a[j] = ljj;
        if (lane > j) a[j] = a[j] / ljj;
#pragma unroll
        for (int c = j + 1; c < 7; ++c) {
          const V lcj = __shfl_sync(0xffffffffu, a[j], c);
          if (lane >= c) a[c] -= a[j] * lcj;
        }
      }
      if (lane < 7) {
#pragma unroll
        for (int c = 0; c < 7; ++c) Akk[lane * 7 + c] = c <= lane ? a[c] : V(0);
        V dl = a[0];
#pragma unroll
        for (int c = 1; c < 7; ++c)
          if (c == lane) dl = a[c];
        s_rdiag[lane] = V(1) / dl;
      }
      if (lane == 0 && !ok) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    // 2. panel: every row of the band blocks (k+1..k+nr, k) and of the
    // separators' blocks (s, k) solves x L_kk^T = a by forward substitution
    // (one thread per row; it reads and writes only its own row); L_kk goes out
    const int nr = min(w, nb - 1 - k);
    for (int t = tid; t < (nr + ns) * 7; t += nt) {
      const int b = t / 7, r = t - 7 * b;
      V* X = (b < nr ? win + ((size_t)((k + 1 + b) % W1) * W1 + (b + 1)) * 49
                     : bwin + ((size_t)(b - nr) * W1 + (k % W1)) * 49) + r * 7;
      V x[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        V v = X[c];
#pragma unroll
        for (int q = 0; q < c; ++q) v -= x[q] * Akk[c * 7 + q];
        x[c] = v * s_rdiag[c];
      }
#pragma unroll
      for (int c = 0; c < 7; ++c) X[c] = x[c];
    }
    // the stored pivot block keeps the reciprocals on its diagonal (the solves multiply)
    for (int t = tid; t < 49; t += nt)
      S[((size_t)k * W1) * 49 + t] = (t % 8 == 0) ? s_rdiag[t / 8] : Akk[t];
    __syncthreads();
    // 3. rank-7 updates: band A_ij -= L_ik L_jk^T (k < j <= i <= k+w), separator
    // rows C_sj -= L_sk L_jk^T (k < j <= k+w), corner D_st -= L_sk L_tk^T (t <= s);
    // column k retires to global memory in the same phase (it is only read here)
    {
      const int nband = nr * (nr + 1) / 2, nsep = ns * nr, ncorner = ns * (ns + 1) / 2;
      const int tasks = nband + nsep + ncorner;
      // one output block per thread: L_j in registers, then row by row of L_i
      for (int b = tid; b < tasks; b += nt) {
        const V *Li, *Lj;
        V* Y;
        if (b < nband) {
          // (ii, jj) with 0 <= jj <= ii < nr: rows i = k+1+ii, j = k+1+jj
          int ii = (int)((sqrtf(8.0f * b + 1.0f) - 1.0f) * 0.5f);
          while ((ii + 1) * (ii + 2) / 2 <= b) ++ii;
          while (ii * (ii + 1) / 2 > b) --ii;
          const int jj = b - ii * (ii + 1) / 2;
          const int i = k + 1 + ii, j = k + 1 + jj;
          Li = win + ((size_t)(i % W1) * W1 + (i - k)) * 49;
          Lj = win + ((size_t)(j % W1) * W1 + (j - k)) * 49;
          Y = win + ((size_t)(i % W1) * W1 + (i - j)) * 49;
        } else if (b < nband + nsep) {
          const int q = b - nband, s = q / nr, jj = q - s * nr, j = k + 1 + jj;
          Li = bwin + ((size_t)s * W1 + (k % W1)) * 49;
          Lj = win + ((size_t)(j % W1) * W1 + (j - k)) * 49;
          Y = bwin + ((size_t)s * W1 + (j % W1)) * 49;
        } else {
          const int q = b - nband - nsep;
          int s = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
          while ((s + 1) * (s + 2) / 2 <= q) ++s;
          while (s * (s + 1) / 2 > q) --s;
          const int u = q - s * (s + 1) / 2;
          Li = bwin + ((size_t)s * W1 + (k % W1)) * 49;
          Lj = bwin + ((size_t)u * W1 + (k % W1)) * 49;
          Y = corner + ((size_t)s * ns + u) * 49;
        }
        V lj[49];
#pragma unroll
        for (int e = 0; e < 49; ++e) lj[e] = Lj[e];
#pragma unroll
        for (int r = 0; r < 7; ++r) {
          V li[7];
#pragma unroll
          for (int q = 0; q < 7; ++q) li[q] = Li[r * 7 + q];
#pragma unroll
          for (int c = 0; c < 7; ++c) {
            V acc = V(0);
#pragma unroll
            for (int q = 0; q < 7; ++q) acc += li[q] * lj[c * 7 + q];
            Y[r * 7 + c] -= acc;
          }
        }
      }
      for (int t = tid; t < nr * 49; t += nt) {
        const int b = t / 49 + 1, i = k + b;
        S[((size_t)i * W1 + b) * 49 + t % 49] = win[((size_t)(i % W1) * W1 + b) * 49 + t % 49];
      }
      for (int t = tid; t < ns * 49; t += nt) {
        const int s = t / 49;
        S[D.border0 + ((size_t)s * nb + k) * 49 + t % 49] = bwin[((size_t)s * W1 + (k % W1)) * 49 + t % 49];
      }
    }
    __syncthreads();
    // 4. the prefetched row and separator column take the slot of row k
    if (rn < nb) {
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        const int t = tid + u * nt;
        if (t >= pre_n) continue;
        if (t < W1 * 49) win[((size_t)(rn % W1) * W1 + t / 49) * 49 + t % 49] = pre[u];
        else {
          const int q = t - W1 * 49;
          bwin[((size_t)(q / 49) * W1 + (rn % W1)) * 49 + q % 49] = pre[u];
        }
      }
    }
    __syncthreads();
  }
  // 5. dense Cholesky of the updated corner (7 ns x 7 ns, lower), column by column
  const int m = 7 * ns;
  auto cidx = [&](int R, int C) -> V& { return corner[((size_t)(R / 7) * ns + (C / 7)) * 49 + (R % 7) * 7 + (C % 7)]; };
  for (int j = 0; j < m && !s_fail; ++j) {
    if (tid == 0) {
      V d = cidx(j, j);
      if (!(d > V(0))) {   // as for the band pivots
        if (sizeof(V) == 8) s_fail = 1;
        d = V(1e-30);
      }
      cidx(j, j) = sqrt(d);
    }
    __syncthreads();
    if (s_fail) break;
    const V dj = cidx(j, j);
    for (int i = j + 1 + tid; i < m; i += nt) cidx(i, j) /= dj;
    __syncthreads();
    for (int t = tid; t < (m - j - 1) * (m - j - 1); t += nt) {
      const int i = j + 1 + t / (m - j - 1), c = j + 1 + t % (m - j - 1);
      if (c <= i) cidx(i, c) -= cidx(i, j) * cidx(c, j);
    }
    __syncthreads();
  }
  for (int t = tid; t < ns * ns * 49; t += nt) S[D.corner0 + t] = corner[t];
  if (tid == 0 && s_fail) {
    st->status = PGO_ERR_NUMERICAL;
    st->stop_reason = 4;
    st->done = 1;
  }
}

// ---- forward and backward substitution -------------------------------------------
// rhs: -b (from_residual = 0) or the FP64 refinement residual; x = (H + lambda I)^-1 rhs
// in the graph's vertex order (fixed vertex 0).  One thread block of 512.  The
// band sweeps are sequential: warp 0 carries them (lane l < 7 owns component l
// of the current row) while warps 1..15 stage the factor blocks each row needs
// into a ring of shared-memory slots ahead of it (a row's blocks (r, r - o)
// forward, a column's blocks (r + o, r) backward).  A slot holds sweep index i
// when ring_row[slot] == i; warp 0 publishes how many indices it has consumed.
// Every wait is bounded; a wait that runs out reports a numerical failure.
constexpr int kSolveThreads = 512;
constexpr long long kSpinLimit = 1ll << 26;

template <class V>
__device__ __forceinline__ void stage_slot(const V* S, V* slot, int r, int nb, int W1, int forward, int lane) {
  for (int t = lane; t < W1 * 49; t += 32) {
    const int o = t / 49;
    V v = V(0);
    if (forward) {
      if (o <= r) v = S[((size_t)r * W1 + o) * 49 + t % 49];          // block (r, r - o)
    } else {
      if (r + o < nb) v = S[((size_t)(r + o) * W1 + o) * 49 + t % 49];  // block (r + o, r)
    }
    slot[t] = v;
  }
}

template <class V>
__global__ void __launch_bounds__(kSolveThreads, 1) k_direct_solve(DevGraph g, DirectDev D, int from_residual,
                                                                   int ring) {
  SolverState* st = g.st;
  if (st->done || (from_residual && st->ref_done)) return;
  const int nb = D.nb, w = D.w, ns = D.ns, W1 = D.w + 1, m = 7 * ns;
  const V* S = DV<V>::store(D);
  V* x = DV<V>::x(g);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* slots = reinterpret_cast<V*>(smem_raw);         // ring x W1 x 49
  V* y = slots + (size_t)ring * W1 * 49;             // band values, 7 per band row (nb * 7)
  V* ys = y + (size_t)nb * 7;                        // separator values (m)
  __shared__ int ring_row[32];
  __shared__ int consumed, s_fail;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  if (tid < 32) ring_row[tid] = -1;
  if (tid == 0) {
    consumed = 0;
    s_fail = 0;
  }
  // gather the right-hand side in the factor's order
  for (int t = tid; t < (nb + ns) * 7; t += nt) {
    const int r = t / 7, a = t % 7;
    const int v = r < nb ? __ldg(D.band_v + r) : __ldg(D.sep_v + (r - nb));
    const double rv = from_residual ? g.res64[(size_t)v * VEC + a] : -g.b[(size_t)v * VEC + a];
    y[t] = V(rv);
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    const int forward = pass == 0;
    if (warp > 0) {
      // producers: warp p stages sweep indices p - 1, p - 1 + (nwarps - 1), ...
      for (int i = warp - 1; i < nb; i += nwarps - 1) {
        long long spins = 0;
        while (*(volatile int*)&consumed <= i - ring && !*(volatile int*)&s_fail && ++spins < kSpinLimit) {
        }
        if (spins >= kSpinLimit || *(volatile int*)&s_fail) {
          if (lane == 0) s_fail = 1;
          break;
        }
        const int r = forward ? i : nb - 1 - i;
        stage_slot<V>(S, slots + (size_t)(i % ring) * W1 * 49, r, nb, W1, forward, lane);
        __syncwarp();
        __threadfence_block();
        if (lane == 0) *(volatile int*)&ring_row[i % ring] = i;
        if (*(volatile int*)&s_fail) break;
      }
    } else {
      for (int i = 0; i < nb; ++i) {
        long long spins = 0;
        while (*(volatile int*)&ring_row[i % ring] != i && !*(volatile int*)&s_fail && ++spins < kSpinLimit) {
        }
        if (spins >= kSpinLimit || *(volatile int*)&s_fail) {
          if (lane == 0) s_fail = 1;
          break;
        }
        __threadfence_block();
        const V* sl = slots + (size_t)(i % ring) * W1 * 49;
        const int r = forward ? i : nb - 1 - i;
        V acc = V(0);
        if (forward) {
          // y_r = L_rr^-1 (y_r - sum_o L_{r,r-o} y_{r-o})
          if (lane < 7)
            for (int o = 1; o <= min(w, r); ++o) {
              const V* L = sl + (size_t)o * 49 + lane * 7;
              const V* yy = y + (size_t)(r - o) * 7;
#pragma unroll
              for (int q = 0; q < 7; ++q) acc += L[q] * yy[q];
            }
          V val = lane < 7 ? y[(size_t)r * 7 + lane] - acc : V(0);
#pragma unroll
          for (int a = 0; a < 7; ++a) {
            const V ya = __shfl_sync(0xffffffffu, val, a) * sl[a * 7 + a];
            if (lane == a) val = ya;
            if (lane > a && lane < 7) val -= sl[lane * 7 + a] * ya;
          }
          if (lane < 7) y[(size_t)r * 7 + lane] = val;
        } else {
          // x_r = L_rr^-T (y_r - sum_o L_{r+o,r}^T x_{r+o})
          if (lane < 7)
            for (int o = 1; o <= min(w, nb - 1 - r); ++o) {
              const V* L = sl + (size_t)o * 49;
              const V* xx = y + (size_t)(r + o) * 7;
#pragma unroll
              for (int q = 0; q < 7; ++q) acc += L[q * 7 + lane] * xx[q];
            }
          V val = lane < 7 ? y[(size_t)r * 7 + lane] - acc : V(0);
#pragma unroll
          for (int a = 6; a >= 0; --a) {
            const V xa = __shfl_sync(0xffffffffu, val, a) * sl[a * 7 + a];
            if (lane == a) val = xa;
            if (lane < a) val -= sl[a * 7 + lane] * xa;
          }
          if (lane < 7) y[(size_t)r * 7 + lane] = val;
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) *(volatile int*)&consumed = i + 1;
        if (*(volatile int*)&s_fail) break;
      }
    }
    __syncthreads();
    if (s_fail) break;
    if (tid < 32) ring_row[tid] = -1;
    if (tid == 0) consumed = 0;
    if (forward) {
      // separators: ys -= L_C y_B, one warp per separator row (lanes over the
      // band columns, then a shuffle reduction), then the dense forward and
      // backward solves with L_D on warp 0 (lanes over the row's entries)
      for (int R = warp; R < m; R += nwarps) {
        const int sR = R / 7, a = R % 7;
        V acc = V(0);
        for (int t = lane; t < nb * 7; t += 32) {
          const int c = t / 7, q = t % 7;
          acc += S[D.border0 + ((size_t)sR * nb + c) * 49 + a * 7 + q] * y[t];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) ys[R] -= acc;
      }
      __syncthreads();
      auto LD = [&](int R, int C) -> V {
        return S[D.corner0 + ((size_t)(R / 7) * ns + C / 7) * 49 + (R % 7) * 7 + C % 7];
      };
      if (tid < 32) {
        for (int R = 0; R < m; ++R) {
          V acc = V(0);
          for (int C = lane; C < R; C += 32) acc += LD(R, C) * ys[C];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) ys[R] = (ys[R] - acc) / LD(R, R);
          __syncwarp();
        }
        for (int R = m - 1; R >= 0; --R) {
          V acc = V(0);
          for (int C = R + 1 + lane; C < m; C += 32) acc += LD(C, R) * ys[C];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) ys[R] = (ys[R] - acc) / LD(R, R);
          __syncwarp();
        }
      }
      __syncthreads();
      // y_B -= L_C^T x_S (band columns in parallel)
      for (int t = tid; t < nb * 7; t += nt) {
        const int c = t / 7, a = t % 7;
        V acc = V(0);
        for (int s2 = 0; s2 < ns; ++s2) {
          const V* L = S + D.border0 + ((size_t)s2 * nb + c) * 49;
#pragma unroll
          for (int q = 0; q < 7; ++q) acc += L[q * 7 + a] * ys[s2 * 7 + q];
        }
        y[t] -= acc;
      }
      __syncthreads();
    }
  }
  if (s_fail) {
    if (tid == 0) {
      st->status = PGO_ERR_NUMERICAL;
      st->stop_reason = 4;
      st->done = 1;
    }
    return;
  }
  // scatter to the vertex order; the fixed vertex stays 0
  for (int t = tid; t < g.N * VEC; t += nt) x[t] = V(0);
  __syncthreads();
  for (int t = tid; t < (nb + ns) * 7; t += nt) {
    const int r = t / 7, a = t % 7;
    const int v = r < nb ? __ldg(D.band_v + r) : __ldg(D.sep_v + (r - nb));
    x[(size_t)v * VEC + a] = r < nb ? y[t] : ys[t - nb * 7];
  }
}

size_t factor_smem(int w, int ns, size_t vbytes) {
  const size_t W1 = (size_t)w + 1;
  return (W1 * W1 + (size_t)ns * W1 + (size_t)ns * ns) * 49 * vbytes;
}

int solve_ring(size_t vbytes) { return vbytes == 4 ? 16 : 8; }

size_t solve_smem(int nb, int ns, int w, size_t vbytes) {
  return ((size_t)solve_ring(vbytes) * (w + 1) * 49 + (size_t)nb * 7 + 7 * (size_t)ns) * vbytes;
}

int smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 48 * 1024;
  }
  return v;
}

}  // namespace

// ---- host analysis ------------------------------------------------------------------
DirectHost* direct_build(int N, int fixed, const int* inc_ptr, const int* inc_code, const int* inc_other,
                         cudaStream_t s, const char** why) {
  *why = nullptr;
  // edges between free vertices, from the side-0 incidence entries
  std::vector<int> ei, ej, eid;
  for (int v = 0; v < N; ++v)
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k)
      if ((inc_code[k] & 1) == 0) {
        const int u = inc_other[k];
        if (v == fixed || u == fixed) continue;
        ei.push_back(v);
        ej.push_back(u);
        eid.push_back(inc_code[k] >> 1);
      }
  const int E = (int)ei.size();
  std::vector<int> sid(N, -1);
  std::vector<int> sep;
  for (int e = 0; e < E; ++e)
    if (std::abs(ei[e] - ej[e]) > kBandCap)
      for (int v : {ei[e], ej[e]})
        if (sid[v] < 0) {
          sid[v] = 0;
          sep.push_back(v);
        }
  std::sort(sep.begin(), sep.end());
  if ((int)sep.size() > kMaxSep) {
    *why = "too many long-range edge endpoints for the direct solver";
    return nullptr;
  }
  for (size_t q = 0; q < sep.size(); ++q) sid[sep[q]] = (int)q;
  std::vector<int> pos(N, -1), band;
  for (int v = 0; v < N; ++v)
    if (v != fixed && sid[v] < 0) {
      pos[v] = (int)band.size();
      band.push_back(v);
    }
  const int nb = (int)band.size(), ns = (int)sep.size();
  if (nb < 1) {
    *why = "no band vertex";
    return nullptr;
  }
  int w = 1;
  for (int e = 0; e < E; ++e)
    if (pos[ei[e]] >= 0 && pos[ej[e]] >= 0) w = std::max(w, std::abs(pos[ei[e]] - pos[ej[e]]));
  const int W1 = w + 1;
  // targets: band (r, o) -> r * W1 + o; border (s, c) -> B0 + s * nb + c; corner (s, t) -> C0 + s * ns + t
  const size_t B0 = (size_t)nb * W1, C0 = B0 + (size_t)ns * nb, nblk = C0 + (size_t)ns * ns;
  std::vector<std::vector<int>> rec;   // per target (sparse map below)
  std::vector<size_t> tdst;
  std::vector<int> tindex(nblk, -1);
  auto add = [&](size_t dst, int code) {
    if (tindex[dst] < 0) {
      tindex[dst] = (int)tdst.size();
      tdst.push_back(dst);
      rec.emplace_back();
    }
    rec[tindex[dst]].push_back(code);
  };
  for (int v = 0; v < N; ++v) {
    if (v == fixed) continue;
    if (pos[v] >= 0) add((size_t)pos[v] * W1, -(v + 1));
    else add(C0 + (size_t)sid[v] * ns + sid[v], -(v + 1));
  }
  for (int e = 0; e < E; ++e) {
    const int i = ei[e], j = ej[e], code = 2 * eid[e];
    const bool bi = pos[i] >= 0, bj = pos[j] >= 0;
    if (bi && bj) {
      // lower block (row = larger position): H_ij as stored if i is the row
      if (pos[i] > pos[j]) add((size_t)pos[i] * W1 + (pos[i] - pos[j]), code);
      else add((size_t)pos[j] * W1 + (pos[j] - pos[i]), code | 1);
    } else if (!bi && bj) {
      add(B0 + (size_t)sid[i] * nb + pos[j], code);
    } else if (bi && !bj) {
      add(B0 + (size_t)sid[j] * nb + pos[i], code | 1);
    } else {
      if (sid[i] > sid[j]) add(C0 + (size_t)sid[i] * ns + sid[j], code);
      else add(C0 + (size_t)sid[j] * ns + sid[i], code | 1);
    }
  }
  std::vector<int> r_ptr(tdst.size() + 1, 0), r_code, r_dst(tdst.size());
  for (size_t t = 0; t < tdst.size(); ++t) {
    r_ptr[t + 1] = r_ptr[t] + (int)rec[t].size();
    r_code.insert(r_code.end(), rec[t].begin(), rec[t].end());
    r_dst[t] = (int)tdst[t];
  }
  DirectHost* H = new DirectHost();
  DirectDev& D = H->host_view;
  D.nb = nb;
  D.ns = ns;
  D.w = w;
  D.n_targets = (int)tdst.size();
  D.border0 = B0 * 49;
  D.corner0 = C0 * 49;
  D.n_blocks = (long long)nblk;
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t bytes = a256(sizeof(int) * nb) + a256(sizeof(int) * (ns > 0 ? ns : 1)) + a256(sizeof(int) * r_ptr.size()) +
                       a256(sizeof(int) * (r_code.empty() ? 1 : r_code.size())) + a256(sizeof(int) * r_dst.size()) +
                       a256(sizeof(float) * 49 * nblk) + a256(sizeof(double) * 49 * nblk);
  if (cudaMalloc(&H->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete H;
    *why = "device allocation failed";
    return nullptr;
  }
  char* p = H->mem;
  auto take = [&](size_t b) { char* q = p; p += a256(b); return q; };
  int* d_band = reinterpret_cast<int*>(take(sizeof(int) * nb));
  int* d_sep = reinterpret_cast<int*>(take(sizeof(int) * (ns > 0 ? ns : 1)));
  int* d_rptr = reinterpret_cast<int*>(take(sizeof(int) * r_ptr.size()));
  int* d_rcode = reinterpret_cast<int*>(take(sizeof(int) * (r_code.empty() ? 1 : r_code.size())));
  int* d_rdst = reinterpret_cast<int*>(take(sizeof(int) * r_dst.size()));
  D.s32 = reinterpret_cast<float*>(take(sizeof(float) * 49 * nblk));
  D.s64 = reinterpret_cast<double*>(take(sizeof(double) * 49 * nblk));
  D.band_v = d_band;
  D.sep_v = d_sep;
  D.r_ptr = d_rptr;
  D.r_code = d_rcode;
  D.r_dst = d_rdst;
  bool ok = true;
  ok &= cudaMemcpyAsync(d_band, band.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (ns) ok &= cudaMemcpyAsync(d_sep, sep.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(d_rptr, r_ptr.data(), sizeof(int) * r_ptr.size(), cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!r_code.empty())
    ok &= cudaMemcpyAsync(d_rcode, r_code.data(), sizeof(int) * r_code.size(), cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(d_rdst, r_dst.data(), sizeof(int) * r_dst.size(), cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    direct_free(H);
    *why = "upload failed";
    return nullptr;
  }
  H->blocks = nblk;
  return H;
}

void direct_free(DirectHost* H) {
  if (!H) return;
  if (H->mem) cudaFree(H->mem);
  delete H;
}

const DirectDev* direct_desc(const DirectHost* H) { return &H->host_view; }

bool direct_fits(const DirectHost* H, int mixed, const char** why) {
  const DirectDev& D = H->host_view;
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  if (factor_smem(D.w, D.ns, vb) + 1024 > (size_t)smem_optin()) {
    *why = "the band window and separator rows exceed shared memory";
    return false;
  }
  if (solve_smem(D.nb, D.ns, D.w, vb) + 1024 > (size_t)smem_optin()) {
    *why = "the band vector exceeds shared memory";
    return false;
  }
  return true;
}

cudaError_t launch_direct_factor(const DevGraph& g, const DirectDev& D, int mixed, cudaStream_t s) {
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  const size_t bytes = (size_t)D.n_blocks * 49 * vb;
  cudaError_t e = cudaMemsetAsync(mixed ? (void*)D.s32 : (void*)D.s64, 0, bytes, s);
  if (e != cudaSuccess) return e;
  const long long tasks = (long long)D.n_targets * 49;
  const int blocks = (int)((tasks + 255) / 256);
  const size_t smem = factor_smem(D.w, D.ns, vb);
  if (mixed) {
    k_direct_assemble<float><<<blocks, 256, 0, s>>>(g, D);
    e = cudaFuncSetAttribute(k_direct_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct_factor<float><<<1, kFactorThreads, smem, s>>>(g, D);
  } else {
    k_direct_assemble<double><<<blocks, 256, 0, s>>>(g, D);
    e = cudaFuncSetAttribute(k_direct_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct_factor<double><<<1, kFactorThreads, smem, s>>>(g, D);
  }
  return cudaGetLastError();
}

cudaError_t launch_direct_solve(const DevGraph& g, const DirectDev& D, int mixed, int from_residual, cudaStream_t s) {
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  const size_t smem = solve_smem(D.nb, D.ns, D.w, vb);
  const int ring = solve_ring(vb);
  cudaError_t e;
  if (mixed) {
    e = cudaFuncSetAttribute(k_direct_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct_solve<float><<<1, kSolveThreads, smem, s>>>(g, D, from_residual, ring);
  } else {
    e = cudaFuncSetAttribute(k_direct_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct_solve<double><<<1, kSolveThreads, smem, s>>>(g, D, from_residual, ring);
  }
  return cudaGetLastError();
}

}  // namespace pgo
