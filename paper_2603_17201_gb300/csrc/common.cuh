// Shared device helpers: vector types, pose loads, deterministic reductions.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "sim3.cuh"

namespace pgo {

__device__ __forceinline__ Sim3T<double> load_pose(const DevGraph& g, int buf, int v) {
  D4 q = g.pq[buf][v];
  D4 t = g.pt[buf][v];
  Sim3T<double> P;
  P.q[0] = q.x; P.q[1] = q.y; P.q[2] = q.z; P.q[3] = q.w;
  P.t[0] = t.x; P.t[1] = t.y; P.t[2] = t.z; P.s = t.w;
  return P;
}

__device__ __forceinline__ void store_pose(const DevGraph& g, int buf, int v, const Sim3T<double>& P) {
  D4 q = {P.q[0], P.q[1], P.q[2], P.q[3]};
  D4 t = {P.t[0], P.t[1], P.t[2], P.s};
  g.pq[buf][v] = q;
  g.pt[buf][v] = t;
}

__device__ __forceinline__ Sim3T<double> load_meas(const DevGraph& g, int e) {
  D4 q = g.zq[e];
  D4 t = g.zt[e];
  Sim3T<double> P;
  P.q[0] = q.x; P.q[1] = q.y; P.q[2] = q.z; P.q[3] = q.w;
  P.t[0] = t.x; P.t[1] = t.y; P.t[2] = t.z; P.s = t.w;
  return P;
}

// Warp-level sum.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of K values per thread into sh[K] (thread 0 holds the
// result after the call; every thread must call).  Deterministic: fixed
// shuffle tree inside each warp, fixed-order sum over warps.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh /* >= 32*K */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w * K + k];
      v[k] = s;
    }
  }
  __syncthreads();
}

template <int K>
__device__ __forceinline__ void block_max(double (&v)[K], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_max(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = sh[k];
      for (int w = 1; w < nw; ++w) s = fmax(s, sh[w * K + k]);
      v[k] = s;
    }
  }
  __syncthreads();
}

// Publish this block's K partial values and take a ticket.  Returns true (in
// every thread) for the block that arrives last; that block then sees every
// other block's partials (read them with __ldcg).  The ticket is reset by
// the last block so the kernel can be relaunched.
template <int K>
__device__ __forceinline__ bool publish_partials(const double (&v)[K], double* partial,
                                                 unsigned* ticket) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partial[blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
    if (is_last) {
      __threadfence();
      *ticket = 0u;
    }
  }
  __syncthreads();
  return is_last;
}

// Fixed-order sum of the published partials by the last block (all threads
// participate; thread 0 gets the result).
template <int K>
__device__ __forceinline__ void gather_partials_sum(const double* partial, double (&out)[K],
                                                    double* sh) {
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = 0.0;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] += __ldcg(partial + b * K + k);
  }
  block_sum<K>(out, sh);
}

template <int K>
__device__ __forceinline__ void gather_partials_max(const double* partial, double (&out)[K],
                                                    double* sh) {
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = 0.0;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = fmax(out[k], __ldcg(partial + b * K + k));
  }
  block_max<K>(out, sh);
}

__device__ __forceinline__ void set_cond(unsigned long long h, bool v) {
  if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v ? 1u : 0u);
}

}  // namespace pgo
