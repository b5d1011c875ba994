// Loop-correction steps around the pose graph optimisation (Sec. III-B,
// "Loop Correction"): before the optimisation the keyframes connected to the
// keyframe that closed the loop take the loop's Sim(3) correction; after it
// (and for the connected keyframes' points before it) map points follow
// their reference keyframe.  Both are independent per keyframe and per point
// (the data parallelism of Sec. IV-D), so each is one thread per item:
//
//   k_copy_poses / k_propagate   S_k' = (S_k S_c^-1) S_c' for the listed k;
//   k_point_table                per keyframe r the similarity
//                                M_r = S_after[r]^-1 S_before[r] as x -> A x + b
//                                (A = (s_b / s_a) R_a^T R_b, b = R_a^T (t_b - t_a) / s_a);
//   k_apply_points               x' = A_r x + b_r (FP64: 9 fused multiply-adds
//                                and 3 adds per point, 52 bytes of traffic).
#include <cuda_runtime.h>

#include <cstdio>

#include "common.cuh"

namespace pgo {

namespace {

__device__ __forceinline__ Sim3T<double> load_pose8(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  const double2 c = __ldg(reinterpret_cast<const double2*>(p) + 2);
  const double2 d = __ldg(reinterpret_cast<const double2*>(p) + 3);
  Sim3T<double> S;
  S.q[0] = a.x; S.q[1] = a.y; S.q[2] = b.x; S.q[3] = b.y;
  S.t[0] = c.x; S.t[1] = c.y; S.t[2] = d.x; S.s = d.y;
  qnormalize(S.q);
  return S;
}

// k_copy_poses: out = in (pose8 rows, 16-byte vector copies).
__global__ void __launch_bounds__(256) k_copy_poses(int n, const double2* in, double2* out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * 4; t += gridDim.x * blockDim.x) out[t] = in[t];
}

// k_propagate: one thread per listed keyframe k, S_k' = (S_k S_c^-1) S_c',
// quaternion normalised with w >= 0.  Indices outside [0, n) are skipped
// and counted.
__global__ void __launch_bounds__(128) k_propagate(int n, const double* poses, int current, const double* corrected,
                                                   int n_conn, const int* conn, double* out, int* bad) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_conn) return;
  const int k = conn[a];
  if (k < 0 || k >= n) {
    if (bad) atomicAdd(bad, 1);
    return;
  }
  const Sim3T<double> Sc = load_pose8(poses + (size_t)current * 8);
  const Sim3T<double> Sn = load_pose8(corrected);
  const Sim3T<double> Sk = load_pose8(poses + (size_t)k * 8);
  Sim3T<double> R = compose(compose(Sk, inverse(Sc)), Sn);
  qnormalize(R.q);
  const double sg = R.q[3] < 0.0 ? -1.0 : 1.0;
  double* o = out + (size_t)k * 8;
  reinterpret_cast<double2*>(o)[0] = make_double2(sg * R.q[0], sg * R.q[1]);
  reinterpret_cast<double2*>(o)[1] = make_double2(sg * R.q[2], sg * R.q[3]);
  reinterpret_cast<double2*>(o)[2] = make_double2(R.t[0], R.t[1]);
  reinterpret_cast<double2*>(o)[3] = make_double2(R.t[2], R.s);
}

// Per-keyframe similarity of the point correction, 16 doubles per row:
// A (row-major 3x3), b, pad.
constexpr int kTableStride = 16;

__global__ void __launch_bounds__(128) k_point_table(int n, const double* before, const double* after,
                                                     double* table) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const Sim3T<double> Sb = load_pose8(before + (size_t)v * 8);
  const Sim3T<double> Sa = load_pose8(after + (size_t)v * 8);
  const Sim3T<double> M = compose(inverse(Sa), Sb);
  // A = s R(q) column by column: the images of the unit vectors
  double A[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double e[3] = {0.0, 0.0, 0.0}, col[3];
    e[c] = 1.0;
    qrot(M.q, e, col);
#pragma unroll
    for (int r = 0; r < 3; ++r) A[r * 3 + c] = M.s * col[r];
  }
  double2* row = reinterpret_cast<double2*>(table + (size_t)v * kTableStride);
  row[0] = make_double2(A[0], A[1]);
  row[1] = make_double2(A[2], A[3]);
  row[2] = make_double2(A[4], A[5]);
  row[3] = make_double2(A[6], A[7]);
  row[4] = make_double2(A[8], M.t[0]);
  row[5] = make_double2(M.t[1], M.t[2]);
  row[6] = make_double2(0.0, 0.0);
  row[7] = make_double2(0.0, 0.0);
}

// One thread per point: x' = A_r x + b_r; r < 0 copies the point, r >= n
// copies it and counts it.  The points are (P, 3) doubles; a block stages its
// 256 points (6 KB) through shared memory with 16-byte loads and stores so
// that the global accesses are whole coalesced lines (in place is allowed:
// every point is read before it is written, by the same block).
constexpr int kPointThreads = 256;

__global__ void __launch_bounds__(kPointThreads) k_apply_points(int n, int P, const double* X, const int* ref,
                                                                const double* table, double* out, int* bad) {
  __shared__ __align__(16) double sx[kPointThreads * 3];
  int nbad = 0;
  for (long long base = (long long)blockIdx.x * kPointThreads; base < P; base += (long long)gridDim.x * kPointThreads) {
    const int cnt = (int)min((long long)kPointThreads, (long long)P - base);
    const double* src = X + base * 3;
    // 16-byte staging when the block's span is 16-byte aligned (base even)
    const bool vec = ((reinterpret_cast<unsigned long long>(src) & 15ull) == 0) && ((cnt * 3) % 2 == 0);
    __syncthreads();
    if (vec) {
      for (int t = threadIdx.x; t < cnt * 3 / 2; t += kPointThreads)
        reinterpret_cast<double2*>(sx)[t] = __ldcs(reinterpret_cast<const double2*>(src) + t);
    } else {
      for (int t = threadIdx.x; t < cnt * 3; t += kPointThreads) sx[t] = __ldcs(src + t);
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int p = (int)base + threadIdx.x;
      const int r = __ldcs(ref + p);
      if (r >= 0 && r < n) {
        const double2* row = reinterpret_cast<const double2*>(table + (size_t)r * kTableStride);
        const double2 m0 = __ldg(row), m1 = __ldg(row + 1), m2 = __ldg(row + 2);
        const double2 m3 = __ldg(row + 3), m4 = __ldg(row + 4), m5 = __ldg(row + 5);
        // A = [m0.x m0.y m1.x; m1.y m2.x m2.y; m3.x m3.y m4.x], b = (m4.y, m5.x, m5.y)
        const double x = sx[threadIdx.x * 3], y = sx[threadIdx.x * 3 + 1], z = sx[threadIdx.x * 3 + 2];
        sx[threadIdx.x * 3 + 0] = fma(m0.x, x, fma(m0.y, y, fma(m1.x, z, m4.y)));
        sx[threadIdx.x * 3 + 1] = fma(m1.y, x, fma(m2.x, y, fma(m2.y, z, m5.x)));
        sx[threadIdx.x * 3 + 2] = fma(m3.x, x, fma(m3.y, y, fma(m4.x, z, m5.y)));
      } else if (r >= n) {
        ++nbad;
      }
    }
    __syncthreads();
    double* dst = out + base * 3;
    const bool vec_out = ((reinterpret_cast<unsigned long long>(dst) & 15ull) == 0) && ((cnt * 3) % 2 == 0);
    if (vec_out) {
      for (int t = threadIdx.x; t < cnt * 3 / 2; t += kPointThreads)
        __stcs(reinterpret_cast<double2*>(dst) + t, reinterpret_cast<const double2*>(sx)[t]);
    } else {
      for (int t = threadIdx.x; t < cnt * 3; t += kPointThreads) __stcs(dst + t, sx[t]);
    }
  }
  if (bad && nbad) atomicAdd(bad, nbad);
}

int num_sms_correction() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace

cudaError_t launch_propagate_correction(int n, const double* poses, int current, const double* corrected, int n_conn,
                                        const int* conn, double* out, int* bad, cudaStream_t s) {
  if (bad) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (n * 4 + 255) / 256;
  k_copy_poses<<<blocks, 256, 0, s>>>(n, reinterpret_cast<const double2*>(poses), reinterpret_cast<double2*>(out));
  if (n_conn > 0) k_propagate<<<(n_conn + 127) / 128, 128, 0, s>>>(n, poses, current, corrected, n_conn, conn, out, bad);
  return cudaGetLastError();
}

size_t point_table_bytes(int n) { return (size_t)n * kTableStride * sizeof(double); }

cudaError_t launch_correct_points(int n, const double* before, const double* after, int P, const double* X,
                                  const int* ref, double* table, double* out, int* bad, cudaStream_t s) {
  if (bad) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  k_point_table<<<(n + 127) / 128, 128, 0, s>>>(n, before, after, table);
  if (P > 0) {
    // resident blocks: 8 per SM at 256 threads; grid-stride beyond that
    const long long need = ((long long)P + kPointThreads - 1) / kPointThreads;
    const long long cap = (long long)num_sms_correction() * 8;
    const int blocks = (int)(need < cap ? need : cap);
    k_apply_points<<<blocks, kPointThreads, 0, s>>>(n, P, X, ref, table, out, bad);
  }
  return cudaGetLastError();
}

}  // namespace pgo
