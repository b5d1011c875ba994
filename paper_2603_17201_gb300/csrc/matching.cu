// Projection search and loop fusion (Sec. IV-D): map points projected into
// keyframes and matched to their features by 256-bit descriptor distance.
//
// Keyframe features live on the device in a frames object (the resident
// keyframe storage of Sec. IV-E): per keyframe, its features bucketed into a
// 64 x 48 image grid (counting sort at creation), with positions, octaves,
// descriptors and the caller's feature index in grid order.
//
// One call evaluates every (keyframe, map point) pair in parallel -- the data
// parallelism of Sec. IV-D, over points for the projection searches and over
// points and connected keyframes for loop fusion:
//   k_kf_setup      per keyframe: the pose in single precision, R(q / |q|) and
//                   the camera centre;
//   k_match_pairs   per pair: projection, image, distance and viewing-angle
//                   checks, predicted octave and search radius, then the grid
//                   cells around the projection, the best candidate by
//                   Hamming distance (ties to the lower feature index), and a
//                   claim on the chosen feature (64-bit atomicMin of
//                   (distance, point index));
//   k_match_resolve per pair: the conflict rule -- a search keeps the match
//                   only if it won the feature; fusion records the map point
//                   a loop point fuses with.
// Every floating-point step of the geometry is an explicit round-to-nearest
// single-precision operation in a fixed order (no contraction), so the
// decisions are those of the same IEEE operations on the host.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace pgo {

namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }

// Per keyframe: R (9), t (3), s, camera centre O (3) -- 16 floats.
__global__ void __launch_bounds__(64) k_kf_setup(int K, const double* poses, float* tab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double* p = poses + (size_t)k * 8;
  const float qx = __double2float_rn(p[0]), qy = __double2float_rn(p[1]);
  const float qz = __double2float_rn(p[2]), qw = __double2float_rn(p[3]);
  const float t0 = __double2float_rn(p[4]), t1 = __double2float_rn(p[5]), t2 = __double2float_rn(p[6]);
  const float s = __double2float_rn(p[7]);
  const float n = __fsqrt_rn(fa(fa(fa(fm(qx, qx), fm(qy, qy)), fm(qz, qz)), fm(qw, qw)));
  const float x = fd(qx, n), y = fd(qy, n), z = fd(qz, n), w = fd(qw, n);
  float R[9];
  R[0] = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
  R[1] = fm(2.0f, fs(fm(x, y), fm(w, z)));
  R[2] = fm(2.0f, fa(fm(x, z), fm(w, y)));
  R[3] = fm(2.0f, fa(fm(x, y), fm(w, z)));
  R[4] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
  R[5] = fm(2.0f, fs(fm(y, z), fm(w, x)));
  R[6] = fm(2.0f, fs(fm(x, z), fm(w, y)));
  R[7] = fm(2.0f, fa(fm(y, z), fm(w, x)));
  R[8] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(y, y))));
  // O = -(R^T t) / s
  const float ox = fd(-fa(fa(fm(R[0], t0), fm(R[3], t1)), fm(R[6], t2)), s);
  const float oy = fd(-fa(fa(fm(R[1], t0), fm(R[4], t1)), fm(R[7], t2)), s);
  const float oz = fd(-fa(fa(fm(R[2], t0), fm(R[5], t1)), fm(R[8], t2)), s);
  float4* o = reinterpret_cast<float4*>(tab + (size_t)k * 16);
  o[0] = make_float4(R[0], R[1], R[2], R[3]);
  o[1] = make_float4(R[4], R[5], R[6], R[7]);
  o[2] = make_float4(R[8], t0, t1, t2);
  o[3] = make_float4(s, ox, oy, oz);
}

__device__ __forceinline__ int hamming(const uint4& a0, const uint4& a1, const uint4& b0, const uint4& b1) {
  return __popc(a0.x ^ b0.x) + __popc(a0.y ^ b0.y) + __popc(a0.z ^ b0.z) + __popc(a0.w ^ b0.w) +
         __popc(a1.x ^ b1.x) + __popc(a1.y ^ b1.y) + __popc(a1.z ^ b1.z) + __popc(a1.w ^ b1.w);
}

// MODE 0: projection search, 1: loop fusion.  Thread per (keyframe
// blockIdx.y, point).
template <int MODE>
__global__ void __launch_bounds__(128) k_match_pairs(FramesDev F, MatchParams mp, const float* tab,
                                                     const unsigned char* matched, PointsDev pts, int* match,
                                                     int* dist, unsigned long long* win) {
  const int k = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pts.n) return;
  const size_t o = (size_t)k * pts.n + p;
  const int kbase = __ldg(F.kf_ptr + k);
  int best = -1, bd = 256;
  bool ok = true;
  if (MODE == 1) {
    // the keyframe already observes this point: skipped
    const int id = __ldg(pts.id + p);
    int lo = __ldg(F.obs_ptr + k), hi = __ldg(F.obs_ptr + k + 1);
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const int v = __ldg(F.obs_ids + mid);
      if (v < id) lo = mid + 1;
      else hi = mid;
    }
    if (lo < __ldg(F.obs_ptr + k + 1) && __ldg(F.obs_ids + lo) == id) ok = false;
  }
  if (ok) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(tab) + 4 * k);
    const float4 b = __ldg(reinterpret_cast<const float4*>(tab) + 4 * k + 1);
    const float4 c = __ldg(reinterpret_cast<const float4*>(tab) + 4 * k + 2);
    const float4 d = __ldg(reinterpret_cast<const float4*>(tab) + 4 * k + 3);
    const float R0 = a.x, R1 = a.y, R2 = a.z, R3 = a.w, R4 = b.x, R5 = b.y, R6 = b.z, R7 = b.w, R8 = c.x;
    const float t0 = c.y, t1 = c.z, t2 = c.w, s = d.x, ox = d.y, oy = d.z, oz = d.w;
    const float X0 = __ldg(pts.xyz + 3 * (size_t)p), X1 = __ldg(pts.xyz + 3 * (size_t)p + 1);
    const float X2 = __ldg(pts.xyz + 3 * (size_t)p + 2);
    const float px = fa(fm(s, fa(fa(fm(R0, X0), fm(R1, X1)), fm(R2, X2))), t0);
    const float py = fa(fm(s, fa(fa(fm(R3, X0), fm(R4, X1)), fm(R5, X2))), t1);
    const float pz = fa(fm(s, fa(fa(fm(R6, X0), fm(R7, X1)), fm(R8, X2))), t2);
    ok = pz > 0.0f;
    float u = 0.f, v = 0.f;
    if (ok) {
      u = fa(fd(fm(mp.fx, px), pz), mp.cx);
      v = fa(fd(fm(mp.fy, py), pz), mp.cy);
      ok = !(u < mp.min_x || u >= mp.max_x || v < mp.min_y || v >= mp.max_y);
    }
    float dist3 = 0.f, maxd = 0.f;
    if (ok) {
      const float dx = fs(X0, ox), dy = fs(X1, oy), dz = fs(X2, oz);
      dist3 = __fsqrt_rn(fa(fa(fm(dx, dx), fm(dy, dy)), fm(dz, dz)));
      const float mind = __ldg(pts.min_dist + p);
      maxd = __ldg(pts.max_dist + p);
      ok = !(dist3 < mind || dist3 > maxd);
      if (ok) {
        const float n0 = __ldg(pts.normal + 3 * (size_t)p), n1 = __ldg(pts.normal + 3 * (size_t)p + 1);
        const float n2 = __ldg(pts.normal + 3 * (size_t)p + 2);
        ok = !(fa(fa(fm(dx, n0), fm(dy, n1)), fm(dz, n2)) < fm(mp.cos_min, dist3));
      }
    }
    if (ok) {
      int level = 0;
      float sc = 1.0f;
      while (level < mp.n_levels - 1 && maxd > fm(dist3, sc)) {
        sc = fm(sc, mp.scale_factor);
        ++level;
      }
      const float r = fm(mp.th, sc);
      // grid cells that can hold a feature within r of (u, v), one cell of margin
      const int cx0 = max(0, (int)floorf((u - r - mp.min_x) * F.inv_cw) - 1);
      const int cx1 = min(kGridCols - 1, (int)floorf((u + r - mp.min_x) * F.inv_cw) + 1);
      const int cy0 = max(0, (int)floorf((v - r - mp.min_y) * F.inv_ch) - 1);
      const int cy1 = min(kGridRows - 1, (int)floorf((v + r - mp.min_y) * F.inv_ch) + 1);
      const uint4* pd = reinterpret_cast<const uint4*>(pts.desc) + 2 * (size_t)p;
      const uint4 q0 = __ldg(pd), q1 = __ldg(pd + 1);
      const int* cell = F.cell_ptr + (size_t)k * (kGridCols * kGridRows);
      for (int cy = cy0; cy <= cy1; ++cy) {
        const int j0 = __ldg(cell + cy * kGridCols + cx0), j1 = __ldg(cell + cy * kGridCols + cx1 + 1);
        for (int j = j0; j < j1; ++j) {   // the cells of one grid row are contiguous
          const int oc = __ldg(F.oct + j);
          if (oc < level - 1 || oc > level) continue;
          const int orig = __ldg(F.orig + j);
          if (MODE == 0 && matched && matched[kbase + orig]) continue;
          const float2 uv = __ldg(F.uv + j);
          if (!(fabsf(fs(uv.x, u)) < r) || !(fabsf(fs(uv.y, v)) < r)) continue;
          const uint4* fdsc = F.desc + 2 * (size_t)j;
          const int h = hamming(__ldg(fdsc), __ldg(fdsc + 1), q0, q1);
          if (h < bd || (h == bd && orig < best)) {
            bd = h;
            best = orig;
          }
        }
      }
    }
  }
  const int m = (best >= 0 && bd <= mp.th_low) ? best : -1;
  match[o] = m;
  dist[o] = bd;
  if (m >= 0) atomicMin(win + kbase + m, ((unsigned long long)(unsigned)bd << 32) | (unsigned)p);
}

template <int MODE>
__global__ void __launch_bounds__(128) k_match_resolve(FramesDev F, PointsDev pts, int* match, int* dist, int* fuse,
                                                       const unsigned long long* win) {
  const int k = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pts.n) return;
  const size_t o = (size_t)k * pts.n + p;
  const int m = match[o];
  if (MODE == 1) {
    int f = -1;
    if (m >= 0) {
      const int kbase = __ldg(F.kf_ptr + k);
      const int existing = __ldg(F.mp + kbase + m);
      const unsigned w = (unsigned)(win[kbase + m] & 0xffffffffull);
      f = existing >= 0 ? existing : ((int)w != p ? __ldg(pts.id + w) : -1);
    }
    fuse[o] = f;
    return;
  }
  if (m < 0) return;
  const int kbase = __ldg(F.kf_ptr + k);
  const unsigned w = (unsigned)(win[kbase + m] & 0xffffffffull);
  if ((int)w != p) {
    match[o] = -1;
    dist[o] = 256;
  }
}

}  // namespace

cudaError_t launch_project_match(const FramesDev& F, const MatchParams& mp, int mode, const double* poses,
                                 const unsigned char* matched, const PointsDev& pts, int* match, int* dist, int* fuse,
                                 cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(F.win, 0xff, sizeof(unsigned long long) * (size_t)(F.n_features > 0 ? F.n_features : 1), s);
  if (e != cudaSuccess) return e;
  k_kf_setup<<<(F.K + 63) / 64, 64, 0, s>>>(F.K, poses, F.kf_tab);
  if (pts.n > 0) {
    dim3 grid((pts.n + 127) / 128, F.K);
    if (mode == 0) {
      k_match_pairs<0><<<grid, 128, 0, s>>>(F, mp, F.kf_tab, matched, pts, match, dist, F.win);
      k_match_resolve<0><<<grid, 128, 0, s>>>(F, pts, match, dist, fuse, F.win);
    } else {
      k_match_pairs<1><<<grid, 128, 0, s>>>(F, mp, F.kf_tab, nullptr, pts, match, dist, F.win);
      k_match_resolve<1><<<grid, 128, 0, s>>>(F, pts, match, dist, fuse, F.win);
    }
  }
  return cudaGetLastError();
}

}  // namespace pgo
