// Precision accessors of the multigrid hierarchy (shared by the setup and
// the V-cycle inside the PCG kernel).
#pragma once
#include "internal.cuh"

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
  static __device__ __forceinline__ float* cinv(const AmgDev& A) { return A.cinv32; }
  static __device__ __forceinline__ float* pw(const AmgDev& A, int k) { return A.pw32[k]; }
  static __device__ __forceinline__ float* vr(const AmgLevel& L) { return L.vr32; }
  static __device__ __forceinline__ float* vx(const AmgLevel& L) { return L.vx32; }
  static __device__ __forceinline__ float* vs(const AmgLevel& L) { return L.vs32; }
  static __device__ __forceinline__ float* vy(const AmgLevel& L) { return L.vy32; }
  static __device__ __forceinline__ float* pv(const AmgLevel& L) { return L.pv32; }
};

}  // namespace pgo
