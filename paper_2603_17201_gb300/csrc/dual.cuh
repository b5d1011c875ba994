// Forward-mode dual numbers for the device-side automatic differentiation of
// the Sim(3) log map (the paper's Graphite backend differentiates its edge
// residuals automatically, Sec. IV-F).  Dual<T, N> carries a value and N
// tangent components; T may itself be a Dual (nested forward mode gives the
// second derivatives the implicit adjoint needs).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace pgo {

template <class T, int N>
struct Dual {
  T v;
  T d[N];
};

// ---- value of any (possibly nested) scalar: used for branch decisions ----
__host__ __device__ __forceinline__ double val(double x) { return x; }
__host__ __device__ __forceinline__ float val(float x) { return x; }
template <class T, int N>
__host__ __device__ __forceinline__ auto val(const Dual<T, N>& x) { return val(x.v); }

// ---- plain-scalar math (overloads picked by the generic code below) ----
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double datan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float datan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ float dlog(float x) { return logf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float dexpm1(float x) { return expm1f(x); }
__device__ __forceinline__ double dsin(double x) { return sin(x); }
__device__ __forceinline__ float dsin(float x) { return sinf(x); }
__device__ __forceinline__ double dcos(double x) { return cos(x); }
__device__ __forceinline__ float dcos(float x) { return cosf(x); }

template <class T, int N>
__device__ __forceinline__ Dual<T, N> dconst(const T& c);

// Promote a plain constant to scalar type S (double/float or any Dual).
template <class S>
struct Lift {
  __device__ __forceinline__ static S from(double c) { return S(c); }
};
template <class T, int N>
struct Lift<Dual<T, N>> {
  __device__ __forceinline__ static Dual<T, N> from(double c) { return dconst<T, N>(Lift<T>::from(c)); }
};
template <class S>
__device__ __forceinline__ S lift(double c) { return Lift<S>::from(c); }

// ---- construction ----
template <class D>
struct DualTraits;
template <class T, int N>
struct DualTraits<Dual<T, N>> {
  using base = T;
  static constexpr int n = N;
};

template <class T, int N>
__device__ __forceinline__ Dual<T, N> dconst(const T& c) {
  Dual<T, N> r;
  r.v = c;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = lift<T>(0.0);
  return r;
}

// ---- arithmetic ----
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  T inv = lift<T>(1.0) / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
  return r;
}
// mixed with the base scalar
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, const T& c) {
  Dual<T, N> r;
  r.v = a.v * c;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * c;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const T& c, const Dual<T, N>& a) { return a * c; }
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, const T& c) {
  Dual<T, N> r = a;
  r.v = a.v + c;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const T& c, const Dual<T, N>& a) { return a + c; }
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, const T& c) {
  Dual<T, N> r = a;
  r.v = a.v - c;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const T& c, const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = c - a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, const T& c) {
  T inv = lift<T>(1.0) / c;
  return a * inv;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const T& c, const Dual<T, N>& b) {
  Dual<T, N> r;
  T inv = lift<T>(1.0) / b.v;
  r.v = c * inv;
  T f = -r.v * inv;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = f * b.d[k];
  return r;
}

// Scale by / add a plain double constant without widening it to a dual.
__device__ __forceinline__ double scal(double x, double c) { return x * c; }
__device__ __forceinline__ float scal(float x, double c) { return x * (float)c; }
template <class T, int N>
__device__ __forceinline__ Dual<T, N> scal(const Dual<T, N>& x, double c) {
  Dual<T, N> r;
  r.v = scal(x.v, c);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = scal(x.d[k], c);
  return r;
}
__device__ __forceinline__ double addc(double x, double c) { return x + c; }
__device__ __forceinline__ float addc(float x, double c) { return x + (float)c; }
template <class T, int N>
__device__ __forceinline__ Dual<T, N> addc(const Dual<T, N>& x, double c) {
  Dual<T, N> r = x;
  r.v = addc(x.v, c);
  return r;
}

// ---- elementary functions (chain rule) ----
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dsqrt(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dsqrt(a.v);
  T f = lift<T>(0.5) / r.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * f;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> datan2(const Dual<T, N>& y, const Dual<T, N>& x) {
  Dual<T, N> r;
  r.v = datan2(y.v, x.v);
  T inv = lift<T>(1.0) / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * inv;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dlog(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dlog(a.v);
  T inv = lift<T>(1.0) / a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * inv;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dexp(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dexp(a.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * r.v;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dexpm1(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dexpm1(a.v);
  T e = addc(r.v, 1.0);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * e;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dsin(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dsin(a.v);
  T c = dcos(a.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * c;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dcos(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dcos(a.v);
  T s = -dsin(a.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * s;
  return r;
}

}  // namespace pgo
