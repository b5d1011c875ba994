// Device Sim(3) arithmetic for the essential-graph residuals (Sec. III-B,
// IV-F).  A pose S = (q, t, s) maps world to camera, x -> s R(q) x + t.
// Tangent vectors are ordered [omega(3), upsilon(3), sigma(1)] and poses are
// perturbed on the left, S <- exp(xi) S.
//
// Everything is templated on the scalar S (double, float or a forward-mode
// dual) so that one log map serves the residual, its exact Jacobian and the
// second derivatives of the implicit adjoint.  Branch decisions read the
// value part only; every branch is a smooth formula (the small-angle and
// small-scale branches are truncated Taylor series of the same function), so
// the derivatives carried by the duals stay consistent across thresholds.
#pragma once
#include "dual.cuh"

namespace pgo {

template <class S>
struct Sim3T {
  S q[4];  // x, y, z, w
  S t[3];
  S s;
};

// Hamilton product a * b of quaternions stored (x, y, z, w).
template <class S>
__device__ __forceinline__ void qmul(const S* a, const S* b, S* c) {
  S x = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  S y = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  S z = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  S w = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
  c[0] = x; c[1] = y; c[2] = z; c[3] = w;
}

// v' = R(q) v for a unit quaternion: v + w t + u x t with t = 2 u x v.
template <class S>
__device__ __forceinline__ void qrot(const S* q, const S* v, S* out) {
  S tx = scal(q[1] * v[2] - q[2] * v[1], 2.0);
  S ty = scal(q[2] * v[0] - q[0] * v[2], 2.0);
  S tz = scal(q[0] * v[1] - q[1] * v[0], 2.0);
  S ox = v[0] + q[3] * tx + (q[1] * tz - q[2] * ty);
  S oy = v[1] + q[3] * ty + (q[2] * tx - q[0] * tz);
  S oz = v[2] + q[3] * tz + (q[0] * ty - q[1] * tx);
  out[0] = ox; out[1] = oy; out[2] = oz;
}

// a * b = (q_a q_b, s_a R_a t_b + t_a, s_a s_b)
template <class S>
__device__ __forceinline__ Sim3T<S> compose(const Sim3T<S>& a, const Sim3T<S>& b) {
  Sim3T<S> c;
  qmul(a.q, b.q, c.q);
  S rt[3];
  qrot(a.q, b.t, rt);
#pragma unroll
  for (int k = 0; k < 3; ++k) c.t[k] = a.s * rt[k] + a.t[k];
  c.s = a.s * b.s;
  return c;
}

// a^-1 = (q*, -R^T t / s, 1 / s)
template <class S>
__device__ __forceinline__ Sim3T<S> inverse(const Sim3T<S>& a) {
  Sim3T<S> c;
  c.q[0] = -a.q[0]; c.q[1] = -a.q[1]; c.q[2] = -a.q[2]; c.q[3] = a.q[3];
  S rt[3];
  qrot(c.q, a.t, rt);
  S inv = lift<S>(1.0) / a.s;
#pragma unroll
  for (int k = 0; k < 3; ++k) c.t[k] = -(rt[k] * inv);
  c.s = inv;
  return c;
}

// Reciprocals 1/m, m = 1..76 (c_rcp[m - 1]), rounded once by the compiler:
// the moment series below scales by them with a loop-dependent m, where a
// division would cost a full FP64 divide per term.
static __device__ __constant__ double c_rcp[76] = {
    1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8,
    1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16,
    1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24,
    1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32,
    1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40,
    1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48,
    1.0 / 49, 1.0 / 50, 1.0 / 51, 1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55, 1.0 / 56,
    1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61, 1.0 / 62, 1.0 / 63, 1.0 / 64,
    1.0 / 65, 1.0 / 66, 1.0 / 67, 1.0 / 68, 1.0 / 69, 1.0 / 70, 1.0 / 71, 1.0 / 72,
    1.0 / 73, 1.0 / 74, 1.0 / 75, 1.0 / 76};

// Moments I_n(sigma) = int_0^1 tau^n e^(sigma tau) dtau for n = 1..10 from
// the power series sum_k sigma^k / (k! (n + k + 1)), summed until the term
// is below 1e-18 of the leading moment (at most 64 terms).
template <class S>
__device__ __forceinline__ void moments(const S& sigma, S* I /* I[1..10] in I[0..9] */) {
#pragma unroll
  for (int n = 0; n < 10; ++n) I[n] = lift<S>(1.0 / (n + 2));
  S term = lift<S>(1.0);
  double av = fabs((double)val(sigma));
  double mag = 1.0;
  for (int k = 1; k < 64; ++k) {
    term = scal(term * sigma, c_rcp[k - 1]);
    mag *= av * c_rcp[k - 1];
#pragma unroll
    for (int n = 0; n < 10; ++n) I[n] = I[n] + scal(term, c_rcp[n + k + 1]);
    if (mag < 1e-19) break;
  }
}

// Coefficients of W = A I + B w^ + C w^2 with W = int_0^1 exp(tau (w^ + sigma I)) dtau,
// given th2 = |w|^2:
//   A = (e^sigma - 1) / sigma
//   B = [e^sigma (sigma sin th - th cos th) + th] / (th (sigma^2 + th^2))
//   C = [A - (e^sigma (sigma cos th + th sin th) - sigma) / (sigma^2 + th^2)] / th^2
// with the Taylor series in th^2 over the moments I_n(sigma) below th = 0.1:
//   B = sum_m (-1)^m th^2m I_{2m+1} / (2m+1)!,
//   C = sum_m (-1)^m th^2m I_{2m+2} / (2m+2)!.
template <class S>
__device__ __forceinline__ void wcoeffs(const S& th2, const S& sigma, S& A, S& B, S& C) {
  double sv = (double)val(sigma);
  if (fabs(sv) < 1e-4) {
    // (e^s - 1)/s = 1 + s/2 + s^2/6 + s^3/24 + s^4/120
    A = addc(sigma * (addc(sigma * (addc(sigma * (addc(scal(sigma, 1.0 / 120.0), 1.0 / 24.0)), 1.0 / 6.0)), 0.5)), 1.0);
  } else {
    A = dexpm1(sigma) / sigma;
  }
  if ((double)val(th2) < 0.01) {
    S I[10];
    moments(sigma, I);
    // B: I1 - th2 I3/6 + th2^2 I5/120 - th2^3 I7/5040 + th2^4 I9/362880
    B = I[0] + th2 * (scal(I[2], -1.0 / 6.0) + th2 * (scal(I[4], 1.0 / 120.0) +
          th2 * (scal(I[6], -1.0 / 5040.0) + th2 * scal(I[8], 1.0 / 362880.0))));
    // C: I2/2 - th2 I4/24 + th2^2 I6/720 - th2^3 I8/40320 + th2^4 I10/3628800
    C = scal(I[1], 0.5) + th2 * (scal(I[3], -1.0 / 24.0) + th2 * (scal(I[5], 1.0 / 720.0) +
          th2 * (scal(I[7], -1.0 / 40320.0) + th2 * scal(I[9], 1.0 / 3628800.0))));
  } else {
    S th = dsqrt(th2);
    S sn = dsin(th), cs = dcos(th), es = dexp(sigma);
    S den = sigma * sigma + th2;
    B = (es * (sigma * sn - th * cs) + th) / (th * den);
    C = (A - (es * (sigma * cs + th * sn) - sigma) / den) / th2;
  }
}

// log of (q, t, s), q of unit norm: omega = rotation vector of q,
// sigma = ln s, upsilon = W(omega, sigma)^-1 t.
template <class S>
__device__ __forceinline__ void sim3_log(const Sim3T<S>& T, S* xi) {
  S qx = T.q[0], qy = T.q[1], qz = T.q[2], qw = T.q[3];
  if ((double)val(qw) < 0.0) { qx = -qx; qy = -qy; qz = -qz; qw = -qw; }
  S n2 = qx * qx + qy * qy + qz * qz;
  S w2 = qw * qw;
  S f;  // omega = f * (qx, qy, qz), f = 2 atan2(|v|, w) / |v|
  if ((double)val(n2) < 1e-6 * (double)val(w2)) {
    // 2 atan(x)/(x w) with x^2 = n2/w2: (2/w) (1 - x^2/3 + x^4/5 - x^6/7)
    S x2 = n2 / w2;
    S poly = addc(x2 * (addc(x2 * (addc(scal(x2, -1.0 / 7.0), 1.0 / 5.0)), -1.0 / 3.0)), 1.0);
    f = scal(poly / qw, 2.0);
  } else {
    S n = dsqrt(n2);
    f = scal(datan2(n, qw), 2.0) / n;
  }
  S w[3] = {f * qx, f * qy, f * qz};
  S th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  S sigma = dlog(T.s);
  S A, B, C;
  wcoeffs(th2, sigma, A, B, C);
  // W^-1 = a I + b w^ + c w^2 with a = 1/A,
  // b = -a A B / det, c = a (B^2 - P C) / det, P = A - th2 C, det = P^2 + th2 B^2
  S a = lift<S>(1.0) / A;
  S P = A - th2 * C;
  S det = P * P + th2 * B * B;
  S b = -(a * A * B) / det;
  S c = a * (B * B - P * C) / det;
  S wxt[3] = {w[1] * T.t[2] - w[2] * T.t[1], w[2] * T.t[0] - w[0] * T.t[2], w[0] * T.t[1] - w[1] * T.t[0]};
  S wwxt[3] = {w[1] * wxt[2] - w[2] * wxt[1], w[2] * wxt[0] - w[0] * wxt[2], w[0] * wxt[1] - w[1] * wxt[0]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xi[k] = w[k];
    xi[3 + k] = a * T.t[k] + b * wxt[k] + c * wwxt[k];
  }
  xi[6] = sigma;
}

// exp of xi (plain FP64): q = (sin(th/2) w/th, cos(th/2)), s = e^sigma,
// t = W(w, sigma) upsilon.
__device__ __forceinline__ Sim3T<double> sim3_exp(const double* xi) {
  Sim3T<double> E;
  double th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
  double h;   // sin(th/2)/th
  double cw;  // cos(th/2)
  if (th2 < 1e-8) {
    h = 0.5 - th2 / 48.0 + th2 * th2 / 3840.0;
    cw = 1.0 - th2 / 8.0 + th2 * th2 / 384.0;
  } else {
    double th = sqrt(th2);
    double sh, ch;
    sincos(0.5 * th, &sh, &ch);
    h = sh / th;
    cw = ch;
  }
  E.q[0] = h * xi[0]; E.q[1] = h * xi[1]; E.q[2] = h * xi[2]; E.q[3] = cw;
  double A, B, C;
  wcoeffs<double>(th2, xi[6], A, B, C);
  const double* w = xi;
  const double* u = xi + 3;
  double wxu[3] = {w[1] * u[2] - w[2] * u[1], w[2] * u[0] - w[0] * u[2], w[0] * u[1] - w[1] * u[0]};
  double wwxu[3] = {w[1] * wxu[2] - w[2] * wxu[1], w[2] * wxu[0] - w[0] * wxu[2], w[0] * wxu[1] - w[1] * wxu[0]};
#pragma unroll
  for (int k = 0; k < 3; ++k) E.t[k] = A * u[k] + B * wxu[k] + C * wwxu[k];
  E.s = exp(xi[6]);
  return E;
}

// Rotation matrix of a unit quaternion (row-major).
template <class S>
__device__ __forceinline__ void qmat(const S* q, S* R) {
  S x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// Seed the 7 left-generator directions on T: T(eps) = (I + sum eps_k G_k) T,
// i.e. dq = 1/2 (e_k, 0) q, dt = e_k x t (rotations), dt = e_k (translations),
// ds = s, dt = t (scale).
template <class T>
__device__ __forceinline__ Sim3T<Dual<T, 7>> seed_left(const Sim3T<T>& P) {
  Sim3T<Dual<T, 7>> D;
#pragma unroll
  for (int c = 0; c < 4; ++c) D.q[c] = dconst<T, 7>(P.q[c]);
#pragma unroll
  for (int c = 0; c < 3; ++c) D.t[c] = dconst<T, 7>(P.t[c]);
  D.s = dconst<T, 7>(P.s);
  const T* v = P.q;
  const T qw = P.q[3];
  // rotation generators k = 0, 1, 2: (e_k, 0) * q = (w e_k + e_k x v, -v_k)
  // e_0 x v = (0, -v2, v1), e_1 x v = (v2, 0, -v0), e_2 x v = (-v1, v0, 0)
  D.q[0].d[0] = scal(qw, 0.5);      D.q[1].d[0] = scal(-v[2], 0.5);  D.q[2].d[0] = scal(v[1], 0.5);  D.q[3].d[0] = scal(-v[0], 0.5);
  D.q[0].d[1] = scal(v[2], 0.5);    D.q[1].d[1] = scal(qw, 0.5);     D.q[2].d[1] = scal(-v[0], 0.5); D.q[3].d[1] = scal(-v[1], 0.5);
  D.q[0].d[2] = scal(-v[1], 0.5);   D.q[1].d[2] = scal(v[0], 0.5);   D.q[2].d[2] = scal(qw, 0.5);    D.q[3].d[2] = scal(-v[2], 0.5);
  const T* t = P.t;
  D.t[0].d[1] = t[2];  D.t[0].d[2] = -t[1];
  D.t[1].d[0] = -t[2]; D.t[1].d[2] = t[0];
  D.t[2].d[0] = t[1];  D.t[2].d[1] = -t[0];
  D.t[0].d[3] = lift<T>(1.0); D.t[1].d[4] = lift<T>(1.0); D.t[2].d[5] = lift<T>(1.0);
  D.t[0].d[6] = t[0]; D.t[1].d[6] = t[1]; D.t[2].d[6] = t[2];
  D.s.d[6] = P.s;
  return D;
}

template <class S>
__device__ __forceinline__ void qnormalize(S* q) {
  S inv = lift<S>(1.0) / dsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  q[0] = q[0] * inv; q[1] = q[1] * inv; q[2] = q[2] * inv; q[3] = q[3] * inv;
}

}  // namespace pgo
