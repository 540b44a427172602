// dual.cuh -- forward-mode derivatives by operator overloading: a value and
// its derivatives with respect to K inputs, FP64.  Each elementary function
// applies its own derivative (chain rule); used where a short sequential
// computation needs the exact Jacobian with respect to a few parameters
// (the single-orbit fits).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace nb {

template <int K>
struct Dual {
  double v;
  double d[K];
};

template <int K>
__device__ __forceinline__ Dual<K> dconst(double c) {
  Dual<K> r;
  r.v = c;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = 0.0;
  return r;
}

// the input k (seed d_k = 1)
template <int K>
__device__ __forceinline__ Dual<K> dvar(double c, int k) {
  Dual<K> r = dconst<K>(c);
  r.d[k] = 1.0;
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator*(double c, const Dual<K>& a) {
  Dual<K> r;
  r.v = c * a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = c * a.d[k];
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator+(double c, const Dual<K>& a) {
  Dual<K> r = a;
  r.v += c;
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, double c) {
  Dual<K> r = a;
  r.v -= c;
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> operator-(double c, const Dual<K>& a) {
  return c + (-a);
}

// f(a) with f(a.v) = fv and f'(a.v) = fp
template <int K>
__device__ __forceinline__ Dual<K> dchain(const Dual<K>& a, double fv, double fp) {
  Dual<K> r;
  r.v = fv;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = fp * a.d[k];
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> dsqrt(const Dual<K>& a) {
  const double s = sqrt(a.v);
  return dchain(a, s, 0.5 / s);
}

template <int K>
__device__ __forceinline__ Dual<K> dlog1p(const Dual<K>& a) {
  return dchain(a, log1p(a.v), 1.0 / (1.0 + a.v));
}

template <int K>
__device__ __forceinline__ Dual<K> datan2(const Dual<K>& y, const Dual<K>& x) {
  // d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
  Dual<K> r;
  r.v = atan2(y.v, x.v);
  const double q = 1.0 / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * q;
  return r;
}

template <int K>
__device__ __forceinline__ Dual<K> dasin(const Dual<K>& a) {
  return dchain(a, asin(a.v), 1.0 / sqrt(1.0 - a.v * a.v));
}

template <int K>
__device__ __forceinline__ Dual<K> dsin(const Dual<K>& a) {
  return dchain(a, sin(a.v), cos(a.v));
}

template <int K>
__device__ __forceinline__ Dual<K> dcos(const Dual<K>& a) {
  return dchain(a, cos(a.v), -sin(a.v));
}

}  // namespace nb

namespace nb {

// Second order: value, gradient and the upper triangle of the Hessian with
// respect to K inputs (hyper-dual numbers); products and the chain rule
// carry the second derivatives exactly:
//   (ab)_ij = a_ij b + a_i b_j + a_j b_i + a b_ij,
//   f(a)_ij = f'(a) a_ij + f''(a) a_i a_j.
template <int K>
struct HDual {
  static constexpr int NH = K * (K + 1) / 2;
  double v;
  double d[K];
  double h[NH];  // (i, j), i <= j, row by row
};

template <int K>
__device__ __forceinline__ HDual<K> hconst(double c) {
  HDual<K> r;
  r.v = c;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = 0.0;
#pragma unroll
  for (int k = 0; k < HDual<K>::NH; ++k) r.h[k] = 0.0;
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> operator+(const HDual<K>& a, const HDual<K>& b) {
  HDual<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
#pragma unroll
  for (int k = 0; k < HDual<K>::NH; ++k) r.h[k] = a.h[k] + b.h[k];
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> operator-(const HDual<K>& a) {
  HDual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
#pragma unroll
  for (int k = 0; k < HDual<K>::NH; ++k) r.h[k] = -a.h[k];
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> operator-(const HDual<K>& a, const HDual<K>& b) {
  return a + (-b);
}

template <int K>
__device__ __forceinline__ HDual<K> operator*(const HDual<K>& a, const HDual<K>& b) {
  HDual<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  int q = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = i; j < K; ++j, ++q)
      r.h[q] = a.h[q] * b.v + a.d[i] * b.d[j] + a.d[j] * b.d[i] + a.v * b.h[q];
  return r;
}

// f(a) with f(a.v) = fv, f' = f1, f'' = f2
template <int K>
__device__ __forceinline__ HDual<K> hchain(const HDual<K>& a, double fv, double f1, double f2) {
  HDual<K> r;
  r.v = fv;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = f1 * a.d[k];
  int q = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = i; j < K; ++j, ++q) r.h[q] = f1 * a.h[q] + f2 * a.d[i] * a.d[j];
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> hrcp(const HDual<K>& a) {
  const double i = 1.0 / a.v;
  return hchain(a, i, -i * i, 2.0 * i * i * i);
}

template <int K>
__device__ __forceinline__ HDual<K> operator/(const HDual<K>& a, const HDual<K>& b) {
  return a * hrcp(b);
}

template <int K>
__device__ __forceinline__ HDual<K> operator*(double c, const HDual<K>& a) {
  HDual<K> r;
  r.v = c * a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = c * a.d[k];
#pragma unroll
  for (int k = 0; k < HDual<K>::NH; ++k) r.h[k] = c * a.h[k];
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> operator+(double c, const HDual<K>& a) {
  HDual<K> r = a;
  r.v += c;
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> operator-(const HDual<K>& a, double c) {
  HDual<K> r = a;
  r.v -= c;
  return r;
}

template <int K>
__device__ __forceinline__ HDual<K> operator-(double c, const HDual<K>& a) {
  return c + (-a);
}

template <int K>
__device__ __forceinline__ HDual<K> dsqrt(const HDual<K>& a) {
  const double s = sqrt(a.v);
  return hchain(a, s, 0.5 / s, -0.25 / (s * a.v));
}

template <int K>
__device__ __forceinline__ HDual<K> dlog1p(const HDual<K>& a) {
  const double i = 1.0 / (1.0 + a.v);
  return hchain(a, log1p(a.v), i, -i * i);
}

template <int K>
__device__ __forceinline__ HDual<K> dasin(const HDual<K>& a) {
  const double w = 1.0 - a.v * a.v;
  const double iw = 1.0 / sqrt(w);
  return hchain(a, asin(a.v), iw, a.v * iw / w);
}

// atan2(y, x): first derivatives (x, -y)/q, second derivatives
// d2/dy2 = -2xy/q^2, d2/dx2 = 2xy/q^2, d2/dxdy = (y^2 - x^2)/q^2, q = x^2 + y^2
template <int K>
__device__ __forceinline__ HDual<K> datan2(const HDual<K>& y, const HDual<K>& x) {
  HDual<K> r;
  const double q = x.v * x.v + y.v * y.v, iq = 1.0 / q, iq2 = iq * iq;
  const double fy = x.v * iq, fx = -y.v * iq;
  const double fyy = -2.0 * x.v * y.v * iq2, fxx = 2.0 * x.v * y.v * iq2;
  const double fxy = (y.v * y.v - x.v * x.v) * iq2;
  r.v = atan2(y.v, x.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = fy * y.d[k] + fx * x.d[k];
  int p = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = i; j < K; ++j, ++p)
      r.h[p] = fy * y.h[p] + fx * x.h[p] + fyy * y.d[i] * y.d[j] + fxx * x.d[i] * x.d[j] +
               fxy * (x.d[i] * y.d[j] + y.d[i] * x.d[j]);
  return r;
}

}  // namespace nb
