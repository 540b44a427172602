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
