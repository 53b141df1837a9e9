// Forward-mode dual numbers with K directions: a value and its K first
// derivatives.  Products follow the Leibniz rule, quotients the quotient rule;
// sqrt and sincos use their derivatives.  Used by the adjoint kernels, in FP64
// for the retraction and in FP32 for the per-edge terms.  Mixed operations
// take a scalar of the dual's own type, so an FP32 dual never widens to FP64.
#pragma once
#include <cuda_runtime.h>

template <class F, int K>
struct Dual {
  F v;
  F g[K];
};

template <class F, int K>
__device__ __forceinline__ Dual<F, K> dual_const(F v) {
  Dual<F, K> r;
  r.v = v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = F(0);
  return r;
}

template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator+(const Dual<F, K>& a, const Dual<F, K>& b) {
  Dual<F, K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = a.g[q] + b.g[q];
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator-(const Dual<F, K>& a, const Dual<F, K>& b) {
  Dual<F, K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = a.g[q] - b.g[q];
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator-(const Dual<F, K>& a) {
  Dual<F, K> r;
  r.v = -a.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = -a.g[q];
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator*(const Dual<F, K>& a, const Dual<F, K>& b) {
  Dual<F, K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = a.g[q] * b.v + a.v * b.g[q];
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator/(const Dual<F, K>& a, const Dual<F, K>& b) {
  Dual<F, K> r;
  const F ib = F(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = (a.g[q] - r.v * b.g[q]) * ib;
  return r;
}

// dual (op) scalar and scalar (op) dual
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator+(const Dual<F, K>& a, F b) {
  Dual<F, K> r = a;
  r.v = a.v + b;
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator+(F a, const Dual<F, K>& b) {
  return b + a;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator-(const Dual<F, K>& a, F b) {
  Dual<F, K> r = a;
  r.v = a.v - b;
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator-(F a, const Dual<F, K>& b) {
  Dual<F, K> r;
  r.v = a - b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = -b.g[q];
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator*(const Dual<F, K>& a, F b) {
  Dual<F, K> r;
  r.v = a.v * b;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = a.g[q] * b;
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator*(F a, const Dual<F, K>& b) {
  return b * a;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator/(F a, const Dual<F, K>& b) {
  Dual<F, K> r;
  const F ib = F(1) / b.v;
  r.v = a * ib;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = -r.v * b.g[q] * ib;
  return r;
}
template <class F, int K>
__device__ __forceinline__ Dual<F, K> operator/(const Dual<F, K>& a, F b) {
  return a * (F(1) / b);
}

// hooks used by the generic SE(3) retraction
template <class F, int K>
__device__ __forceinline__ F dpv_value(const Dual<F, K>& a) {
  return a.v;
}
template <int K>
__device__ __forceinline__ Dual<double, K> dpv_sqrt(const Dual<double, K>& a) {
  Dual<double, K> r;
  r.v = sqrt(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.g[q] = a.g[q] * h;
  return r;
}
template <int K>
__device__ __forceinline__ void dpv_sincos(const Dual<double, K>& a, Dual<double, K>& s, Dual<double, K>& c) {
  double sv, cv;
  sincos(a.v, &sv, &cv);
  s.v = sv;
  c.v = cv;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    s.g[q] = cv * a.g[q];
    c.g[q] = -sv * a.g[q];
  }
}
