// SE(3) retraction T <- Exp(xi) T in FP64 (device function).
//
// Exp(xi) = [ R(phi)  V(phi) rho ; 0 1 ] for xi = (rho, phi), th = |phi|:
//   R(phi) from the unit quaternion (a phi, c), a = sin(th/2)/th, c = cos(th/2);
//   V = I + B [phi]x + C [phi]x^2,  B = (1 - cos th)/th^2,  C = (th - sin th)/th^3.
// Gauss-Newton steps are small, so below th = 0.1 the four coefficients are
// evaluated as their Maclaurin series in th^2 up to th^8 (the first omitted
// term is below 3e-19 there): pure multiply-adds, no transcendental calls.
// Above, the closed forms are used with B = 2 sin^2(th/2) / th^2.
#pragma once
#include "internal.cuh"

__device__ __forceinline__ double dpv_value(double x) { return x; }
__device__ __forceinline__ double dpv_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void dpv_sincos(double x, double& s, double& c) { sincos(x, &s, &c); }
template <class T>
__device__ __forceinline__ void dpv_quat_rot_t(const T* q, T* R) {
  const T x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - z * w); R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w); R[7] = 2.0 * (y * z + x * w); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// T is double for the step itself; the adjoint instantiates it with FP64 dual
// numbers (operators +, -, *, /, sqrt, sincos, and quaternion-to-rotation for T).
template <class T>
__device__ __forceinline__ void dpv_se3_retract_t(const T* __restrict__ x, T* __restrict__ P) {
  const T r0 = x[0], r1 = x[1], r2 = x[2], p0 = x[3], p1 = x[4], p2 = x[5];
  const T t2 = p0 * p0 + p1 * p1 + p2 * p2;
  T a, c, B, C;
  if (dpv_value(t2) < 1e-2) {
    a = 0.5 + t2 * (-1.0 / 48.0 + t2 * (1.0 / 3840.0 + t2 * (-1.0 / 645120.0 + t2 * (1.0 / 185794560.0))));
    c = 1.0 + t2 * (-1.0 / 8.0 + t2 * (1.0 / 384.0 + t2 * (-1.0 / 46080.0 + t2 * (1.0 / 10321920.0))));
    B = 0.5 + t2 * (-1.0 / 24.0 + t2 * (1.0 / 720.0 + t2 * (-1.0 / 40320.0 + t2 * (1.0 / 3628800.0))));
    C = 1.0 / 6.0 + t2 * (-1.0 / 120.0 + t2 * (1.0 / 5040.0 + t2 * (-1.0 / 362880.0 + t2 * (1.0 / 39916800.0))));
  } else {
    const T th = dpv_sqrt(t2);
    T sh, ch;
    dpv_sincos(0.5 * th, sh, ch);
    a = sh / th;
    c = ch;
    B = 2.0 * sh * sh / t2;
    C = (th - 2.0 * sh * ch) / (t2 * th);
  }
  const T qe[4] = {a * p0, a * p1, a * p2, c};
  // phi x rho and phi x (phi x rho)
  const T u0 = p1 * r2 - p2 * r1, u1 = p2 * r0 - p0 * r2, u2 = p0 * r1 - p1 * r0;
  const T v0 = p1 * u2 - p2 * u1, v1 = p2 * u0 - p0 * u2, v2 = p0 * u1 - p1 * u0;
  T Re[9];
  dpv_quat_rot_t(qe, Re);
  const T t0 = P[0], t1 = P[1], tt2 = P[2];
  P[0] = Re[0] * t0 + Re[1] * t1 + Re[2] * tt2 + r0 + B * u0 + C * v0;
  P[1] = Re[3] * t0 + Re[4] * t1 + Re[5] * tt2 + r1 + B * u1 + C * v1;
  P[2] = Re[6] * t0 + Re[7] * t1 + Re[8] * tt2 + r2 + B * u2 + C * v2;
  const T bx = P[3], by = P[4], bz = P[5], bw = P[6];
  T nq[4];
  nq[0] = qe[3] * bx + qe[0] * bw + qe[1] * bz - qe[2] * by;
  nq[1] = qe[3] * by - qe[0] * bz + qe[1] * bw + qe[2] * bx;
  nq[2] = qe[3] * bz + qe[0] * by - qe[1] * bx + qe[2] * bw;
  nq[3] = qe[3] * bw - qe[0] * bx - qe[1] * by - qe[2] * bz;
  const T inv = 1.0 / dpv_sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
#pragma unroll
  for (int m = 0; m < 4; ++m) P[3 + m] = nq[m] * inv;
}

__device__ __forceinline__ void dpv_se3_retract(const double* __restrict__ x, double* __restrict__ P) {
  dpv_se3_retract_t<double>(x, P);
}
