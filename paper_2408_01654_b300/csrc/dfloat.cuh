// Double-float arithmetic on the FP32 pipe, and the per-edge linearisation of
// Eq. 2-3 carried in it (the mixed-precision path).
//
// A value is an unevaluated pair hi + lo of floats (~48 significant bits).
// The building blocks are the error-free transformations of Knuth (TwoSum:
// the exact rounding error of a sum) and of Dekker with a fused multiply-add
// (TwoProd: fma(a, b, -a*b) is the exact rounding error of a product), and
// Dekker's 1971 double-length algorithms for the product, quotient and square
// root (one FP32 estimate, then a correction from the exactly computed
// remainder).  B300 runs FP64 at ~1/64 of the FP32 rate; these cost 3-20 FP32
// operations each.  Every operation uses the _rn intrinsics so that the
// compiler does not contract a product into the following sum, which would
// change the error terms.
//
// Why the loop-closure systems need it: S = B + lambda I - E Ct^-1 E^T is the
// small difference of two large, nearly equal sums per patch, and the
// 1000-keyframe system has an equilibrated condition number of ~2e7 with
// patches whose inverse depth lies near the clamp.  Rounding the per-patch
// Schur terms e_k, C_k, w_k to FP32 alone moves the GN step of a 400-frame
// loop-closure graph by ~1e-4 (depth, relative); rounding the relative pose,
// the back-projected ray, the point, the residual or the Jacobians to FP32
// moves the 1000-frame step by up to 7e-4 at such patches (measured with the
// FP64 reference implementation rounded at each of these places).  Carried in
// double-float they move it by ~1e-9.
#pragma once
#include "internal.cuh"

// ---- error-free transformations and double-float operations --------------
__device__ __forceinline__ DF dd_two_sum(float a, float b) {  // exactly a + b
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}
__device__ __forceinline__ DF dd_fast_two_sum(float a, float b) {  // exactly a + b when |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF dd_prod(float a, float b) {  // exactly a * b
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF dd_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF dd_norm(DF a) { return dd_fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ DF dd_add(DF a, DF b) {
  const DF s = dd_two_sum(a.hi, b.hi);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF dd_sub(DF a, DF b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ DF dd_add_f(DF a, float b) {
  const DF s = dd_two_sum(a.hi, b);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ DF dd_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p, e);
}
__device__ __forceinline__ DF dd_mul_f(DF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return dd_fast_two_sum(p, e);
}
// acc += a * b with the pair left unnormalised (hi carries the rounded sum,
// lo every rounding error); read it through dd_norm.  12 operations.
__device__ __forceinline__ void dd_acc(DF& acc, DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const DF s = dd_two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void dd_acc_add(DF& acc, DF b) {  // acc += b, unnormalised
  const DF s = dd_two_sum(acc.hi, b.hi);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, b.lo));
}
// Dekker's quotient: q1 = a / b in FP32, then q2 from the remainder a - q1 b
// (formed to double-float accuracy).
__device__ __forceinline__ DF dd_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF r = dd_sub(a, dd_mul_f(b, q1));
  return dd_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ DF dd_rcp(DF b) { return dd_div(DF{1.f, 0.f}, b); }
// Dekker's square root: s = sqrt(a) in FP32, then (a - s^2) / (2 s).
__device__ __forceinline__ DF dd_sqrt(DF a) {
  const float s = __fsqrt_rn(a.hi);
  const DF r = dd_sub(a, dd_prod(s, s));
  return dd_fast_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.f, s)));
}
__device__ __forceinline__ DF dd_ld(const float2 v) { return DF{v.x, v.y}; }
__device__ __forceinline__ float2 dd_st(DF a) { return make_float2(a.hi, a.lo); }
// the pair as one FP64 value (integer conversions and one FP64 add)
__device__ __forceinline__ double dd_to_f64(DF a) { return dpv_f2d_bits(a.hi) + dpv_f2d_bits(a.lo); }

// ---- relative pose in double-float ----------------------------------------
// T_ij = T_j T_i^-1 from two rows of the pose table (R and the camera centre
// as double-float pairs):  R = R_j R_i^T,  t = R_j (c_i - c_j);  and the
// translation-rotation block [t]x R of Ad(T_ij).
struct RelPoseDD {
  DF R[9], t[3], txR[9];
};
__device__ __forceinline__ void dpv_relative_pose_dd(const float* Pi, const float* Pj, RelPoseDD& o) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      DF acc = {0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 3; ++k)
        dd_acc(acc, DF{Pj[3 * r + k], Pj[9 + 3 * r + k]}, DF{Pi[3 * c + k], Pi[9 + 3 * c + k]});
      o.R[3 * r + c] = dd_norm(acc);
    }
  DF dc[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) dc[m] = dd_sub(DF{Pi[18 + m], Pi[21 + m]}, DF{Pj[18 + m], Pj[21 + m]});
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    DF acc = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k) dd_acc(acc, DF{Pj[3 * r + k], Pj[9 + 3 * r + k]}, dc[k]);
    o.t[r] = dd_norm(acc);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.txR[0 + c] = dd_sub(dd_mul(o.t[1], o.R[6 + c]), dd_mul(o.t[2], o.R[3 + c]));
    o.txR[3 + c] = dd_sub(dd_mul(o.t[2], o.R[0 + c]), dd_mul(o.t[0], o.R[6 + c]));
    o.txR[6 + c] = dd_sub(dd_mul(o.t[0], o.R[3 + c]), dd_mul(o.t[1], o.R[0 + c]));
  }
}

// ---- per-edge linearisation of Eq. 3 in double-float (target side) -------
//   X = R xb + t d  (xb = ((u-cx)/fx, (v-cy)/fy, 1), homogeneous 4th entry d)
//   r = (target - c) - f X/Z   (per component)
//   Jj = dproj/dX [ d I | -[X]x ],  Jd = dproj/dX t
// written with x = X/Z, y = Y/Z:  dproj/dX [d I] = f/Z [d, 0, -x d], the
// rotation part f [-x y, 1 + x^2, -y] (u row) and f [-(1 + y^2), x y, x]
// (v row), and Jd = f/Z (t_0 - x t_2, t_1 - y t_2).  The source-pose Jacobian
// Ji = -Jj Ad(T_ij) is not formed: every product with it is taken through
// Ad(T_ij)^T once per run or per edge (dpv_adT_dd).
// T: the relative pose as pairs in shared memory, floats [2m, 2m+1] for
// R[m] (row-major), [18 + 2m, 19 + 2m] for t[m], [24 + 2m, 25 + 2m] for
// ([t]x R)[m].
struct EdgeLinDD {
  DF r[2];
  DF Jj[2][6], Jd[2];  // Jj[0][1] = Jj[1][0] = 0
  bool valid;
};

__device__ __forceinline__ DF dd_sm(const float* T, int i) { return DF{T[2 * i], T[2 * i + 1]}; }

__device__ __forceinline__ void dpv_edge_linearize_dd(const float* T, DF xb0, DF xb1, float d, float tu, float tv,
                                                      const float* K, float z_min, bool self_edge, EdgeLinDD& o) {
  DF X[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    DF acc = dd_sm(T, 3 * r + 2);
    dd_acc(acc, dd_sm(T, 3 * r), xb0);
    dd_acc(acc, dd_sm(T, 3 * r + 1), xb1);
    dd_acc(acc, dd_sm(T, 9 + r), DF{d, 0.f});
    X[r] = dd_norm(acc);
  }
  o.valid = !self_edge && (X[2].hi > z_min * d);
  const float fx = K[0], fy = K[1];
  const DF iz = dd_rcp(X[2]);
  const DF xz = dd_mul(X[0], iz), yz = dd_mul(X[1], iz);
  o.r[0] = dd_sub(dd_two_sum(tu, -K[2]), dd_mul_f(xz, fx));
  o.r[1] = dd_sub(dd_two_sum(tv, -K[3]), dd_mul_f(yz, fy));
  const DF id = dd_mul_f(iz, d);
  const DF xy = dd_mul(xz, yz);
  const DF zero = {0.f, 0.f};
  o.Jj[0][0] = dd_mul_f(id, fx);
  o.Jj[0][1] = zero;
  o.Jj[0][2] = dd_neg(dd_mul_f(dd_mul(xz, id), fx));
  o.Jj[0][3] = dd_neg(dd_mul_f(xy, fx));
  o.Jj[0][4] = dd_mul_f(dd_add_f(dd_mul(xz, xz), 1.f), fx);
  o.Jj[0][5] = dd_neg(dd_mul_f(yz, fx));
  o.Jj[1][0] = zero;
  o.Jj[1][1] = dd_mul_f(id, fy);
  o.Jj[1][2] = dd_neg(dd_mul_f(dd_mul(yz, id), fy));
  o.Jj[1][3] = dd_neg(dd_mul_f(dd_add_f(dd_mul(yz, yz), 1.f), fy));
  o.Jj[1][4] = dd_mul_f(xy, fy);
  o.Jj[1][5] = dd_mul_f(xz, fy);
  o.Jd[0] = dd_mul(dd_mul_f(iz, fx), dd_sub(dd_sm(T, 9), dd_mul(xz, dd_sm(T, 11))));
  o.Jd[1] = dd_mul(dd_mul_f(iz, fy), dd_sub(dd_sm(T, 10), dd_mul(yz, dd_sm(T, 11))));
}

// out = Ad(T_ij)^T v for a 6-vector v (translation part first):
// Ad = [ R  [t]x R ; 0  R ]  =>  out[c] = sum_m R[m][c] v[m],
// out[3 + c] = sum_m (([t]x R)[m][c] v[m] + R[m][c] v[3 + m]).
__device__ __forceinline__ void dpv_adT_dd(const float* T, const DF* v, DF* out) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    DF a = {0.f, 0.f}, b = {0.f, 0.f};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      dd_acc(a, dd_sm(T, 3 * m + c), v[m]);
      dd_acc(b, dd_sm(T, 12 + 3 * m + c), v[m]);
      dd_acc(b, dd_sm(T, 3 * m + c), v[3 + m]);
    }
    out[c] = dd_norm(a);
    out[3 + c] = dd_norm(b);
  }
}

// The back-projected ray coordinate (p - c) / f of a float pixel p in
// double-float: p - c is exact as a pair (TwoSum), the division Dekker's.
__device__ __forceinline__ DF dpv_ray_dd(float p, float c, float f) { return dd_div(dd_two_sum(p, -c), DF{f, 0.f}); }
