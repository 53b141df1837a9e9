// Proximity loop edges (ba_proximity_edges): Sec. 3.2 "Proximity Loop
// Closure" and "Constructing the Patch Graph".  A loop is detected from how
// close the camera comes to where an older frame was; the loop is closed with
// uni-directional edges from the stored patches of the old frame to the
// recent frame, so only the recent frame's dense features are needed.
//
// Rule, for each query frame b in [b0, b1):
//   candidates : frames a with b - a > gap;
//   selection  : the candidate whose camera centre c = -R^T t is nearest to
//                c_b (the lowest index among equal distances), if its squared
//                distance is < radius^2;
//   edges      : (ii, jj, kk) = (a, b, a*M + m) for the patches m of frame a
//                whose centre pixel, reprojected by Eq. 2 at its current
//                inverse depth, lies more than z_min in front of frame b and
//                inside [0, width) x [0, height);
//   order      : by b, then m.
//
// Precision.  FP64 issues at a small fraction of the FP32 rate on this GPU and
// a warp's FP64 instruction chain is long, so the only FP64 work is splitting
// the FP64 poses into float pairs hi + lo (and the rare fallback below).
// Everything else runs in double-float arithmetic on the FP32 pipe
// (error-free transformations: Knuth's TwoSum, and the exact product error
// fma(a, b, -ab)), about 44 significant bits:
//   - selection: float32 distances with a rigorous rounding interval (below)
//     discard every candidate that cannot be the nearest; the survivors (one
//     to three per query) are measured again in double-float, and the argmin,
//     the lowest-index rule and the radius test are taken on those values;
//   - reprojection: Y = T (u, v, 1, d)^T in double-float; a test is taken from
//     the pair when it lies farther from its threshold than 2^-40 of the sum
//     of the magnitudes of its terms, else the patch is redone in FP64.
// The decisions therefore agree with exact arithmetic whenever the exact value
// is more than ~1e-12 (relative) from its threshold.
//
// Two launches, both on the handle's stream, the second a programmatic
// dependent launch (its CTAs start while the first grid runs and wait for it
// before reading the tables):
//   k_prox_frames  eight threads per frame: the FP64 pose split into pairs
//                  (one thread per component), then in double-float the
//                  rotation and, three per thread, the centre c = -R^T t and
//                  the reprojection factors A = R^T K^-1, B = K R, e = K t;
//   k_prox_main    one warp per query frame, 8 per CTA (the CTA stages the
//                  candidates' float32 centres in shared memory):
//     selection    as above;
//     reprojection lanes 0..11 form the query's 3x4 transform
//                  T = [B_b A_a | B_b c_a + e_b] (one entry each); Y is the
//                  pixel times Z d, so the depth test is Y_z > z_min d and the
//                  image test 0 <= Y_x < width Y_z, 0 <= Y_y < height Y_z (no
//                  division); kept pixels are the pair quotients rounded to
//                  float;
//     compaction   the CTA's kept count is published at once and its output
//                  offset found by looking back over the earlier CTAs'
//                  published counts and prefixes (decoupled look-back); CTAs
//                  take their query blocks from a ticket counter, so a CTA
//                  only ever waits on CTAs that started before it, and every
//                  wait is bounded.  The last CTA to finish writes the total
//                  (or -1 after a timed-out wait) and resets the counters.
//
// Distance interval.  With u = 2^-24, float32 centres c~ (the hi parts of the
// pairs, so each component is c rounded once to float), the float32
// difference and sum of squares s of a pair (a, b) give
// |sqrt(s) - |c_a - c_b|| <= 1.01 u (|c_a|_1 + |c_b|_1) + 3.5 u sqrt(s).  The
// kernel takes r = s * rsqrt(s) (an approximate reciprocal square root, a few
// ulps) and widens the bound to eta = 16 u (W_a + W_b + r), W the float32 L1
// norms, which also covers the reciprocal square root and the rounding of
// forming r +- eta many times over.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <climits>

namespace {

constexpr int PX_WARPS = 8;             // queries per CTA
constexpr int PX_THREADS = 32 * PX_WARPS;
constexpr int PX_MAX_M = 1024;          // patches per frame
constexpr int PX_XT = 48;               // floats per frame in the transform table: 21 pairs (hi block, lo block)
constexpr int PX_FR = 32;               // frames per CTA of k_prox_frames
constexpr int PX_TILE = 2048;           // candidate centres staged in shared memory per pass
constexpr float PX_SLACK = 16.0f / 16777216.0f;           // 16 u
constexpr float PX_DF_BOUND = 1.0f / 1099511627776.0f;    // 2^-40
constexpr unsigned long long PX_PREFIX = 1ull << 31;
constexpr size_t PX_SOLO_SMEM = 96 * 1024;  // dynamic shared memory that keeps k_prox_main alone on its SM

// ---- double-float arithmetic (value = hi + lo, |lo| <= ulp(hi) / 2) -------
// The _rn intrinsics keep the compiler from contracting products into sums,
// which would break the error terms.
__device__ __forceinline__ DF px_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF px_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF px_add(DF a, DF b) {
  DF s = px_two_sum(a.hi, b.hi);
  const DF t = px_two_sum(a.lo, b.lo);
  s = px_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return px_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ DF px_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF px_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return px_fast_two_sum(p, e);
}
__device__ __forceinline__ DF px_scale2(DF a, float s) { return DF{a.hi * s, a.lo * s}; }  // s a power of two
__device__ __forceinline__ bool px_less(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ DF px_dot3(DF a0, DF a1, DF a2, DF b0, DF b1, DF b2) {
  return px_add(px_add(px_mul(a0, b0), px_mul(a1, b1)), px_mul(a2, b2));
}

struct ProxArgs {
  int M, MW, b0, Q, gap, nblk;
  float fx, fy, cx, cy;       // intrinsics (exact floats)
  DF ifx, ify, cxifx, cyify;  // 1/fx, 1/fy, cx/fx, cy/fy
  DF r2;                      // radius^2
  float zf[2], wf[2], hf[2];  // z_min, width, height as pairs
  double z_min, width, height;
  long long timeout;
};

struct ProxSync {
  unsigned* words;            // [0] ticket, [1] finished CTAs, [2] epoch, [3] timed out
  unsigned long long* flags;  // [nblk] (epoch << 32) | prefix bit | count
};

__device__ __forceinline__ void px_st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long px_ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long px_ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Per-frame tables.  c32[a] = (c~, |c~|_1), clo[a] = (lo parts of c, 0), and
// xt[a] = A (9 pairs, row-major), B (9 pairs), e (3 pairs): hi parts in
// floats 0..20, lo parts in 24..44.  Eight threads per frame: first each
// splits one FP64 pose component, then each forms the rotation and three of
// the frame's 24 output pairs (A, B, e, c), which keeps every thread's chain
// of dependent operations short.
__device__ DF px_frame_out(int k, const DF* R, const DF* t, const ProxArgs& A) {
  const DF fx = {A.fx, 0.f}, fy = {A.fy, 0.f}, cx = {A.cx, 0.f}, cy = {A.cy, 0.f};
  if (k < 9) {  // A = R^T K^-1: row r from column r of R
    const int r = k / 3, c = k % 3;
    if (c == 0) return px_mul(R[r], A.ifx);
    if (c == 1) return px_mul(R[3 + r], A.ify);
    return px_add(R[6 + r], px_neg(px_add(px_mul(R[r], A.cxifx), px_mul(R[3 + r], A.cyify))));
  }
  if (k < 18) {  // B = K R
    const int r = (k - 9) / 3, c = (k - 9) % 3;
    if (r == 0) return px_add(px_mul(fx, R[c]), px_mul(cx, R[6 + c]));
    if (r == 1) return px_add(px_mul(fy, R[3 + c]), px_mul(cy, R[6 + c]));
    return R[6 + c];
  }
  if (k == 18) return px_add(px_mul(fx, t[0]), px_mul(cx, t[2]));  // e = K t
  if (k == 19) return px_add(px_mul(fy, t[1]), px_mul(cy, t[2]));
  if (k == 20) return t[2];
  const int m = k - 21;  // centre c = -R^T t
  return px_neg(px_dot3(R[m], R[3 + m], R[6 + m], t[0], t[1], t[2]));
}

__global__ void __launch_bounds__(PX_FR * 8) k_prox_frames(int n, const double* __restrict__ poses, ProxArgs A,
                                                           float4* __restrict__ c32, float4* __restrict__ clo,
                                                           float* __restrict__ xt) {
  __shared__ float s_h[PX_FR][8], s_l[PX_FR][8];
  __shared__ DF s_cen[PX_FR][3];
  // k_prox_main may be scheduled now; it waits for this grid before reading
  // the tables (programmatic dependent launch)
  asm volatile("griddepcontrol.launch_dependents;");
  const int f0 = blockIdx.x * PX_FR;
  const int fl = threadIdx.x >> 3, k = threadIdx.x & 7;
  const int a = f0 + fl;
  {  // split: thread (frame, component) -> pair
    float h = 0.f, l = 0.f;
    if (k < 7 && a < n) {
      const double x = poses[7 * (size_t)a + k];
      h = __double2float_rn(x);
      l = __double2float_rn(x - (double)h);
    }
    s_h[fl][k] = h;
    s_l[fl][k] = l;
  }
  __syncthreads();
  if (a < n) {
    DF t[3], q[4];
#pragma unroll
    for (int j = 0; j < 3; ++j) t[j] = DF{s_h[fl][j], s_l[fl][j]};
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = DF{s_h[fl][3 + j], s_l[fl][3 + j]};
    // rotation of the unit quaternion (x, y, z, w)
    const DF xx = px_mul(q[0], q[0]), yy = px_mul(q[1], q[1]), zz = px_mul(q[2], q[2]);
    const DF xy = px_mul(q[0], q[1]), xz = px_mul(q[0], q[2]), yz = px_mul(q[1], q[2]);
    const DF xw = px_mul(q[0], q[3]), yw = px_mul(q[1], q[3]), zw = px_mul(q[2], q[3]);
    const DF one = {1.f, 0.f};
    DF R[9];
    R[0] = px_add(one, px_scale2(px_add(yy, zz), -2.f));
    R[1] = px_scale2(px_add(xy, px_neg(zw)), 2.f);
    R[2] = px_scale2(px_add(xz, yw), 2.f);
    R[3] = px_scale2(px_add(xy, zw), 2.f);
    R[4] = px_add(one, px_scale2(px_add(xx, zz), -2.f));
    R[5] = px_scale2(px_add(yz, px_neg(xw)), 2.f);
    R[6] = px_scale2(px_add(xz, px_neg(yw)), 2.f);
    R[7] = px_scale2(px_add(yz, xw), 2.f);
    R[8] = px_add(one, px_scale2(px_add(xx, yy), -2.f));
    float* o = xt + PX_XT * (size_t)a;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int out = k + 8 * j;  // 0..23
      const DF v = px_frame_out(out, R, t, A);
      if (out < 21) {
        o[out] = v.hi;
        o[24 + out] = v.lo;
      } else {
        s_cen[fl][out - 21] = v;
      }
    }
  }
  __syncthreads();
  if (k == 0 && a < n) {
    const DF c0 = s_cen[fl][0], c1 = s_cen[fl][1], c2 = s_cen[fl][2];
    c32[a] = make_float4(c0.hi, c1.hi, c2.hi, fabsf(c0.hi) + fabsf(c1.hi) + fabsf(c2.hi));
    clo[a] = make_float4(c0.lo, c1.lo, c2.lo, 0.f);
  }
}

// float32 distance of a pair and its rounding slack
__device__ __forceinline__ void px_dist32(const float4& c, const float4& cb, float& r, float& eta) {
  const float dx = c.x - cb.x, dy = c.y - cb.y, dz = c.z - cb.z;
  const float s = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  r = s > 0.f ? s * rsqrtf(s) : 0.f;
  eta = PX_SLACK * (c.w + cb.w + r);
}

// keep the smallest lower end (and its index) and the second smallest
__device__ __forceinline__ void px_track(float lo, int idx, float& lo1, int& i1, float& lo2) {
  if (lo < lo1) {
    lo2 = lo1;
    lo1 = lo;
    i1 = idx;
  } else if (lo < lo2) {
    lo2 = lo;
  }
}

// copy n float4 from global to shared memory with asynchronous 16-byte
// copies (no register round trip, all in flight together), then wait and
// synchronise the CTA
__device__ __forceinline__ void px_stage(float4* dst, const float4* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src + i) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
}

// squared distance of two centres in double-float
__device__ __forceinline__ DF px_dist2_df(const float4& ca, const float4& la, const float4& cb, const float4& lb) {
  const DF dx = px_add(DF{ca.x, la.x}, DF{-cb.x, -lb.x});
  const DF dy = px_add(DF{ca.y, la.y}, DF{-cb.y, -lb.y});
  const DF dz = px_add(DF{ca.z, la.z}, DF{-cb.z, -lb.z});
  return px_dot3(dx, dy, dz, dx, dy, dz);
}

// (d2, a) before (e2, b): the nearer, then the lower index
__device__ __forceinline__ bool px_before(DF d2, int a, DF e2, int b) {
  return px_less(d2, e2) || (d2.hi == e2.hi && d2.lo == e2.lo && a < b);
}

// ---- double-float reprojection ------------------------------------------
struct DFT {
  float h[12], l[12];
};

// acc = T[c0] u + T[c1] v + T[c2] + T[c3] d as a pair, with sum |terms| in S
__device__ __forceinline__ DF px_row(const DFT& T, int c0, int c1, int c2, int c3, float u, float v, float d,
                                     float& S) {
  DF acc = {T.h[c2], T.l[c2]};
  df_fma(acc, T.h[c0], u);
  acc.lo = __fmaf_rn(T.l[c0], u, acc.lo);
  df_fma(acc, T.h[c1], v);
  acc.lo = __fmaf_rn(T.l[c1], v, acc.lo);
  df_fma(acc, T.h[c3], d);
  acc.lo = __fmaf_rn(T.l[c3], d, acc.lo);
  S = fabsf(T.h[c0] * u) + fabsf(T.h[c1] * v) + fabsf(T.h[c2]) + fabsf(T.h[c3] * d);
  return acc;
}

// x - w y for pairs x, y and a constant pair w
__device__ __forceinline__ DF px_sub_scaled(DF x, float wh, float wl, const DF& y) {
  df_fma(x, -wh, y.hi);
  x.lo = __fmaf_rn(-wh, y.lo, __fmaf_rn(-wl, y.hi, x.lo));
  return x;
}

// the quotient x / y of two pairs rounded to float: q = x_hi / y_hi, then one
// correction from the exact residual x_hi - q y_hi
__device__ __forceinline__ float px_div(const DF& x, const DF& y) {
  const float q = __fdiv_rn(x.hi, y.hi);
  const float r = __fmaf_rn(-q, y.hi, x.hi);
  const float rr = __fadd_rn(r, __fmaf_rn(-q, y.lo, x.lo));
  return __fadd_rn(q, __fdiv_rn(rr, y.hi));
}

// the same patch in FP64, with the transform T = hi + lo read from shared
// memory behind a compiler barrier, so that its conversion stays in this
// rarely taken branch instead of being hoisted out of the patch loop
__device__ bool px_project64(const float* Th, const float* Tl, double u, double v, double d, const ProxArgs& A,
                             float2& uv) {
  asm volatile("" ::: "memory");
  double T[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) T[k] = (double)Th[k] + (double)Tl[k];
  const double Yx = fma(T[0], u, fma(T[1], v, fma(T[9], d, T[2])));
  const double Yy = fma(T[3], u, fma(T[4], v, fma(T[10], d, T[5])));
  const double Yz = fma(T[6], u, fma(T[7], v, fma(T[11], d, T[8])));
  if (!(Yz > A.z_min * d)) return false;
  bool keep;
  if (Yz > 0.0) {
    keep = Yx >= 0.0 && Yx < A.width * Yz && Yy >= 0.0 && Yy < A.height * Yz;
  } else {  // only with a non-positive inverse depth
    const double pu = Yx / Yz, pv = Yy / Yz;
    keep = pu >= 0.0 && pu < A.width && pv >= 0.0 && pv < A.height;
  }
  if (keep) uv = make_float2((float)(Yx / Yz), (float)(Yy / Yz));
  return keep;
}

__global__ void __launch_bounds__(PX_THREADS, 1) k_prox_main(ProxArgs A, const float4* __restrict__ c32,
                                                             const float4* __restrict__ clo,
                                                             const float* __restrict__ xt,
                                                             const float* __restrict__ patches,
                                                             int* __restrict__ match, int* __restrict__ ii,
                                                             int* __restrict__ jj, int* __restrict__ kk,
                                                             float2* __restrict__ coords, long long cap,
                                                             int* __restrict__ count, ProxSync Y) {
  extern __shared__ __align__(16) unsigned char px_smem[];
  __shared__ float4 s_c[PX_TILE];
  __shared__ float s_Th[PX_WARPS][12], s_Tl[PX_WARPS][12];
  __shared__ int s_tk, s_wc[PX_WARPS], s_sel[PX_WARPS], s_ok;
  __shared__ unsigned s_epoch;
  __shared__ long long s_base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* s_uv = reinterpret_cast<float2*>(px_smem);                                          // [PX_WARPS][M]
  unsigned* s_mask = reinterpret_cast<unsigned*>(px_smem + sizeof(float2) * PX_WARPS * A.M);  // [PX_WARPS][MW]
  if (threadIdx.x == 0) {
    s_tk = (int)atomicAdd(&Y.words[0], 1u);
    s_epoch = *(volatile unsigned*)&Y.words[2] + 1u;
    s_ok = 1;
  }
  __syncthreads();
  const int cta = s_tk;
  const unsigned epoch = s_epoch;
  // the frame tables of k_prox_frames (launched before this grid, which may
  // start early) are complete and visible after this
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int q = cta * PX_WARPS + w;
  const int b = A.b0 + q;
  // ---- nearest older centre ----
  // candidates 0 .. na-1 of this warp's query; the CTA's queries are
  // consecutive frames, so its last valid query has the most
  const int na = q < A.Q ? max(0, b - A.gap) : 0;
  const int na_cta = max(0, A.b0 + min(cta * PX_WARPS + PX_WARPS - 1, A.Q - 1) - A.gap);
  const float4 cb = q < A.Q ? c32[b] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 lb = q < A.Q ? clo[b] : make_float4(0.f, 0.f, 0.f, 0.f);
  // pass 1 (float32): the smallest upper end U of the candidates' intervals
  // (four independent minima per lane), and per lane the smallest lower end
  // (with its index) and the second smallest
  float U0 = INFINITY, U1 = INFINITY, U2 = INFINITY, U3 = INFINITY;
  float lo1 = INFINITY, lo2 = INFINITY;
  int i1 = -1;
  for (int t0 = 0; t0 < na_cta; t0 += PX_TILE) {
    const int tn = min(PX_TILE, na_cta - t0);
    __syncthreads();
    px_stage(s_c, c32 + t0, tn);
    const int hi = min(tn, na - t0);
    int i = lane;
    for (; i + 96 < hi; i += 128) {
      float r[4], eta[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) px_dist32(s_c[i + 32 * k], cb, r[k], eta[k]);
      U0 = fminf(U0, r[0] + eta[0]);
      U1 = fminf(U1, r[1] + eta[1]);
      U2 = fminf(U2, r[2] + eta[2]);
      U3 = fminf(U3, r[3] + eta[3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) px_track(r[k] - eta[k], t0 + i + 32 * k, lo1, i1, lo2);
    }
    for (; i < hi; i += 32) {
      float r, eta;
      px_dist32(s_c[i], cb, r, eta);
      U0 = fminf(U0, r + eta);
      px_track(r - eta, t0 + i, lo1, i1, lo2);
    }
  }
  float U = fminf(fminf(U0, U1), fminf(U2, U3));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) U = fminf(U, __shfl_xor_sync(0xffffffffu, U, o));
  // pass 2: double-float distances of the candidates whose lower end reaches
  // below U.  When no lane has two of them (the usual case) they are the
  // lanes' smallest lower ends; otherwise the candidates are scanned again,
  // in increasing index per lane (the lane keeps its lowest index among
  // equal values).
  DF best = {INFINITY, 0.f};
  int ba = INT_MAX;
  // (CTA-wide decision: the rescan may restage tiles behind barriers)
  if (!__syncthreads_or(lo2 < INFINITY && lo2 <= U)) {
    if (i1 >= 0 && lo1 <= U) {
      best = px_dist2_df(c32[i1], clo[i1], cb, lb);
      ba = i1;
    }
  } else {
    for (int t0 = 0; t0 < na_cta; t0 += PX_TILE) {
      const int tn = min(PX_TILE, na_cta - t0);
      if (na_cta > PX_TILE) {  // with one tile it is still in shared memory
        __syncthreads();
        px_stage(s_c, c32 + t0, tn);
      }
      const int hi = min(tn, na - t0);
      for (int i = lane; i < hi; i += 32) {
        float r, eta;
        px_dist32(s_c[i], cb, r, eta);
        if (r - eta <= U) {
          const DF d2 = px_dist2_df(s_c[i], clo[t0 + i], cb, lb);
          if (px_less(d2, best)) {
            best = d2;
            ba = t0 + i;
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const DF ob = {__shfl_xor_sync(0xffffffffu, best.hi, o), __shfl_xor_sync(0xffffffffu, best.lo, o)};
    const int oa = __shfl_xor_sync(0xffffffffu, ba, o);
    if (px_before(ob, oa, best, ba)) {
      best = ob;
      ba = oa;
    }
  }
  int kept = 0, sel = -1;
  if (q < A.Q) {
    sel = (ba != INT_MAX && px_less(best, A.r2)) ? ba : -1;
    if (lane == 0 && match) match[q] = sel;
    if (sel >= 0) {
      // the first rounds of patch centres, loaded before T is formed so that
      // their memory latency overlaps it
      const float* pk0 = patches + (size_t)sel * A.M * 27;
      constexpr int PF = 4;
      float pu[PF], pv[PF], pd[PF];
#pragma unroll
      for (int r = 0; r < PF; ++r) {
        const int m = 32 * r + lane;
        pu[r] = pv[r] = pd[r] = 0.f;
        if (r < A.MW && m < A.M) {
          const float* pk = pk0 + (size_t)m * 27;
          pu[r] = pk[4];
          pv[r] = pk[13];
          pd[r] = pk[22];
        }
      }
      // T = [B_b A_a | B_b c_a + e_b], one entry per lane 0..11
      DF tv = {0.f, 0.f};
      if (lane < 12) {
        const float* Xa = xt + PX_XT * (size_t)sel;
        const float* Xb = xt + PX_XT * (size_t)b;
        const int r = lane < 9 ? lane / 3 : lane - 9;
        const DF b0 = {Xb[9 + 3 * r], Xb[33 + 3 * r]}, b1 = {Xb[10 + 3 * r], Xb[34 + 3 * r]},
                 b2 = {Xb[11 + 3 * r], Xb[35 + 3 * r]};
        if (lane < 9) {
          const int c = lane % 3;
          tv = px_dot3(b0, b1, b2, DF{Xa[c], Xa[24 + c]}, DF{Xa[3 + c], Xa[27 + c]}, DF{Xa[6 + c], Xa[30 + c]});
        } else {
          const float4 ch = c32[sel], cl = clo[sel];
          tv = px_add(px_dot3(b0, b1, b2, DF{ch.x, cl.x}, DF{ch.y, cl.y}, DF{ch.z, cl.z}),
                      DF{Xb[18 + r], Xb[42 + r]});
        }
      }
      if (lane < 12) {
        s_Th[w][lane] = tv.hi;
        s_Tl[w][lane] = tv.lo;
      }
      DFT T;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        T.h[k] = __shfl_sync(0xffffffffu, tv.hi, k);
        T.l[k] = __shfl_sync(0xffffffffu, tv.lo, k);
      }
      // T[0..8] = rows of B_b A_a, T[9..11] = B_b c_a + e_b
      const float zh = A.zf[0], zl = A.zf[1], wh = A.wf[0], wl = A.wf[1], hh = A.hf[0], hl = A.hf[1];
      for (int r = 0; r < A.MW; ++r) {
        const int m = 32 * r + lane;
        bool keep = false, fallback = false;
        float u = 0.f, v = 0.f, d = 0.f;
        if (m < A.M) {
          if (r < PF) {
            u = r == 0 ? pu[0] : r == 1 ? pu[1] : r == 2 ? pu[2] : pu[3];
            v = r == 0 ? pv[0] : r == 1 ? pv[1] : r == 2 ? pv[2] : pv[3];
            d = r == 0 ? pd[0] : r == 1 ? pd[1] : r == 2 ? pd[2] : pd[3];
          } else {
            const float* pk = pk0 + (size_t)m * 27;
            u = pk[4];
            v = pk[13];
            d = pk[22];
          }
          float Sx, Sy, Sz;
          const DF Yx = px_row(T, 0, 1, 2, 9, u, v, d, Sx);
          const DF Yy = px_row(T, 3, 4, 5, 10, u, v, d, Sy);
          const DF Yz = px_row(T, 6, 7, 8, 11, u, v, d, Sz);
          const DF Dz = px_sub_scaled(Yz, zh, zl, DF{d, 0.f});  // Yz - z_min d
          const DF Dx = px_sub_scaled(Yx, wh, wl, Yz);           // Yx - width Yz
          const DF Dy = px_sub_scaled(Yy, hh, hl, Yz);           // Yy - height Yz
          const float bz = PX_DF_BOUND * (Sz + zh * fabsf(d)), bx = PX_DF_BOUND * Sx, by = PX_DF_BOUND * Sy;
          const float bxw = PX_DF_BOUND * (Sx + wh * Sz), byh = PX_DF_BOUND * (Sy + hh * Sz);
          // (the float sum hi + lo has the sign of the pair)
          const float vz = Dz.hi + Dz.lo, vx = Yx.hi + Yx.lo, vy = Yy.hi + Yy.lo;
          const float vxw = Dx.hi + Dx.lo, vyh = Dy.hi + Dy.lo, yz = Yz.hi + Yz.lo;
          if (vz > bz && yz > PX_DF_BOUND * Sz) {  // clearly in front, Yz > 0
            if (fabsf(vx) > bx && fabsf(vy) > by && fabsf(vxw) > bxw && fabsf(vyh) > byh) {
              keep = vx > 0.f && vxw < 0.f && vy > 0.f && vyh < 0.f;
              if (keep) s_uv[w * A.M + m] = make_float2(px_div(Yx, Yz), px_div(Yy, Yz));
            } else {
              fallback = true;
            }
          } else if (!(vz < -bz)) {  // not clearly behind z_min either
            fallback = true;
          }
        }
        if (__any_sync(0xffffffffu, fallback)) {  // warp-uniform: FP64 only where needed
          if (fallback) {
            float2 uv;
            keep = px_project64(s_Th[w], s_Tl[w], u, v, d, A, uv);
            if (keep) s_uv[w * A.M + m] = uv;
          }
        }
        const unsigned bits = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_mask[w * A.MW + r] = bits;
        kept += __popc(bits);
      }
    }
  }
  if (lane == 0) {
    s_wc[w] = kept;
    s_sel[w] = sel;
  }
  __syncthreads();
  // ---- output offset of this CTA (decoupled look-back over earlier CTAs) ----
  // Warp 0 reads 256 earlier flags per round, eight consecutive ones per lane
  // (lane 0 the nearest); the nearest flag holding a prefix ends the look-back,
  // adding its prefix and the counts after it.  The counts travel inside the
  // flag words, so plain (relaxed) loads suffice; polls back off briefly, which
  // keeps the 125-odd CTAs from saturating the few cache lines of the flags.
  if (w == 0) {
    long long agg = 0;
#pragma unroll
    for (int k = 0; k < PX_WARPS; ++k) agg += s_wc[k];
    if (lane == 0)
      px_st_release(Y.flags + cta, ((unsigned long long)epoch << 32) | (cta == 0 ? PX_PREFIX : 0ull) |
                                       (unsigned long long)agg);
    long long excl = 0;
    bool ok = true;
    int j = cta - 1;
    const long long t0 = clock64();
    while (j >= 0) {
      unsigned long long f[8];
      while (true) {
        bool ready = true;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int idx = j - 8 * lane - k;
          f[k] = idx >= 0 ? px_ld_relaxed(Y.flags + idx) : 0ull;
          ready = ready && (idx < 0 || (unsigned)(f[k] >> 32) == epoch);
        }
        if (__all_sync(0xffffffffu, ready)) break;
        if (__any_sync(0xffffffffu, clock64() - t0 > A.timeout)) {  // warp-uniform
          ok = false;
          break;
        }
        __nanosleep(128);
      }
      if (!ok) break;
      int kp = 8;  // nearest prefix among this lane's flags
#pragma unroll
      for (int k = 7; k >= 0; --k)
        if (j - 8 * lane - k >= 0 && (f[k] & PX_PREFIX)) kp = k;
      long long mine = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k <= kp && j - 8 * lane - k >= 0) mine += (long long)(f[k] & (PX_PREFIX - 1));
      const unsigned pm = __ballot_sync(0xffffffffu, kp < 8);
      const int stop = pm ? __ffs(pm) - 1 : 31;
      long long v = lane <= stop ? mine : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      excl += v;
      if (pm) break;
      j -= 256;
    }
    if (lane == 0) {
      if (cta > 0)
        px_st_release(Y.flags + cta, ((unsigned long long)epoch << 32) | PX_PREFIX |
                                         (unsigned long long)((excl + agg) & (PX_PREFIX - 1)));
      if (!ok) {
        atomicExch(&Y.words[3], 1u);
        s_ok = 0;
      }
      s_base = excl;
    }
  }
  __syncthreads();
  // ---- write this CTA's edges ----
  if (s_ok && q < A.Q && s_wc[w] > 0) {
    long long off = s_base;
    for (int k = 0; k < w; ++k) off += s_wc[k];
    const int a = s_sel[w];
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < A.MW; ++r) {
      const unsigned bits = s_mask[w * A.MW + r];
      if ((bits >> lane) & 1u) {
        const long long pos = off + __popc(bits & lt);
        const int m = 32 * r + lane;
        if (pos < cap) {
          ii[pos] = a;
          jj[pos] = b;
          kk[pos] = a * A.M + m;
          if (coords) coords[pos] = s_uv[w * A.M + m];
        }
      }
      off += __popc(bits);
    }
  }
  // ---- the last CTA to finish: the total, then the counters for the next call ----
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&Y.words[1], 1u) == (unsigned)A.nblk - 1u) {
      __threadfence();
      const unsigned long long f = px_ld_acquire(Y.flags + (A.nblk - 1));
      const bool good = *(volatile unsigned*)&Y.words[3] == 0u && (unsigned)(f >> 32) == epoch && (f & PX_PREFIX);
      *count = good ? (int)(f & (PX_PREFIX - 1)) : -1;
      Y.words[0] = 0u;
      Y.words[1] = 0u;
      Y.words[3] = 0u;
      Y.words[2] = epoch;
      __threadfence();
    }
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

DF split_pair(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}

}  // namespace

extern "C" ba_status_t ba_proximity_edges(ba_handle_t h, int N, int M, const double* poses, const float* patches,
                                          const float* intrinsics, int b0, int b1, int gap, double radius,
                                          double width, double height, int* ii, int* jj, int* kk, float* coords,
                                          long long cap, int* match, int* count, long long* n_host) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!poses || !patches || !intrinsics || !count || (cap > 0 && (!ii || !jj || !kk)))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: null pointer");
  if (N < 1 || M < 1 || M > PX_MAX_M || (long long)N * M > INT_MAX || b0 < 0 || b1 < b0 || b1 > N || gap < 0 ||
      cap < 0 || !(radius >= 0.0) || !std::isfinite(radius) || !(width > 0.0) || !(height > 0.0))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: sizes or thresholds out of range");
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, intrinsics) != cudaSuccess) cudaGetLastError();
  if (pa.type == cudaMemoryTypeDevice)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: intrinsics must be host memory");
  if (coords && (reinterpret_cast<uintptr_t>(coords) & 7u))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: coords must be 8-byte aligned");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DPV_CUDA(h, cudaStreamIsCapturing(h->stream, &cs));
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  if (capturing && n_host)
    return dpv_fail(h, BA_ERR_STATE, "ba_proximity_edges: cannot return the count to the host during capture");
  const int Q = b1 - b0;
  if (Q == 0) {
    DPV_CUDA(h, cudaMemsetAsync(count, 0, sizeof(int), h->stream));
    if (n_host) {
      DPV_CUDA(h, cudaStreamSynchronize(h->stream));
      *n_host = 0;
    }
    return BA_OK;
  }
  const int MW = (M + 31) / 32;
  const int nblk = (Q + PX_WARPS - 1) / PX_WARPS;
  // scratch: counters (256 B) | CTA flags | float32 centres | their lo parts |
  // transforms.  The counters and flags carry state from call to call (the
  // epoch), so the flag region never moves while it is in use: growing it
  // reallocates and clears the whole scratch.
  Workspace* ws = h->ws;
  DBuf<unsigned char>& buf = ws->prox;
  if (!buf.p || nblk > ws->prox_blocks || b1 > ws->prox_frames) {
    // nothing captured by the handle refers to this scratch, so growing it
    // leaves the handle's graphs valid
    if (capturing || h->capturing)
      return dpv_fail(h, BA_ERR_STATE, "ba_proximity_edges: scratch must grow; call once outside graph capture");
    const long long blocks = std::max<long long>(nblk, ws->prox_blocks);
    const long long frames = std::max<long long>(b1, ws->prox_frames);
    const size_t bytes = 256 + align256(8 * (size_t)blocks) + 2 * align256(16 * (size_t)frames) +
                         align256(4 * PX_XT * (size_t)frames);
    if (buf.p) {
      DPV_CUDA(h, cudaStreamSynchronize(h->stream));
      cudaFree(buf.p);
      buf.p = nullptr;
      buf.cap = 0;
      ws->prox_blocks = ws->prox_frames = 0;
    }
    DPV_CUDA(h, cudaMalloc((void**)&buf.p, bytes));
    buf.cap = (long long)bytes;
    DPV_CUDA(h, cudaMemsetAsync(buf.p, 0, bytes, h->stream));
    ws->prox_blocks = blocks;
    ws->prox_frames = frames;
  }
  unsigned char* base = buf.p;
  ProxSync Y;
  Y.words = reinterpret_cast<unsigned*>(base);
  Y.flags = reinterpret_cast<unsigned long long*>(base + 256);
  unsigned char* pc = base + 256 + align256(8 * (size_t)ws->prox_blocks);
  const size_t cbytes = align256(16 * (size_t)ws->prox_frames);
  float4* c32 = reinterpret_cast<float4*>(pc);
  float4* clo = reinterpret_cast<float4*>(pc + cbytes);
  float* xt = reinterpret_cast<float*>(pc + 2 * cbytes);
  ProxArgs A;
  A.M = M;
  A.MW = MW;
  A.b0 = b0;
  A.Q = Q;
  A.gap = gap;
  A.nblk = nblk;
  A.fx = intrinsics[0];
  A.fy = intrinsics[1];
  A.cx = intrinsics[2];
  A.cy = intrinsics[3];
  A.ifx = split_pair(1.0 / (double)A.fx);
  A.ify = split_pair(1.0 / (double)A.fy);
  A.cxifx = split_pair((double)A.cx / (double)A.fx);
  A.cyify = split_pair((double)A.cy / (double)A.fy);
  A.r2 = split_pair(radius * radius);
  A.z_min = h->opt.z_min;
  A.width = width;
  A.height = height;
  const DF zp = split_pair(A.z_min), wp = split_pair(width), hp = split_pair(height);
  A.zf[0] = zp.hi;
  A.zf[1] = zp.lo;
  A.wf[0] = wp.hi;
  A.wf[1] = wp.lo;
  A.hf[0] = hp.hi;
  A.hf[1] = hp.lo;
  A.timeout = h->opt.timeout_cycles;
  size_t smem = PX_WARPS * ((size_t)M * sizeof(float2) + (size_t)MW * sizeof(unsigned));
  // With at most one CTA per SM to place, ask for enough shared memory that
  // the scheduler cannot put two on one SM: a pair shares the SM's issue
  // slots and finishes last, and every later CTA's offset waits for it.
  if (nblk <= h->num_sms) smem = std::max<size_t>(smem, PX_SOLO_SMEM);
  static bool smem_set = false;
  if (!smem_set) {
    DPV_CUDA(h, cudaFuncSetAttribute(k_prox_main, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(PX_SOLO_SMEM, PX_WARPS * (PX_MAX_M * sizeof(float2) +
                                                                                     PX_MAX_M / 32 * sizeof(unsigned)))));
    smem_set = true;
  }
  dpv_prof_begin(h, BA_KERNEL_PROXIMITY);
  k_prox_frames<<<(b1 + PX_FR - 1) / PX_FR, PX_FR * 8, 0, h->stream>>>(b1, poses, A, c32, clo, xt);
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk);
    cfg.blockDim = dim3(PX_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DPV_CUDA(h, cudaLaunchKernelEx(&cfg, k_prox_main, A, (const float4*)c32, (const float4*)clo, (const float*)xt,
                                   patches, match, ii, jj, kk, reinterpret_cast<float2*>(coords), cap, count, Y));
  }
  dpv_prof_end(h);
  h->launches += 2;
  DPV_CUDA(h, cudaGetLastError());
  if (n_host) {
    int c = 0;
    DPV_CUDA(h, cudaMemcpyAsync(&c, count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DPV_CUDA(h, cudaStreamSynchronize(h->stream));
    *n_host = c;
    if (c < 0) return dpv_fail(h, BA_ERR_TIMEOUT, "ba_proximity_edges: a device-side wait ran out");
    if (c > cap) return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: more edges than the output capacity");
  }
  return BA_OK;
}
