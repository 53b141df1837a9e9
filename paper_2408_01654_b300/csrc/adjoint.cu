// Adjoint (reverse mode) of the recorded Gauss-Newton iterations of Eq. 3
// (Sec. 3.1), i.e. the derivative of a loss on the final poses and inverse
// depths with respect to the targets and weights that the update operator
// feeds into the bundle adjustment (Sec. 3.1: the layer is differentiable and
// trained end to end; gradients flow through the unrolled iterations).
//
// One iteration maps the state x_s (poses, inverse depths) to
//   x_{s+1} = R(x_s, Delta),  H(x_s) Delta = g(x_s),
//   H = sum_e J_e^T W_e J_e + damping,  g = sum_e J_e^T W_e r_e,
// with R the retraction T <- Exp(dxi) T and the clamp d <- max(d + dd, d_min).
// Pose cotangents are kept in the left-perturbation tangent space of each pose
// (xi = (rho, phi), T <- Exp(xi) T); depth cotangents per patch.  Given the
// cotangent of x_{s+1}, the step goes:
//   1. retraction adjoint: Delta_bar = (dR/dDelta)^T x_bar_{s+1}, and the part
//      of x_bar_s that passes through R (k_adj_retract, FP64 duals);
//   2. lambda = H^-1 Delta_bar: the same Schur elimination, Cholesky solve and
//      back-substitution as the forward step, with (Delta_bar_xi, Delta_bar_d)
//      as the right-hand side (H is symmetric);
//   3. per edge, with a = J lambda, b = J Delta (2-vectors):
//        target_bar += W a,   weight_bar_c += a_c (r_c - b_c),
//        x_bar_s += d/dx [ sum_c w_c a_c (r_c - b_c) ]  (lambda, Delta held),
//      the last through FP32 dual numbers in the 6 directions of a left
//      perturbation of the edge's relative pose and the patch's inverse depth
//      (k_adj_edges); the pose part is reduced per (source, target) run and
//      added to the two poses in FP64.
// Masked edges (self edges, points behind z_min) contribute nothing, and fixed
// poses have no cotangent.
#include "internal.cuh"

#include "dual.cuh"
#include "retract.cuh"

namespace {

constexpr int ADJ_THREADS = 256;
constexpr int ADJ_WARPS = ADJ_THREADS / 32;

using D2 = Dual<double, 2>;
using D7 = Dual<float, 7>;

// First-order change (dt, dq) of a pose p = (t, q) under T <- Exp(eps e_k) T:
// dt = rho + omega x t, dq = 1/2 (omega, 0) (x) q.
__device__ void left_change(int k, const double* p, double* dt, double* dq) {
  double rho[3] = {0.0, 0.0, 0.0}, om[3] = {0.0, 0.0, 0.0};
  if (k < 3) rho[k] = 1.0;
  else om[k - 3] = 1.0;
  dt[0] = rho[0] + om[1] * p[2] - om[2] * p[1];
  dt[1] = rho[1] + om[2] * p[0] - om[0] * p[2];
  dt[2] = rho[2] + om[0] * p[1] - om[1] * p[0];
  const double qx = p[3], qy = p[4], qz = p[5], qw = p[6];
  dq[0] = 0.5 * (qw * om[0] + om[1] * qz - om[2] * qy);
  dq[1] = 0.5 * (qw * om[1] + om[2] * qx - om[0] * qz);
  dq[2] = 0.5 * (qw * om[2] + om[0] * qy - om[1] * qx);
  dq[3] = -0.5 * (om[0] * qx + om[1] * qy + om[2] * qz);
}

// Tangent (rho, omega) of a first-order change (dt, dq) at the unit pose p:
// omega = 2 vec(dq (x) q*), rho = dt - omega x t.
__device__ void tangent_of(const double* p, const double* dt, const double* dq, double* eta) {
  const double qx = p[3], qy = p[4], qz = p[5], qw = p[6];
  // vec(dq (x) q*) with q* = (-q_v, q_w)
  const double w0 = -dq[3] * qx + qw * dq[0] - (dq[1] * qz - dq[2] * qy);
  const double w1 = -dq[3] * qy + qw * dq[1] - (dq[2] * qx - dq[0] * qz);
  const double w2 = -dq[3] * qz + qw * dq[2] - (dq[0] * qy - dq[1] * qx);
  const double om[3] = {2.0 * w0, 2.0 * w1, 2.0 * w2};
  eta[3] = om[0];
  eta[4] = om[1];
  eta[5] = om[2];
  eta[0] = dt[0] - (om[1] * p[2] - om[2] * p[1]);
  eta[1] = dt[1] - (om[2] * p[0] - om[0] * p[2]);
  eta[2] = dt[2] - (om[0] * p[1] - om[1] * p[0]);
}

// Cotangent of the final poses, given per coordinate of (t, q), mapped to the
// tangent space: xb[a][k] = <grad_a, d(t, q)/d xi_k>.  Fixed poses get 0.
__global__ void k_adj_init(int N, const int* __restrict__ fdx, const double* __restrict__ poses,
                           const double* __restrict__ grad, double* __restrict__ xb, const int* status) {
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 6 * N) return;
  const int a = q / 6, k = q - 6 * a;
  if (fdx[a] < 0) {
    xb[q] = 0.0;
    return;
  }
  double dt[3], dq[4];
  left_change(k, poses + 7 * (size_t)a, dt, dq);
  const double* g = grad + 7 * (size_t)a;
  xb[q] = g[0] * dt[0] + g[1] * dt[1] + g[2] * dt[2] + g[3] * dq[0] + g[4] * dq[1] + g[5] * dq[2] + g[6] * dq[3];
}

// Step 1 for iteration s.  Pose part, thread (a, k) of a free pose a:
//   vext[k]  = sum_m M[m][k] xb_next[a][m],   M = d tangent(T_{s+1}) / d dxi  (the
//              SE(3) left Jacobian at dxi),
//   xb_cur[k] = sum_m A[m][k] xb_next[a][m],  A = d tangent(T_{s+1}) / d tangent(T_s)
//              (= Ad(Exp(dxi))),
// both columns from one run of the retraction in 2-direction FP64 dual numbers.
// Depth part, thread k: the full cotangent of d_{s+1,k} (the part that passed
// the clamp + the per-edge terms of iteration s+1, patch-major) times the
// clamp's derivative [d_s + dd_s > d_min].
__global__ void k_adj_retract(int N, const int* __restrict__ fdx, int P, float d_min,
                              const double* __restrict__ xb_next,
                              const double* __restrict__ dx_s, const double* __restrict__ poses_s,
                              double* __restrict__ vext, double* __restrict__ xb_cur,
                              const float* __restrict__ db_next, const float* __restrict__ gd,
                              const int* __restrict__ pptr, const float* __restrict__ patches_s,
                              const float* __restrict__ dd_s, float* __restrict__ wext, const int* status) {
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 6 * N) {
    const int a = q / 6, k = q - 6 * a;
    const int o = fdx[a];
    if (o < 0) {
      xb_cur[q] = 0.0;
      return;
    }
    D2 x[6], T[7];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      x[m] = dual_const<double, 2>(dx_s[o + m]);
      if (m == k) x[m].g[0] = 1.0;
    }
    const double* p = poses_s + 7 * (size_t)a;
    double dt[3], dq[4];
    left_change(k, p, dt, dq);
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      T[m] = dual_const<double, 2>(p[m]);
      T[m].g[1] = m < 3 ? dt[m] : dq[m - 3];
    }
    dpv_se3_retract_t(x, T);
    double pv[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) pv[m] = T[m].v;
    const double* xn = xb_next + 6 * (size_t)a;
    double out[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double ct[3], cq[4], eta[6];
#pragma unroll
      for (int m = 0; m < 3; ++m) ct[m] = T[m].g[c];
#pragma unroll
      for (int m = 0; m < 4; ++m) cq[m] = T[3 + m].g[c];
      tangent_of(pv, ct, cq, eta);
      out[c] = 0.0;
#pragma unroll
      for (int m = 0; m < 6; ++m) out[c] += eta[m] * xn[m];
    }
    vext[o + k] = out[0];
    xb_cur[q] = out[1];
    return;
  }
  const int k = q - 6 * N;
  if (k >= P) return;
  float db = db_next[k];
  if (gd)
    for (int e = pptr[k]; e < pptr[k + 1]; ++e) db += gd[e];
  const float dn = patches_s[27 * (size_t)k + 22] + dd_s[k];
  wext[k] = dn > d_min ? db : 0.f;
}

// Cotangent of the initial inverse depths: the clamp-passed part + the
// per-edge terms of iteration 0.
__global__ void k_adj_final(int P, const float* __restrict__ db, const float* __restrict__ gd,
                            const int* __restrict__ pptr, float* __restrict__ out, const int* status) {
  if (dpv_status(status)) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  float v = db[k];
  if (gd)
    for (int e = pptr[k]; e < pptr[k + 1]; ++e) v += gd[e];
  out[k] = v;
}

// e_q x v
__device__ __forceinline__ void ecross(int q, const float* v, float* o) {
  o[0] = q == 1 ? v[2] : (q == 2 ? -v[1] : 0.f);
  o[1] = q == 0 ? -v[2] : (q == 2 ? v[0] : 0.f);
  o[2] = q == 0 ? v[1] : (q == 1 ? -v[0] : 0.f);
}

__device__ __forceinline__ void dcross(const D7* a, const D7* b, D7* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// v (6) under a left perturbation delta of the relative pose, to first order:
// Ad(Exp(delta) T) v_i = (I + ad(delta)) m,  m = Ad(T) v_i, and the step of the
// target frame is fixed, so  mu = v_j - m - ad(delta) m  with
// ad(rho, phi) m = (phi x m_rho + rho x m_phi, phi x m_phi).
__device__ __forceinline__ void perturbed_diff(const float* vj, const float* m, D7* mu) {
#pragma unroll
  for (int c = 0; c < 6; ++c) mu[c] = dual_const<float, 7>(vj[c] - m[c]);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float e1[3], e2[3], e3[3];
    ecross(q, m + 3, e1);  // d/d rho_q of the rho part: -(e_q x m_phi)
    ecross(q, m, e2);      // d/d phi_q of the rho part: -(e_q x m_rho)
    ecross(q, m + 3, e3);  // d/d phi_q of the phi part: -(e_q x m_phi)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mu[c].g[q] = -e1[c];
      mu[c].g[3 + q] = -e2[c];
      mu[3 + c].g[3 + q] = -e3[c];
    }
  }
}

// Ad(T) v for T = (R, t) with txR = [t]x R:  (R v_rho + txR v_phi, R v_phi)
__device__ __forceinline__ void adjoint_apply(const RelPose& T, const float* v, float* o) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    o[r] = T.R[3 * r] * v[0] + T.R[3 * r + 1] * v[1] + T.R[3 * r + 2] * v[2] + T.txR[3 * r] * v[3] +
           T.txR[3 * r + 1] * v[4] + T.txR[3 * r + 2] * v[5];
    o[3 + r] = T.R[3 * r] * v[3] + T.R[3 * r + 1] * v[4] + T.R[3 * r + 2] * v[5];
  }
}

// Step 3 for iteration s: one CTA per patch group, one warp per (source,
// target) run, one lane per edge.
// PIX residual pixels per edge (1: the patch centre; 9: the whole patch,
// targets and their cotangents [E,9,2]): the edge's terms are the sums over
// its pixels, each pixel masked on its own as in the forward assembly.
template <int PIX>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_edges(
    int G, int P, const int* __restrict__ fdx, const int* __restrict__ gprob, float z_min,
    const int* __restrict__ gptr,
    const int* __restrict__ grun,
    const int* __restrict__ gnr, const unsigned* __restrict__ eslot, const int* __restrict__ perm,
    const int* __restrict__ pmpos, const int* __restrict__ win, const float* __restrict__ posef,
    const float* __restrict__ patches, const float* __restrict__ targets, const float* __restrict__ weights,
    const float* __restrict__ intr, const float* __restrict__ lam_p, const float* __restrict__ lam_d,
    const double* __restrict__ dx_s, const float* __restrict__ dd_s, float* __restrict__ gT, float* __restrict__ gW,
    float* __restrict__ gd, double* __restrict__ xb, const int* status) {
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gs = gptr[g], nruns = gnr[g];
  const int* runptr = grun + (size_t)g * (DPV_RMAX + 1);
  const int* wf = win + (size_t)g * DPV_WMAX;
  const float* Kg = intr + 4 * gprob[g];  // the group's problem's intrinsics
  const float fx = Kg[0], fy = Kg[1], cx = Kg[2], cy = Kg[3];
  for (int r = wid; r < nruns; r += ADJ_WARPS) {
    const int s0 = gs + runptr[r], s1 = gs + runptr[r + 1];
    const unsigned sw0 = eslot[s0];
    const int si = dpv_slot_i(sw0), sj = dpv_slot_j(sw0);
    if (si == sj) {  // self edges are masked in the forward step
      for (int s = s0 + lane; s < s1; s += 32) gd[pmpos[s]] = 0.f;
      continue;
    }
    const int fi = wf[si], fj = wf[sj];
    RelPose T;  // as in the forward assembly (the pose table is the one of x_s)
    dpv_relative_pose_df(posef + DPV_POSE_ROW * (size_t)fi, posef + DPV_POSE_ROW * (size_t)fj, T);
    const int oi = fdx[fi], oj = fdx[fj];
    float li[6], lj[6], di[6], dj[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      li[m] = oi >= 0 ? lam_p[oi + m] : 0.f;
      lj[m] = oj >= 0 ? lam_p[oj + m] : 0.f;
      di[m] = oi >= 0 ? dpv_d2f_bits(dx_s[oi + m]) : 0.f;
      dj[m] = oj >= 0 ? dpv_d2f_bits(dx_s[oj + m]) : 0.f;
    }
    float ml[6], md[6];
    adjoint_apply(T, li, ml);
    adjoint_apply(T, di, md);
    float gdel[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = s0 + lane; s < s1; s += 32) {
      const int kl = dpv_slot_k(eslot[s]);
      const int k = g * G + kl;
      const int e = perm[s];
      const float* pk = patches + 27 * (size_t)k;
      const float d = pk[22];
      const float2 wt = *reinterpret_cast<const float2*>(weights + 2 * (size_t)e);
      const float ld = lam_d[k], Dd = dd_s[k];
      float gdk = 0.f, gw0 = 0.f, gw1 = 0.f;
#pragma unroll 1
      for (int px = 0; px < PIX; ++px) {
        const int pp = PIX == 1 ? 4 : px;
        const float xb0 = (pk[pp] - cx) / fx, xb1 = (pk[9 + pp] - cy) / fy;
        // the forward step's point and mask, bit for bit
        const float X = fmaf(T.R[0], xb0, fmaf(T.R[1], xb1, fmaf(T.t[0], d, T.R[2])));
        const float Y = fmaf(T.R[3], xb0, fmaf(T.R[4], xb1, fmaf(T.t[1], d, T.R[5])));
        const float Z = fmaf(T.R[6], xb0, fmaf(T.R[7], xb1, fmaf(T.t[2], d, T.R[8])));
        if (!(Z > z_min * d)) continue;
        const size_t te = (size_t)e * PIX + px;
        const float2 tg = *reinterpret_cast<const float2*>(targets + 2 * te);
        // point, translation and depth as duals in (rho, phi, d)
        const float Xv[3] = {X, Y, Z};
        D7 Xd[3], td[3], dd;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Xd[c] = dual_const<float, 7>(Xv[c]);
          Xd[c].g[c] = d;
          td[c] = dual_const<float, 7>(T.t[c]);
          td[c].g[c] = 1.f;
          Xd[c].g[6] = T.t[c];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float ex[3], et[3];
          ecross(q, Xv, ex);
          ecross(q, T.t, et);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Xd[c].g[3 + q] = ex[c];
            td[c].g[3 + q] = et[c];
          }
        }
        dd = dual_const<float, 7>(d);
        dd.g[6] = 1.f;
        // A = d mu_rho + mu_phi x X + lambda_d t (a = D A), B likewise with the step
        D7 A[3], B[3];
        {
          D7 mu[6], cr[3];
          perturbed_diff(lj, ml, mu);
          dcross(mu + 3, Xd, cr);
#pragma unroll
          for (int c = 0; c < 3; ++c) A[c] = dd * mu[c] + cr[c] + ld * td[c];
          perturbed_diff(dj, md, mu);
          dcross(mu + 3, Xd, cr);
#pragma unroll
          for (int c = 0; c < 3; ++c) B[c] = dd * mu[c] + cr[c] + Dd * td[c];
        }
        const D7 iz = 1.f / Xd[2];
        const D7 u = Xd[0] * iz, v = Xd[1] * iz;
        const D7 a0 = fx * iz * (A[0] - u * A[2]), a1 = fy * iz * (A[1] - v * A[2]);
        const D7 b0 = fx * iz * (B[0] - u * B[2]), b1 = fy * iz * (B[1] - v * B[2]);
        D7 r0 = tg.x - (fx * u + cx), r1 = tg.y - (fy * v + cy);
        const float izv = 1.0f / Z;  // the forward step's residual value
        r0.v = tg.x - fmaf(fx * X, izv, cx);
        r1.v = tg.y - fmaf(fy * Y, izv, cy);
        const D7 phi = wt.x * (a0 * (r0 - b0)) + wt.y * (a1 * (r1 - b1));
        float2* pT = reinterpret_cast<float2*>(gT + 2 * te);
        float2 t2 = *pT;
        t2.x += wt.x * a0.v;
        t2.y += wt.y * a1.v;
        *pT = t2;
        gw0 += a0.v * (r0.v - b0.v);
        gw1 += a1.v * (r1.v - b1.v);
        gdk += phi.g[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) gdel[m] += phi.g[m];
      }
      float2* pW = reinterpret_cast<float2*>(gW + 2 * (size_t)e);
      float2 w2 = *pW;
      w2.x += gw0;
      w2.y += gw1;
      *pW = w2;
      gd[pmpos[s]] = gdk;
    }
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) gdel[m] += __shfl_xor_sync(0xffffffffu, gdel[m], o);
    if (lane == 0) {
      if (oj >= 0)
        for (int m = 0; m < 6; ++m) atomicAdd(xb + 6 * (size_t)fj + m, dpv_f2d_bits(gdel[m]));
      if (oi >= 0) {
        // d delta / d xi_i = -Ad(T_ij):  xb_i -= Ad^T gdel = (R^T g_rho, txR^T g_rho + R^T g_phi)
        for (int c = 0; c < 3; ++c) {
          const float pr = T.R[c] * gdel[0] + T.R[3 + c] * gdel[1] + T.R[6 + c] * gdel[2];
          const float pp = T.txR[c] * gdel[0] + T.txR[3 + c] * gdel[1] + T.txR[6 + c] * gdel[2] +
                           T.R[c] * gdel[3] + T.R[3 + c] * gdel[4] + T.R[6 + c] * gdel[5];
          atomicAdd(xb + 6 * (size_t)fi + c, dpv_f2d_bits(-pr));
          atomicAdd(xb + 6 * (size_t)fi + 3 + c, dpv_f2d_bits(-pp));
        }
      }
    }
  }
}

// Restores the handle's state pointers when the backward pass leaves.
struct StateGuard {
  ba_handle_t h;
  double* poses;
  float* patches;
  ~StateGuard() {
    h->poses = poses;
    h->patches = patches;
  }
};

}  // namespace

// Tape of one recorded ba_step call: x_s before each iteration, x_K after the
// last, and each iteration's step (dxi in FP64, dd in FP32).
ba_status_t dpv_tape_reserve(ba_handle_t h, int iters) {
  Workspace* ws = h->ws;
  ba_status_t s;
  if ((s = dpv_grow(h, ws->tp_poses, 7LL * h->N * (iters + 1), "tape poses")) ||
      (s = dpv_grow(h, ws->tp_patches, 27LL * h->P * iters, "tape patches")) ||
      (s = dpv_grow(h, ws->tp_dx, (long long)h->n_pad * iters, "tape steps")) ||
      (s = dpv_grow(h, ws->tp_dd, (long long)h->P * iters, "tape depth steps")))
    return s;
  return BA_OK;
}

ba_status_t dpv_tape_state(ba_handle_t h, int it) {
  Workspace* ws = h->ws;
  DPV_CUDA(h, cudaMemcpyAsync(ws->tp_poses.p + 7LL * h->N * it, h->poses, sizeof(double) * 7 * h->N,
                              cudaMemcpyDeviceToDevice, h->stream));
  if (it < h->tape_iters_pending)
    DPV_CUDA(h, cudaMemcpyAsync(ws->tp_patches.p + 27LL * h->P * it, h->patches, sizeof(float) * 27 * h->P,
                                cudaMemcpyDeviceToDevice, h->stream));
  return BA_OK;
}

ba_status_t dpv_tape_step(ba_handle_t h, int it) {
  Workspace* ws = h->ws;
  DPV_CUDA(h, cudaMemcpyAsync(ws->tp_dx.p + (long long)h->n_pad * it, ws->dx.p, sizeof(double) * h->n_pad,
                              cudaMemcpyDeviceToDevice, h->stream));
  DPV_CUDA(h, cudaMemcpyAsync(ws->tp_dd.p + (long long)h->P * it, ws->dd.p, sizeof(float) * h->P,
                              cudaMemcpyDeviceToDevice, h->stream));
  return BA_OK;
}

extern "C" ba_status_t ba_set_record(ba_handle_t h, int on) {
  if (!h) return BA_ERR_INVALID_ARG;
  h->record = on ? 1 : 0;
  return BA_OK;
}

extern "C" ba_status_t ba_backward(ba_handle_t h, const double* grad_poses, const float* grad_depths,
                                   float* grad_targets, float* grad_weights, double* grad_tangent0,
                                   float* grad_depths0) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!h->have_graph || !h->tape_valid)
    return dpv_fail(h, BA_ERR_STATE, "ba_backward: no recorded ba_step (call ba_set_record(h, 1) before ba_step)");
  if (h->patches_padded)
    return dpv_fail(h, BA_ERR_UNSUPPORTED,
                    "ba_backward: a batched binding whose patch counts are not multiples of the group size "
                    "(the library works on a padded copy of the patches) has no adjoint; choose a group size "
                    "that divides every problem's patch count");
  if ((reinterpret_cast<uintptr_t>(grad_targets) | reinterpret_cast<uintptr_t>(grad_weights)) & 7)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_backward: grad_targets/grad_weights must be 8-byte aligned");
  Workspace* ws = h->ws;
  const int N = h->N, P = h->P, E = h->E, K = h->tape_iters;
  ba_status_t s;
  // the system geometry of the recorded call (a later ba_step may have used another fixed count)
  if ((s = dpv_ensure_system(h, h->tape_fixed))) return s;
  const int* fdx = ws->fdx.p;
  const long long E2 = 2LL * (E > 0 ? E : 1);
  if ((s = dpv_grow(h, ws->ad_xb, 12LL * N, "pose cotangents")) ||
      (s = dpv_grow(h, ws->ad_w, 2LL * P, "depth cotangents")) ||
      (s = dpv_grow(h, ws->ad_gd, E > 0 ? E : 1, "edge depth cotangents")) ||
      (s = dpv_grow(h, ws->ad_lamd, P, "depth multipliers")) ||
      (s = dpv_grow(h, ws->ad_v, h->n_pad, "adjoint rhs")) ||
      (!grad_targets && (s = dpv_grow(h, ws->ad_gt, E2 * h->opt.residual_pixels, "target cotangents"))) ||
      (!grad_weights && (s = dpv_grow(h, ws->ad_gw, E2, "weight cotangents"))))
    return s;
  DPV_CUDA(h, cudaMemsetAsync(ws->ad_v.p, 0, sizeof(double) * h->n_pad, h->stream));
  float* gT = grad_targets ? grad_targets : ws->ad_gt.p;
  float* gW = grad_weights ? grad_weights : ws->ad_gw.p;
  if (E > 0) {
    DPV_CUDA(h, cudaMemsetAsync(gT, 0, sizeof(float) * 2 * E * h->opt.residual_pixels, h->stream));
    DPV_CUDA(h, cudaMemsetAsync(gW, 0, sizeof(float) * 2 * E, h->stream));
  }
  double* xbn = ws->ad_xb.p;
  double* xbc = ws->ad_xb.p + 6LL * N;
  float* wn = ws->ad_w.p;
  float* wc = ws->ad_w.p + P;
  dpv_prof_begin(h, BA_KERNEL_ADJOINT);
  if (grad_poses) {
    k_adj_init<<<(6 * N + 127) / 128, 128, 0, h->stream>>>(N, fdx, ws->tp_poses.p + 7LL * N * K, grad_poses, xbn,
                                                             ws->status);
    ++h->launches;
  } else {
    DPV_CUDA(h, cudaMemsetAsync(xbn, 0, sizeof(double) * 6 * N, h->stream));
  }
  if (grad_depths) DPV_CUDA(h, cudaMemcpyAsync(wn, grad_depths, sizeof(float) * P, cudaMemcpyDefault, h->stream));
  else DPV_CUDA(h, cudaMemsetAsync(wn, 0, sizeof(float) * P, h->stream));
  dpv_prof_end(h);
  DPV_CUDA(h, cudaGetLastError());
  const float* gdp = nullptr;  // per-edge depth terms of the iteration after s
  StateGuard guard{h, h->poses, h->patches};
  for (int it = K - 1; it >= 0; --it) {
    const double* poses_s = ws->tp_poses.p + 7LL * N * it;
    float* patches_s = ws->tp_patches.p + 27LL * P * it;
    const double* dx_s = ws->tp_dx.p + (long long)h->n_pad * it;
    const float* dd_s = ws->tp_dd.p + (long long)P * it;
    dpv_prof_begin(h, BA_KERNEL_ADJOINT);
    const int nthr = 6 * N + P;
    k_adj_retract<<<(nthr + 127) / 128, 128, 0, h->stream>>>(N, fdx, P, h->opt.d_min, xbn, dx_s, poses_s,
                                                               ws->ad_v.p, xbc, wn, gdp, ws->pptr.p, patches_s, dd_s,
                                                               wc, ws->status);
    ++h->launches;
    dpv_prof_end(h);
    DPV_CUDA(h, cudaGetLastError());
    // lambda = H(x_s)^-1 (vext, wext): the forward elimination at x_s
    h->poses = const_cast<double*>(poses_s);
    h->patches = patches_s;
    if ((s = dpv_assemble_ext(h, -1, ws->ad_v.p, wc))) return s;
    int retracted = 0;
    dpv_prof_begin(h, BA_KERNEL_SOLVE);
    s = dpv_solve(h, &retracted);
    dpv_prof_end(h);
    if (s) return s;
    dpv_prof_begin(h, BA_KERNEL_BACKSUB);
    s = dpv_backsub_ext(h, wc, ws->ad_lamd.p);
    dpv_prof_end(h);
    if (s) return s;
    dpv_prof_begin(h, BA_KERNEL_ADJOINT);
    auto adj_edges = h->opt.residual_pixels == 9 ? k_adj_edges<9> : k_adj_edges<1>;
    adj_edges<<<h->ngroups, ADJ_THREADS, 0, h->stream>>>(
        h->G, P, fdx, ws->gprob.p, h->opt.z_min, ws->gptr.p, ws->grun.p, ws->gnr.p, ws->eslot.p, ws->perm.p, ws->pmpos.p,
        ws->win.p, ws->posef.p, patches_s, h->targets, h->weights, ws->intr, ws->tmpv.p, ws->ad_lamd.p, dx_s, dd_s,
        gT, gW, ws->ad_gd.p, xbc, ws->status);
    ++h->launches;
    dpv_prof_end(h);
    DPV_CUDA(h, cudaGetLastError());
    gdp = ws->ad_gd.p;
    double* tx = xbn; xbn = xbc; xbc = tx;
    float* tw = wn; wn = wc; wc = tw;
  }
  if (grad_tangent0)
    DPV_CUDA(h, cudaMemcpyAsync(grad_tangent0, xbn, sizeof(double) * 6 * N, cudaMemcpyDefault, h->stream));
  if (grad_depths0) {
    k_adj_final<<<(P + 127) / 128, 128, 0, h->stream>>>(P, wn, gdp, ws->pptr.p, grad_depths0, ws->status);
    ++h->launches;
    DPV_CUDA(h, cudaGetLastError());
  }
  return BA_OK;
}
