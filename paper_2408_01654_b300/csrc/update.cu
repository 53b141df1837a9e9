// State update of one Gauss-Newton iteration (Sec. 3.1 Eq. 3, Schur form of
// Sec. 3.2): back-substitution of the inverse depths and SE(3) retraction of
// the free poses.
//
//   dd_k = Ct_k^-1 ( w_k - sum_a e_{a,k}^T dxi_a ),  d_k <- max(d_k + dd_k, d_min)
//   T_a <- Exp(dxi_a) T_a   (FP64, left perturbation, xi = (rho, phi))
//
// The back-substitution re-linearises the group's edges (same run layout and
// arithmetic as the assembly kernel, so e_{a,k} is reproduced exactly) rather
// than storing the E blocks: 12 bytes of edge data re-read per edge instead
// of 48 bytes written and read back.
#include "internal.cuh"

namespace {

constexpr int BS_THREADS = 256;
constexpr int BS_WARPS = BS_THREADS / 32;

__global__ void __launch_bounds__(BS_THREADS) k_backsub(
    int G, int P, int fixed, float z_min, float d_min, const int* __restrict__ gseg, const int* __restrict__ runptr,
    const unsigned* __restrict__ eslot, const int* __restrict__ perm, const int* __restrict__ win,
    const int* __restrict__ wlen, const double* __restrict__ poses, float* __restrict__ patches,
    const float* __restrict__ weights, const float* __restrict__ intr, const double* __restrict__ dx,
    const float* __restrict__ Ct, const float* __restrict__ wk, float* __restrict__ dd_out, const int* status) {
  __shared__ float pd[3 * DPV_GMAX];
  __shared__ float acc[DPV_GMAX];
  __shared__ float rp[BS_WARPS][24];
  __shared__ int wf[DPV_WMAX];
  __shared__ float xi[6 * DPV_WMAX];
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int w = wlen[g];
  float K[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) K[q] = intr[q];
  for (int q = tid; q < w; q += BS_THREADS) wf[q] = win[g * DPV_WMAX + q];
  for (int q = tid; q < G; q += BS_THREADS) {
    const int k = g * G + q;
    float x0 = 0.f, x1 = 0.f, d = 1.f;
    if (k < P) {
      const float* pk = patches + 27 * (size_t)k;
      x0 = (pk[4] - K[2]) / K[0];
      x1 = (pk[13] - K[3]) / K[1];
      d = pk[22];
    }
    pd[3 * q] = x0;
    pd[3 * q + 1] = x1;
    pd[3 * q + 2] = d;
    acc[q] = 0.f;
  }
  __syncthreads();
  for (int q = tid; q < 6 * w; q += BS_THREADS) {
    const int f = wf[q / 6];
    xi[q] = f >= fixed ? (float)dx[6 * (f - fixed) + (q % 6)] : 0.f;
  }
  __syncthreads();

  const int r0 = gseg[g], r1 = gseg[g + 1];
  for (int r = r0 + wid; r < r1; r += BS_WARPS) {
    const int s0 = runptr[r], s1 = runptr[r + 1];
    const unsigned sw0 = eslot[s0];
    const int si = dpv_slot_i(sw0), sj = dpv_slot_j(sw0);
    if (si == sj) continue;
    if (lane == 0) {
      RelPose T;
      dpv_relative_pose(poses + 7 * (size_t)wf[si], poses + 7 * (size_t)wf[sj], T);
#pragma unroll
      for (int m = 0; m < 9; ++m) rp[wid][m] = T.R[m];
#pragma unroll
      for (int m = 0; m < 3; ++m) rp[wid][9 + m] = T.t[m];
#pragma unroll
      for (int m = 0; m < 9; ++m) rp[wid][12 + m] = T.txR[m];
    }
    __syncwarp();
    RelPose T;
#pragma unroll
    for (int m = 0; m < 9; ++m) T.R[m] = rp[wid][m];
#pragma unroll
    for (int m = 0; m < 3; ++m) T.t[m] = rp[wid][9 + m];
#pragma unroll
    for (int m = 0; m < 9; ++m) T.txR[m] = rp[wid][12 + m];
    __syncwarp();
    float xa[6], xb[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      xa[m] = xi[6 * si + m];
      xb[m] = xi[6 * sj + m];
    }
    for (int s = s0 + lane; s < s1; s += 32) {
      const int kl = dpv_slot_k(eslot[s]);
      const int e = perm[s];
      const float2 wt = *reinterpret_cast<const float2*>(weights + 2 * (size_t)e);
      EdgeLin L;
      dpv_edge_linearize(T, pd[3 * kl], pd[3 * kl + 1], pd[3 * kl + 2], 0.f, 0.f, K, z_min, false, L);
      if (!L.valid) continue;
      const float wJd0 = wt.x * L.Jd[0], wJd1 = wt.y * L.Jd[1];
      float q = 0.f;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        q = fmaf(L.Ji[0][m] * wJd0 + L.Ji[1][m] * wJd1, xa[m], q);
        q = fmaf(L.Jj[0][m] * wJd0 + L.Jj[1][m] * wJd1, xb[m], q);
      }
      atomicAdd(&acc[kl], q);
    }
  }
  __syncthreads();
  for (int q = tid; q < G; q += BS_THREADS) {
    const int k = g * G + q;
    if (k >= P) continue;
    const float dd = (wk[k] - acc[q]) / Ct[k];
    const float dn = fmaxf(pd[3 * q + 2] + dd, d_min);
    dd_out[k] = dd;
    float* pk = patches + 27 * (size_t)k + 18;
#pragma unroll
    for (int m = 0; m < 9; ++m) pk[m] = dn;
  }
}

// T <- Exp(xi) T for every free pose, FP64.  Exp(xi) = [R(phi) V(phi) rho; 0 1]
// with R from the unit quaternion (sin(th/2)/th phi, cos(th/2)) and
// V = I + B [phi]x + C [phi]x^2, B = (1 - cos th)/th^2 = 2 sin^2(th/2)/th^2,
// C = (th - sin th)/th^3; the coefficients switch to their Taylor series in
// th^2 below th = 1e-3.
__global__ void k_retract(int N, int fixed, const double* __restrict__ dx, double* __restrict__ poses,
                          const int* status) {
  if (dpv_status(status)) return;
  const int f = fixed + blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= N) return;
  const double* x = dx + 6 * (f - fixed);
  const double r0 = x[0], r1 = x[1], r2 = x[2], p0 = x[3], p1 = x[4], p2 = x[5];
  const double th2 = p0 * p0 + p1 * p1 + p2 * p2;
  double a, c, B, C;
  if (th2 < 1e-6) {
    a = 0.5 - th2 * (1.0 / 48.0) + th2 * th2 * (1.0 / 3840.0);
    c = 1.0 - th2 * 0.125 + th2 * th2 * (1.0 / 384.0);
    B = 0.5 - th2 * (1.0 / 24.0) + th2 * th2 * (1.0 / 720.0);
    C = 1.0 / 6.0 - th2 * (1.0 / 120.0) + th2 * th2 * (1.0 / 5040.0);
  } else {
    const double th = sqrt(th2);
    double sh, ch;
    sincos(0.5 * th, &sh, &ch);
    a = sh / th;
    c = ch;
    B = 2.0 * sh * sh / th2;
    C = (th - sin(th)) / (th2 * th);
  }
  const double qe[4] = {a * p0, a * p1, a * p2, c};
  double* P = poses + 7 * (size_t)f;
  // phi x rho and phi x (phi x rho)
  const double u0 = p1 * r2 - p2 * r1, u1 = p2 * r0 - p0 * r2, u2 = p0 * r1 - p1 * r0;
  const double v0 = p1 * u2 - p2 * u1, v1 = p2 * u0 - p0 * u2, v2 = p0 * u1 - p1 * u0;
  double Re[9];
  dpv_quat_rot64(qe, Re);
  const double t0 = P[0], t1 = P[1], t2 = P[2];
  P[0] = Re[0] * t0 + Re[1] * t1 + Re[2] * t2 + r0 + B * u0 + C * v0;
  P[1] = Re[3] * t0 + Re[4] * t1 + Re[5] * t2 + r1 + B * u1 + C * v1;
  P[2] = Re[6] * t0 + Re[7] * t1 + Re[8] * t2 + r2 + B * u2 + C * v2;
  const double bx = P[3], by = P[4], bz = P[5], bw = P[6];
  double nq[4];
  nq[0] = qe[3] * bx + qe[0] * bw + qe[1] * bz - qe[2] * by;
  nq[1] = qe[3] * by - qe[0] * bz + qe[1] * bw + qe[2] * bx;
  nq[2] = qe[3] * bz + qe[0] * by - qe[1] * bx + qe[2] * bw;
  nq[3] = qe[3] * bw - qe[0] * bx - qe[1] * by - qe[2] * bz;
  const double inv = 1.0 / sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
#pragma unroll
  for (int m = 0; m < 4; ++m) P[3 + m] = nq[m] * inv;
}

}  // namespace

ba_status_t dpv_backsub(ba_handle_t h) {
  Workspace* ws = h->ws;
  k_backsub<<<h->ngroups, BS_THREADS, 0, h->stream>>>(
      h->G, h->P, h->fixed, h->opt.z_min, h->opt.d_min, ws->gseg.p, ws->runptr.p, ws->eslot.p, ws->perm.p, ws->win.p,
      ws->wlen.p, h->poses, h->patches, h->weights, ws->intr, ws->dx.p, ws->Ct.p, ws->wk.p, ws->dd.p, ws->status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

ba_status_t dpv_retract(ba_handle_t h) {
  const int nf = h->N - h->fixed;
  if (nf <= 0) return BA_OK;
  k_retract<<<(nf + 127) / 128, 128, 0, h->stream>>>(h->N, h->fixed, h->ws->dx.p, h->poses, h->ws->status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
