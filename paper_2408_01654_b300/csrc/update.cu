// State update of one Gauss-Newton iteration (Sec. 3.1 Eq. 3, Schur form of
// Sec. 3.2): back-substitution of the inverse depths and SE(3) retraction of
// the free poses.
//
//   dd_k = Ct_k^-1 ( w_k - sum_a e_{a,k}^T dxi_a ),  d_k <- max(d_k + dd_k, d_min)
//   T_a <- Exp(dxi_a) T_a   (FP64, left perturbation, xi = (rho, phi))
//
// The back-substitution reads the per-edge depth terms that the assembly
// kernel wrote in patch-major order (J_i^T W Jd, J_j^T W Jd for every edge,
// 64 bytes per edge, contiguous per patch), so it needs neither the poses nor
// a second linearisation.
#include "internal.cuh"

#include "retract.cuh"

namespace {

__global__ void k_backsub(int P, int G, int fixed, float d_min, const int* __restrict__ pptr,
                          const float4* __restrict__ pterm, const int* __restrict__ win,
                          const float* __restrict__ dxf, const float* __restrict__ Ct, const float* __restrict__ wk,
                          float* __restrict__ patches, float* __restrict__ dd_out, int N, const double* __restrict__ dx,
                          double* __restrict__ poses, int write_depth, const int* status) {
  if (dpv_status(status)) return;
  if (N > fixed && blockIdx.x == gridDim.x - 1) {
    // the extra last CTA retracts the free poses (FP64) while the others back-substitute
    for (int f = fixed + threadIdx.x; f < N; f += blockDim.x)
      dpv_se3_retract(dx + 6 * (f - fixed), poses + 7 * (size_t)f);
    return;
  }
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const int* wf = win + (k / G) * DPV_WMAX;
  DF acc = {wk[k], 0.f};
  for (int p = pptr[k]; p < pptr[k + 1]; ++p) {
    const float4 a = pterm[4 * (size_t)p], b = pterm[4 * (size_t)p + 1], c = pterm[4 * (size_t)p + 2],
                 d = pterm[4 * (size_t)p + 3];
    const int sl = __float_as_int(d.z);
    const int fi = wf[sl & 0xff] - fixed, fj = wf[sl >> 8] - fixed;
    if (fi >= 0) {
      const float* x = dxf + 6 * fi;
      df_fma(acc, -a.x, x[0]); df_fma(acc, -a.y, x[1]); df_fma(acc, -a.z, x[2]);
      df_fma(acc, -a.w, x[3]); df_fma(acc, -b.x, x[4]); df_fma(acc, -b.y, x[5]);
    }
    if (fj >= 0) {
      const float* x = dxf + 6 * fj;
      df_fma(acc, -b.z, x[0]); df_fma(acc, -b.w, x[1]); df_fma(acc, -c.x, x[2]);
      df_fma(acc, -c.y, x[3]); df_fma(acc, -c.z, x[4]); df_fma(acc, -c.w, x[5]);
    }
  }
  const float dd = df_val(acc) / Ct[k];
  dd_out[k] = dd;
  if (!write_depth) return;
  float* pk = patches + 27 * (size_t)k;
  const float dn = fmaxf(pk[22] + dd, d_min);
#pragma unroll
  for (int m = 18; m < 27; ++m) pk[m] = dn;
}

__global__ void k_retract(int N, int fixed, const double* __restrict__ dx, double* __restrict__ poses,
                          const int* status) {
  if (dpv_status(status)) return;
  const int f = fixed + blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= N) return;
  dpv_se3_retract(dx + 6 * (f - fixed), poses + 7 * (size_t)f);
}

}  // namespace

// Back-substitution of the depths; with `retract` the kernel also updates the
// poses (one extra CTA).
ba_status_t dpv_backsub(ba_handle_t h, int retract) {
  Workspace* ws = h->ws;
  const int nb = (h->P + 127) / 128 + (retract ? 1 : 0);
  k_backsub<<<nb, 128, 0, h->stream>>>(h->P, h->G, h->fixed, h->opt.d_min, ws->pptr.p, ws->pterm.p, ws->win.p,
                                       ws->tmpv.p, ws->Ct.p, ws->wk.p, h->patches, ws->dd.p,
                                       retract ? h->N : h->fixed, ws->dx.p, h->poses, 1, ws->status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

// The adjoint's depth part of lambda: out_k = Ct_k^-1 (w_ext_k - sum_a e_ak^T lambda_a),
// with lambda_a in the solver's output; no state is changed.
ba_status_t dpv_backsub_ext(ba_handle_t h, const float* w_ext, float* out) {
  Workspace* ws = h->ws;
  const int nb = (h->P + 127) / 128;
  k_backsub<<<nb, 128, 0, h->stream>>>(h->P, h->G, h->fixed, h->opt.d_min, ws->pptr.p, ws->pterm.p, ws->win.p,
                                       ws->tmpv.p, ws->Ct.p, w_ext, h->patches, out, h->fixed, ws->dx.p, h->poses, 0,
                                       ws->status);
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
