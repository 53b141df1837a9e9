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
#include "dfloat.cuh"
#include "internal.cuh"

#include "retract.cuh"

namespace {

constexpr int BS_THREADS = 256;
constexpr int BS_WARPS = BS_THREADS / 32;

// One warp per patch (lanes over its edges, compensated warp sum).  With
// `retract`, thread 0 of CTA f < N also retracts pose f when it is free
// (FP64) and, when `posef` is given, refreshes its row of the linearisation
// table; one pose per CTA spreads the FP64 work (1/64 of the FP32 rate) over
// the SMs.  fdx maps a frame to its unknowns in dx / dxf (-1: fixed).
__global__ void __launch_bounds__(BS_THREADS) k_backsub(
    int P, int G, const int* __restrict__ fdx, float d_min, const int* __restrict__ pptr,
    const float4* __restrict__ pterm, const int* __restrict__ win, const float* __restrict__ dxf,
    const float* __restrict__ Ct, const float* __restrict__ wk, float* __restrict__ patches,
    float* __restrict__ dd_out, int N, int retract, const double* __restrict__ dx, double* __restrict__ poses,
    float* __restrict__ posef, int write_depth, const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int lane = threadIdx.x & 31;
  if (retract && threadIdx.x == 0 && (int)blockIdx.x < N) {
    const int f = blockIdx.x;
    const int o = fdx[f];
    if (o >= 0) {
      dpv_se3_retract(dx + o, poses + 7 * (size_t)f);
      if (posef) dpv_pose_table_row(poses + 7 * (size_t)f, posef + DPV_POSE_ROW * (size_t)f);
    }
  }
  const int k = blockIdx.x * BS_WARPS + (threadIdx.x >> 5);
  if (k >= P) return;
  const int* wf = win + (k / G) * DPV_WMAX;
  DF acc = {0.f, 0.f};
  for (int p = pptr[k] + lane; p < pptr[k + 1]; p += 32) {
    const float4 a = pterm[4 * (size_t)p], b = pterm[4 * (size_t)p + 1], c = pterm[4 * (size_t)p + 2],
                 d = pterm[4 * (size_t)p + 3];
    const int sl = __float_as_int(d.z);
    const int fi = fdx[wf[sl & 0xff]], fj = fdx[wf[sl >> 8]];
    if (fi >= 0) {
      const float* x = dxf + fi;
      df_fma(acc, -a.x, x[0]); df_fma(acc, -a.y, x[1]); df_fma(acc, -a.z, x[2]);
      df_fma(acc, -a.w, x[3]); df_fma(acc, -b.x, x[4]); df_fma(acc, -b.y, x[5]);
    }
    if (fj >= 0) {
      const float* x = dxf + fj;
      df_fma(acc, -b.z, x[0]); df_fma(acc, -b.w, x[1]); df_fma(acc, -c.x, x[2]);
      df_fma(acc, -c.y, x[3]); df_fma(acc, -c.z, x[4]); df_fma(acc, -c.w, x[5]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const DF t = {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
    df_add_df(acc, t);
  }
  if (lane == 0) {
    df_add(acc, wk[k]);
    const float dd = df_val(acc) / Ct[k];
    dd_out[k] = dd;
    if (write_depth) {
      float* pk = patches + 27 * (size_t)k;
      const float dn = fmaxf(pk[22] + dd, d_min);
#pragma unroll
      for (int m = 18; m < 27; ++m) pk[m] = dn;
    }
  }
}

// The pose step as double-float pairs (once per solve, for the double-float
// back-substitution: splitting it there would repeat the split for every edge).
__global__ void k_dx_pairs(int n, const double* __restrict__ dx, float2* __restrict__ dx2, const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) dx2[q] = dpv_d2df_bits(dx[q]);
}

// The same in double-float (the BA_MIXED path): the depth terms are pairs
// (128 bytes per edge, assemble_df.cu), the pose step comes as pairs
// (k_dx_pairs), Ct and w are pairs, and the new depth d + dd is rounded to
// float once.  Two patches per warp, 16 lanes each (a patch has about a dozen
// edges), each lane's six depth-term loads issued beside its slot load.
__global__ void __launch_bounds__(BS_THREADS) k_backsub_dd(
    int P, int G, const int* __restrict__ fdx, float d_min, const int* __restrict__ pptr,
    const float4* __restrict__ pterm, const int* __restrict__ win, const float2* __restrict__ dxv,
    const float2* __restrict__ Ct2, const float2* __restrict__ wk2, const float* __restrict__ w_ext,
    float* __restrict__ patches, float* __restrict__ dd_out, int N, int retract, const double* __restrict__ dx,
    double* __restrict__ poses, float* __restrict__ posef, int write_depth, const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int lane = threadIdx.x & 31;
  if (retract && threadIdx.x == 0 && (int)blockIdx.x < N) {
    const int f = blockIdx.x;
    const int o = fdx[f];
    if (o >= 0) {
      dpv_se3_retract(dx + o, poses + 7 * (size_t)f);
      if (posef) dpv_pose_table_row(poses + 7 * (size_t)f, posef + DPV_POSE_ROW * (size_t)f);
    }
  }
  const int hl = lane & 15;
  const int k = 2 * (blockIdx.x * BS_WARPS + (threadIdx.x >> 5)) + (lane >> 4);
  if (2 * (blockIdx.x * BS_WARPS + (threadIdx.x >> 5)) >= P) return;  // (uniform over the warp)
  const bool mine = k < P;
  DF acc = {0.f, 0.f};
  if (mine) {
    const int* wf = win + (k / G) * DPV_WMAX;
    const int p1 = pptr[k + 1];
    for (int p = pptr[k] + hl; p < p1; p += 16) {
      const float4* t4 = pterm + 8 * (size_t)p;
      float4 e[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) e[q] = t4[q];
      const int sl = __float_as_int(t4[7].x);
      const int fi = fdx[wf[sl & 0xff]], fj = fdx[wf[sl >> 8]];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int fo = side == 0 ? fi : fj;
        if (fo < 0) continue;
        const float4* x = reinterpret_cast<const float4*>(dxv + fo);  // fo is even: 16-byte aligned
#pragma unroll
        for (int h2 = 0; h2 < 3; ++h2) {
          const float4 v = e[3 * side + h2], xv = x[h2];
          dd_acc(acc, DF{-v.x, -v.y}, DF{xv.x, xv.y});
          dd_acc(acc, DF{-v.z, -v.w}, DF{xv.z, xv.w});
        }
      }
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) dd_acc_add(acc, DF{__shfl_xor_sync(0xffffffffu, acc.hi, o),
                                                    __shfl_xor_sync(0xffffffffu, acc.lo, o)});
  if (hl == 0 && mine) {
    const DF wv = w_ext ? DF{w_ext[k], 0.f} : dd_ld(wk2[k]);
    const DF ddk = dd_div(dd_add(dd_norm(acc), wv), dd_ld(Ct2[k]));
    dd_out[k] = ddk.hi + ddk.lo;
    if (write_depth) {
      float* pk = patches + 27 * (size_t)k;
      const DF s = dd_add_f(ddk, pk[22]);
      const float dn = fmaxf(s.hi + s.lo, d_min);
#pragma unroll
      for (int m = 18; m < 27; ++m) pk[m] = dn;
    }
  }
}

unsigned backsub_grid(ba_handle_t h, int retract, int per_warp = 1) {
  const long long wb = ((long long)h->P + per_warp * BS_WARPS - 1) / (per_warp * BS_WARPS);
  const long long rb = retract ? (long long)h->N : 0;
  return (unsigned)(wb > rb ? wb : rb);
}

}  // namespace

// Back-substitution of the depths; with `retract` the kernel also updates the
// poses and their rows of the linearisation table.
ba_status_t dpv_backsub(ba_handle_t h, int retract) {
  Workspace* ws = h->ws;
  if (retract && dpv_use_dense(h)) return dpv_dense_backsub(h);  // the dense form (dense.cu)
  if (h->opt.precision == BA_MIXED) {
    DPV_CUDA(h, dpv_launch_pdl(k_dx_pairs, dim3((h->n_pad + 255) / 256), dim3(256), 0, h->stream, h->n_pad,
                               (const double*)ws->dx.p, ws->dx2.p, (const int*)ws->status));
    ++h->launches;
    DPV_CUDA(h, dpv_launch_pdl(k_backsub_dd, dim3(backsub_grid(h, retract, 2)), dim3(BS_THREADS), 0, h->stream, h->P,
                               h->G, ws->fdx.p, h->opt.d_min, ws->pptr.p, ws->pterm.p, ws->win.p,
                               (const float2*)ws->dx2.p, (const float2*)ws->Ct2.p, (const float2*)ws->wk2.p,
                               (const float*)nullptr, h->patches, ws->dd.p, h->N, retract, (const double*)ws->dx.p,
                               h->poses, ws->posef.p, 1, (const int*)ws->status));
    ++h->launches;
    DPV_CUDA(h, cudaGetLastError());
    return BA_OK;
  }
  DPV_CUDA(h, dpv_launch_pdl(k_backsub, dim3(backsub_grid(h, retract)), dim3(BS_THREADS), 0, h->stream, h->P, h->G,
                             ws->fdx.p, h->opt.d_min, ws->pptr.p, ws->pterm.p, ws->win.p, ws->tmpv.p, ws->Ct.p,
                             ws->wk.p, h->patches, ws->dd.p, h->N, retract, ws->dx.p, h->poses, ws->posef.p, 1,
                             ws->status));
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

// The adjoint's depth part of lambda: out_k = Ct_k^-1 (w_ext_k - sum_a e_ak^T lambda_a),
// with lambda_a in the solver's output; no state is changed.
ba_status_t dpv_backsub_ext(ba_handle_t h, const float* w_ext, float* out) {
  Workspace* ws = h->ws;
  if (h->opt.precision == BA_MIXED) {
    k_dx_pairs<<<(h->n_pad + 255) / 256, 256, 0, h->stream>>>(h->n_pad, ws->dx.p, ws->dx2.p, ws->status);
    ++h->launches;
    k_backsub_dd<<<backsub_grid(h, 0, 2), BS_THREADS, 0, h->stream>>>(
        h->P, h->G, ws->fdx.p, h->opt.d_min, ws->pptr.p, ws->pterm.p, ws->win.p, ws->dx2.p, ws->Ct2.p, ws->wk2.p,
        w_ext, h->patches, out, h->N, 0, ws->dx.p, h->poses, nullptr, 0, ws->status);
    ++h->launches;
    DPV_CUDA(h, cudaGetLastError());
    return BA_OK;
  }
  k_backsub<<<backsub_grid(h, 0), BS_THREADS, 0, h->stream>>>(
      h->P, h->G, ws->fdx.p, h->opt.d_min, ws->pptr.p, ws->pterm.p, ws->win.p, ws->tmpv.p, ws->Ct.p, w_ext,
      h->patches, out, h->N, 0, ws->dx.p, h->poses, nullptr, 0, ws->status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
