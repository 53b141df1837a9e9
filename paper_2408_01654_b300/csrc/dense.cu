// The dense form of one Gauss-Newton iteration for small patch graphs.
//
// The appendix "Bundle-Adjustment Efficiency" compares DPVO's dense bundle
// adjustment with the block-sparse one of Sec. 3.2 ("Efficient Global
// Optimization"): for very small, highly connected graphs (the odometry
// window) the dense form wins because it needs no block indexing, and the
// system switches between the two on the fly by size.  This file is that
// dense form, for one problem of at most DPV_SMALL_N pose unknowns:
//
//   k_dense_lin      one thread per edge: the FP32 linearisation of Eq. 3 at
//                    the patch centre (dpv_edge_linearize), and every product
//                    scattered with FP64 atomics into dense arrays: the pose
//                    blocks H_ii, H_ij, H_jj and v into the system S, y, the
//                    pose-depth columns J_i^T W J_d, J_j^T W J_d into the dense
//                    matrix E [P][n_pad] (one column per patch), C and w into
//                    [P][2];
//   k_dense_schur    sixteen patches per CTA: their columns scaled by
//                    Ct^-1/2 (double-float), then S -= E_hat E_hat^T (one
//                    thread per entry of the lower triangle, double-float
//                    sums) and y -= E_hat (w Ct^-1/2), added with FP64 atomics;
//   the one-CTA solver of the block-sparse path;
//   k_dense_backsub  one warp per patch: dd_k = (w_k - E[k] . dxi) / Ct_k over
//                    the dense column (double-float), the depth clamp, and
//                    the retraction of the poses (one per CTA).
//
// No per-run reduction, no window tables: the edges are visited in the
// binding's order only to reach their frames, and every sum is an atomic on
// a dense array.  Exact products are not needed here (the graphs are small
// and well conditioned); each FP32 product enters an FP64 sum.
//
// Measured on B300 (two-iteration step with the binding, L2 flushed between
// steps), the block-sparse form is the faster one at every size: 237 vs 172
// us at 8 keyframes, 497 vs 229 us at 22, 1337 vs 570 us at 44.  The FP64
// atomics on the dense arrays (about 60 per edge) cost more than the
// block-sparse form's shared-memory window reductions, so the automatic
// policy keeps the block-sparse form and this one runs when asked for.
#include "dfloat.cuh"
#include "retract.cuh"

#include <algorithm>

namespace {

constexpr int DL_THREADS = 256;
constexpr int DS_PATCHES = 16;  // patches per Schur CTA
constexpr int DS_THREADS = 256;
constexpr int DB_THREADS = 256;

__device__ __forceinline__ void red_f(double* p, float v) {
  if (v != 0.f) dpv_red_add(p, dpv_f2d_bits(v));
}

__global__ void __launch_bounds__(DL_THREADS) k_dense_lin(
    int G, int n_pad, const int* __restrict__ fdx, float z_min, const int* __restrict__ gptr,
    const unsigned* __restrict__ eslot, const int* __restrict__ perm, const int* __restrict__ win,
    const float* __restrict__ posef, const float* __restrict__ patches, const float* __restrict__ targets,
    const float* __restrict__ weights, const float* __restrict__ intr, double* __restrict__ S, int TS,
    double* __restrict__ y, double* __restrict__ Ed, double* __restrict__ Cw, double* __restrict__ cost,
    const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int s0 = gptr[g], s1 = gptr[g + 1];
  const int* wf = win + (size_t)g * DPV_WMAX;
  float K[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) K[q] = intr[q];
  float cst = 0.f;
  for (int s = s0 + threadIdx.x; s < s1; s += DL_THREADS) {
    const unsigned sw = eslot[s];
    const int si = dpv_slot_i(sw), sj = dpv_slot_j(sw);
    const int k = g * G + dpv_slot_k(sw);
    const int e = perm[s];
    const int fi = wf[si], fj = wf[sj];
    RelPose T;
    dpv_relative_pose_df(posef + DPV_POSE_ROW * (size_t)fi, posef + DPV_POSE_ROW * (size_t)fj, T);
    const float* pk = patches + 27 * (size_t)k;
    const float xb0 = (pk[4] - K[2]) / K[0], xb1 = (pk[13] - K[3]) / K[1];
    const float2 tg = *reinterpret_cast<const float2*>(targets + 2 * (size_t)e);
    const float2 wt = *reinterpret_cast<const float2*>(weights + 2 * (size_t)e);
    EdgeLin L;
    dpv_edge_linearize(T, xb0, xb1, pk[22], tg.x, tg.y, K, z_min, si == sj, L);
    if (!L.valid) continue;
    const float wc[2] = {wt.x, wt.y};
    cst += wc[0] * L.r[0] * L.r[0] + wc[1] * L.r[1] * L.r[1];
    const int oi = fdx[fi], oj = fdx[fj];
    // pose-depth columns, C and w
    const float wJd0 = wc[0] * L.Jd[0], wJd1 = wc[1] * L.Jd[1];
    double* col = Ed + (size_t)k * n_pad;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      if (oi >= 0) red_f(col + oi + m, fmaf(L.Ji[0][m], wJd0, L.Ji[1][m] * wJd1));
      if (oj >= 0) red_f(col + oj + m, fmaf(L.Jj[0][m], wJd0, L.Jj[1][m] * wJd1));
    }
    red_f(Cw + 2 * (size_t)k, fmaf(L.Jd[0], wJd0, L.Jd[1] * wJd1));
    red_f(Cw + 2 * (size_t)k + 1, fmaf(L.r[0], wJd0, L.r[1] * wJd1));
    // the pose blocks and the pose gradient (lower triangle of S)
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const float wi0 = wc[0] * L.Ji[0][a], wi1 = wc[1] * L.Ji[1][a];
      const float wj0 = wc[0] * L.Jj[0][a], wj1 = wc[1] * L.Jj[1][a];
      if (oi >= 0) red_f(y + oi + a, fmaf(wi0, L.r[0], wi1 * L.r[1]));
      if (oj >= 0) red_f(y + oj + a, fmaf(wj0, L.r[0], wj1 * L.r[1]));
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        if (oi >= 0 && b <= a) red_f(S + dpv_s_index(oi + a, oi + b, TS), fmaf(wi0, L.Ji[0][b], wi1 * L.Ji[1][b]));
        if (oj >= 0 && b <= a) red_f(S + dpv_s_index(oj + a, oj + b, TS), fmaf(wj0, L.Jj[0][b], wj1 * L.Jj[1][b]));
        if (oi >= 0 && oj >= 0) {  // H_ij[a][b]: row of frame i, column of frame j
          const float h = fmaf(wi0, L.Jj[0][b], wi1 * L.Jj[1][b]);
          red_f(S + (oi > oj ? dpv_s_index(oi + a, oj + b, TS) : dpv_s_index(oj + b, oi + a, TS)), h);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cst += __shfl_xor_sync(0xffffffffu, cst, o);
  if (cost && (threadIdx.x & 31) == 0 && cst != 0.f) atomicAdd(cost, (double)cst);
}

__global__ void __launch_bounds__(DS_THREADS) k_dense_schur(
    int P, int n, int n_pad, float lambda_d, const double* __restrict__ Ed, const double* __restrict__ Cw,
    double* __restrict__ S, int TS, double* __restrict__ y, float* __restrict__ Ct_out, float* __restrict__ wk_out,
    const int* status) {
  extern __shared__ float2 smd[];
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  float2* col = smd;                               // [DS_PATCHES][n_pad] e_k Ct^-1/2
  float2* sc = col + (size_t)DS_PATCHES * n_pad;   // [DS_PATCHES] Ct^-1/2, w Ct^-1/2
  const int k0 = blockIdx.x * DS_PATCHES;
  const int np = min(DS_PATCHES, P - k0);
  if (threadIdx.x < DS_PATCHES) {
    const int q = threadIdx.x;
    DF sq = {0.f, 0.f}, wsq = {0.f, 0.f};
    if (q < np) {
      const int k = k0 + q;
      const float2 c2 = dpv_d2df_bits(Cw[2 * (size_t)k]), w2 = dpv_d2df_bits(Cw[2 * (size_t)k + 1]);
      const DF ct = dd_add_f(DF{c2.x, c2.y}, lambda_d);
      sq = dd_rcp(dd_sqrt(ct));
      wsq = dd_mul(DF{w2.x, w2.y}, sq);
      Ct_out[k] = ct.hi + ct.lo;
      wk_out[k] = w2.x + w2.y;
    }
    sc[2 * q] = dd_st(sq);
    sc[2 * q + 1] = dd_st(wsq);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < DS_PATCHES * n_pad; t += DS_THREADS) {
    const int q = t / n_pad, r = t - q * n_pad;
    DF v = {0.f, 0.f};
    if (q < np && r < n) {
      const float2 e2 = dpv_d2df_bits(Ed[(size_t)(k0 + q) * n_pad + r]);
      v = dd_mul(DF{e2.x, e2.y}, dd_ld(sc[2 * q]));
    }
    col[t] = dd_st(v);
  }
  __syncthreads();
  // lower triangle, one entry per thread
  const int ntri = n * (n + 1) / 2;
  for (int t = threadIdx.x; t < ntri; t += DS_THREADS) {
    int r = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    const int c = t - r * (r + 1) / 2;
    DF acc = {0.f, 0.f};
    for (int q = 0; q < np; ++q) dd_acc(acc, dd_neg(dd_ld(col[q * n_pad + r])), dd_ld(col[q * n_pad + c]));
    acc = dd_norm(acc);
    if (acc.hi != 0.f) dpv_red_add(S + dpv_s_index(r, c, TS), dd_to_f64(acc));
  }
  for (int r = threadIdx.x; r < n; r += DS_THREADS) {
    DF acc = {0.f, 0.f};
    for (int q = 0; q < np; ++q) dd_acc(acc, dd_neg(dd_ld(col[q * n_pad + r])), dd_ld(sc[2 * q + 1]));
    acc = dd_norm(acc);
    if (acc.hi != 0.f) dpv_red_add(y + r, dd_to_f64(acc));
  }
}

__global__ void __launch_bounds__(DB_THREADS) k_dense_backsub(
    int P, int n_pad, const int* __restrict__ fdx, float d_min, const double* __restrict__ Ed,
    const double* __restrict__ Cw, float lambda_d, const double* __restrict__ dx, float* __restrict__ patches,
    float* __restrict__ dd_out, int N, double* __restrict__ poses, float* __restrict__ posef, const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0 && (int)blockIdx.x < N) {  // the retraction, one pose per CTA
    const int f = blockIdx.x;
    const int o = fdx[f];
    if (o >= 0) {
      dpv_se3_retract(dx + o, poses + 7 * (size_t)f);
      dpv_pose_table_row(poses + 7 * (size_t)f, posef + DPV_POSE_ROW * (size_t)f);
    }
  }
  const int k = blockIdx.x * (DB_THREADS / 32) + (threadIdx.x >> 5);
  if (k >= P) return;
  const double* col = Ed + (size_t)k * n_pad;
  DF acc = {0.f, 0.f};
  for (int r = lane; r < n_pad; r += 32) {
    const double e = col[r];
    if (e != 0.0) {
      const float2 e2 = dpv_d2df_bits(e), x2 = dpv_d2df_bits(dx[r]);
      dd_acc(acc, DF{-e2.x, -e2.y}, DF{x2.x, x2.y});
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    dd_acc_add(acc, DF{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
  if (lane == 0) {
    const float2 c2 = dpv_d2df_bits(Cw[2 * (size_t)k]), w2 = dpv_d2df_bits(Cw[2 * (size_t)k + 1]);
    const DF ct = dd_add_f(DF{c2.x, c2.y}, lambda_d);
    const DF ddk = dd_div(dd_add(dd_norm(acc), DF{w2.x, w2.y}), ct);
    dd_out[k] = ddk.hi + ddk.lo;
    float* pk = patches + 27 * (size_t)k;
    const DF s = dd_add_f(ddk, pk[22]);
    const float dn = fmaxf(s.hi + s.lo, d_min);
#pragma unroll
    for (int m = 18; m < 27; ++m) pk[m] = dn;
  }
}

size_t schur_smem(int n_pad) { return sizeof(float2) * ((size_t)DS_PATCHES * n_pad + 2 * DS_PATCHES); }

}  // namespace

// Whether the next iterations of this binding take the dense form: one
// problem, the FP32 linearisation at the patch centre, 6 <= n <= DPV_SMALL_N
// unknowns, no tape being recorded (the adjoint runs on the block-sparse
// form), and a dense E of at most DPV_DENSE_MAX_ENTRIES; then by the policy
// (BA_DENSE_AUTO: at most DPV_DENSE_AUTO_EDGES edges, the measured crossover).
bool dpv_use_dense(ba_handle_t h) {
  if (h->opt.dense_policy == BA_DENSE_NEVER) return false;
  if (h->nprob != 1 || h->opt.precision != BA_FP32 || h->opt.residual_pixels != 1 || h->record) return false;
  if (h->n < 6 || h->n > DPV_SMALL_N || (long long)h->n_pad * h->P > DPV_DENSE_MAX_ENTRIES) return false;
  if (h->opt.dense_policy == BA_DENSE_ALWAYS) return true;
  return h->E <= DPV_DENSE_AUTO_EDGES;
}

ba_status_t dpv_dense_reserve(ba_handle_t h) {
  ba_status_t s;
  if ((s = dpv_grow(h, h->ws->dE, (long long)h->n_pad * h->P, "dense pose-depth columns")) ||
      (s = dpv_grow(h, h->ws->dCw, 2LL * h->P, "dense C and w")))
    return s;
  return BA_OK;
}

// The dense assembly (after k_init_system has prepared S, y and the pose table).
ba_status_t dpv_dense_assemble(ba_handle_t h, double* cost) {
  Workspace* ws = h->ws;
  ba_status_t s = dpv_dense_reserve(h);
  if (s) return s;
  static bool attr = false;
  if (!attr) {
    DPV_CUDA(h, cudaFuncSetAttribute(k_dense_schur, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)schur_smem(DPV_SMALL_N)));
    attr = true;
  }
  DPV_CUDA(h, cudaMemsetAsync(ws->dE.p, 0, sizeof(double) * (size_t)h->n_pad * h->P, h->stream));
  DPV_CUDA(h, cudaMemsetAsync(ws->dCw.p, 0, sizeof(double) * 2 * (size_t)h->P, h->stream));
  const SysDesc& sd = h->sys[0];
  DPV_CUDA(h, dpv_launch_pdl(k_dense_lin, dim3(h->ngroups), dim3(DL_THREADS), 0, h->stream, h->G, h->n_pad,
                             (const int*)ws->fdx.p, h->opt.z_min, (const int*)ws->gptr.p,
                             (const unsigned*)ws->eslot.p, (const int*)ws->perm.p, (const int*)ws->win.p,
                             (const float*)ws->posef.p, (const float*)h->patches, h->targets, h->weights,
                             (const float*)ws->intr, ws->S.p, sd.TS, ws->y.p, ws->dE.p, ws->dCw.p, cost,
                             (const int*)ws->status));
  ++h->launches;
  DPV_CUDA(h, dpv_launch_pdl(k_dense_schur, dim3((h->P + DS_PATCHES - 1) / DS_PATCHES), dim3(DS_THREADS),
                             schur_smem(h->n_pad), h->stream, h->P, h->n, h->n_pad, h->opt.lambda_depth,
                             (const double*)ws->dE.p, (const double*)ws->dCw.p, ws->S.p, sd.TS, ws->y.p, ws->Ct.p,
                             ws->wk.p, (const int*)ws->status));
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

// The dense back-substitution with the retraction of the poses.
ba_status_t dpv_dense_backsub(ba_handle_t h) {
  Workspace* ws = h->ws;
  const unsigned grid = (unsigned)std::max<long long>((h->P + DB_THREADS / 32 - 1) / (DB_THREADS / 32), h->N);
  DPV_CUDA(h, dpv_launch_pdl(k_dense_backsub, dim3(grid), dim3(DB_THREADS), 0, h->stream, h->P, h->n_pad,
                             (const int*)ws->fdx.p, h->opt.d_min, (const double*)ws->dE.p, (const double*)ws->dCw.p,
                             h->opt.lambda_depth, (const double*)ws->dx.p, h->patches, ws->dd.p, h->N, h->poses,
                             ws->posef.p, (const int*)ws->status));
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
