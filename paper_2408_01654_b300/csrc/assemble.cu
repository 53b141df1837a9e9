// Linearisation + block reduction + Schur complement (one fused kernel).
//
// For one Gauss-Newton iteration of Eq. 3 (Sec. 3.1) with the inverse depths
// eliminated (Sec. 3.2 "Efficient Global Optimization", appendix
// "Bundle-Adjustment Efficiency"):
//
//   H = [ B  E ; E^T  C ],  g = [ v ; w ],   S = B + lambda_p I - E Ct^-1 E^T,
//   y = v - E Ct^-1 w,  Ct = C + lambda_d  (C diagonal: one depth per patch).
//
// Because every patch has a single inverse depth, E Ct^-1 E^T is a sum of
// rank-1 terms e_k e_k^T / Ct_k over patches.  A CTA owns one *group* of G
// consecutive patches and the window W of frames its edges touch (at most
// DPV_WMAX).  It
//   1. linearises every edge of the group (one warp per (source, target) run,
//      per-lane register accumulation of the 6x6 B blocks and 6x1 v blocks,
//      one warp reduction per run) and accumulates, in shared memory, the
//      window-local B, v and the per-patch columns e_k and scalars C_k, w_k;
//   2. scales e_k by Ct_k^-1/2 and forms the window-local Schur complement
//      B - E_hat E_hat^T and y - E_hat w_hat (a small dense SYRK over the G
//      patches of the group);
//   3. adds the window-local result into the global tiled lower-triangular S
//      and y with fire-and-forget red.global.add; each entry of S receives at
//      most one add per group whose window covers it.
#include "internal.cuh"

namespace {

constexpr int AS_THREADS = 256;
constexpr int AS_WARPS = AS_THREADS / 32;
constexpr int EH_STRIDE = 6 * DPV_WMAX + 1;   // floats per patch column of E_hat
constexpr int NV = 90;                        // run accumulator length

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

struct AsmSmem {
  static constexpr int SB = tri(6 * DPV_WMAX, 0);  // packed lower (6W)(6W+1)/2
};

size_t assemble_smem_bytes(int G) {
  return sizeof(float) * ((size_t)AsmSmem::SB + (size_t)G * EH_STRIDE + 6 * DPV_WMAX + 2 * G + 3 * G + 2 * G +
                          AS_WARPS * 24) +
         sizeof(int) * DPV_WMAX;
}

__device__ __forceinline__ int pair_a(int p) {
  int a = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while (tri(a + 1, 0) <= p) ++a;
  while (tri(a, 0) > p) --a;
  return a;
}

__global__ void __launch_bounds__(AS_THREADS) k_assemble(
    int G, int P, int fixed, int TS, float lambda_d, float z_min, const int* __restrict__ gseg,
    const int* __restrict__ runptr, const unsigned* __restrict__ eslot, const int* __restrict__ perm,
    const int* __restrict__ win, const int* __restrict__ wlen, const double* __restrict__ poses,
    const float* __restrict__ patches, const float* __restrict__ targets, const float* __restrict__ weights,
    const float* __restrict__ intr, float* __restrict__ S, float* __restrict__ y, float* __restrict__ Ct_out,
    float* __restrict__ wk_out, double* __restrict__ cost, int* status) {
  extern __shared__ float sm[];
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int w = wlen[g];
  const int nr = 6 * w;
  const int nsb = tri(nr, 0);

  float* SB = sm;                              // packed lower of the window's B
  float* Eh = SB + AsmSmem::SB;                // [G][EH_STRIDE]
  float* yl = Eh + (size_t)G * EH_STRIDE;      // [6W]
  float* Cw = yl + 6 * DPV_WMAX;               // [G][2] C_k, w_k
  float* pd = Cw + 2 * G;                      // [G][3] xb0, xb1, d
  float* sc = pd + 3 * G;                      // [G][2] Ct^-1/2, w Ct^-1/2
  float* rp = sc + 2 * G;                      // [warps][24] relative pose of the warp's run
  int* wf = (int*)(rp + AS_WARPS * 24);        // [W] window frames

  float K[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) K[q] = intr[q];

  // ---- phase 0: clear accumulators, stage window and patch centres -------
  for (int q = tid; q < nsb; q += AS_THREADS) SB[q] = 0.f;
  for (int q = tid; q < G * EH_STRIDE; q += AS_THREADS) Eh[q] = 0.f;
  for (int q = tid; q < 6 * DPV_WMAX; q += AS_THREADS) yl[q] = 0.f;
  for (int q = tid; q < 2 * G; q += AS_THREADS) Cw[q] = 0.f;
  for (int q = tid; q < w; q += AS_THREADS) wf[q] = win[g * DPV_WMAX + q];
  for (int q = tid; q < G; q += AS_THREADS) {
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
  }
  __syncthreads();

  // ---- phase 1: one warp per (source, target) run -------------------------
  float cst = 0.f;
  const int r0 = gseg[g], r1 = gseg[g + 1];
  for (int r = r0 + wid; r < r1; r += AS_WARPS) {
    const int s0 = runptr[r], s1 = runptr[r + 1];
    const unsigned sw0 = eslot[s0];
    const int si = dpv_slot_i(sw0), sj = dpv_slot_j(sw0);
    if (si == sj) continue;  // self edges are masked (warp-uniform)
    float* rpw = rp + wid * 24;
    if (lane == 0) {
      RelPose T;
      dpv_relative_pose(poses + 7 * (size_t)wf[si], poses + 7 * (size_t)wf[sj], T);
#pragma unroll
      for (int m = 0; m < 9; ++m) rpw[m] = T.R[m];
#pragma unroll
      for (int m = 0; m < 3; ++m) rpw[9 + m] = T.t[m];
#pragma unroll
      for (int m = 0; m < 9; ++m) rpw[12 + m] = T.txR[m];
    }
    __syncwarp();
    RelPose T;
#pragma unroll
    for (int m = 0; m < 9; ++m) T.R[m] = rpw[m];
#pragma unroll
    for (int m = 0; m < 3; ++m) T.t[m] = rpw[9 + m];
#pragma unroll
    for (int m = 0; m < 9; ++m) T.txR[m] = rpw[12 + m];
    __syncwarp();

    float acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.f;
    for (int s = s0 + lane; s < s1; s += 32) {
      const int kl = dpv_slot_k(eslot[s]);
      const int e = perm[s];
      const float2 tg = *reinterpret_cast<const float2*>(targets + 2 * (size_t)e);
      const float2 wt = *reinterpret_cast<const float2*>(weights + 2 * (size_t)e);
      EdgeLin L;
      dpv_edge_linearize(T, pd[3 * kl], pd[3 * kl + 1], pd[3 * kl + 2], tg.x, tg.y, K, z_min, false, L);
      if (!L.valid) continue;
      const float wc[2] = {wt.x, wt.y};
      cst += wc[0] * L.r[0] * L.r[0] + wc[1] * L.r[1] * L.r[1];
      // per-patch depth terms
      const float wJd0 = wc[0] * L.Jd[0], wJd1 = wc[1] * L.Jd[1];
      atomicAdd(&Cw[2 * kl], wJd0 * L.Jd[0] + wJd1 * L.Jd[1]);
      atomicAdd(&Cw[2 * kl + 1], wJd0 * L.r[0] + wJd1 * L.r[1]);
      float* ek = Eh + (size_t)kl * EH_STRIDE;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        atomicAdd(&ek[6 * si + m], L.Ji[0][m] * wJd0 + L.Ji[1][m] * wJd1);
        atomicAdd(&ek[6 * sj + m], L.Jj[0][m] * wJd0 + L.Jj[1][m] * wJd1);
      }
      // run blocks: Hii (lower), Hij, Hjj (lower), vi, vj
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float wi[6], wj[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          wi[m] = wc[c] * L.Ji[c][m];
          wj[m] = wc[c] * L.Jj[c][m];
        }
        int q = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b) acc[q++] += wi[a] * L.Ji[c][b];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b < 6; ++b) acc[q++] += wi[a] * L.Jj[c][b];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b) acc[q++] += wj[a] * L.Jj[c][b];
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[q++] += wi[a] * L.r[c];
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[q++] += wj[a] * L.r[c];
      }
    }
    // warp reduction of the run accumulators, then scatter into the window
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      float v = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[q] = v;
    }
    const int bi = 6 * si, bj = 6 * sj;
    int q = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b, ++q)
        if ((q & 31) == lane) atomicAdd(&SB[tri(bi + a, bi + b)], acc[q]);
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b, ++q)
        if ((q & 31) == lane) {
          const int R = bi + a, C = bj + b;
          atomicAdd(&SB[R >= C ? tri(R, C) : tri(C, R)], acc[q]);
        }
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b, ++q)
        if ((q & 31) == lane) atomicAdd(&SB[tri(bj + a, bj + b)], acc[q]);
#pragma unroll
    for (int a = 0; a < 6; ++a, ++q)
      if ((q & 31) == lane) atomicAdd(&yl[bi + a], acc[q]);
#pragma unroll
    for (int a = 0; a < 6; ++a, ++q)
      if ((q & 31) == lane) atomicAdd(&yl[bj + a], acc[q]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cst += __shfl_xor_sync(0xffffffffu, cst, o);
  if (lane == 0 && cst != 0.f) atomicAdd(cost, (double)cst);
  __syncthreads();

  // ---- phase 2: per patch Ct = C + lambda_d, scale E_hat columns ----------
  for (int q = tid; q < G; q += AS_THREADS) {
    const int k = g * G + q;
    const float ct = Cw[2 * q] + lambda_d;
    const float s = 1.0f / sqrtf(ct);
    sc[2 * q] = s;
    sc[2 * q + 1] = Cw[2 * q + 1] * s;
    if (k < P) {
      Ct_out[k] = ct;
      wk_out[k] = Cw[2 * q + 1];
    }
  }
  __syncthreads();
  for (int q = tid; q < G * nr; q += AS_THREADS) {
    const int kl = q / nr, row = q - kl * nr;
    Eh[(size_t)kl * EH_STRIDE + row] *= sc[2 * kl];
  }
  __syncthreads();

  // ---- phase 3: window Schur complement, scattered into the global S ------
  const int npair_all = w * (w + 1) / 2;
  for (int p = tid; p < npair_all; p += AS_THREADS) {
    const int a = pair_a(p), b = p - tri(a, 0);
    const int fa = wf[a], fb = wf[b];
    if (fa < fixed || fb < fixed) continue;
    float acc[36];
#pragma unroll
    for (int q = 0; q < 36; ++q) acc[q] = 0.f;
    for (int kl = 0; kl < G; ++kl) {
      const float* ek = Eh + (size_t)kl * EH_STRIDE;
      float ea[6], eb[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        ea[m] = ek[6 * a + m];
        eb[m] = ek[6 * b + m];
      }
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[6 * r + c] = fmaf(ea[r], eb[c], acc[6 * r + c]);
    }
    const int gr = 6 * (fa - fixed), gc = 6 * (fb - fixed);
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (a == b && c > r) continue;
        const float v = SB[tri(6 * a + r, 6 * b + c)] - acc[6 * r + c];
        dpv_red_add(S + dpv_s_index(gr + r, gc + c, TS), v);
      }
  }
  for (int R = tid; R < nr; R += AS_THREADS) {
    const int fa = wf[R / 6];
    if (fa < fixed) continue;
    float v = yl[R];
    for (int kl = 0; kl < G; ++kl) v = fmaf(-Eh[(size_t)kl * EH_STRIDE + R], sc[2 * kl + 1], v);
    dpv_red_add(y + 6 * (fa - fixed) + (R % 6), v);
  }
}

// S <- 0 with lambda_p on the free diagonal and 1 on the padding diagonal; y <- 0
__global__ void k_init_system(float* __restrict__ S, size_t nS, float* __restrict__ y, int n, int n_pad, int TS,
                              float lambda_p, const int* status) {
  if (dpv_status(status)) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t n4 = nS / 4;
  float4* S4 = reinterpret_cast<float4*>(S);
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride)
    S4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)n_pad; q += stride) y[q] = 0.f;
}

__global__ void k_init_diag(float* __restrict__ S, int n, int n_pad, int TS, float lambda_p, const int* status) {
  if (dpv_status(status)) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_pad) S[dpv_s_index(r, r, TS)] = r < n ? lambda_p : 1.0f;
}

__global__ void k_export_S(const float* __restrict__ S, int n, int TS, float* __restrict__ out) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int r = (int)(q / n), c = (int)(q % n);
  out[q] = c <= r ? S[dpv_s_index(r, c, TS)] : 0.f;
}

}  // namespace

size_t dpv_assemble_smem(int G) { return assemble_smem_bytes(G); }

ba_status_t dpv_assemble(ba_handle_t h, int it) {
  Workspace* ws = h->ws;
  const size_t nS = (size_t)h->T * (h->T + 1) / 2 * h->TS * h->TS;
  dpv_prof_begin(h, BA_KERNEL_INIT);
  k_init_system<<<2 * h->num_sms, 256, 0, h->stream>>>(ws->S.p, nS, ws->y.p, h->n, h->n_pad, h->TS,
                                                        h->opt.lambda_pose, ws->status);
  ++h->launches;
  k_init_diag<<<(h->n_pad + 255) / 256, 256, 0, h->stream>>>(ws->S.p, h->n, h->n_pad, h->TS, h->opt.lambda_pose,
                                                              ws->status);
  ++h->launches;
  dpv_prof_end(h);
  const size_t smem = assemble_smem_bytes(h->G);
  static bool attr_set = false;
  if (!attr_set) {
    DPV_CUDA(h, cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)assemble_smem_bytes(DPV_GMAX)));
    attr_set = true;
  }
  double* cost = ws->cost + (it < ws->cost_cap ? it : ws->cost_cap - 1);
  dpv_prof_begin(h, BA_KERNEL_ASSEMBLE);
  k_assemble<<<h->ngroups, AS_THREADS, smem, h->stream>>>(
      h->G, h->P, h->fixed, h->TS, h->opt.lambda_depth, h->opt.z_min, ws->gseg.p, ws->runptr.p, ws->eslot.p, ws->perm.p,
      ws->win.p, ws->wlen.p, h->poses, h->patches, h->targets, h->weights, ws->intr, ws->S.p, ws->y.p, ws->Ct.p, ws->wk.p,
      cost, ws->status);
  ++h->launches;
  dpv_prof_end(h);
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

ba_status_t dpv_export_S(ba_handle_t h, float* dst) {
  const size_t nn = (size_t)h->n * h->n;
  if (nn == 0) return BA_OK;
  k_export_S<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(h->ws->S.p, h->n, h->TS, dst);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
