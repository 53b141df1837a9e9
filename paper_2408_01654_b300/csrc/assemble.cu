// Linearisation + block reduction + Schur complement (one fused kernel).
//
// For one Gauss-Newton iteration of Eq. 3 (Sec. 3.1) with the inverse depths
// eliminated (Sec. 3.2 "Efficient Global Optimization", appendix
// "Bundle-Adjustment Efficiency"):
//
//   H = [ B  E ; E^T  C ],  g = [ v ; w ],   S = B + lambda_p I - E Ct^-1 E^T,
//   y = v - E Ct^-1 w,  Ct = C + lambda_d  (C diagonal: one depth per patch).
//
// Every patch has a single inverse depth, so E Ct^-1 E^T is a sum of rank-1
// terms e_k e_k^T / Ct_k.  A CTA owns one *group* of G consecutive patches and
// the window W (at most DPV_WMAX frames) its edges touch:
//
//   phase 0  relative pose of each (source, target) run of the group, from the
//            per-pose table (R, camera centre in double-float);
//   phase 1  one warp per run: each lane linearises an edge, stages its
//            sqrt(w)-scaled Jacobian rows in shared memory and writes the
//            edge's depth terms (J^T W Jd, Jd^T W Jd, Jd^T W r) to the
//            patch-major table; the lanes then reduce the run's 6x6 blocks
//            Hii, Hij, Hjj and vectors vi, vj with compensated sums;
//   phase 2  one thread per patch sums its edges' depth terms (compensated)
//            into e_k, C_k, w_k and forms the column e_k / sqrt(Ct_k);
//   phase 3  one thread per entry of the window's lower triangle forms
//            B_ab - sum_k e_a e_b / Ct_k with compensated sums and adds it to
//            the global tiled S with red.global.add.f64 (likewise y).
//
// Why compensated sums: S is the small difference of two large, nearly equal
// sums (B and E Ct^-1 E^T).  Rounding each FP32 product is harmless; each
// group's compensated contribution goes to FP64 whole (rounding it to FP32
// costs 1.3e-5 of the step at 708 unknowns) and the sum across groups (up to
// ~150 groups per entry with small groups) is carried in FP64 by the L2
// atomics (in FP32 it alone costs ~6e-6 of the step).  Inside
// a group the long sums (run blocks over a run's edges, the window product
// over the group's patches) are Kahan-compensated with the product fused into
// the compensation step; the short per-patch sums use TwoSum pairs.  The FP64
// operand of each atomic is built from the pair with integer conversions and
// one FP64 add (FP64 arithmetic runs at ~1/64 of the FP32 rate on this part).
#include "internal.cuh"

#include <algorithm>

namespace {

constexpr int AS_THREADS = 512;
constexpr int AS_WARPS = AS_THREADS / 32;
constexpr int EH_STRIDE = 6 * DPV_WMAX + 1;  // floats per patch column of E_hat
constexpr int NV = 90;                       // run block entries: Hii 21, Hij 36, Hjj 21, vi 6, vj 6
constexpr int ROWF = 27;                     // staged floats per edge: 13 per residual component + pad

// (row a, row b) of the staged per-edge vector [sqrt(w) Ji (6), sqrt(w) Jj (6), sqrt(w) r]
// whose product gives run entry q
__constant__ unsigned char c_pa[NV], c_pb[NV];

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// the phase-2b tables live in the phase-1 staging rows
static_assert(DPV_WMAX * DPV_WMAX + 8 * (DPV_WMAX * 21 + DPV_WMAX * 6) <= 4 * AS_WARPS * 32 * ROWF,
              "phase-2b tables exceed the staging space");

// staged floats per patch: (xb0, xb1, d) of the centre, or the nine pixels'
// xb0, then their xb1, then d (whole-patch residual)
__host__ __device__ constexpr int pd_stride(int pix) { return pix == 1 ? 3 : 19; }

size_t assemble_smem_bytes(int G, int pix) {
  return sizeof(float) * ((size_t)DPV_RMAX * NV * 2 + (size_t)DPV_RMAX * 21 + (size_t)G * EH_STRIDE + 2 * G +
                          (size_t)pd_stride(pix) * G + (size_t)AS_WARPS * 32 * ROWF) +
         sizeof(int) * (DPV_RMAX + 2 * DPV_WMAX);
}

__device__ __forceinline__ int tri_row(int t) {
  int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (tri(a + 1, 0) <= t) ++a;
  while (tri(a, 0) > t) --a;
  return a;
}

// PIX residual pixels per edge: 1 (the patch centre) or 9 (the whole patch,
// targets [E,9,2], the edge's weights shared by its pixels)
template <int PIX>
__global__ void __launch_bounds__(AS_THREADS) k_assemble(
    int G, int P, const int* __restrict__ fdx, const int* __restrict__ gprob, const SysDesc* __restrict__ sysd,
    float lambda_d, float z_min, const int* __restrict__ gptr,
    const int* __restrict__ grun, const int* __restrict__ gnr, const unsigned* __restrict__ eslot,
    const int* __restrict__ perm,
    const int* __restrict__ pmpos, const int* __restrict__ pptr, const int* __restrict__ win,
    const int* __restrict__ wlen, const float* __restrict__ posef, const float* __restrict__ patches,
    const float* __restrict__ targets, const float* __restrict__ weights, const float* __restrict__ intr,
    float4* __restrict__ pterm, double* __restrict__ S, double* __restrict__ y, float* __restrict__ Ct_out,
    float* __restrict__ wk_out, double* __restrict__ cost, const float* __restrict__ w_ext, int* status) {
  extern __shared__ float sm[];
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int w = wlen[g];
  const int nr = 6 * w;
  const int gs = gptr[g], nruns = gnr[g];
  const int* runptr = grun + (size_t)g * (DPV_RMAX + 1);  // run starts relative to gs

  float2* runv = reinterpret_cast<float2*>(sm);            // [RMAX][NV] (hi, lo)
  float* rpose = sm + DPV_RMAX * NV * 2;                    // [RMAX][21]
  float* Eh = rpose + DPV_RMAX * 21;                        // [G][EH_STRIDE]
  float* sc = Eh + (size_t)G * EH_STRIDE;                   // [G][2]  Ct^-1/2, w Ct^-1/2
  constexpr int PDS = pd_stride(PIX);
  float* pd = sc + 2 * G;                                   // [G][PDS]  xb0, xb1, d
  float* rows = pd + PDS * G;                               // [warps][32][ROWF]
  int* rsl = reinterpret_cast<int*>(rows + AS_WARPS * 32 * ROWF);  // [RMAX] si | sj << 8
  int* wf = rsl + DPV_RMAX;                                 // [W] window frames
  int* fr = wf + DPV_WMAX;                                  // [W] unknown row in the group's system, -1 fixed
  // the group's pose system (every frame of a group belongs to one problem)
  const SysDesc sd = sysd[gprob[g]];

  float K[4];  // the group's problem's intrinsics
#pragma unroll
  for (int q = 0; q < 4; ++q) K[q] = intr[4 * gprob[g] + q];

  // ---- phase 0 ------------------------------------------------------------
  for (int q = tid; q < G * EH_STRIDE; q += AS_THREADS) Eh[q] = 0.f;
  for (int q = tid; q < w; q += AS_THREADS) {
    const int f = win[g * DPV_WMAX + q];
    const int o = fdx[f];
    wf[q] = f;
    fr[q] = o < 0 ? -1 : o - sd.voff;
  }
  if (PIX == 1) {
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
  } else {
    for (int t = tid; t < G * 9; t += AS_THREADS) {
      const int q = t / 9, px = t - 9 * q;
      const int k = g * G + q;
      float x0 = 0.f, x1 = 0.f, d = 1.f;
      if (k < P) {
        const float* pk = patches + 27 * (size_t)k;
        x0 = (pk[px] - K[2]) / K[0];
        x1 = (pk[9 + px] - K[3]) / K[1];
        d = pk[22];
      }
      pd[PDS * q + px] = x0;
      pd[PDS * q + 9 + px] = x1;
      if (px == 4) pd[PDS * q + 18] = d;
    }
  }
  __syncthreads();
  for (int r = tid; r < nruns; r += AS_THREADS) {
    const unsigned sw = eslot[gs + runptr[r]];
    const int si = dpv_slot_i(sw), sj = dpv_slot_j(sw);
    rsl[r] = si | (sj << 8);
    RelPose T;  // accurate to rounding: its error is shared by the whole run
    dpv_relative_pose_df(posef + DPV_POSE_ROW * (size_t)wf[si], posef + DPV_POSE_ROW * (size_t)wf[sj], T);
    float* o = rpose + 21 * r;
#pragma unroll
    for (int m = 0; m < 9; ++m) o[m] = T.R[m];
#pragma unroll
    for (int m = 0; m < 3; ++m) o[9 + m] = T.t[m];
#pragma unroll
    for (int m = 0; m < 9; ++m) o[12 + m] = T.txR[m];
  }
  __syncthreads();

  // ---- phase 1: one warp per run ------------------------------------------
  float cst = 0.f;
  float* rw = rows + wid * 32 * ROWF;
  // this lane's run entries q = lane + 32 t: staged-row operands, read once
  // (lanes read different table entries, which the constant cache serialises)
  int pa[3], pb[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int q = lane + 32 * t;
    pa[t] = q < NV ? c_pa[q] : 0;
    pb[t] = q < NV ? c_pb[q] : 0;
  }
  for (int r = wid; r < nruns; r += AS_WARPS) {
    const int s0 = gs + runptr[r], s1 = gs + runptr[r + 1];
    const int si = rsl[r] & 0xff, sj = rsl[r] >> 8;
    const bool self_run = si == sj;  // masked edges: they contribute nothing
    RelPose T;
    {
      const float* o = rpose + 21 * r;
#pragma unroll
      for (int m = 0; m < 9; ++m) T.R[m] = o[m];
#pragma unroll
      for (int m = 0; m < 3; ++m) T.t[m] = o[9 + m];
#pragma unroll
      for (int m = 0; m < 9; ++m) T.txR[m] = o[12 + m];
    }
    KS acc[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) acc[t] = KS{0.f, 0.f};
    for (int b = s0; b < s1; b += 32) {
      const int s = b + lane;
      const int nb = min(32, s1 - b);
      float* row = rw + lane * ROWF;
      int kl = 0, e = 0;
      float2 wt = make_float2(0.f, 0.f);
      if (s < s1) {
        kl = dpv_slot_k(eslot[s]);
        e = perm[s];
        wt = *reinterpret_cast<const float2*>(weights + 2 * (size_t)e);
      }
      float Ei[6], Ej[6], Ce = 0.f, we = 0.f;
#pragma unroll
      for (int m = 0; m < 6; ++m) Ei[m] = Ej[m] = 0.f;
      // one residual pixel at a time: each lane stages its edge's two rows,
      // then the warp adds every staged edge's products to the run's blocks
#pragma unroll 1
      for (int px = 0; px < PIX; ++px) {
        if (s < s1) {
          const float2 tg = *reinterpret_cast<const float2*>(targets + 2 * ((size_t)e * PIX + px));
          const float xb0 = PIX == 1 ? pd[3 * kl] : pd[PDS * kl + px];
          const float xb1 = PIX == 1 ? pd[3 * kl + 1] : pd[PDS * kl + 9 + px];
          const float dk = PIX == 1 ? pd[3 * kl + 2] : pd[PDS * kl + 18];
          EdgeLin L;
          dpv_edge_linearize(T, xb0, xb1, dk, tg.x, tg.y, K, z_min, self_run, L);
          if (L.valid) {
            const float wc[2] = {wt.x, wt.y};
            cst += wc[0] * L.r[0] * L.r[0] + wc[1] * L.r[1] * L.r[1];
            const float wJd0 = wc[0] * L.Jd[0], wJd1 = wc[1] * L.Jd[1];
            Ce += wJd0 * L.Jd[0] + wJd1 * L.Jd[1];
            we += wJd0 * L.r[0] + wJd1 * L.r[1];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
              Ei[m] += L.Ji[0][m] * wJd0 + L.Ji[1][m] * wJd1;
              Ej[m] += L.Jj[0][m] * wJd0 + L.Jj[1][m] * wJd1;
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const float sw = sqrtf(wc[c]);
#pragma unroll
              for (int m = 0; m < 6; ++m) {
                row[13 * c + m] = sw * L.Ji[c][m];
                row[13 * c + 6 + m] = sw * L.Jj[c][m];
              }
              row[13 * c + 12] = sw * L.r[c];
            }
          } else {
#pragma unroll
            for (int m = 0; m < 26; ++m) row[m] = 0.f;
          }
        }
        __syncwarp();
        for (int q = 0; q < nb; ++q) {
          const float* re = rw + q * ROWF;
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            if (lane + 32 * t < NV) {
              ks_fma(acc[t], re[pa[t]], re[pb[t]]);
              ks_fma(acc[t], re[13 + pa[t]], re[13 + pb[t]]);
            }
          }
        }
        __syncwarp();
      }
      if (s < s1) {
        float4* pt = pterm + 4 * (size_t)pmpos[s];
        pt[0] = make_float4(Ei[0], Ei[1], Ei[2], Ei[3]);
        pt[1] = make_float4(Ei[4], Ei[5], Ej[0], Ej[1]);
        pt[2] = make_float4(Ej[2], Ej[3], Ej[4], Ej[5]);
        pt[3] = make_float4(Ce, we, __int_as_float(si | (sj << 8)), 0.f);
      }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int q = lane + 32 * t;
      if (q < NV) runv[r * NV + q] = make_float2(acc[t].s, -acc[t].c);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cst += __shfl_xor_sync(0xffffffffu, cst, o);
  if (cost && lane == 0 && cst != 0.f) atomicAdd(cost, (double)cst);
  __syncthreads();

  // ---- phase 2: per patch e_k, C_k, w_k (compensated) ---------------------
  // one warp per patch, one lane per edge; the target-frame columns of E_hat
  // are added with shared-memory atomics (two edges of a patch may share a
  // target), the source-frame column and C, w by a compensated warp sum
  for (int q = wid; q < G; q += AS_WARPS) {
    const int k = g * G + q;
    float* col = Eh + (size_t)q * EH_STRIDE;
    DF ei[6], C = {0.f, 0.f}, wv = {0.f, 0.f};
#pragma unroll
    for (int m = 0; m < 6; ++m) ei[m] = DF{0.f, 0.f};
    int si = -1;
    if (k < P) {
      for (int p = pptr[k] + lane; p < pptr[k + 1]; p += 32) {
        const float4 a = pterm[4 * (size_t)p], b = pterm[4 * (size_t)p + 1], c = pterm[4 * (size_t)p + 2],
                     d = pterm[4 * (size_t)p + 3];
        const int sl = __float_as_int(d.z);
        si = sl & 0xff;
        const int sj = sl >> 8;
        df_add(ei[0], a.x); df_add(ei[1], a.y); df_add(ei[2], a.z);
        df_add(ei[3], a.w); df_add(ei[4], b.x); df_add(ei[5], b.y);
        float* cj = col + 6 * sj;
        atomicAdd(cj + 0, b.z); atomicAdd(cj + 1, b.w); atomicAdd(cj + 2, c.x);
        atomicAdd(cj + 3, c.y); atomicAdd(cj + 4, c.z); atomicAdd(cj + 5, c.w);
        df_add(C, d.x);
        df_add(wv, d.y);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const DF t = {__shfl_xor_sync(0xffffffffu, ei[m].hi, o), __shfl_xor_sync(0xffffffffu, ei[m].lo, o)};
        df_add_df(ei[m], t);
      }
      const DF tc = {__shfl_xor_sync(0xffffffffu, C.hi, o), __shfl_xor_sync(0xffffffffu, C.lo, o)};
      const DF tw = {__shfl_xor_sync(0xffffffffu, wv.hi, o), __shfl_xor_sync(0xffffffffu, wv.lo, o)};
      df_add_df(C, tc);
      df_add_df(wv, tw);
      si = max(si, __shfl_xor_sync(0xffffffffu, si, o));
    }
    df_add(C, lambda_d);
    __syncwarp();
    // lane 0's sums for every lane (the butterfly may differ in the last bit across lanes)
    const float ct = __shfl_sync(0xffffffffu, df_val(C), 0);
    const float wf_ = w_ext ? (k < P ? w_ext[k] : 0.f) : __shfl_sync(0xffffffffu, df_val(wv), 0);
    if (lane == 0 && si >= 0) {
#pragma unroll
      for (int m = 0; m < 6; ++m) col[6 * si + m] += df_val(ei[m]);
    }
    __syncwarp();
    const float sq = 1.0f / sqrtf(ct);
    for (int m = lane; m < nr; m += 32) col[m] *= sq;
    if (lane == 0) {
      sc[2 * q] = sq;
      sc[2 * q + 1] = wf_ * sq;
      if (k < P) {
        Ct_out[k] = ct;
        wk_out[k] = wf_;
      }
    }
  }
  __syncthreads();

  // ---- phase 2b: run sums per window block (in the phase-1 staging space) ---
  // prt[a * w + b] = the run with (source, target) slots (a, b), or -1;
  // dgb[a][e] = sum of the runs' Hii (a = source) and Hjj (a = target) lower
  // entries; yrn[a][m] likewise for vi / vj.
  signed char* prt = reinterpret_cast<signed char*>(rows);
  float2* dgb = reinterpret_cast<float2*>(rows + DPV_WMAX * DPV_WMAX / 4);
  float2* yrn = dgb + DPV_WMAX * 21;
  for (int q = tid; q < w * w; q += AS_THREADS) prt[q] = -1;
  __syncthreads();
  for (int r = tid; r < nruns; r += AS_THREADS) {
    const int si = rsl[r] & 0xff, sj = rsl[r] >> 8;
    if (si != sj) prt[si * w + sj] = (signed char)r;
  }
  for (int q = tid; q < 27 * w; q += AS_THREADS) {
    const int a = q / 27, e = q - 27 * a;
    const int oi = e < 21 ? e : 78 + (e - 21), oj = e < 21 ? 57 + e : 84 + (e - 21);
    DF acc = {0.f, 0.f};
    for (int r = 0; r < nruns; ++r) {
      const int si = rsl[r] & 0xff, sj = rsl[r] >> 8;
      if (si == sj) continue;
      const float2* rv = runv + r * NV;
      if (si == a) df_add_df(acc, DF{rv[oi].x, rv[oi].y});
      if (sj == a) df_add_df(acc, DF{rv[oj].x, rv[oj].y});
    }
    if (e < 21) dgb[a * 21 + e] = make_float2(acc.hi, acc.lo);
    else yrn[a * 6 + (e - 21)] = make_float2(acc.hi, acc.lo);
  }
  __syncthreads();

  // ---- phase 3: window Schur complement into the global S and y -----------
  // one thread per 3x3 sub-block (rows 3ha.. of frame a, columns 3hb.. of
  // frame b, a >= b): nine independent compensated sums over the patches.
  const int nblk = tri(w, 0);
  for (int t = tid; t < 4 * nblk; t += AS_THREADS) {
    const int blk = t >> 2, ha = (t >> 1) & 1, hb = t & 1;
    const int a = tri_row(blk), b = blk - tri(a, 0);
    if (a == b && hb > ha) continue;
    const int ra0 = fr[a], rb0 = fr[b];
    if (ra0 < 0 || rb0 < 0) continue;
    const int R0 = 6 * a + 3 * ha, C0 = 6 * b + 3 * hb;
    DF acc[3][3];
    {
      KS ks[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) ks[i][j] = KS{0.f, 0.f};
      for (int kl = 0; kl < G; ++kl) {
        const float* col = Eh + (size_t)kl * EH_STRIDE;
        const float er[3] = {-col[R0], -col[R0 + 1], -col[R0 + 2]};
        const float ec[3] = {col[C0], col[C0 + 1], col[C0 + 2]};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) ks_fma(ks[i][j], er[i], ec[j]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[i][j] = ks_df(ks[i][j]);
    }
    if (a == b) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (3 * hb + j <= 3 * ha + i) {
            const float2 v = dgb[a * 21 + tri(3 * ha + i, 3 * hb + j)];
            df_add_df(acc[i][j], DF{v.x, v.y});
          }
    } else {
      const int r1 = prt[a * w + b], r2 = prt[b * w + a];
      if (r1 >= 0) {  // run a -> b: Hij rows belong to a
        const float2* rv = runv + r1 * NV + 21;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float2 v = rv[6 * (3 * ha + i) + 3 * hb + j];
            df_add_df(acc[i][j], DF{v.x, v.y});
          }
      }
      if (r2 >= 0) {  // run b -> a: Hij rows belong to b (transposed)
        const float2* rv = runv + r2 * NV + 21;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float2 v = rv[6 * (3 * hb + j) + 3 * ha + i];
            df_add_df(acc[i][j], DF{v.x, v.y});
          }
      }
    }
    const int gr = ra0 + 3 * ha, gc = rb0 + 3 * hb;
    double* Sg = S + sd.soff;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (a != b || 3 * hb + j <= 3 * ha + i)
          dpv_red_add(Sg + dpv_s_index(gr + i, gc + j, sd.TS), dpv_f2d_bits(acc[i][j].hi) + dpv_f2d_bits(acc[i][j].lo));
  }
  for (int R = tid; R < nr; R += AS_THREADS) {
    const int a = R / 6, ra = R - 6 * a;
    if (fr[a] < 0) continue;
    DF acc = {0.f, 0.f};
    if (!w_ext) acc = DF{yrn[R].x, yrn[R].y};  // with an external right-hand side v comes from y's init
    for (int kl = 0; kl < G; ++kl) df_fma(acc, -Eh[(size_t)kl * EH_STRIDE + R], sc[2 * kl + 1]);
    dpv_red_add(y + sd.voff + fr[a] + ra, dpv_f2d_bits(acc.hi) + dpv_f2d_bits(acc.lo));
  }
}

// S <- 0, y <- 0 (or the given right-hand side), and the per-pose table for
// this iteration (R and the camera centre as double-float pairs).  With
// diag_pad > 0 (one system held in one tile of edge diag_pad) the diagonal is
// written here as well: lambda_p on the first diag_n entries, 1 on the
// padding; otherwise k_init_diag follows.  The first iteration of a step also
// clears the step's ncost cost slots (cost_zero).
__global__ void k_init_system(double* __restrict__ S, size_t nS, double* __restrict__ y, int nv,
                              const double* __restrict__ y_init, const double* __restrict__ poses, int N,
                              float* __restrict__ posef, int diag_n, int diag_pad, float lambda_p,
                              double* __restrict__ cost_zero, int ncost, const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cost_zero && gid < (size_t)ncost) cost_zero[gid] = 0.0;
  if (gid < (size_t)N) dpv_pose_table_row(poses + 7 * gid, posef + DPV_POSE_ROW * gid);
  double2* S2 = reinterpret_cast<double2*>(S);
  const size_t dstep = (size_t)diag_pad + 1;
  for (size_t q = gid; q < nS / 2; q += stride) {
    double2 v = make_double2(0.0, 0.0);
    if (diag_pad > 0) {
      if ((2 * q) % dstep == 0) v.x = (2 * q) / dstep < (size_t)diag_n ? (double)lambda_p : 1.0;
      if ((2 * q + 1) % dstep == 0) v.y = (2 * q + 1) / dstep < (size_t)diag_n ? (double)lambda_p : 1.0;
    }
    S2[q] = v;
  }
  for (size_t q = gid; q < (size_t)nv; q += stride) y[q] = y_init ? y_init[q] : 0.0;
}

// lambda_p on the free diagonal of every system, 1 on its padding diagonal (blockIdx.y = system)
__global__ void k_init_diag(double* __restrict__ S, const SysDesc* __restrict__ sysd, float lambda_p,
                            const int* status) {
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const SysDesc sd = sysd[blockIdx.y];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < sd.n_pad) S[sd.soff + dpv_s_index(r, r, sd.TS)] = r < sd.n ? (double)lambda_p : 1.0;
}

__global__ void k_export_S(const double* __restrict__ S, int n, int TS, double* __restrict__ out) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int r = (int)(q / n), c = (int)(q % n);
  out[q] = c <= r ? S[dpv_s_index(r, c, TS)] : 0.0;
}

bool g_tables_ready = false;

ba_status_t upload_tables(ba_handle_t h) {
  if (g_tables_ready) return BA_OK;
  unsigned char pa[NV], pb[NV];
  int q = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b <= a; ++b, ++q) { pa[q] = a; pb[q] = b; }          // Hii (lower)
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b, ++q) { pa[q] = a; pb[q] = 6 + b; }       // Hij
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b <= a; ++b, ++q) { pa[q] = 6 + a; pb[q] = 6 + b; }  // Hjj (lower)
  for (int a = 0; a < 6; ++a, ++q) { pa[q] = a; pb[q] = 12; }            // vi
  for (int a = 0; a < 6; ++a, ++q) { pa[q] = 6 + a; pb[q] = 12; }        // vj
  DPV_CUDA(h, cudaMemcpyToSymbol(c_pa, pa, NV));
  DPV_CUDA(h, cudaMemcpyToSymbol(c_pb, pb, NV));
  DPV_CUDA(h, cudaFuncSetAttribute(k_assemble<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)assemble_smem_bytes(DPV_GMAX, 1)));
  DPV_CUDA(h, cudaFuncSetAttribute(k_assemble<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)assemble_smem_bytes(DPV_GMAX, 9)));
  g_tables_ready = true;
  return BA_OK;
}

}  // namespace

namespace {
ba_status_t assemble_impl(ba_handle_t h, int it, const double* v_ext, const float* w_ext, int skip_init);
}

ba_status_t dpv_assemble(ba_handle_t h, int it, int skip_init) {
  return assemble_impl(h, it, nullptr, nullptr, skip_init);
}

// Assembly with an external right-hand side (the adjoint): y = v_ext - E Ct^-1 w_ext
// instead of the residual-based v and w.  Both null: the normal assembly.
ba_status_t dpv_assemble_ext(ba_handle_t h, int it, const double* v_ext, const float* w_ext) {  // it < 0: no cost
  return assemble_impl(h, it, v_ext, w_ext, 0);
}

namespace {
ba_status_t assemble_impl(ba_handle_t h, int it, const double* v_ext, const float* w_ext, int skip_init) {
  Workspace* ws = h->ws;
  ba_status_t s = upload_tables(h);
  if (s) return s;
  const size_t nS = (size_t)h->nS;
  if (!skip_init) {
    dpv_prof_begin(h, BA_KERNEL_INIT);
    // one system in one tile: its diagonal is written by the same launch
    const bool one_tile = h->sys.size() == 1 && h->sys[0].T == 1 && h->sys[0].soff == 0;
    // the first iteration of a forward step clears the step's cost slots
    const bool zero_cost = it == 0 && !v_ext && !w_ext;
    DPV_CUDA(h, dpv_launch_pdl(k_init_system, dim3(2 * h->num_sms), dim3(256), 0, h->stream, ws->S.p, nS, ws->y.p,
                               h->n_pad, v_ext, (const double*)h->poses, h->N, ws->posef.p,
                               one_tile ? h->sys[0].n : 0, one_tile ? h->sys[0].n_pad : 0, h->opt.lambda_pose,
                               zero_cost ? ws->cost : (double*)nullptr, (int)ws->cost_cap,
                               (const int*)ws->status));
    ++h->launches;
    if (!one_tile) {
      int maxpad = 0;
      for (const SysDesc& d : h->sys) maxpad = std::max(maxpad, d.n_pad);
      DPV_CUDA(h, dpv_launch_pdl(k_init_diag, dim3((maxpad + 255) / 256, h->nprob), dim3(256), 0, h->stream,
                                 ws->S.p, (const SysDesc*)ws->sysd.p, h->opt.lambda_pose, (const int*)ws->status));
      ++h->launches;
    }
    dpv_prof_end(h);
  }
  double* cost = it < 0 ? nullptr : ws->cost + (it < ws->cost_cap ? it : ws->cost_cap - 1);
  dpv_prof_begin(h, BA_KERNEL_ASSEMBLE);
  if (!v_ext && !w_ext && dpv_use_dense(h)) {  // the dense form of small graphs (dense.cu)
    ba_status_t s2 = dpv_dense_assemble(h, cost);
    dpv_prof_end(h);
    return s2;
  }
  if (h->opt.precision == BA_MIXED) {  // the double-float linearisation (assemble_df.cu)
    ba_status_t s2 = dpv_assemble_dd(h, cost, w_ext);
    dpv_prof_end(h);
    if (s2) return s2;
    DPV_CUDA(h, cudaGetLastError());
    return BA_OK;
  }
  auto kern = h->opt.residual_pixels == 9 ? k_assemble<9> : k_assemble<1>;
  DPV_CUDA(h, dpv_launch_pdl(kern, dim3(h->ngroups), dim3(AS_THREADS),
                             assemble_smem_bytes(h->G, h->opt.residual_pixels), h->stream, h->G, h->P, ws->fdx.p,
                             ws->gprob.p, ws->sysd.p, h->opt.lambda_depth, h->opt.z_min, ws->gptr.p, ws->grun.p,
                             ws->gnr.p, ws->eslot.p, ws->perm.p, ws->pmpos.p, ws->pptr.p, ws->win.p, ws->wlen.p,
                             ws->posef.p, h->patches, h->targets, h->weights, ws->intr, ws->pterm.p, ws->S.p,
                             ws->y.p, ws->Ct.p, ws->wk.p, cost, w_ext, ws->status));
  ++h->launches;
  dpv_prof_end(h);
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
}  // namespace

ba_status_t dpv_export_S(ba_handle_t h, double* dst) {
  const size_t nn = (size_t)h->n * h->n;
  if (nn == 0) return BA_OK;
  k_export_S<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(h->ws->S.p, h->n, h->TS, dst);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
