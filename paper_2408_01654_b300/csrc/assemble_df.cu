// Linearisation + block reduction + Schur complement in double-float
// arithmetic (the BA_MIXED path): the kernel of assemble.cu with every
// quantity of the linearisation carried as a pair of floats.
//
// Same structure and outputs as k_assemble (Sec. 3.1 Eq. 2-3, the Schur
// form of Sec. 3.2 "Efficient Global Optimization"): a CTA owns one group of
// G consecutive patches and the window of frames its edges touch;
//
//   phase 0  the double-float relative pose of each (source, target) run;
//   phase 1  one warp per run, one lane per edge: the double-float residual
//            and target-pose Jacobian J_j (dfloat.cuh), the sqrt(w)-scaled
//            rows [J_j, r] staged in shared memory as pairs, and the run's
//            H_jj (21 entries) and v_j (6) summed as double-float products,
//            one entry per lane.  Every edge of a run shares T_ij and
//            J_i = -J_j Ad(T_ij), so the rest of the run's blocks follow once
//            per run: H_ij = -Ad^T H_jj, H_ii = -H_ij Ad, v_i = -Ad^T v_j
//            (a third of the per-edge products of summing all 90 entries).
//            The edge's depth terms e_j = J_j^T W Jd, e_i = -Ad^T e_j,
//            Jd^T W Jd and Jd^T W r go to the patch-major table as pairs;
//   phase 2  16 lanes per patch: e_k, C_k, w_k summed as pairs (edges of one
//            patch that share a target frame are summed by the first lane of
//            each such set, found with __match_any_sync), the column
//            e_k / sqrt(Ct_k) formed in double-float;
//   phase 3  one thread per 3x3 sub-block of the window's lower triangle:
//            B_ab - sum_k e_a e_b / Ct_k in double-float, added to the global
//            FP64 S with red.global.add.f64 (likewise y).
//
// Shared memory per CTA is ~219 KB at G = 32 (the pairs double the window
// columns), so the path supports G <= DPV_GMAX_DD patches per group; it runs
// 512 threads (one CTA per SM, at most 128 registers per thread).  The
// patch-major table holds 128 bytes per edge
// (two float4 per 6-vector pair of e_i, e_j; C, w; the slots), read again by
// the double-float back-substitution (update.cu).
#include "dfloat.cuh"

#include <algorithm>

namespace {

constexpr int AD_THREADS = 512;
constexpr int AD_WARPS = AD_THREADS / 32;
constexpr int EH_STRIDE = 6 * DPV_WMAX + 1;  // pairs per patch column of E_hat
constexpr int NV = 90;                       // run block entries: Hii 21, Hij 36, Hjj 21, vi 6, vj 6
constexpr int NJ = 27;                       // per-edge run entries: Hjj 21 (lower), vj 6
constexpr int ROWP = 15;                     // staged pairs per edge: [Jj, r] per residual component + pad
constexpr int RPOSE = 42;                    // floats per run's relative pose: R, t, [t]x R as pairs

__constant__ unsigned char c_qa[NJ], c_qb[NJ];

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// staged floats per patch: the centre's ray (x hi, x lo, y hi, y lo) and d,
// or the nine pixels' rays (x pairs, then y pairs) and d
__host__ __device__ constexpr int pd_stride(int pix) { return pix == 1 ? 5 : 37; }

// phase-2b tables (window run map, diagonal and y sums as pairs) and the
// phase-2 scratch of the lanes' target terms live in the phase-1 staging rows
static_assert(DPV_WMAX * DPV_WMAX + 8 * (DPV_WMAX * 21 + DPV_WMAX * 6) <= 8 * AD_WARPS * 32 * ROWP,
              "phase-2b tables exceed the staging space");
static_assert(2 * 36 + 6 <= 32 * ROWP, "run-transform scratch exceeds a warp's staging rows");
static_assert(32 * 12 <= 2 * 32 * ROWP, "phase-2 scratch exceeds a warp's staging rows");

size_t assemble_dd_smem_bytes(int G, int pix) {
  return sizeof(float2) * ((size_t)DPV_RMAX * NV + (size_t)G * EH_STRIDE + 2 * G + (size_t)AD_WARPS * 32 * ROWP) +
         sizeof(float) * ((size_t)DPV_RMAX * RPOSE + (size_t)pd_stride(pix) * G) +
         sizeof(int) * (DPV_RMAX + 2 * DPV_WMAX);
}

__device__ __forceinline__ int tri_row(int t) {
  int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (tri(a + 1, 0) <= t) ++a;
  while (tri(a, 0) > t) --a;
  return a;
}

template <int PIX>
__global__ void __launch_bounds__(AD_THREADS, 1) k_assemble_dd(
    int G, int P, const int* __restrict__ fdx, const int* __restrict__ gprob, const SysDesc* __restrict__ sysd,
    float lambda_d, float z_min, const int* __restrict__ gptr, const int* __restrict__ grun,
    const int* __restrict__ gnr, const unsigned* __restrict__ eslot, const int* __restrict__ perm,
    const int* __restrict__ pmpos, const int* __restrict__ pptr, const int* __restrict__ win,
    const int* __restrict__ wlen, const float* __restrict__ posef, const float* __restrict__ patches,
    const float* __restrict__ targets, const float* __restrict__ weights, const float* __restrict__ intr,
    float4* __restrict__ pterm, double* __restrict__ S, double* __restrict__ y, float* __restrict__ Ct_out,
    float* __restrict__ wk_out, float2* __restrict__ Ct2_out, float2* __restrict__ wk2_out, double* __restrict__ cost,
    const float* __restrict__ w_ext, int* status) {
  extern __shared__ float2 smd[];
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int w = wlen[g];
  const int nr = 6 * w;
  const int gs = gptr[g], nruns = gnr[g];
  const int* runptr = grun + (size_t)g * (DPV_RMAX + 1);

  float2* runv = smd;                                        // [RMAX][NV]
  float2* Eh = runv + DPV_RMAX * NV;                         // [G][EH_STRIDE]
  float2* sc = Eh + (size_t)G * EH_STRIDE;                   // [G][2]  Ct^-1/2, w Ct^-1/2
  float2* rows = sc + 2 * G;                                 // [warps][32][ROWP]
  float* rpose = reinterpret_cast<float*>(rows + AD_WARPS * 32 * ROWP);  // [RMAX][RPOSE]
  constexpr int PDS = pd_stride(PIX);
  float* pd = rpose + DPV_RMAX * RPOSE;                      // [G][PDS]
  int* rsl = reinterpret_cast<int*>(pd + PDS * G);           // [RMAX] si | sj << 8
  int* wf = rsl + DPV_RMAX;                                  // [W] window frames
  int* fr = wf + DPV_WMAX;                                   // [W] unknown row in the group's system, -1 fixed
  const SysDesc sd = sysd[gprob[g]];

  float K[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) K[q] = intr[4 * gprob[g] + q];

  // ---- phase 0 ------------------------------------------------------------
  for (int q = tid; q < G * EH_STRIDE; q += AD_THREADS) Eh[q] = make_float2(0.f, 0.f);
  for (int q = tid; q < w; q += AD_THREADS) {
    const int f = win[g * DPV_WMAX + q];
    const int o = fdx[f];
    wf[q] = f;
    fr[q] = o < 0 ? -1 : o - sd.voff;
  }
  for (int t = tid; t < G * PIX; t += AD_THREADS) {
    const int q = t / PIX, px = t - PIX * q;
    const int k = g * G + q;
    DF x0 = {0.f, 0.f}, x1 = {0.f, 0.f};
    float d = 1.f;
    if (k < P) {
      const float* pk = patches + 27 * (size_t)k;
      const int pix = PIX == 1 ? 4 : px;
      x0 = dpv_ray_dd(pk[pix], K[2], K[0]);
      x1 = dpv_ray_dd(pk[9 + pix], K[3], K[1]);
      d = pk[22];
    }
    float* o = pd + PDS * q;
    if (PIX == 1) {
      o[0] = x0.hi; o[1] = x0.lo; o[2] = x1.hi; o[3] = x1.lo; o[4] = d;
    } else {
      o[2 * px] = x0.hi; o[2 * px + 1] = x0.lo; o[18 + 2 * px] = x1.hi; o[19 + 2 * px] = x1.lo;
      if (px == 4) o[36] = d;
    }
  }
  __syncthreads();
  for (int r = tid; r < nruns; r += AD_THREADS) {
    const unsigned sw = eslot[gs + runptr[r]];
    const int si = dpv_slot_i(sw), sj = dpv_slot_j(sw);
    rsl[r] = si | (sj << 8);
    RelPoseDD T;
    dpv_relative_pose_dd(posef + DPV_POSE_ROW * (size_t)wf[si], posef + DPV_POSE_ROW * (size_t)wf[sj], T);
    float* o = rpose + RPOSE * r;
#pragma unroll
    for (int m = 0; m < 9; ++m) { o[2 * m] = T.R[m].hi; o[2 * m + 1] = T.R[m].lo; }
#pragma unroll
    for (int m = 0; m < 3; ++m) { o[18 + 2 * m] = T.t[m].hi; o[19 + 2 * m] = T.t[m].lo; }
#pragma unroll
    for (int m = 0; m < 9; ++m) { o[24 + 2 * m] = T.txR[m].hi; o[25 + 2 * m] = T.txR[m].lo; }
  }
  __syncthreads();

  // ---- phase 1: one warp per run ------------------------------------------
  float cst = 0.f;
  float2* rw = rows + wid * 32 * ROWP;
  const bool own = lane < NJ;  // this lane's run entry: Hjj (lower) or vj
  const int pa = own ? c_qa[lane] : 0, pb = own ? c_qb[lane] : 0;
  for (int r = wid; r < nruns; r += AD_WARPS) {
    const int s0 = gs + runptr[r], s1 = gs + runptr[r + 1];
    const int si = rsl[r] & 0xff, sj = rsl[r] >> 8;
    const bool self_run = si == sj;
    const float* T = rpose + RPOSE * r;
    DF acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};  // the two residual components
    for (int b = s0; b < s1; b += 32) {
      const int s = b + lane;
      const int nb = min(32, s1 - b);
      float2* row = rw + lane * ROWP;
      int kl = 0, e = 0;
      float2 wt = make_float2(0.f, 0.f);
      if (s < s1) {
        kl = dpv_slot_k(eslot[s]);
        e = perm[s];
        wt = *reinterpret_cast<const float2*>(weights + 2 * (size_t)e);
      }
      DF Ej[6], Ce = {0.f, 0.f}, we = {0.f, 0.f};
#pragma unroll
      for (int m = 0; m < 6; ++m) Ej[m] = DF{0.f, 0.f};
#pragma unroll 1
      for (int px = 0; px < PIX; ++px) {
        if (s < s1) {
          const float2 tg = *reinterpret_cast<const float2*>(targets + 2 * ((size_t)e * PIX + px));
          const float* pq = pd + PDS * kl;
          const DF xb0 = PIX == 1 ? DF{pq[0], pq[1]} : DF{pq[2 * px], pq[2 * px + 1]};
          const DF xb1 = PIX == 1 ? DF{pq[2], pq[3]} : DF{pq[18 + 2 * px], pq[19 + 2 * px]};
          const float dk = PIX == 1 ? pq[4] : pq[36];
          EdgeLinDD L;
          dpv_edge_linearize_dd(T, xb0, xb1, dk, tg.x, tg.y, K, z_min, self_run, L);
          if (L.valid) {
            const float wc[2] = {wt.x, wt.y};
            cst += wc[0] * L.r[0].hi * L.r[0].hi + wc[1] * L.r[1].hi * L.r[1].hi;
            const DF wJd0 = dd_mul_f(L.Jd[0], wc[0]), wJd1 = dd_mul_f(L.Jd[1], wc[1]);
            dd_acc(Ce, wJd0, L.Jd[0]);
            dd_acc(Ce, wJd1, L.Jd[1]);
            dd_acc(we, wJd0, L.r[0]);
            dd_acc(we, wJd1, L.r[1]);
            dd_acc(Ej[0], L.Jj[0][0], wJd0);
            dd_acc(Ej[1], L.Jj[1][1], wJd1);
#pragma unroll
            for (int m = 2; m < 6; ++m) {
              dd_acc(Ej[m], L.Jj[0][m], wJd0);
              dd_acc(Ej[m], L.Jj[1][m], wJd1);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const DF sw = dd_sqrt(DF{wc[c], 0.f});
#pragma unroll
              for (int m = 0; m < 6; ++m) row[7 * c + m] = dd_st(dd_mul(sw, L.Jj[c][m]));
              row[7 * c + 6] = dd_st(dd_mul(sw, L.r[c]));
            }
          } else {
#pragma unroll
            for (int m = 0; m < 14; ++m) row[m] = make_float2(0.f, 0.f);
          }
        }
        __syncwarp();
        if (own) {
          for (int q = 0; q < nb; ++q) {
            const float2* re = rw + q * ROWP;
            dd_acc(acc0, dd_ld(re[pa]), dd_ld(re[pb]));
            dd_acc(acc1, dd_ld(re[7 + pa]), dd_ld(re[7 + pb]));
          }
        }
        __syncwarp();
      }
      if (s < s1) {
#pragma unroll
        for (int m = 0; m < 6; ++m) Ej[m] = dd_norm(Ej[m]);
        DF Ei[6];
        dpv_adT_dd(T, Ej, Ei);  // e_i = -Ad^T e_j
        Ce = dd_norm(Ce);
        we = dd_norm(we);
        float4* pt = pterm + 8 * (size_t)pmpos[s];
        pt[0] = make_float4(-Ei[0].hi, -Ei[0].lo, -Ei[1].hi, -Ei[1].lo);
        pt[1] = make_float4(-Ei[2].hi, -Ei[2].lo, -Ei[3].hi, -Ei[3].lo);
        pt[2] = make_float4(-Ei[4].hi, -Ei[4].lo, -Ei[5].hi, -Ei[5].lo);
        pt[3] = make_float4(Ej[0].hi, Ej[0].lo, Ej[1].hi, Ej[1].lo);
        pt[4] = make_float4(Ej[2].hi, Ej[2].lo, Ej[3].hi, Ej[3].lo);
        pt[5] = make_float4(Ej[4].hi, Ej[4].lo, Ej[5].hi, Ej[5].lo);
        pt[6] = make_float4(Ce.hi, Ce.lo, we.hi, we.lo);
        pt[7] = make_float4(__int_as_float(si | (sj << 8)), 0.f, 0.f, 0.f);
      }
    }
    // the run's blocks from Hjj and vj: Hij = -Ad^T Hjj, Hii = -Hij Ad
    // (row a: -Ad^T applied to row a of Hij), vi = -Ad^T vj; in the warp's
    // staging rows: Hjj full [36], vj [6], Hij [36]
    const DF hq = dd_norm(dd_add(acc0, acc1));
    float2* hs = rw;
    __syncwarp();
    if (own) {
      if (lane < 21) {
        hs[6 * pa + pb] = dd_st(hq);
        hs[6 * pb + pa] = dd_st(hq);
        runv[r * NV + 57 + lane] = dd_st(hq);
      } else {
        hs[36 + pa] = dd_st(hq);
        runv[r * NV + 84 + pa] = dd_st(hq);
      }
    }
    __syncwarp();
    if (lane < 7) {  // lanes 0..5: column `lane` of Hij; lane 6: vi
      DF v[6], o[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) v[m] = dd_ld(lane < 6 ? hs[6 * m + lane] : hs[36 + m]);
      dpv_adT_dd(T, v, o);
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const float2 x = dd_st(dd_neg(o[m]));
        if (lane < 6) {
          hs[42 + 6 * m + lane] = x;
          runv[r * NV + 21 + 6 * m + lane] = x;
        } else {
          runv[r * NV + 78 + m] = x;
        }
      }
    }
    __syncwarp();
    if (lane < 6) {  // row `lane` of Hii, lower part
      DF v[6], o[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) v[m] = dd_ld(hs[42 + 6 * lane + m]);
      dpv_adT_dd(T, v, o);
#pragma unroll
      for (int m = 0; m < 6; ++m)
        if (m <= lane) runv[r * NV + tri(lane, m)] = dd_st(dd_neg(o[m]));
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cst += __shfl_xor_sync(0xffffffffu, cst, o);
  if (cost && lane == 0 && cst != 0.f) atomicAdd(cost, (double)cst);
  __syncthreads();

  // ---- phase 2: per patch e_k, C_k, w_k as pairs ----------------------------
  // 16 lanes per patch (two patches per warp), one lane per edge: the
  // source-frame column and C, w summed over the lanes (pairs), the
  // target-frame 6-vectors added to their slots of the patch's column by the
  // first lane of each set of edges with the same target (found with
  // __match_any_sync; the lanes' terms wait in the warp's staging rows)
  {
    float* scr = reinterpret_cast<float*>(rows) + wid * 32 * 12;
    const int half = lane >> 4, hl = lane & 15;
    for (int q0 = 2 * wid; q0 < G; q0 += 2 * AD_WARPS) {
      const int q = q0 + half;
      const int k = g * G + q;
      const bool mine = q < G && k < P;
      float2* col = Eh + (size_t)(q < G ? q : q0) * EH_STRIDE;
      DF ei[6], C = {0.f, 0.f}, wv = {0.f, 0.f};
#pragma unroll
      for (int m = 0; m < 6; ++m) ei[m] = DF{0.f, 0.f};
      int si = -1;
      const int p0 = mine ? pptr[k] : 0, cnt = mine ? pptr[k + 1] - p0 : 0;
      const int most = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, 16));
      for (int base = 0; base < most; base += 16) {
        const bool act = base + hl < cnt;
        int key = -1 - lane;  // a key no other lane has
        int sj = 0;
        if (act) {
          const float4* t4 = pterm + 8 * (size_t)(p0 + base + hl);
          const float4 a = t4[0], b = t4[1], c = t4[2], d3 = t4[3], d4 = t4[4], d5 = t4[5], d6 = t4[6],
                       d7 = t4[7];
          const int sl = __float_as_int(d7.x);
          si = sl & 0xff;
          sj = sl >> 8;
          key = (half << 8) | sj;
          dd_acc_add(ei[0], DF{a.x, a.y}); dd_acc_add(ei[1], DF{a.z, a.w});
          dd_acc_add(ei[2], DF{b.x, b.y}); dd_acc_add(ei[3], DF{b.z, b.w});
          dd_acc_add(ei[4], DF{c.x, c.y}); dd_acc_add(ei[5], DF{c.z, c.w});
          dd_acc_add(C, DF{d6.x, d6.y});
          dd_acc_add(wv, DF{d6.z, d6.w});
          float* o = scr + 12 * lane;
          o[0] = d3.x; o[1] = d3.y; o[2] = d3.z; o[3] = d3.w;
          o[4] = d4.x; o[5] = d4.y; o[6] = d4.z; o[7] = d4.w;
          o[8] = d5.x; o[9] = d5.y; o[10] = d5.z; o[11] = d5.w;
        }
        const unsigned same = __match_any_sync(0xffffffffu, key);
        __syncwarp();
        if (act && (int)(__ffs(same) - 1) == lane) {
          DF tj[6];
#pragma unroll
          for (int m = 0; m < 6; ++m) tj[m] = DF{0.f, 0.f};
          for (unsigned bits = same; bits; bits &= bits - 1) {
            const float* o = scr + 12 * (__ffs(bits) - 1);
#pragma unroll
            for (int m = 0; m < 6; ++m) dd_acc_add(tj[m], DF{o[2 * m], o[2 * m + 1]});
          }
          float2* cj = col + 6 * sj;
#pragma unroll
          for (int m = 0; m < 6; ++m) cj[m] = dd_st(dd_add(dd_ld(cj[m]), dd_norm(tj[m])));
        }
        __syncwarp();
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
        for (int m = 0; m < 6; ++m)
          dd_acc_add(ei[m], DF{__shfl_xor_sync(0xffffffffu, ei[m].hi, o), __shfl_xor_sync(0xffffffffu, ei[m].lo, o)});
        dd_acc_add(C, DF{__shfl_xor_sync(0xffffffffu, C.hi, o), __shfl_xor_sync(0xffffffffu, C.lo, o)});
        dd_acc_add(wv, DF{__shfl_xor_sync(0xffffffffu, wv.hi, o), __shfl_xor_sync(0xffffffffu, wv.lo, o)});
        si = max(si, __shfl_xor_sync(0xffffffffu, si, o));
      }
      // the first lane of each half's sums for the whole half (the butterfly
      // may differ in the last bit across lanes)
      const int src = half << 4;
      DF ct = dd_add_f(dd_norm(C), lambda_d);
      ct = DF{__shfl_sync(0xffffffffu, ct.hi, src), __shfl_sync(0xffffffffu, ct.lo, src)};
      DF wf_;
      if (w_ext) {
        wf_ = DF{mine ? w_ext[k] : 0.f, 0.f};
      } else {
        wf_ = dd_norm(wv);
        wf_ = DF{__shfl_sync(0xffffffffu, wf_.hi, src), __shfl_sync(0xffffffffu, wf_.lo, src)};
      }
      if (hl == 0 && q < G && si >= 0) {
#pragma unroll
        for (int m = 0; m < 6; ++m) col[6 * si + m] = dd_st(dd_add(dd_ld(col[6 * si + m]), dd_norm(ei[m])));
      }
      __syncwarp();
      if (q < G) {
        const DF sq = dd_rcp(dd_sqrt(ct));
        for (int m = hl; m < nr; m += 16) col[m] = dd_st(dd_mul(dd_ld(col[m]), sq));
        if (hl == 0) {
          sc[2 * q] = dd_st(sq);
          sc[2 * q + 1] = dd_st(dd_mul(wf_, sq));
          if (k < P) {
            Ct_out[k] = ct.hi + ct.lo;
            wk_out[k] = wf_.hi + wf_.lo;
            Ct2_out[k] = dd_st(ct);
            wk2_out[k] = dd_st(wf_);
          }
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();

  // ---- phase 2b: run sums per window block (in the staging space) ----------
  signed char* prt = reinterpret_cast<signed char*>(rows);
  float2* dgb = rows + DPV_WMAX * DPV_WMAX / 8;
  float2* yrn = dgb + DPV_WMAX * 21;
  for (int q = tid; q < w * w; q += AD_THREADS) prt[q] = -1;
  __syncthreads();
  for (int r = tid; r < nruns; r += AD_THREADS) {
    const int si = rsl[r] & 0xff, sj = rsl[r] >> 8;
    if (si != sj) prt[si * w + sj] = (signed char)r;
  }
  for (int q = tid; q < 27 * w; q += AD_THREADS) {
    const int a = q / 27, e = q - 27 * a;
    const int oi = e < 21 ? e : 78 + (e - 21), oj = e < 21 ? 57 + e : 84 + (e - 21);
    DF acc = {0.f, 0.f};
    for (int r = 0; r < nruns; ++r) {
      const int si = rsl[r] & 0xff, sj = rsl[r] >> 8;
      if (si == sj) continue;
      const float2* rv = runv + r * NV;
      if (si == a) dd_acc_add(acc, dd_ld(rv[oi]));
      if (sj == a) dd_acc_add(acc, dd_ld(rv[oj]));
    }
    if (e < 21) dgb[a * 21 + e] = dd_st(dd_norm(acc));
    else yrn[a * 6 + (e - 21)] = dd_st(dd_norm(acc));
  }
  __syncthreads();

  // ---- phase 3: window Schur complement into the global S and y -----------
  const int nblk = tri(w, 0);
  for (int t = tid; t < 4 * nblk; t += AD_THREADS) {
    const int blk = t >> 2, ha = (t >> 1) & 1, hb = t & 1;
    const int a = tri_row(blk), b = blk - tri(a, 0);
    if (a == b && hb > ha) continue;
    const int ra0 = fr[a], rb0 = fr[b];
    if (ra0 < 0 || rb0 < 0) continue;
    const int R0 = 6 * a + 3 * ha, C0 = 6 * b + 3 * hb;
    DF acc[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) acc[i][j] = DF{0.f, 0.f};
    for (int kl = 0; kl < G; ++kl) {
      const float2* col = Eh + (size_t)kl * EH_STRIDE;
      DF er[3], ec[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        er[i] = dd_neg(dd_ld(col[R0 + i]));
        ec[i] = dd_ld(col[C0 + i]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dd_acc(acc[i][j], er[i], ec[j]);
    }
    if (a == b) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (3 * hb + j <= 3 * ha + i) dd_acc_add(acc[i][j], dd_ld(dgb[a * 21 + tri(3 * ha + i, 3 * hb + j)]));
    } else {
      const int r1 = prt[a * w + b], r2 = prt[b * w + a];
      if (r1 >= 0) {  // run a -> b: Hij rows belong to a
        const float2* rv = runv + r1 * NV + 21;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) dd_acc_add(acc[i][j], dd_ld(rv[6 * (3 * ha + i) + 3 * hb + j]));
      }
      if (r2 >= 0) {  // run b -> a: Hij rows belong to b (transposed)
        const float2* rv = runv + r2 * NV + 21;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) dd_acc_add(acc[i][j], dd_ld(rv[6 * (3 * hb + j) + 3 * ha + i]));
      }
    }
    const int gr = ra0 + 3 * ha, gc = rb0 + 3 * hb;
    double* Sg = S + sd.soff;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (a != b || 3 * hb + j <= 3 * ha + i)
          dpv_red_add(Sg + dpv_s_index(gr + i, gc + j, sd.TS), dd_to_f64(dd_norm(acc[i][j])));
  }
  for (int R = tid; R < nr; R += AD_THREADS) {
    const int a = R / 6, ra = R - 6 * a;
    if (fr[a] < 0) continue;
    DF acc = {0.f, 0.f};
    if (!w_ext) acc = dd_ld(yrn[R]);  // with an external right-hand side v comes from y's init
    for (int kl = 0; kl < G; ++kl) dd_acc(acc, dd_neg(dd_ld(Eh[(size_t)kl * EH_STRIDE + R])), dd_ld(sc[2 * kl + 1]));
    dpv_red_add(y + sd.voff + fr[a] + ra, dd_to_f64(dd_norm(acc)));
  }
}

bool g_dd_ready = false;

ba_status_t setup_dd(ba_handle_t h) {
  if (g_dd_ready) return BA_OK;
  unsigned char pa[NJ], pb[NJ];
  int q = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b <= a; ++b, ++q) { pa[q] = a; pb[q] = b; }  // Hjj (lower)
  for (int a = 0; a < 6; ++a, ++q) { pa[q] = a; pb[q] = 6; }     // vj
  DPV_CUDA(h, cudaMemcpyToSymbol(c_qa, pa, NJ));
  DPV_CUDA(h, cudaMemcpyToSymbol(c_qb, pb, NJ));
  DPV_CUDA(h, cudaFuncSetAttribute(k_assemble_dd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)assemble_dd_smem_bytes(DPV_GMAX_DD, 1)));
  DPV_CUDA(h, cudaFuncSetAttribute(k_assemble_dd<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)assemble_dd_smem_bytes(DPV_GMAX_DD, 9)));
  g_dd_ready = true;
  return BA_OK;
}

}  // namespace

// The double-float assembly launch (BA_MIXED); the caller has prepared S, y
// and the pose table as for k_assemble.
ba_status_t dpv_assemble_dd(ba_handle_t h, double* cost, const float* w_ext) {
  Workspace* ws = h->ws;
  ba_status_t s = setup_dd(h);
  if (s) return s;
  if (h->G > DPV_GMAX_DD)
    return dpv_fail(h, BA_ERR_UNSUPPORTED, "the mixed-precision assembly takes at most 32 patches per group");
  auto kern = h->opt.residual_pixels == 9 ? k_assemble_dd<9> : k_assemble_dd<1>;
  DPV_CUDA(h, dpv_launch_pdl(kern, dim3(h->ngroups), dim3(AD_THREADS),
                             assemble_dd_smem_bytes(h->G, h->opt.residual_pixels), h->stream, h->G, h->P, ws->fdx.p,
                             ws->gprob.p, ws->sysd.p, h->opt.lambda_depth, h->opt.z_min, ws->gptr.p, ws->grun.p,
                             ws->gnr.p, ws->eslot.p, ws->perm.p, ws->pmpos.p, ws->pptr.p, ws->win.p, ws->wlen.p,
                             ws->posef.p, h->patches, h->targets, h->weights, ws->intr, ws->pterm.p, ws->S.p,
                             ws->y.p, ws->Ct.p, ws->wk.p, ws->Ct2.p, ws->wk2.p, cost, w_ext, ws->status));
  ++h->launches;
  return BA_OK;
}
