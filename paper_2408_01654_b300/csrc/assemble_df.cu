// Linearisation + block reduction + Schur complement in double-float
// arithmetic (the BA_MIXED path): what k_assemble (assemble.cu) computes, with
// every quantity of the linearisation carried as a pair of floats, in two
// kernels (Sec. 3.1 Eq. 2-3, the Schur form of Sec. 3.2 "Efficient Global
// Optimization"):
//
//   H = [ B  E ; E^T  C ],  g = [ v ; w ],   S = B + lambda_p I - E Ct^-1 E^T,
//   y = v - E Ct^-1 w,  Ct = C + lambda_d.
//
// k_runs_dd: one warp per (source, target) run of a patch group, four
//   independent warps per CTA.  The warp forms the run's relative pose T_ij
//   in double-float (lanes in parallel), each lane linearises one edge (the
//   residual, the target-pose Jacobian J_j and J_d, dfloat.cuh), the
//   sqrt(w)-scaled rows [J_j, r] are staged in shared memory as pairs and the
//   lanes sum the run's H_jj (21 entries) and v_j (6) as double-float
//   products, one entry per lane.  Every edge of a run shares T_ij and
//   J_i = -J_j Ad(T_ij), so the run's other blocks follow once per run:
//   H_ij = -Ad^T H_jj, H_ii = -H_ij Ad, v_i = -Ad^T v_j.  The run's B blocks
//   and v go straight into the FP64 S and y (red.global.add.f64); the edge's
//   depth terms e_j = J_j^T W J_d, e_i = -Ad^T e_j, J_d^T W J_d and J_d^T W r
//   go to the patch-major table as pairs (128 bytes per edge).
// k_schur_dd: one CTA per patch group (G <= DPV_GMAX_DD patches and the
//   window of frames their edges touch): 16 lanes per patch sum e_k, C_k, w_k
//   as pairs (edges of one patch that share a target frame are summed by the
//   first lane of each such set, found with __match_any_sync) and form the
//   column e_k / sqrt(Ct_k); one thread per 3x3 sub-block of the window's
//   lower triangle then adds -sum_k e_a e_b^T / Ct_k (double-float) to the
//   FP64 S with red.global.add.f64, and likewise -E Ct^-1 w to y.
//
// The two parts of each S entry (B, and the Schur product that nearly
// cancels it) reach the FP64 S separately, each accurate to ~48 bits, so
// their difference keeps the double-float accuracy.  Splitting the work this
// way lets four run CTAs and two Schur CTAs share an SM (~16 KB and ~111 KB
// of shared memory) instead of one CTA doing all phases behind barriers.
#include "dfloat.cuh"

#include <algorithm>

namespace {

constexpr int RW = 4;                        // warps (runs in flight) per run CTA
constexpr int SC_THREADS = 256;
constexpr int SC_WARPS = SC_THREADS / 32;
constexpr int EH_STRIDE = 6 * DPV_WMAX + 1;  // pairs per patch column of E_hat
constexpr int NJ = 27;                       // per-edge run entries: Hjj 21 (lower), vj 6
constexpr int ROWP = 15;                     // staged pairs per edge: [Jj, r] per residual component + pad
constexpr int RPOSE = 42;                    // floats of a run's relative pose: R, t, [t]x R as pairs

__constant__ unsigned char c_qa[NJ], c_qb[NJ];

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

static_assert(2 * 36 + 6 <= 32 * ROWP, "run-transform scratch exceeds a warp's staging rows");

size_t runs_smem_bytes() { return (size_t)RW * (sizeof(float2) * 32 * ROWP + sizeof(float) * RPOSE); }
size_t schur_smem_bytes(int G) {
  return sizeof(float2) * ((size_t)G * EH_STRIDE + 2 * G) + sizeof(float) * SC_WARPS * 32 * 12 +
         sizeof(int) * DPV_WMAX;
}

__device__ __forceinline__ int tri_row(int t) {
  int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (tri(a + 1, 0) <= t) ++a;
  while (tri(a, 0) > t) --a;
  return a;
}

// The run's relative pose T_ij = T_j T_i^-1 from two rows of the pose table
// (R and the camera centre as pairs) into T (RPOSE floats: R, t, [t]x R as
// pairs) by the lanes of one warp: R_ij = R_j R_i^T (lanes 0..8),
// t = R_j (c_i - c_j) (lanes 9..11), then [t]x R (lanes 0..8).
__device__ __forceinline__ void rel_pose_warp(const float* __restrict__ Pi, const float* __restrict__ Pj, float* T,
                                              int lane) {
  if (lane < 9) {
    const int r = lane / 3, c = lane - 3 * r;
    DF acc = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dd_acc(acc, DF{Pj[3 * r + k], Pj[9 + 3 * r + k]}, DF{Pi[3 * c + k], Pi[9 + 3 * c + k]});
    const DF v = dd_norm(acc);
    T[2 * lane] = v.hi;
    T[2 * lane + 1] = v.lo;
  } else if (lane < 12) {
    const int r = lane - 9;
    DF acc = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dd_acc(acc, DF{Pj[3 * r + k], Pj[9 + 3 * r + k]},
             dd_sub(DF{Pi[18 + k], Pi[21 + k]}, DF{Pj[18 + k], Pj[21 + k]}));
    const DF v = dd_norm(acc);
    T[18 + 2 * r] = v.hi;
    T[19 + 2 * r] = v.lo;
  }
  __syncwarp();
  if (lane < 9) {  // ([t]x R)[a][c] = t_{a+1} R[a+2][c] - t_{a+2} R[a+1][c] (indices mod 3)
    const int a = lane / 3, c = lane - 3 * a;
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    const DF v = dd_sub(dd_mul(dd_sm(T, 9 + a1), dd_sm(T, 3 * a2 + c)), dd_mul(dd_sm(T, 9 + a2), dd_sm(T, 3 * a1 + c)));
    T[24 + 2 * lane] = v.hi;
    T[25 + 2 * lane] = v.lo;
  }
  __syncwarp();
}

// PIX residual pixels per edge: 1 (the patch centre) or 9 (the whole patch).
// Five CTAs per SM for PIX = 1 (96 registers, no spills; the kernel issues
// on about half of its cycles, so more resident warps help), four for 9.
template <int PIX>
__global__ void __launch_bounds__(RW * 32, PIX == 1 ? 5 : 4) k_runs_dd(
    int G, int P, const int* __restrict__ fdx, const int* __restrict__ gprob, const SysDesc* __restrict__ sysd,
    float z_min, const int* __restrict__ gptr, const int* __restrict__ grun, const int* __restrict__ gnr,
    const unsigned* __restrict__ eslot, const int* __restrict__ perm, const int* __restrict__ pmpos,
    const int* __restrict__ win, const float* __restrict__ posef, const float* __restrict__ patches,
    const float* __restrict__ targets, const float* __restrict__ weights, const float* __restrict__ intr,
    float4* __restrict__ pterm, double* __restrict__ S, double* __restrict__ y, double* __restrict__ cost,
    int add_v, int* status) {
  extern __shared__ float2 smr[];
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gs = gptr[g], nruns = gnr[g];
  const int* runptr = grun + (size_t)g * (DPV_RMAX + 1);
  const int* wf = win + (size_t)g * DPV_WMAX;
  float2* rw = smr + wid * 32 * ROWP;
  float* T = reinterpret_cast<float*>(smr + RW * 32 * ROWP) + wid * RPOSE;
  const int prob = gprob[g];
  const SysDesc sd = sysd[prob];
  float K[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) K[q] = intr[4 * prob + q];
  const bool own = lane < NJ;  // this lane's run entry: Hjj (lower) or vj
  const int pa = own ? c_qa[lane] : 0, pb = own ? c_qb[lane] : 0;
  float cst = 0.f;
  for (int r = wid; r < nruns; r += RW) {
    const int s0 = gs + runptr[r], s1 = gs + runptr[r + 1];
    const unsigned sw0 = eslot[s0];
    const int si = dpv_slot_i(sw0), sj = dpv_slot_j(sw0);
    const int fi = wf[si], fj = wf[sj];
    const bool self_run = si == sj;
    rel_pose_warp(posef + DPV_POSE_ROW * (size_t)fi, posef + DPV_POSE_ROW * (size_t)fj, T, lane);
    DF acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};  // the two residual components
    for (int b = s0; b < s1; b += 32) {
      const int s = b + lane;
      const int nb = min(32, s1 - b);
      float2* row = rw + lane * ROWP;
      int k = 0, e = 0;
      float2 wt = make_float2(0.f, 0.f);
      if (s < s1) {
        k = g * G + dpv_slot_k(eslot[s]);
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
          const float* pk = patches + 27 * (size_t)k;
          const int pix = PIX == 1 ? 4 : px;
          const DF xb0 = dpv_ray_dd(pk[pix], K[2], K[0]);
          const DF xb1 = dpv_ray_dd(pk[9 + pix], K[3], K[1]);
          EdgeLinDD L;
          dpv_edge_linearize_dd(T, xb0, xb1, pk[22], tg.x, tg.y, K, z_min, self_run, L);
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
              const DF swc = dd_sqrt(DF{wc[c], 0.f});
#pragma unroll
              for (int m = 0; m < 6; ++m) row[7 * c + m] = dd_st(dd_mul(swc, L.Jj[c][m]));
              row[7 * c + 6] = dd_st(dd_mul(swc, L.r[c]));
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
    if (self_run) continue;  // masked edges: nothing to add (warp-uniform)
    // the run's blocks from Hjj and vj into S and y: Hjj full [36], vj [6],
    // then Hij [36] in the warp's staging rows
    const int o0 = fdx[fi], o1 = fdx[fj];
    const int oi = o0 < 0 ? -1 : o0 - sd.voff, oj = o1 < 0 ? -1 : o1 - sd.voff;
    if (oi < 0 && oj < 0) continue;  // both poses held (warp-uniform)
    double* Sg = S + sd.soff;
    const DF hq = dd_norm(dd_add(acc0, acc1));
    float2* hs = rw;
    __syncwarp();
    if (own) {
      if (lane < 21) {
        hs[6 * pa + pb] = dd_st(hq);
        hs[6 * pb + pa] = dd_st(hq);
        if (oj >= 0) dpv_red_add(Sg + dpv_s_index(oj + pa, oj + pb, sd.TS), dd_to_f64(hq));
      } else {
        hs[36 + pa] = dd_st(hq);
        if (oj >= 0 && add_v) dpv_red_add(y + sd.voff + oj + pa, dd_to_f64(hq));
      }
    }
    __syncwarp();
    if (lane < 7) {  // lanes 0..5: column `lane` of Hij = -Ad^T Hjj; lane 6: vi = -Ad^T vj
      DF v[6], o[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) v[m] = dd_ld(lane < 6 ? hs[6 * m + lane] : hs[36 + m]);
      dpv_adT_dd(T, v, o);
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const DF x = dd_neg(o[m]);
        if (lane < 6) {
          hs[42 + 6 * m + lane] = dd_st(x);
          // Hij[m][lane]: row m of frame i, column `lane` of frame j, into the lower triangle of S
          if (oi >= 0 && oj >= 0) {
            const size_t at = oi > oj ? dpv_s_index(oi + m, oj + lane, sd.TS) : dpv_s_index(oj + lane, oi + m, sd.TS);
            dpv_red_add(Sg + at, dd_to_f64(x));
          }
        } else if (oi >= 0 && add_v) {
          dpv_red_add(y + sd.voff + oi + m, dd_to_f64(x));
        }
      }
    }
    __syncwarp();
    if (lane < 6 && oi >= 0) {  // row `lane` of Hii = -Hij Ad, lower part
      DF v[6], o[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) v[m] = dd_ld(hs[42 + 6 * lane + m]);
      dpv_adT_dd(T, v, o);
#pragma unroll
      for (int m = 0; m < 6; ++m)
        if (m <= lane) dpv_red_add(Sg + dpv_s_index(oi + lane, oi + m, sd.TS), dd_to_f64(dd_neg(o[m])));
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cst += __shfl_xor_sync(0xffffffffu, cst, o);
  if (cost && lane == 0 && cst != 0.f) atomicAdd(cost, (double)cst);
}

__global__ void __launch_bounds__(SC_THREADS) k_schur_dd(
    int G, int P, const int* __restrict__ fdx, const int* __restrict__ gprob, const SysDesc* __restrict__ sysd,
    float lambda_d, const int* __restrict__ pptr, const int* __restrict__ win, const int* __restrict__ wlen,
    const float4* __restrict__ pterm, double* __restrict__ S, double* __restrict__ y, float* __restrict__ Ct_out,
    float* __restrict__ wk_out, float2* __restrict__ Ct2_out, float2* __restrict__ wk2_out,
    const float* __restrict__ w_ext, int* status) {
  extern __shared__ float2 sms[];
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int w = wlen[g];
  const int nr = 6 * w;
  float2* Eh = sms;                                       // [G][EH_STRIDE]
  float2* sc = Eh + (size_t)G * EH_STRIDE;                // [G][2]  Ct^-1/2, w Ct^-1/2
  float* scr_all = reinterpret_cast<float*>(sc + 2 * G);  // [warps][32][12]
  int* fr = reinterpret_cast<int*>(scr_all + SC_WARPS * 32 * 12);  // [W] unknown row in the group's system, -1 fixed
  const SysDesc sd = sysd[gprob[g]];
  for (int q = tid; q < G * EH_STRIDE; q += SC_THREADS) Eh[q] = make_float2(0.f, 0.f);
  for (int q = tid; q < w; q += SC_THREADS) {
    const int o = fdx[win[g * DPV_WMAX + q]];
    fr[q] = o < 0 ? -1 : o - sd.voff;
  }
  __syncthreads();

  // ---- per patch e_k, C_k, w_k as pairs: 16 lanes per patch -----------------
  {
    float* scr = scr_all + wid * 32 * 12;
    const int half = lane >> 4, hl = lane & 15;
    for (int q0 = 2 * wid; q0 < G; q0 += 2 * SC_WARPS) {
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

  // ---- the window's Schur product into S and y ------------------------------
  // one thread per 3x3 sub-block (rows 3ha.. of frame a, columns 3hb.. of
  // frame b, a >= b): nine independent double-float sums over the patches
  const int nblk = tri(w, 0);
  double* Sg = S + sd.soff;
  for (int t = tid; t < 4 * nblk; t += SC_THREADS) {
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
    const int gr = ra0 + 3 * ha, gc = rb0 + 3 * hb;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (a != b || 3 * hb + j <= 3 * ha + i)
          dpv_red_add(Sg + dpv_s_index(gr + i, gc + j, sd.TS), dd_to_f64(dd_norm(acc[i][j])));
  }
  for (int R = tid; R < nr; R += SC_THREADS) {
    const int a = R / 6, ra = R - 6 * a;
    if (fr[a] < 0) continue;
    DF acc = {0.f, 0.f};
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
  DPV_CUDA(h, cudaFuncSetAttribute(k_schur_dd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)schur_smem_bytes(DPV_GMAX_DD)));
  // all of the unified L1 / shared storage as shared memory: two Schur CTAs per SM at G = 32
  DPV_CUDA(h, cudaFuncSetAttribute(k_schur_dd, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  g_dd_ready = true;
  return BA_OK;
}

}  // namespace

// The double-float assembly launches (BA_MIXED); the caller has prepared S,
// y and the pose table as for k_assemble.  With an external right-hand side
// (w_ext, the adjoint) the runs add no v: y's initial contents stand for it.
ba_status_t dpv_assemble_dd(ba_handle_t h, double* cost, const float* w_ext) {
  Workspace* ws = h->ws;
  ba_status_t s = setup_dd(h);
  if (s) return s;
  if (h->G > DPV_GMAX_DD)
    return dpv_fail(h, BA_ERR_UNSUPPORTED, "the mixed-precision assembly takes at most 32 patches per group");
  auto kern = h->opt.residual_pixels == 9 ? k_runs_dd<9> : k_runs_dd<1>;
  DPV_CUDA(h, dpv_launch_pdl(kern, dim3(h->ngroups), dim3(RW * 32), runs_smem_bytes(), h->stream, h->G, h->P,
                             (const int*)ws->fdx.p, (const int*)ws->gprob.p, (const SysDesc*)ws->sysd.p,
                             h->opt.z_min, (const int*)ws->gptr.p, (const int*)ws->grun.p, (const int*)ws->gnr.p,
                             (const unsigned*)ws->eslot.p, (const int*)ws->perm.p, (const int*)ws->pmpos.p,
                             (const int*)ws->win.p, (const float*)ws->posef.p, (const float*)h->patches, h->targets,
                             h->weights, (const float*)ws->intr, ws->pterm.p, ws->S.p, ws->y.p, cost, w_ext ? 0 : 1,
                             ws->status));
  ++h->launches;
  DPV_CUDA(h, dpv_launch_pdl(k_schur_dd, dim3(h->ngroups), dim3(SC_THREADS), schur_smem_bytes(h->G), h->stream, h->G,
                             h->P, (const int*)ws->fdx.p, (const int*)ws->gprob.p, (const SysDesc*)ws->sysd.p,
                             h->opt.lambda_depth, (const int*)ws->pptr.p, (const int*)ws->win.p,
                             (const int*)ws->wlen.p, (const float4*)ws->pterm.p, ws->S.p, ws->y.p, ws->Ct.p, ws->wk.p,
                             ws->Ct2.p, ws->wk2.p, w_ext, ws->status));
  ++h->launches;
  return BA_OK;
}
