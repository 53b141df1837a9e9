// Dense solve of the reduced pose system S dxi = y for n <= DPV_SMALL_N in
// one CTA (the Cholesky of the pose block of the Schur complement, appendix
// "Bundle-Adjustment Efficiency").
//
// S and y arrive in FP64 (the assembly accumulates them so); S is rounded to
// FP32 into shared memory as a packed lower triangle and factored as
// S = L D L^T (the Cholesky factor is L D^1/2; a pivot D_k <= 0 means S is
// not positive definite) by blocked right-looking elimination, 32 columns at
// a time:
//   1. warp 0 eliminates the 32x32 diagonal block in registers (lane = row);
//      each column reaches the other rows through a shared-memory vector read
//      with 128-bit broadcast loads;
//   2. warp 0 forms the inverse of the block's unit lower factor (lane =
//      column of the inverse);
//   3. the panel below is A_panel L_kk^-T, one warp per row with a lane per
//      output (no dependency chain);
//   4. all threads apply the rank-32 update to the trailing triangle in 4x4
//      register tiles.
// The triangular solves of the refinement run left-looking in warp 0 (lane =
// row of a 32-row block): the rows above (below) enter as a dot product, the
// diagonal block through its inverse.  The retraction of the poses runs in
// the back-substitution kernel, off this single-CTA critical path.
//
// Equilibration: the FP32 copies are scaled to S' = diag(s) S diag(s) with
// s = diag(S)^-1/2 (unit diagonal), which bounds the factorisation error by the
// condition number of S' instead of S (the pose blocks mix rotations and
// translations of very different scale; loop closures make S ill-conditioned).
// The solve works on z = x / s and returns x = s z.
//
// Refinement: sweeps of x += S^-1 (y - S x) with the same factor, until the
// estimated error left in x is below 1e-7 of it (the correction c_s, or
// rho c_s with the contraction rho ~ c_s / c_{s-1}).  In BA_FP32 the sweeps
// compute the residual in compensated FP32 (TwoProd / TwoSum) from the FP32
// copy of S, which removes the factorisation error; in BA_MIXED they compute
// it in FP64 from the FP64 S.
#include "internal.cuh"

#include <algorithm>

namespace {

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

__host__ __device__ constexpr int small_threads(int NQ) { return NQ <= 2 ? 128 : 512; }
// the FP32 copy of S for the compensated residual fits in shared memory up to
// NQ = 5, as a full square with row stride NP + 4 (conflict-free row reads by
// eight rows x four interleaved column parts per warp)
__host__ __device__ constexpr bool keep_sf(int NQ) { return NQ <= 5; }
__host__ __device__ constexpr int sf_stride(int NQ) { return 32 * NQ + 4; }
__host__ __device__ constexpr size_t small_smem(int NQ) {
  return sizeof(float) * ((size_t)tri(32 * NQ, 0) + (keep_sf(NQ) ? (size_t)32 * NQ * sf_stride(NQ) : 0));
}

// CTA b solves system list[b] of the table sysd (its matrix at S + soff, its
// vectors at voff); without a table (sysd == null) one system of n_direct
// unknowns at the given pointers.
template <int NQ>  // NP = 32 NQ
__global__ void __launch_bounds__(small_threads(NQ)) k_solve_small(
    const SysDesc* __restrict__ sysd, const int* __restrict__ list, int n_direct, double* __restrict__ S_,
    double* __restrict__ y_, double* __restrict__ dx_, float* __restrict__ dxf_, int refine32, int refine64,
    float tol, float lambda_p, int reset, int* status) {
  constexpr int NP = 32 * NQ;
  constexpr int NT = small_threads(NQ);
  constexpr int NWARP = NT / 32;
  constexpr int SFS = sf_stride(NQ);
  extern __shared__ float Lsh[];            // packed lower: trailing A, then the unit factor
  float* Sf = Lsh + tri(NP, 0);             // FP32 copy of S, full square, row stride SFS (keep_sf)
  __shared__ float Pb[NP][33];              // unscaled panel of the current block
  __shared__ float Linv[NQ][32][33];        // inverses of the unit diagonal blocks
  __shared__ __align__(16) float ucol[32];  // column broadcast in the diagonal block
  __shared__ float invD[NP];
  __shared__ float rhs[NP];
  __shared__ float sol[NP];
  __shared__ float xhi[NP], xlo[NP];
  __shared__ float yhi[NP], ylo[NP];
  __shared__ float sc[NP];  // equilibration: S' = diag(sc) S diag(sc), sc = 1 / sqrt(diag S)
  __shared__ double xs64[NP], rs64[NP];  // FP64 residual: x and S x
  __shared__ float red[2 * NWARP];
  __shared__ int bad;
  dpv_pdl_enter();
  if (dpv_status(status)) return;
  int n = n_direct;
  double* S = S_;
  double* y = y_;
  double* dx = dx_;
  float* dxf = dxf_;
  if (sysd) {
    const SysDesc sd = sysd[list[blockIdx.x]];
    n = sd.n;
    S += sd.soff;
    y += sd.voff;
    dx += sd.voff;
    dxf += sd.voff;
  }
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) bad = 0;
  {
    // S: FP64 row-major NP x NP (lower triangle valid), read as pairs; warp w
    // takes rows w, w + NWARP, ..., lane the pairs lane, lane + 32, ... of a
    // row.  The loads of the diagonal (for the equilibration scale) and of
    // every row the thread handles are all issued before the first barrier
    // (one memory round trip, up to 16 pairs in flight per thread); then each
    // value is rounded to FP32 with integer operations and equilibrated,
    // s_i S_ij s_j, into the packed factor storage and the square copy.
    constexpr int NPH = NP / 2;
    constexpr int RW = NP / NWARP;        // rows per warp
    constexpr int PL = (NPH + 31) / 32;   // pairs per lane in a row
    constexpr int RB = RW * PL <= 16 ? RW : (PL >= 8 ? 1 : 8 / PL);  // rows per batch
    const double2* S2 = reinterpret_cast<const double2*>(S);
    double2 v[RB][PL];
    auto load_batch = [&](int rb) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int t = 0; t < PL; ++t) {
          const int i = wid + NWARP * (rb + r), p = lane + 32 * t;
          v[r][t] = (rb + r < RW && p < NPH && 2 * p <= i) ? S2[(size_t)i * NPH + p] : make_double2(0.0, 0.0);
        }
    };
    load_batch(0);
    for (int i = tid; i < NP; i += NT) {
      const float d = dpv_d2f_bits(S[(size_t)i * NP + i]);
      sc[i] = (i < n && d > 0.f) ? rsqrtf(d) : 1.f;
    }
    __syncthreads();
    for (int rb = 0; rb < RW; rb += RB) {
      if (rb > 0) load_batch(rb);
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int t = 0; t < PL; ++t) {
          const int i = wid + NWARP * (rb + r), p = lane + 32 * t;
          if (rb + r >= RW || p >= NPH || 2 * p > i) continue;
          const float si = sc[i];
          const float a0 = dpv_d2f_bits(v[r][t].x) * (si * sc[2 * p]);
          Lsh[tri(i, 2 * p)] = a0;
          if (keep_sf(NQ)) {
            Sf[i * SFS + 2 * p] = a0;
            Sf[2 * p * SFS + i] = a0;
          }
          if (2 * p + 1 <= i) {
            const float a1 = dpv_d2f_bits(v[r][t].y) * (si * sc[2 * p + 1]);
            Lsh[tri(i, 2 * p + 1)] = a1;
            if (keep_sf(NQ)) {
              Sf[i * SFS + 2 * p + 1] = a1;
              Sf[(2 * p + 1) * SFS + i] = a1;
            }
          }
        }
    }
  }
  // reset: leave S (lower triangle) as the next assembly expects it: zero,
  // lambda_p on the free diagonal, 1 on the padding diagonal.  Done here when
  // no refinement sweep reads S from global memory again, else at the end.
  const bool s_read_later = refine64 > 0 || (refine32 > 0 && !keep_sf(NQ));
  auto reset_S = [&](int t0, int nt) {
    double2* S2w = reinterpret_cast<double2*>(S);
    for (int q = t0; q < NP * (NP / 2); q += nt) {
      const int i = q / (NP / 2), p = q - (q / (NP / 2)) * (NP / 2);
      if (2 * p > i) continue;
      double2 v = make_double2(0.0, 0.0);
      if (2 * p == i) v.x = i < n ? (double)lambda_p : 1.0;
      if (2 * p + 1 == i) v.y = i < n ? (double)lambda_p : 1.0;
      S2w[q] = v;
    }
  };
  __syncthreads();

  // 4. trailing update by the panel of block r0p, A[i][j] -= sum_c Pb[i][c]
  // L[j][r0p + c] for i >= j >= r0p + 32, on the 4 x 4 tiles whose columns
  // lie in [c0, c1), threads t0, t0 + nt, ...
  auto update_tiles = [&](int r0p, int c0, int c1, int t0, int nt) {
    const int p1 = r0p + 32, mt = (NP - p1) / 4;
    const int b0 = (c0 - p1) / 4, b1 = (c1 - p1) / 4;
    int total = 0;
    for (int bj = b0; bj < b1; ++bj) total += mt - bj;
    for (int t = t0; t < total; t += nt) {
      int bj = b0, bi = t;
      while (bi >= mt - bj) {
        bi -= mt - bj;
        ++bj;
      }
      bi += bj;
      const int i0 = p1 + 4 * bi, j0 = p1 + 4 * bj;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
      for (int c = 0; c < 32; ++c) {
        float pa[4], lb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) pa[a] = Pb[i0 + a][c];
#pragma unroll
        for (int b = 0; b < 4; ++b) lb[b] = Lsh[tri(j0 + b, r0p) + c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(pa[a], lb[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (i0 + a >= j0 + b) Lsh[tri(i0 + a, j0 + b)] -= acc[a][b];
    }
  };
  // Right-looking with one block of lookahead: before block kb is eliminated
  // its own columns receive the previous panel's update (all threads); then
  // warp 0 eliminates and inverts the diagonal block while the other warps
  // apply the previous panel to the columns beyond it (and, for the first
  // block, reset S for the next assembly).
  for (int r0 = 0; r0 < NP; r0 += 32) {
    const int kb = r0 / 32;
    if (kb > 0) {
      update_tiles(r0 - 32, r0, r0 + 32, tid, NT);
      __syncthreads();
    }
    // 1. diagonal block, lane = row r0 + lane
    if (wid == 0) {
      float a[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) a[c] = c <= lane ? Lsh[tri(r0 + lane, r0 + c)] : 0.f;
      bool ok = true;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        ucol[lane] = a[c];
        __syncwarp();
        const float d = ucol[c];
        ok = ok && (d > 0.f);
        float inv;  // approximate reciprocal: the refinement absorbs its last-bit error
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(d));
        const float l = a[c] * inv;
        float u[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 v = reinterpret_cast<const float4*>(ucol)[q];
          u[4 * q] = v.x; u[4 * q + 1] = v.y; u[4 * q + 2] = v.z; u[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int j = c + 1; j < 32; ++j) a[j] = fmaf(-l, u[j], a[j]);
        if (lane == c) invD[r0 + c] = inv;
        if (lane > c) a[c] = l;
        __syncwarp();
      }
      if (!ok && lane == 0) bad = 1;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < lane) Lsh[tri(r0 + lane, r0 + c)] = a[c];
      __syncwarp();
      // 2. inverse of the unit lower block: lane c solves L_kk x = e_c
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < 31; ++k)
#pragma unroll
        for (int i = k + 1; i < 32; ++i) x[i] = fmaf(-Lsh[tri(r0 + i, r0 + k)], x[k], x[i]);
#pragma unroll
      for (int i = 0; i < 32; ++i) Linv[kb][i][lane] = x[i];
    } else {
      if (kb > 0 && r0 + 32 < NP) update_tiles(r0 - 32, r0 + 32, NP, tid - 32, NT - 32);
      if (kb == 0 && reset && !s_read_later) reset_S(tid - 32, NT - 32);
    }
    __syncthreads();
    if (bad) break;
    if (r0 + 32 == NP) break;
    // 3. panel rows below the block: P = A_panel L_kk^-T (lane = output column)
    // (three rows per warp at a time: independent dependency chains)
    for (int i0 = r0 + 32 + wid; i0 < NP; i0 += 3 * NWARP) {
      float p[3] = {0.f, 0.f, 0.f};
      const float* ai[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) ai[u] = Lsh + tri(min(i0 + u * NWARP, NP - 1), r0);
#pragma unroll 8
      for (int cp = 0; cp < 32; ++cp) {
        const float li = Linv[kb][lane][cp];
#pragma unroll
        for (int u = 0; u < 3; ++u) p[u] = fmaf(ai[u][cp], li, p[u]);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = i0 + u * NWARP;
        if (i < NP) {
          Pb[i][lane] = p[u];
          Lsh[tri(i, r0 + lane)] = p[u] * invD[r0 + lane];
        }
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) dpv_set_status(status, DST_NOT_SPD);
    return;
  }
  for (int q = tid; q < NP; q += NT) {
    const double yq = q < n ? y[q] * (double)sc[q] : 0.0;  // the equilibrated right-hand side
    const float yh = (float)yq;
    yhi[q] = yh;
    ylo[q] = (float)(yq - (double)yh);
    rhs[q] = yh;
    xhi[q] = 0.f;
    xlo[q] = 0.f;
  }
  __syncthreads();

  const int sweeps = 1 + refine32 + refine64;
  float cprev = 0.f;  // the previous sweep's largest correction
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    // the two triangular solves in warp 0 (lane = row of a 32-row block);
    // the other warps wait at the barrier.  Forward, left-looking:
    //   u_b = L_bb^-1 (rhs_b - sum_{j<b} L_bj u_j)  (into sol)
    if (wid == 0) {
      float* vb = ucol;
      for (int kb = 0; kb < NQ; ++kb) {
        const int r0 = 32 * kb, r = r0 + lane;
        const float* lr = Lsh + tri(r, 0);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int c = 0; c < r0; c += 4) {
          a0 = fmaf(lr[c], sol[c], a0);
          a1 = fmaf(lr[c + 1], sol[c + 1], a1);
          a2 = fmaf(lr[c + 2], sol[c + 2], a2);
          a3 = fmaf(lr[c + 3], sol[c + 3], a3);
        }
        vb[lane] = rhs[r] - ((a0 + a1) + (a2 + a3));
        __syncwarp();
        float u0 = 0.f, u1 = 0.f, u2 = 0.f, u3 = 0.f;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          u0 = fmaf(Linv[kb][lane][c], vb[c], u0);
          u1 = fmaf(Linv[kb][lane][c + 1], vb[c + 1], u1);
          u2 = fmaf(Linv[kb][lane][c + 2], vb[c + 2], u2);
          u3 = fmaf(Linv[kb][lane][c + 3], vb[c + 3], u3);
        }
        sol[r] = (u0 + u1) + (u2 + u3);
        __syncwarp();
      }
      // backward, left-looking from the bottom (into rhs):
      //   x_b = L_bb^-T (D_b^-1 u_b - sum_{i>b} L_ib^T x_i)
      for (int kb = NQ - 1; kb >= 0; --kb) {
        const int r0 = 32 * kb, r = r0 + lane;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int i = r0 + 32;
        for (; i + 3 < NP; i += 4) {
          a0 = fmaf(Lsh[tri(i, r)], rhs[i], a0);
          a1 = fmaf(Lsh[tri(i + 1, r)], rhs[i + 1], a1);
          a2 = fmaf(Lsh[tri(i + 2, r)], rhs[i + 2], a2);
          a3 = fmaf(Lsh[tri(i + 3, r)], rhs[i + 3], a3);
        }
        vb[lane] = sol[r] * invD[r] - ((a0 + a1) + (a2 + a3));
        __syncwarp();
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          x0 = fmaf(Linv[kb][c][lane], vb[c], x0);
          x1 = fmaf(Linv[kb][c + 1][lane], vb[c + 1], x1);
          x2 = fmaf(Linv[kb][c + 2][lane], vb[c + 2], x2);
          x3 = fmaf(Linv[kb][c + 3][lane], vb[c + 3], x3);
        }
        rhs[r] = (x0 + x1) + (x2 + x3);
        __syncwarp();
      }
    }
    __syncthreads();
    // x += correction (double-float); stop once the correction is below
    // tol of the solution (refinement converged)
    float cmax = 0.f, xmax = 0.f;
    for (int q = tid; q < NP; q += NT) {
      DF a = {xhi[q], xlo[q]};
      df_add(a, rhs[q]);
      xhi[q] = a.hi;
      xlo[q] = a.lo;
      cmax = fmaxf(cmax, fabsf(rhs[q]));
      xmax = fmaxf(xmax, fabsf(a.hi));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
      xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if (lane == 0) {
      red[wid] = cmax;
      red[NWARP + wid] = xmax;
    }
    __syncthreads();
    if (sweep + 1 == sweeps) break;
    {
      float cm = 0.f, xm = 0.f;
      for (int w = 0; w < NWARP; ++w) {
        cm = fmaxf(cm, red[w]);
        xm = fmaxf(xm, red[NWARP + w]);
      }
      // stop once the error left in x is below tol of it: the correction
      // bounds the previous iterate's error, and the current one's is about
      // rho c_s with the contraction rate rho ~ c_s / c_{s-1}
      // (the same decision in every thread)
      if (sweep > 0 && (cm <= tol * xm || cm * cm <= tol * xm * cprev)) break;
      cprev = cm;
    }
    // residual rho = y - S x
    if (sweep < refine32 && keep_sf(NQ)) {
      // compensated FP32 against the FP32 copy of S: four threads per row,
      // each over the columns c = part (mod 4)
      for (int r0 = 0; r0 < NP; r0 += NT / 4) {
        const int r = r0 + (tid >> 2), part = tid & 3;
        DF acc = {0.f, 0.f};
        if (r < n) {
          const float* srow = Sf + r * SFS;
          for (int c = part; c < n; c += 4) {
            const float sv = srow[c];
            df_fma(acc, sv, xhi[c]);
            acc.lo = fmaf(sv, xlo[c], acc.lo);
          }
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, acc.hi, o), ol = __shfl_xor_sync(0xffffffffu, acc.lo, o);
          df_add(acc, oh);
          acc.lo += ol;
        }
        if (part == 0 && r < NP) {
          DF rr = {yhi[r], ylo[r]};
          df_add(rr, -acc.hi);
          rr.lo -= acc.lo;
          rhs[r] = r < n ? df_val(rr) : 0.f;
        }
      }
    } else {
      // FP64 from the FP64 S (lower triangle, symmetric), read row by row
      // (coalesced): entry (r, c), c < r, adds to rows r and c; x in FP64
      for (int q = tid; q < NP; q += NT) {
        xs64[q] = q < n ? (double)sc[q] * ((double)xhi[q] + (double)xlo[q]) : 0.0;
        rs64[q] = 0.0;
      }
      __syncthreads();
      for (int r = wid; r < n; r += NWARP) {
        const double xr = xs64[r];
        const double* srow = S + (size_t)r * NP;
        double acc = 0.0;
        for (int c = lane; c <= r; c += 32) {
          const double sv = srow[c];
          acc += sv * xs64[c];
          if (c < r) atomicAdd(&rs64[c], sv * xr);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(&rs64[r], acc);
      }
      __syncthreads();
      for (int r = tid; r < NP; r += NT) rhs[r] = r < n ? (float)((y[r] - rs64[r]) * (double)sc[r]) : 0.f;
    }
    __syncthreads();
  }
  for (int q = tid; q < n; q += NT) {
    const double xq = (dpv_f2d_bits(xhi[q]) + dpv_f2d_bits(xlo[q])) * dpv_f2d_bits(sc[q]);
    dx[q] = xq;
    dxf[q] = dpv_d2f_bits(xq);
  }
  if (reset) {
    if (s_read_later) {
      __syncthreads();
      reset_S(tid, NT);
    }
    for (int q = tid; q < NP; q += NT) y[q] = 0.0;
  }
}

template <int NQ>
ba_status_t launch_small(ba_handle_t h, cudaStream_t st, int count, const int* list, int refine32, int refine64,
                         int reset) {
  static bool attr = false;
  const size_t smem = small_smem(NQ);
  if (!attr) {
    DPV_CUDA(h, cudaFuncSetAttribute(k_solve_small<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  DPV_CUDA(h, dpv_launch_pdl(k_solve_small<NQ>, dim3(count), dim3(small_threads(NQ)), smem, st, h->ws->sysd.p, list,
                             0, h->ws->S.p, h->ws->y.p, h->ws->dx.p, h->ws->tmpv.p, refine32, refine64,
                             dpv_solve_tol(h), h->opt.lambda_pose, reset, h->ws->status));
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

}  // namespace

ba_status_t dpv_solve_large(ba_handle_t h, int refine);

// Solve every pose system S_b dxi_b = y_b: one launch of the one-CTA solver per
// block count (one CTA per system), then the large systems.
ba_status_t dpv_solve(ba_handle_t h, int* retracted, int reset_system) {
  // refinement sweeps, stopped early once converged: BA_FP32 up to three
  // compensated-FP32 sweeps (small systems), BA_MIXED FP64 sweeps
  const int refine32 = h->opt.precision == BA_MIXED ? 0 : 3;
  const int refine64 = h->opt.precision == BA_MIXED ? h->opt.max_refine : 0;
  *retracted = 0;
  if (h->n == 0) return BA_OK;
  ba_status_t s = BA_OK;
  int buckets = 0;
  for (int nq = 1; nq <= 8; ++nq) buckets += h->small_nq[nq].empty() ? 0 : 1;
  // several block counts: one launch each on its own side stream, forked from
  // and joined back to the handle's stream (the streams and events are made
  // by an eager run, never inside a graph capture)
  bool fork = buckets > 1;
  if (fork && !h->ev_fork) {
    if (h->capturing) {
      fork = false;
    } else {
      DPV_CUDA(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
      for (int q = 0; q < 8; ++q) {
        DPV_CUDA(h, cudaStreamCreateWithFlags(&h->side[q], cudaStreamNonBlocking));
        DPV_CUDA(h, cudaEventCreateWithFlags(&h->ev_join[q], cudaEventDisableTiming));
      }
    }
  }
  if (fork) DPV_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
  int off = 0;
  for (int nq = 1; nq <= 8; ++nq) {
    const int cnt = (int)h->small_nq[nq].size();
    if (!cnt) continue;
    const int* list = h->ws->syslist.p + off;
    cudaStream_t st = h->stream;
    if (fork) {
      st = h->side[nq - 1];
      DPV_CUDA(h, cudaStreamWaitEvent(st, h->ev_fork, 0));
    }
    switch (nq) {
      case 1: s = launch_small<1>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 2: s = launch_small<2>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 3: s = launch_small<3>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 4: s = launch_small<4>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 5: s = launch_small<5>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 6: s = launch_small<6>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 7: s = launch_small<7>(h, st, cnt, list, refine32, refine64, reset_system); break;
      case 8: s = launch_small<8>(h, st, cnt, list, refine32, refine64, reset_system); break;
    }
    if (s) return s;
    if (fork) {
      DPV_CUDA(h, cudaEventRecord(h->ev_join[nq - 1], st));
      DPV_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join[nq - 1], 0));
    }
    off += cnt;
  }
  // large systems, all together: preconditioned conjugate gradients until converged
  return dpv_solve_large(h, std::max(8, refine64));
}

// Launch the one-CTA solver on a system the caller has already laid out as one
// n_pad x n_pad tile (lower triangle, identity on the padding), without the
// retraction.  Used by the allocation-free entry point in noalloc.cu.
namespace {
template <int NQ>
ba_status_t launch_small_raw(cudaStream_t st, int n, const double* S, const double* y, double* dx, float* dxf,
                             int refine, int* status) {
  const size_t smem = small_smem(NQ);
  if (cudaFuncSetAttribute(k_solve_small<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return BA_ERR_CUDA;
  // reset = 0: the kernel only reads S and y
  k_solve_small<NQ><<<1, small_threads(NQ), smem, st>>>(nullptr, nullptr, n, const_cast<double*>(S),
                                                        const_cast<double*>(y), dx, dxf, 0, refine, 1e-7f, 0.f, 0,
                                                        status);
  return cudaGetLastError() == cudaSuccess ? BA_OK : BA_ERR_CUDA;
}
}  // namespace

ba_status_t dpv_launch_small_solver(cudaStream_t st, int n, int n_pad, const double* S, const double* y, double* dx,
                                    float* dxf, int refine, int* status) {
  switch (n_pad / 32) {
    case 1: return launch_small_raw<1>(st, n, S, y, dx, dxf, refine, status);
    case 2: return launch_small_raw<2>(st, n, S, y, dx, dxf, refine, status);
    case 3: return launch_small_raw<3>(st, n, S, y, dx, dxf, refine, status);
    case 4: return launch_small_raw<4>(st, n, S, y, dx, dxf, refine, status);
    case 5: return launch_small_raw<5>(st, n, S, y, dx, dxf, refine, status);
    case 6: return launch_small_raw<6>(st, n, S, y, dx, dxf, refine, status);
    case 7: return launch_small_raw<7>(st, n, S, y, dx, dxf, refine, status);
    case 8: return launch_small_raw<8>(st, n, S, y, dx, dxf, refine, status);
  }
  return BA_ERR_UNSUPPORTED;
}
