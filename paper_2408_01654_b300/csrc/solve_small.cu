// Dense solve of the reduced pose system S dxi = y for n <= DPV_SMALL_N in
// one CTA (the Cholesky of the pose block of the Schur complement, appendix
// "Bundle-Adjustment Efficiency"), followed by the SE(3) retraction of the
// free poses.
//
// S and y arrive in FP64 (the assembly accumulates them so).  S is rounded to
// FP32 into shared memory as a packed lower triangle and factored as
// S = L D L^T (the Cholesky factor is L D^1/2; a pivot D_c <= 0 means S is
// not positive definite) by blocked right-looking elimination with 8-column
// panels:
//   * warp 0 holds the panel in registers (rows lane + 32q) and eliminates its
//     8 columns with shuffles only, then stores it with the scaled copy
//     W = panel D^-1;
//   * all 16 warps apply the rank-8 update A -= panel W^T to the trailing
//     triangle -- two block barriers per panel.
// The triangular solves run in 32-row blocks: warp 0 keeps the block's 32x32
// triangle in registers and solves it with shuffles, all warps update the
// rest of the right-hand side.  In BA_MIXED mode the solution is refined:
// rho = y - S x in FP64 from the FP64 S in global memory, solved with the same
// factor, x += delta.
#include "internal.cuh"

#include "retract.cuh"

namespace {

constexpr int SS_THREADS = 512;
constexpr int SS_WARPS = SS_THREADS / 32;
constexpr int PW = 8;  // panel width

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

template <int NQ>  // NP = 32 NQ
__global__ void __launch_bounds__(SS_THREADS) k_solve_small(int n, const double* __restrict__ S,
                                                            const double* __restrict__ y, double* __restrict__ dx,
                                                            float* __restrict__ dxf, int refine, int N, int fixed,
                                                            double* __restrict__ poses, int* status) {
  constexpr int NP = 32 * NQ;
  extern __shared__ float A[];              // packed lower, tri(NP, 0) floats
  __shared__ float W[PW][NP];               // scaled panel
  __shared__ float invD[NP];
  __shared__ float rhs[NP];
  __shared__ double xs[NP];
  __shared__ int bad;
  if (dpv_status(status)) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = wid; i < NP; i += SS_WARPS)
    for (int j = lane; j <= i; j += 32) A[tri(i, j)] = (float)S[(size_t)i * NP + j];
  if (tid == 0) bad = 0;
  __syncthreads();

  for (int p0 = 0; p0 < NP; p0 += PW) {
    if (wid == 0) {
      // panel rows i = p0 + lane + 32 q, columns p0 .. p0+7, in registers
      float pr[NQ][PW];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int i = p0 + lane + 32 * q;
#pragma unroll
        for (int c = 0; c < PW; ++c) pr[q][c] = (i < NP && i >= p0 + c) ? A[tri(i, p0 + c)] : 0.f;
      }
      bool ok = true;
#pragma unroll
      for (int c = 0; c < PW; ++c) {
        const float dc = __shfl_sync(0xffffffffu, pr[0][c], c);
        ok = ok && (dc > 0.f);
        const float inv = 1.0f / dc;
        if (lane == 0) invD[p0 + c] = inv;
        float ajc[PW];
#pragma unroll
        for (int j = c + 1; j < PW; ++j) ajc[j] = __shfl_sync(0xffffffffu, pr[0][c], j);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int i = p0 + lane + 32 * q;
          const float aic = pr[q][c] * inv;
#pragma unroll
          for (int j = c + 1; j < PW; ++j)
            if (i >= p0 + j) pr[q][j] = fmaf(-aic, ajc[j], pr[q][j]);
        }
      }
      if (!ok && lane == 0) bad = 1;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int i = p0 + lane + 32 * q;
        if (i < NP) {
#pragma unroll
          for (int c = 0; c < PW; ++c) {
            if (i >= p0 + c) A[tri(i, p0 + c)] = pr[q][c];
            W[c][i] = pr[q][c] * invD[p0 + c];
          }
        }
      }
    }
    __syncthreads();
    if (bad) break;
    // rank-PW update of the trailing triangle: A[i][j] -= sum_c A[i][p0+c] W[c][j]
    const int p1 = p0 + PW;
    for (int i = p1 + wid; i < NP; i += SS_WARPS) {
      float ai[PW];
#pragma unroll
      for (int c = 0; c < PW; ++c) ai[c] = A[tri(i, p0 + c)];
      for (int j = p1 + lane; j <= i; j += 32) {
        float s = A[tri(i, j)];
#pragma unroll
        for (int c = 0; c < PW; ++c) s = fmaf(-ai[c], W[c][j], s);
        A[tri(i, j)] = s;
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) dpv_set_status(status, DST_NOT_SPD);
    return;
  }
  // unit lower factor L = A D^-1 (strict lower part, in place)
  for (int i = wid; i < NP; i += SS_WARPS)
    for (int j = lane; j < i; j += 32) A[tri(i, j)] *= invD[j];
  for (int q = tid; q < NP; q += SS_THREADS) {
    rhs[q] = q < n ? (float)y[q] : 0.f;
    xs[q] = 0.0;
  }
  __syncthreads();

  for (int sweep = 0; sweep <= refine; ++sweep) {
    // forward: L u = rhs
    for (int r0 = 0; r0 < NP; r0 += 32) {
      if (wid == 0) {
        float Lrow[32];  // row r0+lane of the diagonal block
#pragma unroll
        for (int c = 0; c < 32; ++c) Lrow[c] = c < lane ? A[tri(r0 + lane, r0 + c)] : 0.f;
        float v = rhs[r0 + lane];
#pragma unroll
        for (int c = 0; c < 32; ++c) v = fmaf(-Lrow[c], __shfl_sync(0xffffffffu, v, c), v);
        rhs[r0 + lane] = v;
      }
      __syncthreads();
      for (int i = r0 + 32 + tid; i < NP; i += SS_THREADS) {
        float v = rhs[i];
        const float* li = A + tri(i, r0);
#pragma unroll 8
        for (int c = 0; c < 32; ++c) v = fmaf(-li[c], rhs[r0 + c], v);
        rhs[i] = v;
      }
      __syncthreads();
    }
    for (int q = tid; q < NP; q += SS_THREADS) rhs[q] *= invD[q];
    __syncthreads();
    // backward: L^T x = v
    for (int r0 = NP - 32; r0 >= 0; r0 -= 32) {
      if (wid == 0) {
        float Lcol[32];  // column r0+lane of the diagonal block
#pragma unroll
        for (int r = 0; r < 32; ++r) Lcol[r] = r > lane ? A[tri(r0 + r, r0 + lane)] : 0.f;
        float v = rhs[r0 + lane];
#pragma unroll
        for (int r = 31; r >= 0; --r) v = fmaf(-Lcol[r], __shfl_sync(0xffffffffu, v, r), v);
        rhs[r0 + lane] = v;
      }
      __syncthreads();
      for (int j = tid; j < r0; j += SS_THREADS) {
        float v = rhs[j];
#pragma unroll 8
        for (int r = 0; r < 32; ++r) v = fmaf(-A[tri(r0 + r, j)], rhs[r0 + r], v);
        rhs[j] = v;
      }
      __syncthreads();
    }
    for (int q = tid; q < NP; q += SS_THREADS) xs[q] += (double)rhs[q];
    __syncthreads();
    if (sweep == refine) break;
    // rho = y - S x in FP64 from the FP64 S (lower triangle, symmetric)
    for (int r = wid; r < NP; r += SS_WARPS) {
      double acc = 0.0;
      if (r < n)
        for (int c = lane; c < n; c += 32) {
          const double sv = c <= r ? S[(size_t)r * NP + c] : S[(size_t)c * NP + r];
          acc += sv * xs[c];
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) rhs[r] = r < n ? (float)(y[r] - acc) : 0.f;
    }
    __syncthreads();
  }
  for (int q = tid; q < n; q += SS_THREADS) {
    dx[q] = xs[q];
    dxf[q] = (float)xs[q];
  }
  // SE(3) retraction of the free poses (FP64)
  for (int f = tid; f < N - fixed; f += SS_THREADS) dpv_se3_retract(xs + 6 * f, poses + 7 * (size_t)(fixed + f));
}

template <int NQ>
ba_status_t launch_small(ba_handle_t h, int refine) {
  static bool attr = false;
  const size_t smem = sizeof(float) * (size_t)tri(32 * NQ, 0);
  if (!attr) {
    DPV_CUDA(h, cudaFuncSetAttribute(k_solve_small<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_solve_small<NQ><<<1, SS_THREADS, smem, h->stream>>>(h->n, h->ws->S.p, h->ws->y.p, h->ws->dx.p, h->ws->tmpv.p,
                                                        refine, h->N, h->fixed, h->poses, h->ws->status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

}  // namespace

ba_status_t dpv_solve_blocked(ba_handle_t h, int refine);

// Solve S dxi = y.  For n <= DPV_SMALL_N this also retracts the poses
// (*retracted = 1); otherwise the caller launches the retraction.
ba_status_t dpv_solve(ba_handle_t h, int* retracted) {
  const int refine = h->opt.precision == BA_MIXED ? h->opt.max_refine : 0;
  *retracted = 0;
  if (h->n == 0) return BA_OK;
  if (h->n > DPV_SMALL_N) return dpv_solve_blocked(h, refine);
  ba_status_t s;
  switch (h->n_pad / 32) {
    case 1: s = launch_small<1>(h, refine); break;
    case 2: s = launch_small<2>(h, refine); break;
    case 3: s = launch_small<3>(h, refine); break;
    case 4: s = launch_small<4>(h, refine); break;
    case 5: s = launch_small<5>(h, refine); break;
    case 6: s = launch_small<6>(h, refine); break;
    case 7: s = launch_small<7>(h, refine); break;
    case 8: s = launch_small<8>(h, refine); break;
    default: return dpv_fail(h, BA_ERR_UNSUPPORTED, "pose system size");
  }
  if (s == BA_OK) *retracted = 1;
  return s;
}

// Launch the one-CTA solver on a system the caller has already laid out as one
// n_pad x n_pad tile (lower triangle, identity on the padding), without the
// retraction.  Used by the allocation-free entry point in noalloc.cu.
namespace {
template <int NQ>
ba_status_t launch_small_raw(cudaStream_t st, int n, const double* S, const double* y, double* dx, float* dxf,
                             int refine, int* status) {
  const size_t smem = sizeof(float) * (size_t)tri(32 * NQ, 0);
  if (cudaFuncSetAttribute(k_solve_small<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return BA_ERR_CUDA;
  k_solve_small<NQ><<<1, SS_THREADS, smem, st>>>(n, S, y, dx, dxf, refine, 0, 0, nullptr, status);
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
