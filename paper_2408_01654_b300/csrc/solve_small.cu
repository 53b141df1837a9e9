// Dense solve of the reduced pose system S dxi = y for n <= DPV_SMALL_N in
// one CTA (the Cholesky of the pose block of the Schur complement, appendix
// "Bundle-Adjustment Efficiency").
//
// S (n_pad x n_pad, one tile, lower triangle) is factored as S = L D L^T by
// right-looking elimination without square roots: after step k, column k+1
// of the trailing matrix is final.  A 32x32 thread grid owns the entries
// (ty + 32a, tx + 32b) in registers; each step reads column k from a
// double-buffered shared vector, updates the owned trailing entries and
// publishes column k+1, so there is one __syncthreads per column.  D > 0 at
// every pivot is exactly S being positive definite (the Cholesky factor is
// L D^1/2).  The two triangular solves run in one warp.  In BA_MIXED mode the
// solution is refined: rho = y - S x in FP64 from the unfactored S, solved
// with the same factor, x += delta.
#include "internal.cuh"

namespace {

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

template <int NB>
__global__ void __launch_bounds__(1024) k_solve_small(int n, const float* __restrict__ S, const float* __restrict__ y,
                                                      double* __restrict__ dx, int refine, int* status) {
  constexpr int NP = NB * 32;
  __shared__ float col[2][NP];
  __shared__ float Dsh[NP];
  __shared__ double xs[NP];
  __shared__ float rhs[NP];
  extern __shared__ float Lsh[];  // packed strictly-lower L (unit), tri(i, j) for i > j
  if (dpv_status(status)) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float A[NB][NB];
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = ty + 32 * a, j = tx + 32 * b;
      A[a][b] = (i >= j) ? S[(size_t)i * NP + j] : 0.f;
    }
  if (tx == 0) {
#pragma unroll
    for (int a = 0; a < NB; ++a) col[0][ty + 32 * a] = A[a][0];
  }
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < NP; ++k) {
    const float* ck = col[k & 1];
    const float akk = ck[k];
    if (!(akk > 0.f)) {  // same value in every thread: uniform exit
      bad = true;
      break;
    }
    const float inv = 1.0f / akk;
    float ci[NB], cj[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) ci[a] = ck[ty + 32 * a];
#pragma unroll
    for (int b = 0; b < NB; ++b) cj[b] = ck[tx + 32 * b] * inv;
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int i = ty + 32 * a, j = tx + 32 * b;
        if (j > k && i >= j) A[a][b] = fmaf(-ci[a], cj[b], A[a][b]);
      }
    const int kn = k + 1;
    if (kn < NP && tx == (kn & 31)) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b == (kn >> 5)) {
#pragma unroll
          for (int a = 0; a < NB; ++a) col[kn & 1][ty + 32 * a] = A[a][b];
        }
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) dpv_set_status(status, DST_NOT_SPD);
    return;
  }
  // pivots, then unit-lower L = A / D
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (ty + 32 * a == tx + 32 * b) Dsh[ty + 32 * a] = A[a][b];
  for (int q = threadIdx.x; q < NP; q += blockDim.x) xs[q] = 0.0;
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = ty + 32 * a, j = tx + 32 * b;
      if (i > j) Lsh[tri(i, j)] = A[a][b] / Dsh[j];
    }
  for (int q = threadIdx.x; q < NP; q += blockDim.x) rhs[q] = q < n ? y[q] : 0.f;
  __syncthreads();

  for (int sweep = 0; sweep <= refine; ++sweep) {
    if (ty == 0) {
      // forward: L u = rhs (unit lower), column oriented
      for (int j = 0; j < NP; ++j) {
        const float uj = rhs[j];
        __syncwarp();
        for (int i = j + 1 + tx; i < NP; i += 32) rhs[i] = fmaf(-Lsh[tri(i, j)], uj, rhs[i]);
        __syncwarp();
      }
      for (int j = tx; j < NP; j += 32) rhs[j] /= Dsh[j];
      __syncwarp();
      // backward: L^T x = v, row oriented (row i of L is contiguous)
      for (int i = NP - 1; i >= 0; --i) {
        const float xi = rhs[i];
        __syncwarp();
        for (int j = tx; j < i; j += 32) rhs[j] = fmaf(-Lsh[tri(i, j)], xi, rhs[j]);
        __syncwarp();
      }
      for (int j = tx; j < NP; j += 32) xs[j] += (double)rhs[j];
    }
    __syncthreads();
    if (sweep == refine) break;
    // rho = y - S x in FP64, S symmetric from its lower triangle
    for (int r = ty; r < n; r += 32) {
      double acc = 0.0;
      for (int c = tx; c < n; c += 32) {
        const float s = c <= r ? S[(size_t)r * NP + c] : S[(size_t)c * NP + r];
        acc += (double)s * xs[c];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (tx == 0) rhs[r] = (float)((double)y[r] - acc);
    }
    for (int q = n + threadIdx.x; q < NP; q += blockDim.x) rhs[q] = 0.f;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) dx[q] = xs[q];
}

template <int NB>
ba_status_t launch_small(ba_handle_t h, int refine) {
  constexpr int NP = NB * 32;
  const size_t smem = sizeof(float) * (size_t)tri(NP, 0);
  static bool set = false;
  if (!set) {
    DPV_CUDA(h, cudaFuncSetAttribute(k_solve_small<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set = true;
  }
  k_solve_small<NB><<<1, 1024, smem, h->stream>>>(h->n, h->ws->S.p, h->ws->y.p, h->ws->dx.p, refine, h->ws->status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

}  // namespace

ba_status_t dpv_solve_blocked(ba_handle_t h, int refine);

ba_status_t dpv_solve(ba_handle_t h) {
  const int refine = h->opt.precision == BA_MIXED ? h->opt.max_refine : 0;
  if (h->n == 0) return BA_OK;
  if (h->n > DPV_SMALL_N) return dpv_solve_blocked(h, refine);
  switch (h->n_pad / 32) {
    case 1: return launch_small<1>(h, refine);
    case 2: return launch_small<2>(h, refine);
    case 3: return launch_small<3>(h, refine);
    case 4: return launch_small<4>(h, refine);
    case 5: return launch_small<5>(h, refine);
    case 6: return launch_small<6>(h, refine);
    case 7: return launch_small<7>(h, refine);
    case 8: return launch_small<8>(h, refine);
  }
  return dpv_fail(h, BA_ERR_UNSUPPORTED, "pose system size");
}
