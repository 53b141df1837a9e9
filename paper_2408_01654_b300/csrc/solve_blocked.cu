// Blocked solve of the reduced pose system for n > DPV_SMALL_N (the global
// loop-closure BA: the dense Cholesky of the pose block of the Schur
// complement that the appendix "Bundle-Adjustment Efficiency" names as the
// memory and runtime bottleneck).
//
// S (FP64, tiled lower triangle) is copied to a dense row-major FP32 matrix
// A (lower triangle used) and factored as S = L D L^T, 64 columns per step:
//   k_lg_diag    one CTA: eliminates the 64x64 diagonal block in shared
//                memory (one barrier per column), writes L and D^-1, and the
//                inverse of the unit block factor;
//   k_lg_panel   one warp per row below: P = A_panel L_kk^-T (unscaled) and
//                L_panel = P D^-1;
//   k_lg_update  64x64 output tiles of the trailing triangle:
//                A_ij -= P_i L_j^T (rank-64, FP32).
// The triangular solves run in 64-row blocks (diagonal block by its inverse,
// then a matrix-vector update of the rows below / above).  Refinement
// sweeps compute rho = y - S x in FP64 from the FP64 S.
#include "internal.cuh"

namespace {

constexpr int NB = 64;
constexpr int TRI64 = NB * (NB + 1) / 2;

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// S (tiled FP64, tile TS) -> dense row-major FP32 lower triangle, ld = n_pad;
// padding rows/cols get the identity
__global__ void k_lg_convert(const double* __restrict__ S, int n, int n_pad, int TS, float* __restrict__ A,
                             const int* status) {
  if (dpv_status(status)) return;
  const size_t total = (size_t)n_pad * n_pad;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n_pad), c = (int)(q % n_pad);
    A[q] = c <= r ? (float)S[dpv_s_index(r, c, TS)] : 0.f;
  }
}

__global__ void __launch_bounds__(512) k_lg_diag(int p0, int n_pad, float* __restrict__ A, float* __restrict__ invD,
                                                 float* __restrict__ Linv, int* status) {
  __shared__ float B[TRI64];
  __shared__ float inv_s[NB];
  __shared__ int bad;
  if (dpv_status(status)) return;
  const int tid = threadIdx.x;
  for (int t = tid; t < TRI64; t += blockDim.x) {
    int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (tri(i + 1, 0) <= t) ++i;
    while (tri(i, 0) > t) --i;
    const int j = t - tri(i, 0);
    B[t] = A[(size_t)(p0 + i) * n_pad + p0 + j];
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  // this thread's entries of the packed block
  int ei[5], ej[5], cnt = 0;
  for (int t = tid; t < TRI64 && cnt < 5; t += blockDim.x, ++cnt) {
    int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (tri(i + 1, 0) <= t) ++i;
    while (tri(i, 0) > t) --i;
    ei[cnt] = i;
    ej[cnt] = t - tri(i, 0);
  }
  for (int c = 0; c < NB; ++c) {
    const float d = B[tri(c, c)];
    if (!(d > 0.f)) {
      if (tid == 0) bad = 1;
      break;
    }
    const float inv = 1.0f / d;
    if (tid == 0) inv_s[c] = inv;
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (q < cnt && ej[q] > c) B[tri(ei[q], ej[q])] -= B[tri(ei[q], c)] * B[tri(ej[q], c)] * inv;
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) dpv_set_status(status, DST_NOT_SPD);
    return;
  }
  // unit factor L = B D^-1 (strict lower), D^-1
  for (int t = tid; t < TRI64; t += blockDim.x) {
    int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (tri(i + 1, 0) <= t) ++i;
    while (tri(i, 0) > t) --i;
    const int j = t - tri(i, 0);
    if (j < i) B[t] *= inv_s[j];
  }
  __syncthreads();
  for (int t = tid; t < TRI64; t += blockDim.x) {
    int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (tri(i + 1, 0) <= t) ++i;
    while (tri(i, 0) > t) --i;
    const int j = t - tri(i, 0);
    A[(size_t)(p0 + i) * n_pad + p0 + j] = B[t];
  }
  if (tid < NB) invD[p0 + tid] = inv_s[tid];
  // inverse of the unit block: thread c solves L x = e_c (column c of L^-1)
  if (tid < NB) {
    const int c = tid;
    float x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) x[i] = (i == c) ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < NB - 1; ++k)
#pragma unroll
      for (int i = k + 1; i < NB; ++i) x[i] = fmaf(-B[tri(i, k)], x[k], x[i]);
    float* out = Linv + (size_t)(p0 / NB) * NB * NB;
#pragma unroll
    for (int i = 0; i < NB; ++i) out[i * NB + c] = x[i];
  }
}

// rows below the block: P[i][c] = sum_c' A[i][p0+c'] Linv[c][c'], L[i][p0+c] = P D^-1
__global__ void __launch_bounds__(256) k_lg_panel(int p0, int n_pad, float* __restrict__ A,
                                                  const float* __restrict__ invD, const float* __restrict__ Linv,
                                                  float* __restrict__ Pg, const int* status) {
  __shared__ float Li[NB][NB + 1];
  if (dpv_status(status)) return;
  const float* lin = Linv + (size_t)(p0 / NB) * NB * NB;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) Li[t / NB][t % NB] = lin[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = p0 + NB + blockIdx.x * nw + wid; i < n_pad; i += gridDim.x * nw) {
    float* ai = A + (size_t)i * n_pad + p0;
    const float a0 = ai[lane], a1 = ai[lane + 32];
    float p0v = 0.f, p1v = 0.f;
#pragma unroll 8
    for (int cp = 0; cp < NB; ++cp) {
      const float acp = __shfl_sync(0xffffffffu, cp < 32 ? a0 : a1, cp & 31);
      p0v = fmaf(acp, Li[lane][cp], p0v);
      p1v = fmaf(acp, Li[lane + 32][cp], p1v);
    }
    Pg[(size_t)i * NB + lane] = p0v;
    Pg[(size_t)i * NB + lane + 32] = p1v;
    ai[lane] = p0v * invD[p0 + lane];
    ai[lane + 32] = p1v * invD[p0 + lane + 32];
  }
}

// trailing update: tiles (bi, bj), bi >= bj, of [p1, n_pad)^2; A_ij -= P_i L_j^T
__global__ void __launch_bounds__(256) k_lg_update(int p0, int n_pad, float* __restrict__ A,
                                                   const float* __restrict__ Pg, const int* status) {
  __shared__ float Ps[NB][NB + 4];
  __shared__ float Ls[NB][NB + 4];
  if (dpv_status(status)) return;
  const int p1 = p0 + NB;
  const int mt = (n_pad - p1) / NB;
  const int t = blockIdx.x;
  int bi = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (tri(bi + 1, 0) <= t) ++bi;
  while (tri(bi, 0) > t) --bi;
  const int bj = t - tri(bi, 0);
  if (bi >= mt) return;
  const int i0 = p1 + NB * bi, j0 = p1 + NB * bj;
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int r = q / NB, c = q % NB;
    Ps[r][c] = Pg[(size_t)(i0 + r) * NB + c];
    Ls[r][c] = A[(size_t)(j0 + r) * n_pad + p0 + c];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  float acc[4][4] = {};
#pragma unroll 8
  for (int c = 0; c < NB; ++c) {
    float pa[4], lb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) pa[a] = Ps[ty + 16 * a][c];
#pragma unroll
    for (int b = 0; b < 4; ++b) lb[b] = Ls[tx + 16 * b][c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(pa[a], lb[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i >= j) A[(size_t)i * n_pad + j] -= acc[a][b];
    }
}

// forward block: u = Linv (rhs_blk); rows below: rhs_i -= L[i][blk] u
__global__ void k_lg_fwd_diag(int p0, float* __restrict__ rhs, const float* __restrict__ Linv, const int* status) {
  __shared__ float r[NB];
  if (dpv_status(status)) return;
  const int c = threadIdx.x;
  r[c] = rhs[p0 + c];
  __syncthreads();
  const float* lin = Linv + (size_t)(p0 / NB) * NB * NB;
  float v = 0.f;
  for (int k = 0; k <= c; ++k) v = fmaf(lin[c * NB + k], r[k], v);
  rhs[p0 + c] = v;
}

__global__ void k_lg_fwd_rows(int p0, int n_pad, const float* __restrict__ A, float* __restrict__ rhs,
                              const int* status) {
  __shared__ float u[NB];
  if (dpv_status(status)) return;
  if (threadIdx.x < NB) u[threadIdx.x] = rhs[p0 + threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = p0 + NB + blockIdx.x * nw + wid; i < n_pad; i += gridDim.x * nw) {
    const float* ai = A + (size_t)i * n_pad + p0;
    float v = ai[lane] * u[lane] + ai[lane + 32] * u[lane + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) rhs[i] -= v;
  }
}

__global__ void k_lg_scale(int n_pad, float* __restrict__ rhs, const float* __restrict__ invD, const int* status) {
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n_pad) rhs[q] *= invD[q];
}

// backward block: x = Linv^T (rhs_blk); columns left: rhs_j -= sum_r L[p0+r][j] x_r
__global__ void k_lg_bwd_diag(int p0, float* __restrict__ rhs, const float* __restrict__ Linv, const int* status) {
  __shared__ float r[NB];
  if (dpv_status(status)) return;
  const int c = threadIdx.x;
  r[c] = rhs[p0 + c];
  __syncthreads();
  const float* lin = Linv + (size_t)(p0 / NB) * NB * NB;
  float v = 0.f;
  for (int k = c; k < NB; ++k) v = fmaf(lin[k * NB + c], r[k], v);
  rhs[p0 + c] = v;
}

__global__ void k_lg_bwd_cols(int p0, int n_pad, const float* __restrict__ A, float* __restrict__ rhs,
                              const int* status) {
  __shared__ float x[NB];
  if (dpv_status(status)) return;
  if (threadIdx.x < NB) x[threadIdx.x] = rhs[p0 + threadIdx.x];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p0) return;
  float v = 0.f;
#pragma unroll 8
  for (int r = 0; r < NB; ++r) v = fmaf(A[(size_t)(p0 + r) * n_pad + j], x[r], v);
  rhs[j] -= v;
}

// refinement: xacc += rhs; then rhs = y - S xacc in FP64 (one warp per row)
__global__ void k_lg_accumulate(int n_pad, const float* __restrict__ rhs, double* __restrict__ xacc, int first,
                                const int* status) {
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n_pad) xacc[q] = (first ? 0.0 : xacc[q]) + (double)rhs[q];
}

__global__ void k_lg_residual(int n, int n_pad, int TS, const double* __restrict__ S, const double* __restrict__ y,
                              const double* __restrict__ x, float* __restrict__ rhs, const int* status) {
  if (dpv_status(status)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = blockIdx.x * nw + wid; r < n_pad; r += gridDim.x * nw) {
    double acc = 0.0;
    if (r < n)
      for (int c = lane; c < n; c += 32) acc += S[c <= r ? dpv_s_index(r, c, TS) : dpv_s_index(c, r, TS)] * x[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rhs[r] = r < n ? (float)(y[r] - acc) : 0.f;
  }
}

__global__ void k_lg_init_rhs(int n, int n_pad, const double* __restrict__ y, float* __restrict__ rhs,
                              const int* status) {
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n_pad) rhs[q] = q < n ? (float)y[q] : 0.f;
}

__global__ void k_lg_output(int n, const double* __restrict__ xacc, double* __restrict__ dx, float* __restrict__ dxf,
                            const int* status) {
  if (dpv_status(status)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) {
    dx[q] = xacc[q];
    dxf[q] = (float)xacc[q];
  }
}

}  // namespace

long long dpv_large_scratch_floats(int n_pad) {
  // dense A, panel, block inverses, D^-1, rhs
  return (long long)n_pad * n_pad + (long long)n_pad * NB + (long long)(n_pad / NB) * NB * NB + 2LL * n_pad;
}

ba_status_t dpv_solve_blocked(ba_handle_t h, int refine) {
  Workspace* ws = h->ws;
  const int n = h->n, n_pad = h->n_pad, TS = h->TS;
  if (n_pad % NB) return dpv_fail(h, BA_ERR_UNSUPPORTED, "large solver needs n_pad % 64 == 0");
  float* A = ws->L.p;
  float* Pg = A + (size_t)n_pad * n_pad;
  float* Linv = Pg + (size_t)n_pad * NB;
  float* invD = Linv + (size_t)(n_pad / NB) * NB * NB;
  float* rhs = invD + n_pad;
  double* xacc = ws->r64.p;
  cudaStream_t st = h->stream;
  int* status = ws->status;
  const int sms = h->num_sms;
  k_lg_convert<<<4 * sms, 256, 0, st>>>(ws->S.p, n, n_pad, TS, A, status);
  ++h->launches;
  for (int p0 = 0; p0 < n_pad; p0 += NB) {
    k_lg_diag<<<1, 512, 0, st>>>(p0, n_pad, A, invD, Linv, status);
    ++h->launches;
    const int rows = n_pad - p0 - NB;
    if (rows > 0) {
      k_lg_panel<<<std::min((rows + 7) / 8, 4 * sms), 256, 0, st>>>(p0, n_pad, A, invD, Linv, Pg, status);
      ++h->launches;
      const int mt = rows / NB;
      k_lg_update<<<mt * (mt + 1) / 2, 256, 0, st>>>(p0, n_pad, A, Pg, status);
      ++h->launches;
    }
  }
  k_lg_init_rhs<<<(n_pad + 255) / 256, 256, 0, st>>>(n, n_pad, ws->y.p, rhs, status);
  ++h->launches;
  for (int sweep = 0; sweep <= refine; ++sweep) {
    for (int p0 = 0; p0 < n_pad; p0 += NB) {
      k_lg_fwd_diag<<<1, NB, 0, st>>>(p0, rhs, Linv, status);
      ++h->launches;
      if (p0 + NB < n_pad) {
        k_lg_fwd_rows<<<std::min((n_pad - p0 - NB + 7) / 8, 4 * sms), 256, 0, st>>>(p0, n_pad, A, rhs, status);
        ++h->launches;
      }
    }
    k_lg_scale<<<(n_pad + 255) / 256, 256, 0, st>>>(n_pad, rhs, invD, status);
    ++h->launches;
    for (int p0 = n_pad - NB; p0 >= 0; p0 -= NB) {
      k_lg_bwd_diag<<<1, NB, 0, st>>>(p0, rhs, Linv, status);
      ++h->launches;
      if (p0 > 0) {
        k_lg_bwd_cols<<<(p0 + 255) / 256, 256, 0, st>>>(p0, n_pad, A, rhs, status);
        ++h->launches;
      }
    }
    k_lg_accumulate<<<(n_pad + 255) / 256, 256, 0, st>>>(n_pad, rhs, xacc, sweep == 0, status);
    ++h->launches;
    if (sweep == refine) break;
    k_lg_residual<<<std::min((n_pad + 7) / 8, 4 * sms), 256, 0, st>>>(n, n_pad, TS, ws->S.p, ws->y.p, xacc, rhs,
                                                                        status);
    ++h->launches;
  }
  k_lg_output<<<(n + 255) / 256, 256, 0, st>>>(n, xacc, ws->dx.p, ws->tmpv.p, status);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
