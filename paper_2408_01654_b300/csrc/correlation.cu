// Patch correlation (ba_patch_correlation): Sec. 3.1 "Patch correlation",
// Eq. 4.  For every edge e = (i, k, j) and patch pixel (v, u),
//   C(e, v, u, a, b) = < g_k(v, u), f_j(P'_e(v, u) + (b - R, a - R)) >,
// the dot product of the patch's correlation feature with the target frame's
// feature map bilinearly sampled on a (2R+1) x (2R+1) grid of integer offsets
// around the reprojected pixel (pixels outside the map are zero).
//
// Bilinear sampling is linear, so each output is a weighted sum of the dot
// products of g with the four surrounding map pixels ("taps"); the 7x7 grid
// of one patch pixel needs an 8x8 block of taps, and the nine pixels of a
// patch, reprojected about one map pixel apart, share most of theirs.  One
// CTA per edge:
//   1. the union box of the nine 8x8 tap blocks (typically 10x10) is staged
//      in shared memory with asynchronous 16-byte copies (zeros outside the
//      map), with the patch's nine feature vectors;
//   2. every tap of the box is dotted with all nine feature vectors at once
//      (a thread per tap, all channels: each map value loaded from shared
//      memory feeds nine FMAs, the feature values are broadcast reads);
//   3. the outputs combine four tap products with the bilinear weights.
// A patch whose box exceeds the staging capacity (a strongly foreshortened
// reprojection) is processed one patch row at a time, and a row that still
// does not fit one pixel at a time.  Edges are taken in an order grouped by
// target frame (a counting sort on the device), so that a frame's map stays
// in L2 while its edges are processed.  Everything is FP32 with FP32
// accumulation; the maps and patch features are read as given (channels last).
#include "internal.cuh"

#include <algorithm>
#include <climits>

namespace {

constexpr int CR_THREADS = 128;
constexpr int CR_MAXPIX = 9;   // p <= 3
constexpr int CR_MAXR = 4;     // radius <= 4: blocks of at most 10x10 taps
constexpr size_t CR_SMEM = 72 * 1024;  // dynamic shared memory of one CTA (three CTAs per SM)

struct CorrArgs {
  int Nf, H, W, D, P, p, E, R, cap;  // cap: taps that fit in the staging buffer
  int DS;                            // shared-memory stride of one tap (D + 4 floats)
};

__device__ __forceinline__ void cr_cp16(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}

// stage the box [by0, by0 + bh) x [bx0, bx0 + bw) of frame j, and the feature
// vectors of the pixels first .. first + npx - 1: one warp per box row (a row
// of the box is contiguous in the map), lanes over the 16-byte chunks of a
// tap; the addresses advance by a tap per step and the taps outside the map
// (a prefix and a suffix of the row) are zero-filled
__device__ void cr_stage(const CorrArgs& A, const float* __restrict__ fmap, const float* __restrict__ gmap, int j,
                         int k, int by0, int bx0, int bh, int bw, int first, int npx, float* s_f, float* s_g) {
  const int c4n = A.D / 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tlo = max(0, -bx0), thi = min(bw, A.W - bx0);  // taps inside the map: [tlo, thi)
  const unsigned s_base = (unsigned)__cvta_generic_to_shared(s_f);
  for (int r = w; r < bh; r += CR_THREADS / 32) {
    const int y = by0 + r;
    const bool row_in = y >= 0 && y < A.H;
    for (int c4 = lane; c4 < c4n; c4 += 32) {
      unsigned sa = s_base + (unsigned)(((size_t)r * bw * A.DS + 4 * c4) * sizeof(float));
      const unsigned sstep = (unsigned)(A.DS * sizeof(float));
      const float* gp = fmap + (((size_t)j * A.H + (row_in ? y : 0)) * A.W + bx0) * A.D + 4 * c4;
      for (int t = 0; t < bw; ++t, sa += sstep, gp += A.D) {
        if (row_in && t >= tlo && t < thi)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gp) : "memory");
        else
          asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};" ::"r"(sa), "f"(0.f) : "memory");
      }
    }
  }
  for (int q = w; q < npx; q += CR_THREADS / 32)
    for (int c4 = lane; c4 < c4n; c4 += 32)
      cr_cp16(s_g + (size_t)q * A.DS + 4 * c4, gmap + ((size_t)k * A.p * A.p + first + q) * A.D + 4 * c4);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
}

// s_dot[q][t] = < g(pixel q), f(tap t) > for the group's NPX pixels and the
// box's ntap taps.  A thread owns one tap and all channels: every map value
// loaded from shared memory feeds NPX FMAs, the feature values are broadcast
// reads, and the eight lanes of a shared-memory phase (eight consecutive taps,
// stride D + 4 floats) start on eight distinct bank groups.  With DT > 0 the
// channel count is a compile-time constant (unrolled loop, immediate offsets).
template <int NPX, int DT>
__device__ void cr_dots(const CorrArgs& A, int ntap, const float* s_f, const float* s_g, float* s_dot) {
  const int D = DT > 0 ? DT : A.D;
  const int DS = DT > 0 ? DT + 4 : A.DS;
  for (int t0 = 0; t0 < ntap; t0 += CR_THREADS) {
    const int t = t0 + threadIdx.x;
    const float* fp = s_f + (size_t)min(t, ntap - 1) * DS;
    float acc[NPX];
#pragma unroll
    for (int q = 0; q < NPX; ++q) acc[q] = 0.f;
#pragma unroll(DT > 0 ? 8 : 2)
    for (int c = 0; c < D; c += 4) {
      const float4 f = *reinterpret_cast<const float4*>(fp + c);
#pragma unroll
      for (int q = 0; q < NPX; ++q) {
        const float4 g = *reinterpret_cast<const float4*>(s_g + q * DS + c);
        acc[q] = fmaf(g.x, f.x, fmaf(g.y, f.y, fmaf(g.z, f.z, fmaf(g.w, f.w, acc[q]))));
      }
    }
    if (t < ntap) {
#pragma unroll
      for (int q = 0; q < NPX; ++q) s_dot[(size_t)q * A.cap + t] = acc[q];
    }
  }
  __syncthreads();
}

// outputs of the pixels first .. first + npx - 1 from the tap products: a
// thread owns one grid offset (a, b) and walks the pixels
__device__ void cr_combine(const CorrArgs& A, int e, int by0, int bx0, int bw, int first, int npx, const int* x0,
                           const int* y0, const float* ax, const float* ay, const float* s_dot,
                           float* __restrict__ out) {
  const int G = 2 * A.R + 1, G2 = G * G;
  for (int ab = threadIdx.x; ab < G2; ab += CR_THREADS) {
    const int a = ab / G, b = ab - a * G;
    float* o = out + ((size_t)e * A.p * A.p + first) * G2 + ab;
    for (int q = 0; q < npx; ++q, o += G2) {
      const int pq = first + q;
      const int ty = y0[pq] - A.R + a - by0, tx = x0[pq] - A.R + b - bx0;
      const float* d = s_dot + (size_t)q * A.cap + ty * bw + tx;
      const float wx = ax[pq], wy = ay[pq];
      *o = (1.f - wy) * ((1.f - wx) * d[0] + wx * d[1]) + wy * ((1.f - wx) * d[bw] + wx * d[bw + 1]);
    }
  }
}

// One group of the patch's pixels (first .. first + npx - 1) of edge e: the
// union box of their tap blocks is staged, dotted and combined.  Returns false
// (having done nothing) when the box exceeds the staging capacity.  Every
// thread takes the same decision (the box comes from shared values).
template <int DT>
__device__ bool cr_group(const CorrArgs& A, const float* __restrict__ fmap, const float* __restrict__ gmap, int e,
                         int j, int k, int first, int npx, const int* x0, const int* y0, const float* ax,
                         const float* ay, float* s_f, float* s_g, float* s_dot, float* __restrict__ out) {
  int xmin = INT_MAX, xmax = INT_MIN, ymin = INT_MAX, ymax = INT_MIN;
  for (int q = first; q < first + npx; ++q) {
    xmin = min(xmin, x0[q]);
    xmax = max(xmax, x0[q]);
    ymin = min(ymin, y0[q]);
    ymax = max(ymax, y0[q]);
  }
  const long long bw = (long long)xmax - xmin + 2 * A.R + 2, bh = (long long)ymax - ymin + 2 * A.R + 2;
  if (bw * bh > A.cap) return false;
  const int by0 = ymin - A.R, bx0 = xmin - A.R, ntap = (int)(bw * bh);
  cr_stage(A, fmap, gmap, j, k, by0, bx0, (int)bh, (int)bw, first, npx, s_f, s_g);
  switch (npx) {
    case 9: cr_dots<9, DT>(A, ntap, s_f, s_g, s_dot); break;
    case 4: cr_dots<4, DT>(A, ntap, s_f, s_g, s_dot); break;
    case 3: cr_dots<3, DT>(A, ntap, s_f, s_g, s_dot); break;
    case 2: cr_dots<2, DT>(A, ntap, s_f, s_g, s_dot); break;
    default: cr_dots<1, DT>(A, ntap, s_f, s_g, s_dot); break;
  }
  cr_combine(A, e, by0, bx0, (int)bw, first, npx, x0, y0, ax, ay, s_dot, out);
  __syncthreads();  // the buffers are restaged next
  return true;
}

// Edges in the order `order`; a patch whose union box does not fit is
// processed row by row of the patch, and a row that does not fit pixel by
// pixel (a (2R+2)^2 block always fits).
template <int DT>
__global__ void __launch_bounds__(CR_THREADS) k_correlation(CorrArgs A, const float* __restrict__ fmap,
                                                            const float* __restrict__ gmap,
                                                            const int* __restrict__ kk, const int* __restrict__ jj,
                                                            const float* __restrict__ coords,
                                                            const int* __restrict__ order, float* __restrict__ out,
                                                            int* __restrict__ status) {
  extern __shared__ __align__(16) float cr_smem[];
  __shared__ int s_x0[CR_MAXPIX], s_y0[CR_MAXPIX];
  __shared__ float s_ax[CR_MAXPIX], s_ay[CR_MAXPIX];
  float* s_f = cr_smem;                           // [cap][DS]
  float* s_g = s_f + (size_t)A.cap * A.DS;        // [CR_MAXPIX][DS]
  float* s_dot = s_g + (size_t)CR_MAXPIX * A.DS;  // [CR_MAXPIX][cap]
  const int np = A.p * A.p, G = 2 * A.R + 1;
  for (int idx = blockIdx.x; idx < A.E; idx += gridDim.x) {
    const int e = order[idx];
    const int k = kk[e], j = jj[e];
    if (k < 0 || k >= A.P || j < 0 || j >= A.Nf) {  // invalid edge: zeros, and the status word
      for (int o = threadIdx.x; o < np * G * G; o += CR_THREADS) out[(size_t)e * np * G * G + o] = 0.f;
      if (threadIdx.x == 0) dpv_set_status(status, DST_BAD_INDEX);
      continue;
    }
    if (threadIdx.x < np) {
      const float x = coords[((size_t)e * np + threadIdx.x) * 2], y = coords[((size_t)e * np + threadIdx.x) * 2 + 1];
      const float fx = floorf(x), fy = floorf(y);
      // coordinates far outside the map are clamped to a point whose whole
      // block is outside too (all outputs then read zeros), which also keeps
      // the integer arithmetic in range
      const float lim = 1.0e6f;
      s_x0[threadIdx.x] = (int)fminf(fmaxf(fx, -lim), lim);
      s_y0[threadIdx.x] = (int)fminf(fmaxf(fy, -lim), lim);
      s_ax[threadIdx.x] = x - fx;
      s_ay[threadIdx.x] = y - fy;
    }
    __syncthreads();
    if (!cr_group<DT>(A, fmap, gmap, e, j, k, 0, np, s_x0, s_y0, s_ax, s_ay, s_f, s_g, s_dot, out)) {
      for (int v = 0; v < A.p; ++v)
        if (!cr_group<DT>(A, fmap, gmap, e, j, k, v * A.p, A.p, s_x0, s_y0, s_ax, s_ay, s_f, s_g, s_dot, out))
          for (int q = v * A.p; q < (v + 1) * A.p; ++q)
            cr_group<DT>(A, fmap, gmap, e, j, k, q, 1, s_x0, s_y0, s_ax, s_ay, s_f, s_g, s_dot, out);
    }
  }
}

// Order of the edges by target frame (a counting sort): hist[b] counts the
// edges of frame b (b = Nf collects invalid frames), then every CTA scans the
// histogram in shared memory and places its edges at their bucket's start
// plus a slot taken with an atomic (the order inside a bucket does not
// matter: the edges are independent).
__global__ void k_corr_hist(int E, int Nf, const int* __restrict__ jj, int* __restrict__ hist) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int j = jj[e];
    atomicAdd(hist + ((j >= 0 && j < Nf) ? j : Nf), 1);
  }
}

__global__ void __launch_bounds__(1024) k_corr_order(int E, int Nf, const int* __restrict__ jj,
                                                     const int* __restrict__ hist, int* __restrict__ cursor,
                                                     int* __restrict__ order) {
  extern __shared__ int s_start[];  // [Nf + 1]
  __shared__ int s_carry, s_w[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 <= Nf; c0 += blockDim.x) {  // chunked exclusive scan
    const int b = c0 + threadIdx.x;
    const int v = b <= Nf ? hist[b] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = lane < nw ? s_w[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_w[lane] = t;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? s_w[w - 1] : 0) + s_carry;
    if (b <= Nf) s_start[b] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = incl;
    __syncthreads();
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int j = jj[e];
    const int bkt = (j >= 0 && j < Nf) ? j : Nf;
    order[s_start[bkt] + atomicAdd(cursor + bkt, 1)] = e;
  }
}

}  // namespace

extern "C" ba_status_t ba_patch_correlation(ba_handle_t h, int Nf, int H, int W, int D, int P, int p, int E,
                                            const float* fmap, const float* gmap, const int* kk, const int* jj,
                                            const float* coords, int radius, float* out) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (E < 0 || Nf < 1 || H < 1 || W < 1 || P < 1 || p < 1 || p > 3 || radius < 0 || radius > CR_MAXR || D < 32 ||
      D % 32 != 0)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_patch_correlation: sizes out of range");
  if (E == 0) return BA_OK;
  if (!fmap || !gmap || !kk || !jj || !coords || !out)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_patch_correlation: null pointer");
  if ((reinterpret_cast<uintptr_t>(fmap) | reinterpret_cast<uintptr_t>(gmap)) & 15u)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_patch_correlation: feature arrays must be 16-byte aligned");
  CorrArgs A;
  A.Nf = Nf;
  A.H = H;
  A.W = W;
  A.D = D;
  A.P = P;
  A.p = p;
  A.E = E;
  A.R = radius;
  A.DS = D + 4;
  // staging capacity: taps that fit beside the feature vectors and the products
  const size_t per_tap = sizeof(float) * ((size_t)A.DS + CR_MAXPIX);
  const long long cap = (long long)((CR_SMEM - sizeof(float) * (size_t)CR_MAXPIX * A.DS) / per_tap);
  const int bs = 2 * radius + 2;
  if (cap < (long long)bs * bs)
    return dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_patch_correlation: feature dimension too large for the staging buffer");
  A.cap = (int)cap;
  const size_t order_smem = sizeof(int) * (size_t)(Nf + 1);
  if (order_smem > 200 * 1024)
    return dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_patch_correlation: too many frames for the edge ordering");
  // scratch for the target-frame order: histogram, cursors (Nf + 1 each), order [E]
  Workspace* ws = h->ws;
  const long long need = 2LL * (Nf + 1) + E;
  if (!ws->corr.p || ws->corr.cap < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DPV_CUDA(h, cudaStreamIsCapturing(h->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone || h->capturing)
      return dpv_fail(h, BA_ERR_STATE, "ba_patch_correlation: scratch must grow; call once outside graph capture");
    if (ws->corr.p) {
      DPV_CUDA(h, cudaStreamSynchronize(h->stream));
      cudaFree(ws->corr.p);
      ws->corr.p = nullptr;
      ws->corr.cap = 0;
    }
    DPV_CUDA(h, cudaMalloc((void**)&ws->corr.p, sizeof(int) * (size_t)need));
    ws->corr.cap = need;
  }
  int* hist = ws->corr.p;
  int* cursor = hist + (Nf + 1);
  int* order = cursor + (Nf + 1);
  // specialised channel counts, else generic
  void (*kern)(CorrArgs, const float*, const float*, const int*, const int*, const float*, const int*, float*,
               int*) =
      D == 128 ? k_correlation<128> : D == 64 ? k_correlation<64> : D == 256 ? k_correlation<256> : k_correlation<0>;
  static bool smem_set[4] = {false, false, false, false};
  const int ki = D == 128 ? 0 : D == 64 ? 1 : D == 256 ? 2 : 3;
  if (!smem_set[ki]) {
    DPV_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CR_SMEM));
    smem_set[ki] = true;
  }
  if (order_smem > 48 * 1024) {
    static bool order_set = false;
    if (!order_set) {
      DPV_CUDA(h, cudaFuncSetAttribute(k_corr_order, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      order_set = true;
    }
  }
  const size_t smem = sizeof(float) * ((size_t)A.cap * A.DS + (size_t)CR_MAXPIX * A.DS + (size_t)CR_MAXPIX * A.cap);
  const int grid = (int)std::min<long long>(E, 64LL * h->num_sms);
  const int ogrid = (int)std::min<long long>((E + 1023) / 1024, 2LL * h->num_sms);
  dpv_prof_begin(h, BA_KERNEL_CORRELATION);
  DPV_CUDA(h, cudaMemsetAsync(hist, 0, sizeof(int) * 2 * (size_t)(Nf + 1), h->stream));
  k_corr_hist<<<ogrid, 1024, 0, h->stream>>>(E, Nf, jj, hist);
  k_corr_order<<<ogrid, 1024, order_smem, h->stream>>>(E, Nf, jj, hist, cursor, order);
  kern<<<grid, CR_THREADS, smem, h->stream>>>(A, fmap, gmap, kk, jj, coords, order, out, h->ws->status);
  dpv_prof_end(h);
  h->launches += 3;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
