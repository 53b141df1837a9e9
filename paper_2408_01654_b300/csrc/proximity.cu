// Proximity loop edges (ba_proximity_edges): Sec. 3.2 "Proximity Loop
// Closure" and "Constructing the Patch Graph".  A loop is detected from how
// close the camera comes to where an older frame was; the loop is closed with
// uni-directional edges from the stored patches of the old frame to the
// recent frame, so only the recent frame's dense features are needed.
//
// Rule, for each query frame b in [b0, b1):
//   candidates : frames a with b - a > gap;
//   selection  : the candidate whose camera centre c = -R^T t is nearest to
//                c_b (the lowest index among equal distances), if its squared
//                distance is < radius^2 (decided in FP64);
//   edges      : (ii, jj, kk) = (a, b, a*M + m) for the patches m of frame a
//                whose centre pixel, reprojected by Eq. 2 at its current
//                inverse depth, lies more than z_min in front of frame b and
//                inside [0, width) x [0, height) (FP64);
//   order      : by b, then m.
//
// Three launches, all on the handle's stream:
//   k_prox_centres  one thread per frame: c = -R^T t (FP64) into a float64x4
//                   table (32 bytes per frame, so one vector load per pair);
//   k_prox_select   one warp per query: strided scan over the candidates with
//                   a running (d^2, a) minimum per lane and a butterfly
//                   reduction; then the selected frame's patches, lane m
//                   reprojecting patch m (and m + 32, ...), a ballot per 32
//                   patches into a keep mask, the reprojected pixels into
//                   scratch, the count per query and per CTA;
//   k_prox_emit     the same warps: the CTA's output offset is the sum of the
//                   earlier CTAs' counts (read by every CTA; there are
//                   Q / 8 of them), each warp's the CTA's plus its
//                   predecessors', and each kept patch lands at its rank
//                   among the set bits of the masks.
// Nothing waits on another CTA, so the kernels have no spin-waits.
#include "internal.cuh"

#include <cmath>
#include <climits>

namespace {

constexpr int PX_WARPS = 8;             // queries per CTA
constexpr int PX_THREADS = 32 * PX_WARPS;
constexpr int PX_MAX_M = 1024;          // patches per frame

struct ProxScratch {
  double4_32a* centre;    // [N]
  int* sel;           // [Q] selected frame or -1
  int* cnt;           // [Q] kept patches
  unsigned* mask;     // [Q][MW]
  float2* uv;         // [Q][M] reprojected centre pixels
  int* block_cnt;     // [ceil(Q / PX_WARPS)]
};

__global__ void __launch_bounds__(256) k_prox_centres(int N, const double* __restrict__ poses,
                                                      double4_32a* __restrict__ centre) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= N) return;
  const double* p = poses + 7 * (size_t)a;
  double R[9];
  dpv_quat_rot64(p + 3, R);
  const double t0 = p[0], t1 = p[1], t2 = p[2];
  centre[a] = make_double4_32a(-(R[0] * t0 + R[3] * t1 + R[6] * t2), -(R[1] * t0 + R[4] * t1 + R[7] * t2),
                           -(R[2] * t0 + R[5] * t1 + R[8] * t2), 0.0);
}

struct ProxArgs {
  int N, M, MW, b0, Q, gap;
  double r2, z_min, width, height;
  double fx, fy, cx, cy;
};

// (d2, a) < (e2, b) in the order that picks the nearest, then the lowest index
__device__ __forceinline__ bool prox_before(double d2, int a, double e2, int b) {
  return d2 < e2 || (d2 == e2 && a < b);
}

__global__ void __launch_bounds__(PX_THREADS) k_prox_select(ProxArgs A, const double* __restrict__ poses,
                                                            const float* __restrict__ patches, ProxScratch S,
                                                            int* __restrict__ match) {
  __shared__ int warp_cnt[PX_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = blockIdx.x * PX_WARPS + w;
  int kept = 0;
  if (q < A.Q) {
    const int b = A.b0 + q;
    const double4_32a cb = S.centre[b];
    // nearest older centre: each lane scans a = lane, lane + 32, ... in
    // increasing order (strict < keeps its lowest index), four loads in flight
    const int na = b - A.gap;  // candidates 0 .. na-1
    double best = INFINITY;
    int ba = INT_MAX;
    int a = lane;
    for (; a + 96 < na; a += 128) {
      double4_32a c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] = S.centre[a + 32 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double dx = c[u].x - cb.x, dy = c[u].y - cb.y, dz = c[u].z - cb.z;
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < best) {
          best = d2;
          ba = a + 32 * u;
        }
      }
    }
    for (; a < na; a += 32) {
      const double4_32a c = S.centre[a];
      const double dx = c.x - cb.x, dy = c.y - cb.y, dz = c.z - cb.z;
      const double d2 = dx * dx + dy * dy + dz * dz;
      if (d2 < best) {
        best = d2;
        ba = a;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, ba, o);
      if (prox_before(ob, oa, best, ba)) {
        best = ob;
        ba = oa;
      }
    }
    const int sel = (ba != INT_MAX && best < A.r2) ? ba : -1;
    if (lane == 0) {
      S.sel[q] = sel;
      if (match) match[q] = sel;
    }
    if (sel >= 0) {
      // T_ab = T_b T_a^-1:  R = R_b R_a^T,  t = t_b - R t_a  (FP64)
      const double* pa = poses + 7 * (size_t)sel;
      const double* pb = poses + 7 * (size_t)b;
      double Ra[9], Rb[9], R[9], t[3];
      dpv_quat_rot64(pa + 3, Ra);
      dpv_quat_rot64(pb + 3, Rb);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          R[3 * r + c] = Rb[3 * r] * Ra[3 * c] + Rb[3 * r + 1] * Ra[3 * c + 1] + Rb[3 * r + 2] * Ra[3 * c + 2];
#pragma unroll
      for (int r = 0; r < 3; ++r) t[r] = pb[r] - (R[3 * r] * pa[0] + R[3 * r + 1] * pa[1] + R[3 * r + 2] * pa[2]);
      const float* pk0 = patches + (size_t)sel * A.M * 27;
      for (int r = 0; r < A.MW; ++r) {
        const int m = 32 * r + lane;
        bool keep = false;
        float2 uv = make_float2(0.f, 0.f);
        if (m < A.M) {
          const float* pk = pk0 + (size_t)m * 27;
          const double u = pk[4], v = pk[13], d = pk[22];
          // homogeneous point in frame b: R (x, y, 1) + t d
          const double xb0 = (u - A.cx) / A.fx, xb1 = (v - A.cy) / A.fy;
          const double X0 = R[0] * xb0 + R[1] * xb1 + R[2] + t[0] * d;
          const double X1 = R[3] * xb0 + R[4] * xb1 + R[5] + t[1] * d;
          const double X2 = R[6] * xb0 + R[7] * xb1 + R[8] + t[2] * d;
          if (X2 > A.z_min * d) {
            const double iz = 1.0 / X2;
            const double pu = A.fx * X0 * iz + A.cx, pv = A.fy * X1 * iz + A.cy;
            keep = pu >= 0.0 && pu < A.width && pv >= 0.0 && pv < A.height;
            uv = make_float2((float)pu, (float)pv);
          }
        }
        const unsigned bits = __ballot_sync(0xffffffffu, keep);
        if (m < A.M) S.uv[(size_t)q * A.M + m] = uv;
        if (lane == 0) S.mask[(size_t)q * A.MW + r] = bits;
        kept += __popc(bits);
      }
    } else if (lane < A.MW) {
      S.mask[(size_t)q * A.MW + lane] = 0u;
    }
    if (lane == 0) S.cnt[q] = kept;
  }
  if (lane == 0) warp_cnt[w] = kept;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
#pragma unroll
    for (int u = 0; u < PX_WARPS; ++u) s += warp_cnt[u];
    S.block_cnt[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(PX_THREADS) k_prox_emit(ProxArgs A, ProxScratch S, int* __restrict__ ii,
                                                          int* __restrict__ jj, int* __restrict__ kk,
                                                          float2* __restrict__ coords, long long cap,
                                                          int* __restrict__ count) {
  __shared__ long long part[PX_WARPS];
  __shared__ int wc[PX_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // offset of this CTA: the counts of all earlier CTAs
  long long s = 0;
  for (int c = threadIdx.x; c < (int)blockIdx.x; c += PX_THREADS) s += S.block_cnt[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[w] = s;
  const int q = blockIdx.x * PX_WARPS + w;
  if (lane == 0) wc[w] = q < A.Q ? S.cnt[q] : 0;
  __syncthreads();
  long long base = 0;
#pragma unroll
  for (int u = 0; u < PX_WARPS; ++u) base += part[u];
  long long off = base;
  for (int u = 0; u < w; ++u) off += wc[u];
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    long long total = base;
#pragma unroll
    for (int u = 0; u < PX_WARPS; ++u) total += wc[u];
    *count = total > INT_MAX ? INT_MAX : (int)total;
  }
  if (q >= A.Q || wc[w] == 0) return;
  const int a = S.sel[q], b = A.b0 + q;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < A.MW; ++r) {
    const unsigned bits = S.mask[(size_t)q * A.MW + r];
    if ((bits >> lane) & 1u) {
      const long long pos = off + __popc(bits & lt);
      const int m = 32 * r + lane;
      if (pos < cap) {
        ii[pos] = a;
        jj[pos] = b;
        kk[pos] = a * A.M + m;
        if (coords) coords[pos] = S.uv[(size_t)q * A.M + m];
      }
    }
    off += __popc(bits);
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" ba_status_t ba_proximity_edges(ba_handle_t h, int N, int M, const double* poses, const float* patches,
                                          const float* intrinsics, int b0, int b1, int gap, double radius,
                                          double width, double height, int* ii, int* jj, int* kk, float* coords,
                                          long long cap, int* match, int* count, long long* n_host) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!poses || !patches || !intrinsics || !count || (cap > 0 && (!ii || !jj || !kk)))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: null pointer");
  if (N < 1 || M < 1 || M > PX_MAX_M || (long long)N * M > INT_MAX || b0 < 0 || b1 < b0 || b1 > N || gap < 0 ||
      cap < 0 || !(radius >= 0.0) || !std::isfinite(radius) || !(width > 0.0) || !(height > 0.0))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: sizes or thresholds out of range");
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, intrinsics) != cudaSuccess) cudaGetLastError();
  if (pa.type == cudaMemoryTypeDevice)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: intrinsics must be host memory");
  if (coords && (reinterpret_cast<uintptr_t>(coords) & 7u))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: coords must be 8-byte aligned");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DPV_CUDA(h, cudaStreamIsCapturing(h->stream, &cs));
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  if (capturing && n_host)
    return dpv_fail(h, BA_ERR_STATE, "ba_proximity_edges: cannot return the count to the host during capture");
  const int Q = b1 - b0;
  if (Q == 0) {
    DPV_CUDA(h, cudaMemsetAsync(count, 0, sizeof(int), h->stream));
    if (n_host) {
      DPV_CUDA(h, cudaStreamSynchronize(h->stream));
      *n_host = 0;
    }
    return BA_OK;
  }
  const int MW = (M + 31) / 32;
  const int nblk = (Q + PX_WARPS - 1) / PX_WARPS;
  const size_t o_centre = 0;
  const size_t o_sel = align256(o_centre + sizeof(double4_32a) * (size_t)N);
  const size_t o_cnt = align256(o_sel + sizeof(int) * (size_t)Q);
  const size_t o_mask = align256(o_cnt + sizeof(int) * (size_t)Q);
  const size_t o_uv = align256(o_mask + sizeof(unsigned) * (size_t)Q * MW);
  const size_t o_blk = align256(o_uv + sizeof(float2) * (size_t)Q * M);
  const size_t bytes = align256(o_blk + sizeof(int) * (size_t)nblk);
  DBuf<unsigned char>& buf = h->ws->prox;
  if (!buf.p || (long long)bytes > buf.cap) {
    // this scratch is not referenced by any captured step, so growing it
    // leaves the handle's graphs valid
    if (capturing || h->capturing)
      return dpv_fail(h, BA_ERR_STATE, "ba_proximity_edges: scratch must grow; call once outside graph capture");
    if (buf.p) {
      DPV_CUDA(h, cudaStreamSynchronize(h->stream));
      cudaFree(buf.p);
      buf.p = nullptr;
      buf.cap = 0;
    }
    DPV_CUDA(h, cudaMalloc((void**)&buf.p, bytes));
    buf.cap = (long long)bytes;
  }
  ProxScratch S;
  S.centre = reinterpret_cast<double4_32a*>(buf.p + o_centre);
  S.sel = reinterpret_cast<int*>(buf.p + o_sel);
  S.cnt = reinterpret_cast<int*>(buf.p + o_cnt);
  S.mask = reinterpret_cast<unsigned*>(buf.p + o_mask);
  S.uv = reinterpret_cast<float2*>(buf.p + o_uv);
  S.block_cnt = reinterpret_cast<int*>(buf.p + o_blk);
  ProxArgs A;
  A.N = N;
  A.M = M;
  A.MW = MW;
  A.b0 = b0;
  A.Q = Q;
  A.gap = gap;
  A.r2 = radius * radius;
  A.z_min = h->opt.z_min;
  A.width = width;
  A.height = height;
  A.fx = intrinsics[0];
  A.fy = intrinsics[1];
  A.cx = intrinsics[2];
  A.cy = intrinsics[3];
  dpv_prof_begin(h, BA_KERNEL_PROXIMITY);
  k_prox_centres<<<(b1 + 255) / 256, 256, 0, h->stream>>>(b1, poses, S.centre);
  k_prox_select<<<nblk, PX_THREADS, 0, h->stream>>>(A, poses, patches, S, match);
  k_prox_emit<<<nblk, PX_THREADS, 0, h->stream>>>(A, S, ii, jj, kk, reinterpret_cast<float2*>(coords), cap, count);
  dpv_prof_end(h);
  h->launches += 3;
  DPV_CUDA(h, cudaGetLastError());
  if (n_host) {
    int c = 0;
    DPV_CUDA(h, cudaMemcpyAsync(&c, count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DPV_CUDA(h, cudaStreamSynchronize(h->stream));
    *n_host = c;
    if (c > cap) return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_proximity_edges: more edges than the output capacity");
  }
  return BA_OK;
}
