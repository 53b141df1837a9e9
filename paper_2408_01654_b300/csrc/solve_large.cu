// Solve of the reduced pose system for n > DPV_SMALL_N (the global
// loop-closure BA: the dense Cholesky of the pose block of the Schur
// complement, which the appendix "Bundle-Adjustment Efficiency" names as the
// memory and runtime bottleneck of global optimisation).
//
// S (FP64, tiled lower triangle, 64 x 64 tiles) is equilibrated (s_i S_ij s_j,
// s = diag(S)^-1/2: the factorisation error then scales with the condition
// number of the equilibrated matrix), rounded to an FP32 copy in the same
// tiled layout and factored as S' = L D L^T by ONE persistent kernel
// that runs a task graph over the tiles:
//   DIAG(k)        factor tile (k,k): unit L_kk, D_k, and the inverse L_kk^-1
//   PANEL(i,k)     L_ik = A_ik L_kk^-T D_k^-1                      (i > k)
//                  and G_ik = L_ik D_k^1/2, stored pre-split for the tensor
//                  cores (TF32 part + FP32 rest, core-matrix layout)
//   UPDATE(i,j,k)  A_ij -= G_ik G_jk^T                             (k < j <= i)
//                  (workers: 2 x 2 tiles at a time, one 128 x 128 x 64
//                  tcgen05 TF32 product with a three-pass split whose
//                  operands arrive by bulk copies)
// Each tile carries a version (the number of updates applied, +1 once it is
// final).  The chain DIAG(k) -> PANEL(k+1,k) -> UPDATE(k+1,k+1,k) -> DIAG(k+1)
// is the critical path, so one CTA, alone on its SM, runs it step after step
// without handing tiles over; the other CTAs take the remaining panels and
// updates from a list in dependency order (lookahead one column) and wait,
// with a bounded spin, only for the versions their task reads.  Every CTA is
// resident (cooperative launch) and each wait is on work that is earlier in
// the critical chain or in the list, so the schedule cannot deadlock.
//
// A second persistent kernel runs conjugate gradients preconditioned by the
// factor: in the triangular solves block row i of the forward solve waits for
// the rows above it (each solved value is published with its pass number in
// one 64-bit word), the backward solve for the rows below; grid barriers
// separate the phases; the products with S run in double-float, until the
// estimated error left in x is below 1e-7 of it (1e-10 with BA_MIXED).
#include "internal.cuh"
#include "tcgen05.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

namespace {

constexpr int NB = 64;  // tile edge, equal to the assembly's tile for n > DPV_SMALL_N
constexpr int TILE = NB * NB;
constexpr int LDX = NB + 1;  // padded row of the tile being factored (column reads by row threads: conflict free)
constexpr int LDS = NB + 4;  // padded row of the product operands: 16-byte rows, and 128-bit accesses of a
                             // quarter warp to 8 consecutive rows hit distinct banks (68 = 4 mod 32)
constexpr int LDC = NB + 1;  // padded row of the solve's staging buffers
constexpr int LG_THREADS = 256;
constexpr int TASK_PANEL = 1, TASK_UPDATE = 2;  // worker task types (the diagonal steps are not listed)
constexpr int LG_MAX_T = 1023;  // tiles per dimension (10-bit task fields)

static_assert(NB == DPV_TILE, "the large solver works on the assembly's tiles");
static_assert(LG_THREADS == 256, "thread layouts of the tile tasks assume 256 threads");

__host__ __device__ inline int tri2(int r) { return r * (r + 1) / 2; }
__host__ __device__ inline unsigned pack_task(int type, int k, int i, int j) {
  return ((unsigned)type << 30) | ((unsigned)k << 20) | ((unsigned)i << 10) | (unsigned)j;
}

// ---------------------------------------------------------------------------
// synchronisation primitives (thread 0 of a CTA; bounded)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *p >= want.  Gives up when another CTA reported an error or when
// `timeout` cycles have passed (then reports DST_TIMEOUT).  Returns success.
__device__ bool wait_geq(const int* p, int want, int* status, long long timeout) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    if (ld_acquire(p) >= want) return true;
    if ((it & 63u) == 63u) {
      if (dpv_status(status)) return false;
      if (clock64() - t0 > timeout) {
        dpv_set_status(status, DST_TIMEOUT);
        return false;
      }
    }
    __nanosleep(64);
  }
}

// Grid-wide barrier of a cooperative launch: count / generation in bar[0..1].
__device__ bool grid_barrier(int* bar, int nblocks, int* status, long long timeout) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const int gen = ld_acquire(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1) == nblocks - 1) {
      bar[0] = 0;
      __threadfence();
      st_release(bar + 1, gen + 1);
    } else {
      ok = wait_geq(bar + 1, gen + 1, status, timeout) ? 1 : 0;
    }
  }
  __syncthreads();
  return ok != 0;
}

// A solved value published with its pass number in one 64-bit word, so that
// a consumer polling the word receives the value with the signal (no
// separate flag, no fence: the word is written and read whole).
__device__ __forceinline__ void st_tagged(unsigned long long* p, unsigned tag, float v) {
  const unsigned long long w = ((unsigned long long)tag << 32) | __float_as_uint(v);
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
// Wait until *p carries `tag`, then return its value in v.  Gives up when
// another CTA reported an error or after `timeout` cycles (DST_TIMEOUT).
__device__ bool wait_tagged(const unsigned long long* p, unsigned tag, float& v, int* status, long long timeout) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    if ((unsigned)(w >> 32) == tag) {
      v = __uint_as_float((unsigned)w);
      return true;
    }
    if ((it & 63u) == 63u) {
      if (dpv_status(status)) return false;
      if (clock64() - t0 > timeout) {
        dpv_set_status(status, DST_TIMEOUT);
        return false;
      }
    }
    if (it > 32) __nanosleep(32);
  }
}

// Two consecutive words p[0], p[1] (see wait_tagged).
__device__ bool wait_tagged2(const unsigned long long* p, unsigned tag, float& v0, float& v1, int* status,
                             long long timeout) {
  const long long t0 = clock64();
  bool h0 = false, h1 = false;
  for (unsigned it = 0;; ++it) {
    unsigned long long w;
    if (!h0) {
      asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
      if ((unsigned)(w >> 32) == tag) {
        v0 = __uint_as_float((unsigned)w);
        h0 = true;
      }
    }
    if (!h1) {
      asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p + 1) : "memory");
      if ((unsigned)(w >> 32) == tag) {
        v1 = __uint_as_float((unsigned)w);
        h1 = true;
      }
    }
    if (h0 && h1) return true;
    if ((it & 63u) == 63u) {
      if (dpv_status(status)) return false;
      if (clock64() - t0 > timeout) {
        dpv_set_status(status, DST_TIMEOUT);
        return false;
      }
    }
    if (it > 32) __nanosleep(32);
  }
}

__device__ __forceinline__ float* tile_ptr(float* A, int i, int j) { return A + (size_t)(tri2(i) + j) * TILE; }

// tile (64 x 64, row-major in global memory, read through L2) -> padded
// shared; all four loads of a thread are issued before the stores
template <int LD>
__device__ __forceinline__ void load_tile(float* dst, const float* src, bool lower_only) {
  constexpr int PER = TILE / 4 / LG_THREADS;
  float4 v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) v[u] = __ldcg(reinterpret_cast<const float4*>(src) + threadIdx.x + u * LG_THREADS);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int q = threadIdx.x + u * LG_THREADS;
    const int r = (4 * q) / NB, c = (4 * q) % NB;
    float* d = dst + r * LD + c;
    if (LD % 4 == 0 && !lower_only) {
      *reinterpret_cast<float4*>(d) = v[u];
    } else {
      d[0] = (!lower_only || c <= r) ? v[u].x : 0.f;
      d[1] = (!lower_only || c + 1 <= r) ? v[u].y : 0.f;
      d[2] = (!lower_only || c + 2 <= r) ? v[u].z : 0.f;
      d[3] = (!lower_only || c + 3 <= r) ? v[u].w : 0.f;
    }
  }
}

// two tiles, eight loads in flight per thread
template <int LD>
__device__ __forceinline__ void load_tiles2(float* d0, const float* s0, float* d1, const float* s1) {
  constexpr int PER = TILE / 4 / LG_THREADS;
  float4 v[2 * PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    v[u] = __ldcg(reinterpret_cast<const float4*>(s0) + threadIdx.x + u * LG_THREADS);
    v[PER + u] = __ldcg(reinterpret_cast<const float4*>(s1) + threadIdx.x + u * LG_THREADS);
  }
#pragma unroll
  for (int u = 0; u < 2 * PER; ++u) {
    const int q = threadIdx.x + (u % PER) * LG_THREADS;
    const int r = (4 * q) / NB, c = (4 * q) % NB;
    float* d = (u < PER ? d0 : d1) + r * LD + c;
    if (LD % 4 == 0) {
      *reinterpret_cast<float4*>(d) = v[u];
    } else {
      d[0] = v[u].x;
      d[1] = v[u].y;
      d[2] = v[u].z;
      d[3] = v[u].w;
    }
  }
}

// acc[a][e] += sum_c X[8w + a][c] Y[l + 32e][c] w[c] for warp w, lane l (X, Y
// with LDS-padded rows, w 16-byte aligned or null): the rows of X are read
// as warp-wide broadcasts, those of Y by quarter warps from distinct banks,
// four values of c per 128-bit load, summed in ascending c.
// LOWER_Y: Y is lower triangular (Y[s][c] = 0 for c > s), so the rows s < 32
// take no products for c >= 32 (exact zeros: the sums are unchanged).
template <bool LOWER_Y>
__device__ __forceinline__ void gemm_rows8(const float* X, const float* Y, const float* w, float acc[8][2]) {
  const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
  const float* xr = X + 8 * wr * LDS;
  const float* y0 = Y + lane * LDS;
  const float* y1 = Y + (lane + 32) * LDS;
#pragma unroll 2
  for (int c = 0; c < (LOWER_Y ? NB / 2 : NB); c += 4) {
    float4 b0 = *reinterpret_cast<const float4*>(y0 + c), b1 = *reinterpret_cast<const float4*>(y1 + c);
    if (w) {
      const float4 wc = *reinterpret_cast<const float4*>(w + c);
      b0.x *= wc.x;
      b0.y *= wc.y;
      b0.z *= wc.z;
      b0.w *= wc.w;
      b1.x *= wc.x;
      b1.y *= wc.y;
      b1.z *= wc.z;
      b1.w *= wc.w;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const float4 x = *reinterpret_cast<const float4*>(xr + a * LDS + c);
      float t0 = fmaf(x.x, b0.x, acc[a][0]), t1 = fmaf(x.x, b1.x, acc[a][1]);
      t0 = fmaf(x.y, b0.y, t0);
      t1 = fmaf(x.y, b1.y, t1);
      t0 = fmaf(x.z, b0.z, t0);
      t1 = fmaf(x.z, b1.z, t1);
      acc[a][0] = fmaf(x.w, b0.w, t0);
      acc[a][1] = fmaf(x.w, b1.w, t1);
    }
  }
  if (LOWER_Y) {  // (w is null here)
#pragma unroll 2
    for (int c = NB / 2; c < NB; c += 4) {
      const float4 b1 = *reinterpret_cast<const float4*>(y1 + c);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const float4 x = *reinterpret_cast<const float4*>(xr + a * LDS + c);
        float t1 = fmaf(x.x, b1.x, acc[a][1]);
        t1 = fmaf(x.y, b1.y, t1);
        t1 = fmaf(x.z, b1.z, t1);
        acc[a][1] = fmaf(x.w, b1.w, t1);
      }
    }
  }
}

// G_ik = L_ik diag(sq) (L_ik in shared memory, padded rows) split into its
// TF32 part and the FP32 rest, each written as one 16 KB operand in the
// K-major core-matrix layout of the tensor cores: 16-byte slot q holds row
// 8 (q >> 7) + (q & 7), columns 4 ((q >> 3) & 15) .. +3.  Coalesced stores.
__device__ __forceinline__ void store_g(const float* Ls, const float* sq, float* g, unsigned char* shi = nullptr,
                                        unsigned char* slo = nullptr) {
#pragma unroll
  for (int u = 0; u < TILE / 4 / LG_THREADS; ++u) {
    const int q = threadIdx.x + u * LG_THREADS;
    const int row = ((q >> 7) << 3) | (q & 7), k0 = ((q >> 3) & 15) << 2;
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) tc_split(Ls[row * LDS + k0 + e] * sq[k0 + e], h[e], l[e]);
    const float4 hv = make_float4(h[0], h[1], h[2], h[3]), lv = make_float4(l[0], l[1], l[2], l[3]);
    reinterpret_cast<float4*>(g)[q] = hv;
    reinterpret_cast<float4*>(g + TILE)[q] = lv;
    if (shi) {  // the same operand for this CTA's own tensor cores
      reinterpret_cast<float4*>(shi)[q] = hv;
      reinterpret_cast<float4*>(slo)[q] = lv;
    }
  }
  tc_fence_global();  // the bulk copies that read G run in the async proxy
}
__device__ __forceinline__ float* g_ptr(float* G, int i, int k) { return G + (size_t)(tri2(i) + k) * 2 * TILE; }

// ---------------------------------------------------------------------------
// the tasks
// ---------------------------------------------------------------------------
struct LgShared {
  float X[NB * LDX];                  // the diagonal tile being factored
  __align__(16) float Y[NB * LDS];    // product operands
  __align__(16) float Z[NB * LDS];
  __align__(16) float ucol[LG_THREADS / 32][32];  // column broadcast of the diagonal factorisation
  float invd[NB];
  float dd[NB];
  __align__(16) float dprev[NB];  // the previous diagonal step's D and D^-1 (critical-path CTA)
  float iprev[NB];
  float sq[NB];     // D_k^1/2 of the panel being written
  int task;
  int bad;
  int pf;  // critical CTA: bit 0 / 1 = tile (k, k-1) / (k, k) of the next step already fetched
};

// LDL^T of the 64 x 64 diagonal tile in sm.X (lower part) by warps 0-3: row
// r = tid % 64 in registers, split by column parity between two threads
// (tid / 64 = the parity, uniform per warp), so that each column's update of
// the entries right of it is shared evenly.  Column c is broadcast through
// shared memory by the threads owning it (double-buffered by the parity of
// c, so one 128-thread named barrier per column suffices: a buffer is
// rewritten two columns later, after every thread passed the barrier in
// between); every thread takes its row's multiplier from the broadcast.
// Writes the unit factor (strict lower) back to sm.X, D and D^-1 to sm.dd /
// sm.invd.  Returns false on a non-positive pivot.
__device__ __noinline__ bool factor64(LgShared& sm) {
  const int r = threadIdx.x & (NB - 1), h = threadIdx.x >> 6;  // threadIdx.x < 128
  float* Xs = sm.X;
  float(*buf)[NB] = reinterpret_cast<float(*)[NB]>(&sm.ucol[0][0]);
  float a[NB / 2];  // a[j]: column 2j + h
#pragma unroll
  for (int j = 0; j < NB / 2; ++j) a[j] = 2 * j + h <= r ? Xs[r * LDX + 2 * j + h] : 0.f;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    float* u = buf[c & 1];
    if (h == (c & 1)) u[r] = a[c >> 1];
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const float d = u[c];
    ok = ok && (d > 0.f);
    float inv;  // approximate reciprocal: the refinement absorbs its last-bit error
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(d));
    const float l = u[r] * inv;
#pragma unroll
    for (int j = c >> 1; j < NB / 2; ++j)  // this thread's columns 2j + h right of c
      if (2 * j > c || (2 * j == c && h == 1)) a[j] = fmaf(-l, u[2 * j + h], a[j]);
    if (h == (c & 1) && r > c) a[c >> 1] = l;
    if (r == c && h == 0) {
      sm.invd[c] = inv;
      sm.dd[c] = d;
    }
  }
#pragma unroll
  for (int j = 0; j < NB / 2; ++j)
    if (2 * j + h < r) Xs[r * LDX + 2 * j + h] = a[j];
  return ok;
}

// Inverse of the unit lower factor in sm.X by 32-row blocks,
//   [L00 0; L10 L11]^-1 = [L00^-1 0; -L11^-1 (L10 L00^-1) L11^-1],
// into sm.Y (padded) and li (global, row-major), by warps 0-3 (a 128-thread
// named barrier, so that warps 4-7 stay free): warps 0 and 1 invert the
// diagonal blocks (lane = column, forward substitution), then the four warps
// form the off-diagonal block through sm.Z (scratch).
__device__ void inverse64(LgShared& sm, float* li) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;  // tid < 128
  if (wid < 2) {
    const int b = 32 * wid;
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < 31; ++k)
#pragma unroll
      for (int i = k + 1; i < 32; ++i) x[i] = fmaf(-sm.X[(b + i) * LDX + b + k], x[k], x[i]);
#pragma unroll
    for (int i = 0; i < 32; ++i) sm.Y[(b + i) * LDS + b + lane] = x[i];
  } else {
    for (int t = tid - 64; t < 32 * 32; t += 64) sm.Y[(t >> 5) * LDS + 32 + (t & 31)] = 0.f;
  }
  asm volatile("bar.sync 3, 128;" ::: "memory");
  // thread: row i, columns j0 + 4e (e < 8) of the 32 x 32 products
  const int i = tid >> 2, j0 = tid & 3;
  {
    // W = L10 L00^-1 (L00^-1 lower: only k >= j contributes; its upper part is 0)
    float w[8] = {};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float x = sm.X[(32 + i) * LDX + k];
#pragma unroll
      for (int e = 0; e < 8; ++e) w[e] = fmaf(x, sm.Y[k * LDS + j0 + 4 * e], w[e]);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) sm.Z[i * LDS + j0 + 4 * e] = w[e];
  }
  asm volatile("bar.sync 3, 128;" ::: "memory");
  {
    // M10 = -L11^-1 W (L11^-1 lower: k <= i)
    float v[8] = {};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float y = k <= i ? sm.Y[(32 + i) * LDS + 32 + k] : 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = fmaf(y, sm.Z[k * LDS + j0 + 4 * e], v[e]);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) sm.Y[(32 + i) * LDS + j0 + 4 * e] = -v[e];
  }
  asm volatile("bar.sync 3, 128;" ::: "memory");
  for (int t = tid; t < TILE; t += 2 * NB) li[t] = sm.Y[(t >> 6) * LDS + (t & 63)];
}

// DIAG(k): the 64 x 64 diagonal tile (in sm.X, lower part) factored by
// factor64 and inverted by inverse64; the unit factor goes to tile (k, k),
// its inverse to Linv (and stays in sm.Y), D and D^-1 to global and to
// sm.dprev / sm.iprev for the next step.
// The critical CTA's buffers for the tiles of its next step, fetched ahead
struct DiagPre {
  float* pa;  // tile (k, k-1), padded rows
  float* pb;  // tile (k, k)
};

// tile (64 x 64, row-major, through L2) -> padded shared, by threads 128..255
__device__ __forceinline__ void load_tile128(float* dst, const float* src) {
  const int t = threadIdx.x - 2 * NB;
  float4 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = __ldcg(reinterpret_cast<const float4*>(src) + t + u * 2 * NB);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = t + u * 2 * NB;
    const int r = (4 * q) / NB, c = (4 * q) % NB;
    *reinterpret_cast<float4*>(dst + r * LDS + c) = v[u];
  }
}
__device__ bool factor_diag(LgShared& sm, const DiagPre& pre, float* A, float* Linv, float* D, float* invD, int k,
                            int T, int* ver, const int* env, int* status, long long timeout) {
  const int tid = threadIdx.x;
  float* tk = tile_ptr(A, k, k);
  if (tid == 0) sm.bad = 0;
  __syncthreads();
  if (tid < 2 * NB) {  // warps 0-3: the factor and its inverse
    const bool ok = factor64(sm);
    if (!ok && tid == 0) sm.bad = 1;
    asm volatile("bar.sync 3, 128;" ::: "memory");
    asm volatile("bar.arrive 4, 256;" ::: "memory");  // (the factor is complete: warps 4-7 store it)
    if (!sm.bad) {
      inverse64(sm, Linv + (size_t)k * TILE);
      if (tid < NB) {
        sm.dprev[tid] = sm.dd[tid];
        sm.iprev[tid] = sm.invd[tid];
      }
    }
    // tile (k, k) final once warps 4-7 have stored the factor too: released
    // here, ahead of the next step's tiles
    asm volatile("bar.sync 6, 256;" ::: "memory");
    if (tid == 0 && !sm.bad) {
      __threadfence();
      st_release(ver + tri2(k) + k, k + 1);
    }
  } else {
    // meanwhile warps 4-7 store the factor (tile (k, k), D, D^-1) once it is
    // complete, then fetch the next step's tiles (k+1, k) and (k+1, k+1)
    // once the workers' updates through step k-1 are complete (those depend
    // only on work published before this step's factorisation)
    asm volatile("bar.sync 4, 256;" ::: "memory");
    if (!sm.bad) {
      for (int t = tid - 2 * NB; t < TILE; t += 2 * NB) {
        const int r = t >> 6, c = t & 63;
        tk[t] = c < r ? sm.X[r * LDX + c] : (c == r ? 1.f : 0.f);
      }
      if (tid < 3 * NB) {
        D[k * NB + tid - 2 * NB] = sm.dd[tid - 2 * NB];
        invD[k * NB + tid - 2 * NB] = sm.invd[tid - 2 * NB];
      }
    }
    asm volatile("bar.arrive 6, 256;" ::: "memory");  // (the stores of the factor are issued)
    if (tid == 2 * NB) {
      int f = 0;
      if (k + 1 < T) {
        bool ok = true;
        if (__ldg(env + k + 1) <= k) {
          ok = wait_geq(ver + tri2(k + 1) + k, k, status, timeout);
          if (ok) f |= 1;
        }
        if (ok && wait_geq(ver + tri2(k + 1) + k + 1, k, status, timeout)) f |= 2;
      }
      sm.pf = f;
    }
    asm volatile("bar.sync 2, 128;" ::: "memory");
    const int f = sm.pf;
    if (f & 1) load_tile128(pre.pa, tile_ptr(A, k + 1, k));
    if (f & 2) load_tile128(pre.pb, tile_ptr(A, k + 1, k + 1));
  }
  __syncthreads();
  return !sm.bad;
}

constexpr uint32_t TC_OP_BYTES = TILE * 4;  // one split part of one tile (16 KB)
constexpr int TC_SMEM = 8 * TC_OP_BYTES;    // A hi, A lo, B hi, B lo: 128 rows (two tiles) each
constexpr uint32_t TC_COLS = 128;           // tensor-memory columns per CTA (128 output columns)

struct TcState {
  uint64_t bar_ld;    // the operand copies
  uint64_t bar_mma;   // the MMAs
  uint32_t tmem;
  uint32_t ph_ld, ph_mma;
  int bad;            // 1: the copies, 2: the MMAs did not complete in time
};

// Byte offset of the tensor-core region in the factorisation kernel's
// dynamic shared memory (after the CUDA-core tasks' LgShared).
constexpr size_t TC_OFF = (sizeof(LgShared) + 1023) / 1024 * 1024;

// Critical-path step k (one dedicated CTA, in order): for k > 0 first the
// panel of tile (k, k-1), L = A_{k,k-1} L_{k-1}^-T D_{k-1}^-1 (from the
// inverse and D of step k-1 kept in shared memory), with its operand G for
// the workers' updates, then the update of tile (k, k) by it, A_kk - L D L^T
// (both on the CUDA cores: one 64 x 64 x 64 product each, no operand split);
// then the factorisation of tile (k, k).  The two tiles the step reads were
// usually fetched during the previous step's elimination (pre.pa / pre.pb
// below, flags in sm.pf); otherwise they are waited for and loaded here.
__device__ bool task_diag_step(LgShared& sm, const DiagPre& pre, float* A, float* G, float* Linv, float* D,
                               float* invD, int k, int T, int* ver, const int* env, int* status, long long timeout) {
  const int tid = threadIdx.x;
  const int pf = sm.pf;  // (written before the previous step's last barrier)
  if (k > 0 && __ldg(env + k) < k) {  // (otherwise tile (k, k-1) lies outside the envelope: no panel, no update)
    float* tp = tile_ptr(A, k, k - 1);
    if (!(pf & 1)) {
      if (tid == 0) sm.bad = wait_geq(ver + tri2(k) + k - 1, k - 1, status, timeout) ? 0 : 1;
      __syncthreads();
      if (sm.bad) return false;
      load_tile<LDS>(pre.pa, tp, false);
    }
    __syncthreads();
    const int lane = tid & 31, r0 = 8 * (tid >> 5);  // (the layout of gemm_rows8)
    {
      float acc[8][2] = {};
      gemm_rows8<true>(pre.pa, sm.Y, nullptr, acc);  // A_{k,k-1} L_{k-1}^-T
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int rr = r0 + a, c = lane + 32 * e;
          const float l = acc[a][e] * sm.iprev[c];
          sm.Z[rr * LDS + c] = l;
          tp[rr * NB + c] = l;
        }
    }
    if (tid < NB) sm.sq[tid] = sqrtf(sm.dprev[tid]);
    __syncthreads();
    store_g(sm.Z, sm.sq, g_ptr(G, k, k - 1));
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(ver + tri2(k) + k - 1, k);  // tile (k, k-1) final
      sm.bad = (pf & 2) || wait_geq(ver + tri2(k) + k, k - 1, status, timeout) ? 0 : 1;
    }
    __syncthreads();
    if (sm.bad) return false;
    if (!(pf & 2)) {
      load_tile<LDS>(pre.pb, tile_ptr(A, k, k), false);
      __syncthreads();
    }
    // A_kk - L D L^T, lower part
    float acc[8][2] = {};
    gemm_rows8<false>(sm.Z, sm.Z, sm.dprev, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int rr = r0 + a, c = lane + 32 * e;
        sm.X[rr * LDX + c] = c <= rr ? pre.pb[rr * LDS + c] - acc[a][e] : 0.f;
      }
  } else {
    load_tile<LDX>(sm.X, tile_ptr(A, k, k), true);
  }
  __syncthreads();
  return factor_diag(sm, pre, A, Linv, D, invD, k, T, ver, env, status, timeout);
}

// PANEL(i,k): L_ik = A_ik L_kk^-T D_k^-1, and the operand G_ik = L_ik D_k^1/2
__device__ void task_panel(LgShared& sm, float* A, float* G, const float* Linv, const float* D, const float* invD,
                           int i, int k) {
  float* t = tile_ptr(A, i, k);
  if (threadIdx.x < NB) {
    sm.invd[threadIdx.x] = __ldcg(invD + k * NB + threadIdx.x);
    sm.sq[threadIdx.x] = sqrtf(__ldcg(D + k * NB + threadIdx.x));
  }
  load_tiles2<LDS>(sm.Z, t, sm.Y, Linv + (size_t)k * TILE);
  __syncthreads();
  float acc[8][2] = {};
  gemm_rows8<true>(sm.Z, sm.Y, nullptr, acc);
  const int lane = threadIdx.x & 31, r0 = 8 * (threadIdx.x >> 5);
  __syncthreads();  // every thread is done reading sm.Z
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int r = r0 + a, c = lane + 32 * e;
      const float l = acc[a][e] * sm.invd[c];
      t[r * NB + c] = l;
      sm.Z[r * LDS + c] = l;
    }
  __syncthreads();
  store_g(sm.Z, sm.sq, g_ptr(G, i, k));
}


// UPDATE of a 2 x 2 block of tiles on the tensor cores: rows i, i+1 and
// columns j, j+1 at step k (each tile only when it lies in the lower triangle
// of a T x T tile grid),
//   A_ab -= G_ak G_bk^T  for a in {i, i+1}, b in {j, j+1},
// as one 128 x 128 x 64 tcgen05 TF32 product with the three-pass split
// (hi*hi + hi*lo + lo*hi, about FP32 accuracy) accumulated in tensor memory.
// The operands, written pre-split by the panels, arrive by bulk copies into
// shared memory while the threads fetch the tiles being updated; one thread
// issues the 24 MMAs.  Operand rows of a missing tile, or of a row whose
// tile in column k lies outside the envelope, hold stale data whose products
// are not read.
__device__ __forceinline__ bool quad_tile(int T, int a, int b) { return a < T && b < T && b <= a; }

__device__ bool task_update_tc(unsigned char* tcbuf, TcState& ts, float* A, const float* G, const int* env,
                               const int* ver, int T, int i, int j, int k, int* status, long long timeout) {
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  unsigned char* a_hi = tcbuf;
  unsigned char* a_lo = a_hi + 2 * TC_OP_BYTES;
  unsigned char* b_hi = a_lo + 2 * TC_OP_BYTES;
  unsigned char* b_lo = b_hi + 2 * TC_OP_BYTES;
  // this thread's 64 outputs: row r of the 128 (tile row i + r / 64), the 64
  // columns of tile column j + wid / 4, read first (only a tile that receives
  // this step: both of its operand rows inside the envelope; the tiles'
  // versions were waited for before the task)
  const int r = 32 * (wid & 3) + lane, cb = wid >> 2;
  const int ta = i + (r >> 6), tb = j + cb, rr = r & 63;
  const bool mine = quad_tile(T, ta, tb) && max(__ldg(env + ta), __ldg(env + tb)) <= k;
  float* ct = tile_ptr(A, mine ? ta : i, mine ? tb : j) + rr * NB;
  float4 cv[16];
#pragma unroll
  for (int q = 0; q < 16; ++q)
    cv[q] = mine ? __ldcg(reinterpret_cast<const float4*>(ct) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    // the operand rows i, i+1 (A) and j, j+1 (B) whose G_ak is nonzero
    // (inside the envelope; the others are not copied), each copied as soon
    // as its panel is final, so that a task waiting for the critical chain's
    // panel has everything else in flight already
    unsigned pending = 0;  // bit q: row (q < 2 ? i : j) + (q & 1)
    uint32_t bytes = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a = (q < 2 ? i : j) + (q & 1);
      if (a < T && __ldg(env + a) <= k) {
        pending |= 1u << q;
        bytes += 2 * TC_OP_BYTES;
      }
    }
    tc_fence_smem();  // this CTA's earlier generic accesses of the buffer are ordered before the copies
    tc_mbar_expect_tx(&ts.bar_ld, bytes);
    const long long t0 = clock64();
    for (unsigned it = 0; pending; ++it) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = (q < 2 ? i : j) + (q & 1);
        if ((pending & (1u << q)) && ld_acquire(ver + tri2(a) + k) >= k + 1) {
          tc_fence_global();  // G was written by other CTAs through the generic proxy
          const float* g = g_ptr(const_cast<float*>(G), a, k);
          unsigned char* d = (q < 2 ? a_hi : b_hi) + (q & 1) * TC_OP_BYTES;
          tc_bulk_g2s(d, g, TC_OP_BYTES, &ts.bar_ld);                            // TF32 part
          tc_bulk_g2s(d + 2 * TC_OP_BYTES, g + TILE, TC_OP_BYTES, &ts.bar_ld);  // FP32 rest
          pending &= ~(1u << q);
        }
      }
      if (!pending) break;
      if ((it & 63u) == 63u && (dpv_status(status) || clock64() - t0 > timeout)) {
        dpv_set_status(status, DST_TIMEOUT);
        ts.bad = 1;  // (the copies issued so far are waited for, bounded, on the way out)
        break;
      }
      __nanosleep(64);
    }
  }
  if (tid == 0 && !ts.bad) {
    if (!tc_mbar_wait(&ts.bar_ld, ts.ph_ld, tc_hw_bound(timeout))) {
      ts.bad = 1;
    } else {
      ts.ph_ld ^= 1u;
      tc_fence_after_sync();
      constexpr uint32_t idesc = tc_idesc_tf32(128, 2 * NB);
      constexpr uint32_t LBO = 128, SBO = (NB / 4) * 128;
      const uint32_t ah0 = tc_smem_addr(a_hi), al0 = tc_smem_addr(a_lo), bh0 = tc_smem_addr(b_hi),
                     bl0 = tc_smem_addr(b_lo);
#pragma unroll
      for (int st = 0; st < NB / 8; ++st) {
        const uint32_t off = st * 256;  // K = 8 TF32 values = two core matrices along K
        const uint64_t ah = tc_desc(ah0 + off, LBO, SBO), al = tc_desc(al0 + off, LBO, SBO);
        const uint64_t bh = tc_desc(bh0 + off, LBO, SBO), bl = tc_desc(bl0 + off, LBO, SBO);
        tc_mma_tf32(ts.tmem, ah, bh, idesc, st > 0);
        tc_mma_tf32(ts.tmem, ah, bl, idesc, 1);
        tc_mma_tf32(ts.tmem, al, bh, idesc, 1);
      }
      tc_commit(&ts.bar_mma);
      if (tc_mbar_wait(&ts.bar_mma, ts.ph_mma, tc_hw_bound(timeout)))
        ts.ph_mma ^= 1u;
      else
        ts.bad = 2;
    }
  }
  __syncthreads();
  if (ts.bad) return false;
  tc_fence_after_sync();
  // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows), columns 64 (w / 4) .. + 63
  const uint32_t taddr = ts.tmem + ((uint32_t)(32 * (wid & 3)) << 16) + (uint32_t)(64 * cb);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float d[32];
    tc_ld32(taddr + 32 * h, d);
    if (mine) {
      const bool diag = ta == tb;  // a diagonal tile keeps only its lower part
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 c = cv[8 * h + q];
        c.x -= d[4 * q];
        c.y -= d[4 * q + 1];
        c.z -= d[4 * q + 2];
        c.w -= d[4 * q + 3];
        float* t = ct + 32 * h + 4 * q;
        if (!diag) {
          *reinterpret_cast<float4*>(t) = c;
        } else {
          const int cc = 32 * h + 4 * q;
          if (cc <= rr) t[0] = c.x;
          if (cc + 1 <= rr) t[1] = c.y;
          if (cc + 2 <= rr) t[2] = c.z;
          if (cc + 3 <= rr) t[3] = c.w;
        }
      }
    }
  }
  tc_fence_before_sync();
  return true;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// One large pose system as the kernels see it (device copy per launch).
struct LgProb {
  float *A, *Linv, *D, *invD, *rhs, *xf, *xb, *sc;  // factor scratch
  float* G;                                        // pre-split update operands [tri(T)][2][64 x 64]
  float2* Sdf;                                     // S as (hi, lo) float pairs, tiled like S
  double *r, *p0, *p1, *u;                         // conjugate gradients: residual, directions, S v
  unsigned long long *tf, *tb;                     // solved rows, tagged: (pass << 32) | value bits
  const double* S;                                 // FP64 tiled lower triangle
  const double* y;                                 // right-hand side
  double *xacc, *dx;                               // refinement accumulator, output
  float* dxf;                                      // FP32 copy of the output
  int* ver;                                        // tile versions [tri(T)]
  int* env;                                        // [T] first tile column of each tile row of S that holds
                                                   // a nonzero (the row envelope; the factor's fill stays in it)
  int* eoff;                                       // [T+1] tiles of the envelope before each tile row
  int T, n, n_pad, rb0;                            // tiles, unknowns, padded size, first global row block
};

// equilibration scale s = diag(S)^-1/2 (1 on the padding); blockIdx.y = system
__global__ void k_lg_scale(const LgProb* __restrict__ probs, const int* status) {
  if (dpv_status(status)) return;
  const LgProb P = probs[blockIdx.y];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.n_pad) return;
  const float d = dpv_d2f_bits(P.S[dpv_s_index(r, r, NB)]);
  P.sc[r] = (r < P.n && d > 0.f) ? rsqrtf(d) : 1.f;
  if (r % NB == 0) P.env[r / NB] = r / NB;  // lowered by k_lg_convert
  P.rhs[r] = r < P.n ? dpv_d2f_bits(P.y[r]) * P.sc[r] : 0.f;
  P.u[r] = 0.0;  // the refinement's product accumulates into u
  P.tf[r] = 0ull;  // no row solved yet in this solve
  P.tb[r] = 0ull;
}

// S (FP64 tiles) -> A (FP32 tiles, identical layout), equilibrated:
// A_ij = s_i S_ij s_j.  CTAs stride over the tiles; blockIdx.y = system.
__global__ void k_lg_convert(const LgProb* __restrict__ probs, const int* status) {
  if (dpv_status(status)) return;
  const LgProb P = probs[blockIdx.y];
  for (int t = blockIdx.x; t < tri2(P.T); t += gridDim.x) {
    int ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (tri2(ti + 1) <= t) ++ti;
    while (tri2(ti) > t) --ti;
    const int tj = t - tri2(ti);
    const double2* src = reinterpret_cast<const double2*>(P.S + (size_t)t * TILE);
    float2* dst = reinterpret_cast<float2*>(P.A + (size_t)t * TILE);
    float4* ddf = reinterpret_cast<float4*>(P.Sdf + (size_t)t * TILE);
    int nz = 0;
    for (int q = threadIdx.x; q < TILE / 2; q += blockDim.x) {
      const int r = (2 * q) / NB, c = (2 * q) % NB;
      const double2 v = src[q];
      nz |= (v.x != 0.0) | (v.y != 0.0);
      const float si = P.sc[ti * NB + r];
      const float2 a = dpv_d2df_bits(v.x), b = dpv_d2df_bits(v.y);
      dst[q] = make_float2(a.x * si * P.sc[tj * NB + c], b.x * si * P.sc[tj * NB + c + 1]);
      ddf[q] = make_float4(a.x, a.y, b.x, b.y);
    }
    // the row envelope: the first tile column holding a nonzero
    if (__syncthreads_or(nz) && threadIdx.x == 0 && tj < ti) atomicMin(P.env + ti, tj);
  }
}

// Whether a factorisation task touches the envelope: PANEL(i,k) when tile
// (i,k) lies in it, an update of rows i, i+1 and columns j, j+1 at step k
// when one of its tiles (a,b) receives that step (both G_ak and G_bk nonzero:
// env_a <= k and env_b <= k).  Outside the envelope L is zero, so a task that
// touches nothing there would only subtract exact zeros.
__device__ __forceinline__ bool task_live(const LgProb* __restrict__ probs, unsigned long long w64) {
  const LgProb& P = probs[(int)(w64 >> 32)];
  const unsigned w = (unsigned)w64;
  const int type = (int)(w >> 30), k = (int)((w >> 20) & 1023u), i = (int)((w >> 10) & 1023u),
            j = (int)(w & 1023u);
  if (type == TASK_PANEL) return __ldg(P.env + i) <= k;
  for (int a = i; a < i + 2 && a < P.T; ++a) {
    if (__ldg(P.env + a) > k) continue;
    for (int b = j; b < j + 2 && b <= a; ++b)
      if (__ldg(P.env + b) <= k) return true;
  }
  return false;
}

constexpr int ENV_THREADS = 256;
constexpr int ENV_MAX_CTAS = 1024;  // CTAs of the envelope's bookkeeping (their counts live in the sync words)

// The envelope's bookkeeping, in two launches over env_ctas CTAs (after
// k_lg_convert has found each tile row's first nonzero tile).  First:
// per system the envelope's tile offsets (the products with S visit only
// its tiles; one warp per system) and the initial tile versions (a tile
// (a,b) of the envelope receives the updates of steps max(env_a, env_b) ..
// b-1 and starts at the first of them; one warp per tile row), and per CTA
// the number of tasks of its share of the dense list that touch the
// envelope (a contiguous share, in list order).
__global__ void __launch_bounds__(ENV_THREADS) k_lg_envelope(const LgProb* __restrict__ probs, int nsys,
                                                             const int* __restrict__ rb_sys, int R,
                                                             const unsigned long long* __restrict__ tasks, int ntasks,
                                                             int* __restrict__ counts, const int* status) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = ENV_THREADS / 32;
  if (dpv_status(status)) return;
  const int gw = blockIdx.x * NW + wid, nw = gridDim.x * NW;  // this warp among all
  for (int p = gw; p < nsys; p += nw) {  // offsets: one warp per system
    const LgProb& P = probs[p];
    int base = 0;
    for (int a0 = 0; a0 < P.T; a0 += 32) {
      const int a = a0 + lane;
      int v = a < P.T ? a - P.env[a] + 1 : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (a < P.T) P.eoff[a + 1] = base + v;
      base += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) P.eoff[0] = 0;
  }
  for (int r = gw; r < R; r += nw) {  // versions: one warp per tile row
    const LgProb& P = probs[rb_sys[r]];
    const int a = r - P.rb0, ea = P.env[a];
    for (int b = ea + lane; b <= a; b += 32) P.ver[tri2(a) + b] = max(ea, P.env[b]);
  }
  const int per = (ntasks + gridDim.x - 1) / gridDim.x;
  const int t0 = min(ntasks, (int)blockIdx.x * per), t1 = min(ntasks, t0 + per);
  int cnt = 0;
  for (int t = t0 + tid; t < t1; t += ENV_THREADS) cnt += task_live(probs, tasks[t]) ? 1 : 0;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  __shared__ int wsum[NW];
  if (lane == 0) wsum[wid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int c = 0;
    for (int w = 0; w < NW; ++w) c += wsum[w];
    counts[blockIdx.x] = c;
  }
}

// Second: each CTA writes the live tasks of its share, in list order, after
// those of the CTAs before it; the last writes the count to live[ntasks].
__global__ void __launch_bounds__(ENV_THREADS) k_lg_compact(const LgProb* __restrict__ probs,
                                                            const unsigned long long* __restrict__ tasks, int ntasks,
                                                            const int* __restrict__ counts,
                                                            unsigned long long* __restrict__ live, const int* status) {
  __shared__ int wsum[ENV_THREADS / 32 + 1];
  __shared__ int base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = ENV_THREADS / 32;
  if (dpv_status(status)) {
    if (blockIdx.x == 0 && tid == 0) live[ntasks] = 0ull;
    return;
  }
  if (tid == 0) {
    int b = 0;
    for (int c = 0; c < (int)blockIdx.x; ++c) b += counts[c];
    base = b;
  }
  __syncthreads();
  const int per = (ntasks + gridDim.x - 1) / gridDim.x;
  const int t0 = min(ntasks, (int)blockIdx.x * per), t1 = min(ntasks, t0 + per);
  for (int r0 = t0; r0 < t1; r0 += ENV_THREADS) {
    const int t = r0 + tid;
    unsigned long long w = 0ull;
    const bool lv = t < t1 && task_live(probs, w = tasks[t]);
    const unsigned m = __ballot_sync(0xffffffffu, lv);
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();
    int before = base;
    for (int q = 0; q < wid; ++q) before += wsum[q];
    if (lv) live[before + __popc(m & ((1u << lane) - 1u))] = w;
    __syncthreads();
    if (tid == 0) {
      int c = 0;
      for (int q = 0; q < NW; ++q) c += wsum[q];
      base += c;
    }
    __syncthreads();
  }
  if (blockIdx.x == gridDim.x - 1 && tid == 0) live[ntasks] = (unsigned long long)base;
}

// The factorisation task graphs of all large systems.  CTA p < nsys runs the
// critical chain of system p (other CTAs on its SM leave when there are SMs
// to spare), then joins the workers; workers take the panels and the
// tensor-core updates of all systems from one list (task: system << 32 |
// type << 30 | k << 20 | i << 10 | j; an update covers rows i, i+1 and
// columns j, j+1).
// Every CTA that stays holds TC_COLS tensor-memory columns, released on every
// way out once its MMAs have completed.
__global__ void __launch_bounds__(LG_THREADS, 1) k_lg_factor(const LgProb* __restrict__ probs, int nsys,
                                                          const unsigned long long* __restrict__ tasks, int cap,
                                                          int* ctr, int* dsm, int isolate, int* status,
                                                          long long timeout) {
  const int ntasks = (int)tasks[cap];  // the live tasks (k_lg_envelope)
  extern __shared__ __align__(1024) float lg_smem[];
  LgShared& sm = *reinterpret_cast<LgShared*>(lg_smem);          // the CUDA-core tasks
  unsigned char* tcbuf = reinterpret_cast<unsigned char*>(lg_smem) + TC_OFF;  // the tensor-core operands
  __shared__ TcState ts;
  __shared__ int role, task, bad;
  if (threadIdx.x == 0) {
    unsigned smid;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    role = 1;
    if ((int)blockIdx.x < nsys) {
      st_release(dsm + blockIdx.x, (int)smid + 1);
    } else if (isolate) {
      for (int c = 0; c < nsys && role > 0; ++c)
        if (!wait_geq(dsm + c, 1, status, timeout) || ld_acquire(dsm + c) == (int)smid + 1) role = -1;
    }
  }
  __syncthreads();
  if (role < 0) return;
  if (threadIdx.x < 32) tc_alloc(&ts.tmem, TC_COLS);
  if (threadIdx.x == 0) {
    tc_mbar_init(&ts.bar_ld, 1);
    tc_mbar_init(&ts.bar_mma, 1);
    ts.ph_ld = ts.ph_mma = 0;
    ts.bad = 0;
  }
  tc_fence_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if ((int)blockIdx.x < nsys) {
    const LgProb& P = probs[blockIdx.x];
    // (the tensor-core operand buffers hold the prefetched tiles on this CTA)
    const DiagPre pre{reinterpret_cast<float*>(tcbuf), reinterpret_cast<float*>(tcbuf) + NB * LDS};
    if (threadIdx.x == 0) sm.pf = 0;
    __syncthreads();
    for (int k = 0; k < P.T; ++k) {
      if (dpv_status(status)) goto done;
      if (!task_diag_step(sm, pre, P.A, P.G, P.Linv, P.D, P.invD, k, P.T, P.ver, P.env, status, timeout)) {
        if (threadIdx.x == 0 && !dpv_status(status)) dpv_set_status(status, DST_NOT_SPD);
        goto done;
      }
      // (tile (k, k) was released inside the step)
    }
  }
  // Each CTA claims its next task while it works on the current one (the
  // claim is an L2 round trip); the versions a task reads are polled by one
  // lane each, and the versions it publishes are released by one lane each.
  // A claimed task waits only for tasks earlier in the list, and the earliest
  // unfinished task is always some CTA's current one, so claiming ahead
  // cannot deadlock.
  if (threadIdx.x == 0) task = dpv_status(status) ? ntasks : atomicAdd(ctr, 1);
  __syncthreads();
  for (;;) {
    tc_fence_smem();  // this thread's generic shared accesses before any later bulk copy into the buffer
    const int t = task;
    __syncthreads();
    if (t >= ntasks) break;
    const unsigned long long w64 = tasks[t];
    const LgProb& P = probs[(int)(w64 >> 32)];
    const unsigned w = (unsigned)w64;
    const int type = (int)(w >> 30), k = (int)((w >> 20) & 1023u), i = (int)((w >> 10) & 1023u),
              j = (int)(w & 1023u);
    int* ver = P.ver;
    const int T = P.T;
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      // lane q waits for the q-th version this task reads: a panel the
      // diagonal tile of column k (final) and its own tile (updated through
      // step k-1); an update its target tiles (updated through step k-1; the
      // panels of its operand rows are waited for inside the task)
      const int* vp = nullptr;
      int want = 0;
      if (type == TASK_PANEL) {
        if (lane == 0) { vp = ver + tri2(k) + k; want = k + 1; }
        if (lane == 1) { vp = ver + tri2(i) + k; want = k; }
      } else if (lane >= 4 && lane < 8) {  // the target tiles (i + (lane >> 1 & 1), j + (lane & 1)) that receive step k
        const int a = i + ((lane >> 1) & 1), b = j + (lane & 1);
        if (quad_tile(T, a, b) && max(__ldg(P.env + a), __ldg(P.env + b)) <= k) { vp = ver + tri2(a) + b; want = k; }
      }
      const bool ok = vp ? wait_geq(vp, want, status, timeout) : true;
      const bool all_ok = __all_sync(0xffffffffu, ok);
      if (lane == 0) {
        bad = all_ok ? 0 : 1;
        // claim the next task now; it is read after this one completes
        task = (!all_ok || dpv_status(status)) ? ntasks : atomicAdd(ctr, 1);
      }
    }
    __syncthreads();
    if (bad) break;
    if (type == TASK_PANEL) {
      task_panel(sm, P.A, P.G, P.Linv, P.D, P.invD, i, k);
    } else if (!task_update_tc(tcbuf, ts, P.A, P.G, P.env, ver, T, i, j, k, status, timeout)) {
      if (threadIdx.x == 0) dpv_set_status(status, DST_TIMEOUT);
      break;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      const int q = threadIdx.x;
      if (type == TASK_PANEL) {
        if (q == 0) {
          __threadfence();
          st_release(ver + tri2(i) + k, k + 1);
        }
      } else {
        const int a = i + (q >> 1), b = j + (q & 1);
        if (quad_tile(T, a, b) && max(__ldg(P.env + a), __ldg(P.env + b)) <= k) {
          __threadfence();
          st_release(ver + tri2(a) + b, k + 1);
        }
      }
    }
  }
done:
  // shared and tensor memory go back once no copy and no MMA of this CTA is in
  // flight: after a timeout, wait (bounded) for the outstanding phase first
  __syncthreads();
  if (threadIdx.x == 0 && ts.bad) tc_mbar_wait(ts.bad == 1 ? &ts.bar_ld : &ts.bar_mma, ts.bad == 1 ? ts.ph_ld : ts.ph_mma,
                                          tc_hw_bound(timeout));
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (threadIdx.x < 32) tc_dealloc(ts.tmem, TC_COLS);
}

// this thread's 4 x 4 block (rows 4 rg.., columns 4 cg..) of a 64 x 64 tile
struct TileRegs {
  float4 m[4];
};
__device__ __forceinline__ TileRegs load_block(const float* M) {
  const int cg = threadIdx.x & 15, rg = threadIdx.x >> 4;
  TileRegs t;
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) t.m[rr] = __ldcg(reinterpret_cast<const float4*>(M + (4 * rg + rr) * NB + 4 * cg));
  return t;
}

// out[r] = sum_c M[r][c] v[c] (trans = false) or out[c] = sum_r M[r][c] v[r]
// (trans = true) for a tile held as per-thread blocks; v, out in shared memory
__device__ void tile_gemv(const TileRegs& t, const float* v, float* out, bool trans, float (*part)[NB + 1]) {
  const int tid = threadIdx.x, cg = tid & 15, rg = tid >> 4;
  if (!trans) {
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
      part[cg][4 * rg + rr] =
          t.m[rr].x * v[4 * cg] + t.m[rr].y * v[4 * cg + 1] + t.m[rr].z * v[4 * cg + 2] + t.m[rr].w * v[4 * cg + 3];
  } else {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const float vr = v[4 * rg + rr];
      s0 = fmaf(t.m[rr].x, vr, s0);
      s1 = fmaf(t.m[rr].y, vr, s1);
      s2 = fmaf(t.m[rr].z, vr, s2);
      s3 = fmaf(t.m[rr].w, vr, s3);
    }
    part[rg][4 * cg] = s0;
    part[rg][4 * cg + 1] = s1;
    part[rg][4 * cg + 2] = s2;
    part[rg][4 * cg + 3] = s3;
  }
  __syncthreads();
  if (tid < NB) {
    float acc = 0.f;
#pragma unroll
    for (int g = 0; g < 16; ++g) acc += part[g][tid];
    out[tid] = acc;
  }
  __syncthreads();
}

// The chains' one product on the critical path, u_i -= M u_{i-1} (and its
// backward counterpart), without a block barrier: M is staged in shared
// memory (row-major, unpadded), warp w takes rows 8w .. 8w+7 and lane l the
// columns 2l, 2l+1, and the lanes read the published vector words
// themselves.
__device__ __forceinline__ void stage_chain(float* dst, const float* M) {
#pragma unroll
  for (int u = 0; u < TILE / 4 / LG_THREADS; ++u)
    reinterpret_cast<float4*>(dst)[threadIdx.x + u * LG_THREADS] =
        __ldcg(reinterpret_cast<const float4*>(M) + threadIdx.x + u * LG_THREADS);
}
// sum_c M[8w + (lane >> 2)][c] x[c] for x[2l] = x0, x[2l+1] = x1 of lane l:
// the eight row partials of each lane are reduced across the warp by halving
// exchanges (lane bits 4, 3, 2 pick the row, bits 1, 0 finish the sum)
__device__ __forceinline__ float chain_product(const float* Ms, float x0, float x1) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float2* M2 = reinterpret_cast<const float2*>(Ms) + (8 * w) * (NB / 2) + lane;
  float s[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const float2 m = M2[r * (NB / 2)];
    s[r] = fmaf(m.x, x0, m.y * x1);
  }
  float t4[4];
  {
    const bool up = lane & 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float send = up ? s[q] : s[q + 4], keep = up ? s[q + 4] : s[q];
      t4[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  float t2[2];
  {
    const bool up = lane & 8;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float send = up ? t4[q] : t4[q + 2], keep = up ? t4[q + 2] : t4[q];
      t2[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  const bool up = lane & 4;
  float t1 = (up ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, up ? t2[0] : t2[1], 4);
  t1 += __shfl_xor_sync(0xffffffffu, t1, 2);
  t1 += __shfl_xor_sync(0xffffffffu, t1, 1);
  return t1;
}
// M = X Y (trans = false) or (X Y)^T, 64 x 64 row-major tiles in global
// memory, staged through gx, gy (padded rows)
__device__ void chain_matrix(const float* X, const float* Y, float* out, bool trans, float* gx, float* gy) {
  load_tiles2<LDC>(gx, X, gy, Y);
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < NB; ++k) {
    float xa[4], yb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xa[a] = gx[(ty + 16 * a) * LDC + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) yb[b] = gy[k * LDC + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], yb[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = ty + 16 * a, c = tx + 16 * b;
      out[trans ? c * NB + r : r * NB + c] = acc[a][b];
    }
  __syncthreads();
}

// The same product for k_lg_chainmat with 128-bit shared loads: X staged
// transposed (xt[k][r]) and Y as is, both with row stride LDS; thread (ty, tx)
// of a 16 x 16 grid owns the 4 x 4 block at rows 4ty, columns 4tx, so one
// k-step is two float4 loads and 16 FMAs, and the block leaves as four float4
// stores (rows, or for the transpose columns, of the output).
__device__ void chain_matrix4(const float* X, const float* Y, float* out, bool trans, float* xt, float* ys) {
  constexpr int PER = TILE / 4 / LG_THREADS;
  float4 vx[PER], vy[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    vx[u] = __ldcg(reinterpret_cast<const float4*>(X) + threadIdx.x + u * LG_THREADS);
    vy[u] = __ldcg(reinterpret_cast<const float4*>(Y) + threadIdx.x + u * LG_THREADS);
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int q = threadIdx.x + u * LG_THREADS;
    const int r = (4 * q) / NB, c = (4 * q) % NB;
    xt[(c + 0) * LDS + r] = vx[u].x;
    xt[(c + 1) * LDS + r] = vx[u].y;
    xt[(c + 2) * LDS + r] = vx[u].z;
    xt[(c + 3) * LDS + r] = vx[u].w;
    *reinterpret_cast<float4*>(ys + r * LDS + c) = vy[u];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < NB; ++k) {
    const float4 xa = *reinterpret_cast<const float4*>(xt + k * LDS + 4 * ty);
    const float4 yb = *reinterpret_cast<const float4*>(ys + k * LDS + 4 * tx);
    const float xv[4] = {xa.x, xa.y, xa.z, xa.w}, yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xv[a], yv[b], acc[a][b]);
  }
  const int r0 = 4 * ty, c0 = 4 * tx;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (trans)  // column c0 + e of the product is row c0 + e of the output
      *reinterpret_cast<float4*>(out + (c0 + e) * NB + r0) = make_float4(acc[0][e], acc[1][e], acc[2][e], acc[3][e]);
    else
      *reinterpret_cast<float4*>(out + (r0 + e) * NB + c0) = make_float4(acc[e][0], acc[e][1], acc[e][2], acc[e][3]);
  }
  __syncthreads();
}

// --- double-float (FP32 pair) arithmetic of the refinement's products -------
struct DFp {
  float h, l;
};
// a += (xh + xl)(yh + yl) to about 2^-44 of the product (xl * yl dropped);
// a is renormalised by the caller (df_norm) after a few terms
__device__ __forceinline__ void df_acc_prod(DFp& a, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float s = a.h + p;
  const float bb = s - a.h;
  a.l += ((a.h - (s - bb)) + (p - bb)) + e;
  a.h = s;
}
__device__ __forceinline__ void df_norm(DFp& a) {
  const float s = a.h + a.l;
  a.l = a.l - (s - a.h);
  a.h = s;
}
__device__ __forceinline__ void df_add2(DFp& a, const DFp& b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  a.l += ((a.h - (s - bb)) + (b.h - bb)) + b.l;
  a.h = s;
  df_norm(a);
}
__device__ __forceinline__ DFp df_shfl_xor(const DFp& a, int o) {
  return DFp{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}
__device__ __forceinline__ void red_df(double* p, const DFp& a) {  // *p += hi + lo, exactly converted
  dpv_red_add(p, dpv_f2d_bits(a.h));
  dpv_red_add(p, dpv_f2d_bits(a.l));
}

// One 64 x 64 tile of the symmetric product u = S v in double-float: rows of
// tile (ti, tj) get S_t v_tj, its columns (off the diagonal) S_t^T v_ti; a
// diagonal tile holds the lower triangle (loaded into registers by
// load_symv_tile).  vr, vc: v of the tile's rows and columns (DF pairs,
// shared memory).  Thread (ty, tx) takes the 4 x 4 block
// at rows 4 ty, columns 4 tx; row sums reduce over tx by shuffles, column sums
// over ty through `part`.  Adds the tile's share of v^T S v to sig (the
// thread's own accumulator).
struct SymvRegs {
  float4 m[4][2];
};
__device__ __forceinline__ void load_symv_tile(const float2* __restrict__ St, SymvRegs& g) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float4* rowp = reinterpret_cast<const float4*>(St + (4 * ty + a) * NB + 4 * tx);
    g.m[a][0] = __ldcs(rowp);
    g.m[a][1] = __ldcs(rowp + 1);
  }
}
__device__ void tile_symv(const SymvRegs& g, const DFp* vr, const DFp* vc, bool diag, double* ur, double* uc,
                          DFp (*part)[NB], DFp& sig) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float4(&m)[4][2] = g.m;
  DFp R[4], C[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) R[q] = C[q] = DFp{0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = 4 * ty + a;
    const float sh[4] = {m[a][0].x, m[a][0].z, m[a][1].x, m[a][1].z};
    const float sl[4] = {m[a][0].y, m[a][0].w, m[a][1].y, m[a][1].w};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = 4 * tx + b;
      if (!diag || c <= r) df_acc_prod(R[a], sh[b], sl[b], vc[c].h, vc[c].l);
      if (!diag || c < r) df_acc_prod(C[b], sh[b], sl[b], vr[r].h, vr[r].l);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    df_norm(R[q]);
    df_norm(C[q]);
  }
  // rows: sum over the 16 tx of the half warp
#pragma unroll
  for (int o = 1; o < 16; o <<= 1)
#pragma unroll
    for (int a = 0; a < 4; ++a) df_add2(R[a], df_shfl_xor(R[a], o));
  if (tx == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * ty + a;
      red_df(ur + r, R[a]);
      df_acc_prod(sig, R[a].h, R[a].l, vr[r].h, vr[r].l);
    }
  }
  // columns: sum over the 16 ty
#pragma unroll
  for (int b = 0; b < 4; ++b) part[ty][4 * tx + b] = C[b];
  __syncthreads();
  if (tid < NB) {
    DFp cs = part[0][tid];
#pragma unroll
    for (int k = 1; k < 16; ++k) df_add2(cs, part[k][tid]);
    red_df((diag ? ur : uc) + tid, cs);
    df_acc_prod(sig, cs.h, cs.l, vc[tid].h, vc[tid].l);
  }
  df_norm(sig);
  __syncthreads();
}

// System p finished after iteration s >= 1: the estimated error left in its
// x is below tol of it (the last step bounds the previous iterate's error;
// the current one's is about rho c_s with rho ~ c_s / c_{s-1}).  A finished
// system takes no further part, so its later maxima stay 0 and it stays
// finished.  The maxima of a completed iteration are final (grid barrier), so
// every CTA reaches the same decision.
// The t-th tile of the envelope in row-major order: its tile row ti and
// column tj, and its index in the tiled lower triangle.
__device__ __forceinline__ int env_tile(const LgProb& P, int t, int& ti, int& tj) {
  int lo = 0, hi = P.T - 1;  // the last row whose envelope starts at or before t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(P.eoff + mid) <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  ti = lo;
  tj = __ldg(P.env + lo) + (t - __ldg(P.eoff + lo));
  return tri2(ti) + tj;
}

__device__ __forceinline__ bool sys_finished(const int* conv, int nsys, int p, int s, float tol) {
  if (s < 1) return false;
  const float cm = __int_as_float(__ldcg(conv + 2 * (s * nsys + p)));
  const float xm = __int_as_float(__ldcg(conv + 2 * (s * nsys + p) + 1));
  const float cp = __int_as_float(__ldcg(conv + 2 * ((s - 1) * nsys + p)));
  return cm <= tol * xm || cm * cm <= tol * xm * cp;
}

// Triangular solves and preconditioned conjugate gradients of all large
// systems.  The FP32 factor M = L D L^T of the equilibrated S' = D_s S D_s
// preconditions CG on S' z = D_s y (x = D_s z):
//   iteration 0:  z = M^-1 y',  r = y' - S' z
//   iteration k:  w = M^-1 r,  rho = r.w,  p = w + (rho / rho_prev) p,
//                 q = S' p,  alpha = rho / p.q,  z += alpha p,  r -= alpha q
// The products with S run in double-float over S_df (FP64-level accuracy
// at FP32 throughput), tile by tile with coalesced reads; r, p, x are FP64.
// rb_sys[r] is the system of global row block r (block i = r - rb0);
// rb_sys[R + q] and rb_sys[2R + q] list the row blocks in forward and
// backward chain order (by i, and by T - 1 - i), and CTA c takes entries
// q = c, c + grid, ... of each; forward rows wait for the rows above them in
// their system, the backward rows for the rows below; grid barriers separate
// the phases.  The iterations stop once every system's estimated error left
// in x is below tol of it (dpv_solve_tol).
__global__ void __launch_bounds__(LG_THREADS, 2) k_lg_solve(const LgProb* __restrict__ probs, int nsys,
                                                            const int* __restrict__ rb_sys, int R, int s0, int s1,
                                                            int sweeps, int ext, int* bar, int* conv, double* red,
                                                            float tol,
                                                            int* status, long long timeout) {
  __shared__ float acc[NB], vj[NB], prod[NB];
  __shared__ float part[16][NB + 1];
  __shared__ DFp dpart[16][NB];
  __shared__ DFp vr[NB], vc[NB];
  __shared__ float wfin[NB];
  __shared__ __align__(16) float gx[NB * LDC];  // (float4 stores, float2 loads: 16-byte aligned)
  __shared__ __align__(16) float gy[NB * LDC];
  __shared__ int ok;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) ok = 1;
  __syncthreads();
  if (dpv_status(status)) return;
  if (ext && s0 > 0) {  // a sweep after every system converged: nothing to do (the same in every CTA)
    bool done = true;
    for (int p = 0; p < nsys && done; ++p) done = sys_finished(conv, nsys, p, s0 - 1, tol);
    if (done) return;
  }
  // the chains' matrices of this CTA's rows, into the update-operand storage
  // G (free once the factorisation is done): Mf_i = L_ii^-1 L_{i,i-1}
  // (forward, tile (i, i-1) in the envelope) at tile i, Mb_i = (L_{i+1,i}
  // L_ii^-1)^T (backward, tile (i+1, i) in the envelope) at tile T + i
  // (ext: the chains run in k_lg_chain, sweeps s0 .. sweeps-1 here)
  for (int q = blockIdx.x; q < R && !ext; q += gridDim.x) {
    const int r = rb_sys[R + q];
    const LgProb& P = probs[rb_sys[r]];
    const int i = r - P.rb0;
    if (__ldg(P.env + i) < i)
      chain_matrix(P.Linv + (size_t)i * TILE, P.A + (size_t)(tri2(i) + i - 1) * TILE, P.G + (size_t)i * TILE, false,
                   gx, gy);
  }
  for (int q = blockIdx.x; q < R && !ext; q += gridDim.x) {
    const int r = rb_sys[2 * R + q];
    const LgProb& P = probs[rb_sys[r]];
    const int i = r - P.rb0;
    if (i + 1 < P.T && __ldg(P.env + i + 1) <= i)
      chain_matrix(P.A + (size_t)(tri2(i + 1) + i) * TILE, P.Linv + (size_t)i * TILE, P.G + (size_t)(P.T + i) * TILE,
                   true, gx, gy);
  }
  for (int sweep = s0; sweep < s1; ++sweep) {
    if (dpv_status(status)) return;
    if (!ext) {
    // ---- forward: L u = rhs; this CTA's row blocks in chain order (all
    // systems' first rows first), so that one system's chain never waits
    // behind another's.  Row i: c_i = L_ii^-1 (rhs_i - sum_{j < i-1} L_ij u_j)
    // while the rows above are solved, then u_i = c_i - Mf_i u_{i-1} as soon
    // as the row above is published (one warp-local product, no barrier)
    for (int q = blockIdx.x; q < R; q += gridDim.x) {
      const int r = rb_sys[R + q];
      if (sys_finished(conv, nsys, rb_sys[r], sweep - 1, tol)) continue;
      const LgProb& P = probs[rb_sys[r]];
      const int i = r - P.rb0;
      const int j0 = __ldg(P.env + i);
      const bool dep = j0 < i;  // tile (i, i-1) lies in the envelope
      if (dep) stage_chain(gx, P.G + (size_t)i * TILE);  // (read after the barriers below)
      if (tid < NB) acc[tid] = __ldcg(P.rhs + i * NB + tid);
      // the tiles do not depend on the solved rows: each is loaded while waiting for the previous row
      TileRegs m = load_block(j0 < i - 1 ? P.A + (size_t)(tri2(i) + j0) * TILE : P.Linv + (size_t)i * TILE);
      for (int j = j0; j < i - 1; ++j) {
        const TileRegs mn =
            load_block(j + 1 < i - 1 ? P.A + (size_t)(tri2(i) + j + 1) * TILE : P.Linv + (size_t)i * TILE);
        if (tid < NB) {
          float v = 0.f;
          if (!wait_tagged(P.tf + j * NB + tid, sweep + 1, v, status, timeout)) ok = 0;
          vj[tid] = v;
        }
        __syncthreads();
        if (!ok) return;
        tile_gemv(m, vj, prod, false, part);
        if (tid < NB) acc[tid] -= prod[tid];
        m = mn;
      }
      __syncthreads();
      tile_gemv(m, acc, prod, false, part);  // c_i
      if (!dep) {
        if (tid < NB) {
          P.xf[i * NB + tid] = prod[tid];
          st_tagged(P.tf + i * NB + tid, sweep + 1, prod[tid]);
        }
      } else {
        float x0 = 0.f, x1 = 0.f;
        if (!wait_tagged2(P.tf + (i - 1) * NB + 2 * lane, sweep + 1, x0, x1, status, timeout)) ok = 0;
        const float sum = chain_product(gx, x0, x1);
        const int row = 8 * wid + (lane >> 2);
        if ((lane & 3) == 0) {
          const float v = prod[row] - sum;
          P.xf[i * NB + row] = v;
          st_tagged(P.tf + i * NB + row, sweep + 1, v);
        }
      }
      __syncthreads();
      if (!ok) return;
    }
    // ---- backward: L^T w = D^-1 u, rows descending; rho = r.w per system
    // (row blocks in chain order from the bottom).  Row i: c_i = L_ii^-T
    // (D_i^-1 u_i - sum_{j > i+1} L_ji^T w_j), then w_i = c_i - Mb_i w_{i+1}
    for (int q = blockIdx.x; q < R; q += gridDim.x) {
      const int r = rb_sys[2 * R + q];
      const int sy = rb_sys[r];
      if (sys_finished(conv, nsys, sy, sweep - 1, tol)) continue;
      const LgProb& P = probs[sy];
      const int i = r - P.rb0, T = P.T;
      const bool dep = i + 1 < T && __ldg(P.env + i + 1) <= i;  // tile (i+1, i) lies in the envelope
      if (dep) stage_chain(gy, P.G + (size_t)(T + i) * TILE);
      // the forward result of this row (solved by whichever CTA owned it in
      // the forward order): taken from its published word
      if (tid < NB) {
        float u = 0.f;
        if (!wait_tagged(P.tf + i * NB + tid, sweep + 1, u, status, timeout)) ok = 0;
        acc[tid] = u * __ldcg(P.invD + i * NB + tid);
      }
      // the rows j > i+1 whose envelope reaches column i (L is zero elsewhere)
      int j = T;
      do { --j; } while (j > i + 1 && __ldg(P.env + j) > i);
      TileRegs m = load_block(j > i + 1 ? P.A + (size_t)(tri2(j) + i) * TILE : P.Linv + (size_t)i * TILE);
      while (j > i + 1) {
        int jn = j;
        do { --jn; } while (jn > i + 1 && __ldg(P.env + jn) > i);
        const TileRegs mn =
            load_block(jn > i + 1 ? P.A + (size_t)(tri2(jn) + i) * TILE : P.Linv + (size_t)i * TILE);
        if (tid < NB) {
          float v = 0.f;
          if (!wait_tagged(P.tb + j * NB + tid, sweep + 1, v, status, timeout)) ok = 0;
          vj[tid] = v;
        }
        __syncthreads();
        if (!ok) return;
        tile_gemv(m, vj, prod, true, part);
        if (tid < NB) acc[tid] -= prod[tid];
        m = mn;
        j = jn;
      }
      __syncthreads();
      if (!ok) return;
      tile_gemv(m, acc, prod, true, part);  // c_i
      if (!dep) {
        if (tid < NB) {
          P.xb[i * NB + tid] = prod[tid];
          st_tagged(P.tb + i * NB + tid, sweep + 1, prod[tid]);
          wfin[tid] = prod[tid];
        }
      } else {
        float x0 = 0.f, x1 = 0.f;
        if (!wait_tagged2(P.tb + (i + 1) * NB + 2 * lane, sweep + 1, x0, x1, status, timeout)) ok = 0;
        const float sum = chain_product(gy, x0, x1);
        const int row = 8 * wid + (lane >> 2);
        if ((lane & 3) == 0) {
          const float v = prod[row] - sum;
          P.xb[i * NB + row] = v;
          st_tagged(P.tb + i * NB + row, sweep + 1, v);
          wfin[row] = v;
        }
      }
      __syncthreads();
      if (!ok) return;
      // off the chain: this block's share of rho = r.w (wfin is rewritten
      // only after the next row's first CTA barrier)
      if (sweep > 0 && wid < 2) {
        const int qq = i * NB + tid;
        double rw = __ldcg(P.r + qq) * dpv_f2d_bits(wfin[tid]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rw += __shfl_xor_sync(0xffffffffu, rw, o);
        if (lane == 0) dpv_red_add(red + 2 * (sweep * nsys + sy), rw);
      }
    }
    if (!grid_barrier(bar, gridDim.x, status, timeout)) return;
    }  // !ext
    if (sweep == 0) {
      // ---- z = w: x = s w, the first correction
      for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const int sy = rb_sys[r];
        const LgProb& P = probs[sy];
        const int q = (r - P.rb0) * NB + tid;
        float cmax = 0.f;
        if (tid < NB) {
          const double x = dpv_f2d_bits(__ldcg(P.xb + q)) * dpv_f2d_bits(P.sc[q]);
          P.xacc[q] = x;
          cmax = fabsf(dpv_d2f_bits(x));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        if (lane == 0 && wid < 2) {  // non-negative floats order like their bit patterns
          atomicMax(conv + 2 * sy, __float_as_int(cmax));
          atomicMax(conv + 2 * sy + 1, __float_as_int(cmax));
        }
      }
      if (sweep + 1 == sweeps) break;
      if (!grid_barrier(bar, gridDim.x, status, timeout)) return;
    }
    // ---- u = S v (double-float), v = s x (iteration 0) or s p; p = w + beta p
    {
      DFp sig{0.f, 0.f};
      for (int sy = 0; sy < nsys; ++sy) {
        if (sys_finished(conv, nsys, sy, sweep - 1, tol)) continue;
        const LgProb& P = probs[sy];
        const double beta =
            sweep > 1 ? __ldcg(red + 2 * (sweep * nsys + sy)) / __ldcg(red + 2 * ((sweep - 1) * nsys + sy)) : 0.0;
        // the tiles of the envelope only (S is zero outside it)
        const int ntile = __ldg(P.eoff + P.T);
        SymvRegs cur, nxt;
        int ti, tj;
        if ((int)blockIdx.x < ntile) load_symv_tile(P.Sdf + (size_t)env_tile(P, blockIdx.x, ti, tj) * TILE, cur);
        for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
          int ti2, tj2;
          if (t + (int)gridDim.x < ntile)
            load_symv_tile(P.Sdf + (size_t)env_tile(P, t + gridDim.x, ti2, tj2) * TILE, nxt);
          env_tile(P, t, ti, tj);
          if (tid < NB) {
            for (int side = 0; side < 2; ++side) {
              const int blk = side ? tj : ti;
              const int q = blk * NB + tid;
              double pv;
              if (sweep == 0) {
                pv = __ldcg(P.xacc + q);  // (s z: already unscaled)
              } else {
                pv = dpv_f2d_bits(__ldcg(P.xb + q)) + (sweep > 1 ? beta * __ldcg(((sweep & 1) ? P.p1 : P.p0) + q) : 0.0);
                // the new direction is written once, by the diagonal tile's CTA
                if (ti == tj && side == 0) (((sweep & 1) ? P.p0 : P.p1))[q] = pv;
                pv *= dpv_f2d_bits(P.sc[q]);
              }
              const float2 d = dpv_d2df_bits(pv);
              (side ? vc : vr)[tid] = DFp{d.x, d.y};
            }
          }
          __syncthreads();
          tile_symv(cur, vr, vc, ti == tj, P.u + ti * NB, P.u + tj * NB, dpart, sig);
          cur = nxt;
        }
        if (sweep > 0) {
          // the CTA's share of p.S'p = v.S v
          __shared__ DFp sred[LG_THREADS / 32];
          DFp a = sig;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) df_add2(a, df_shfl_xor(a, o));
          if (lane == 0) sred[wid] = a;
          __syncthreads();
          if (tid == 0) {
            DFp b = sred[0];
            for (int w = 1; w < LG_THREADS / 32; ++w) df_add2(b, sred[w]);
            if (b.h != 0.f) red_df(red + 2 * (sweep * nsys + sy) + 1, b);
          }
          __syncthreads();
        }
        sig = DFp{0.f, 0.f};
      }
    }
    if (!grid_barrier(bar, gridDim.x, status, timeout)) return;
    // ---- updates: r (iteration 0: r = s (y - u)), or alpha steps of x and r
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
      const int sy = rb_sys[r];
      if (sys_finished(conv, nsys, sy, sweep - 1, tol)) continue;
      const LgProb& P = probs[sy];
      const int q = (r - P.rb0) * NB + tid;
      float cmax = 0.f, xmax = 0.f;
      if (tid < NB) {
        const double s = dpv_f2d_bits(P.sc[q]);
        const double u = __ldcg(P.u + q);
        double rr;
        if (sweep == 0) {
          rr = q < P.n ? s * (P.y[q] - u) : 0.0;
        } else {
          const double rho = __ldcg(red + 2 * (sweep * nsys + sy)), sg = __ldcg(red + 2 * (sweep * nsys + sy) + 1);
          const double alpha = (rho > 0.0 && sg > 0.0) ? rho / sg : 0.0;
          const double pv = __ldcg(((sweep & 1) ? P.p0 : P.p1) + q);
          const double dxq = alpha * s * pv;
          const double x = __ldcg(P.xacc + q) + dxq;
          P.xacc[q] = x;
          rr = q < P.n ? __ldcg(P.r + q) - alpha * s * u : 0.0;
          cmax = fabsf(dpv_d2f_bits(dxq));
          xmax = fabsf(dpv_d2f_bits(x));
        }
        P.r[q] = rr;
        P.rhs[q] = dpv_d2f_bits(rr);
        P.u[q] = 0.0;  // for the next product
      }
      if (sweep > 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
          xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        }
        if (lane == 0 && wid < 2) {
          atomicMax(conv + 2 * (sweep * nsys + sy), __float_as_int(cmax));
          atomicMax(conv + 2 * (sweep * nsys + sy) + 1, __float_as_int(xmax));
        }
      }
    }
    if (!grid_barrier(bar, gridDim.x, status, timeout)) return;
    if (sweep > 0) {
      // per system: the error left in x is below tol of it (the step bounds
      // the previous iterate's error; the current one's is about rho c_s with
      // rho ~ c_s / c_{s-1})
      bool done = true;
      for (int p = 0; p < nsys && done; ++p) done = sys_finished(conv, nsys, p, sweep, tol);
      if (done) break;  // the same decision in every CTA
    }
  }
  // output
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    const LgProb& P = probs[rb_sys[r]];
    const int q = (r - P.rb0) * NB + tid;
    if (tid < NB && q < P.n) {
      const double v = __ldcg(P.xacc + q);
      P.dx[q] = v;
      P.dxf[q] = dpv_d2f_bits(v);
    }
  }
}

// ---------------------------------------------------------------------------
// The triangular-solve chains in one thread-block cluster per system
// ---------------------------------------------------------------------------
// The forward and backward chains of one CG sweep move one 64-row block per
// step from the CTA that solved it to the next; through global memory each
// step costs an L2 round trip of the published words (~1 us per row block
// on this part).  Here the CTAs of one cluster take the row blocks of one
// system round robin (block i on cluster rank i mod C), every CTA holds the
// whole vector as tagged words in its shared memory, and a solved block is
// stored into every CTA's copy through distributed shared memory; the
// consumers poll their own shared memory.  Each solved block is formed from
// per-tile products with the blocks it depends on, the tiles premultiplied
// by the diagonal block's inverse (k_lg_chainmat), so that a warp finishes
// its rows without waiting for the rest of its CTA.

// The chains' matrices, one per tile of the envelope and one CTA per matrix
// (blockIdx.y = system), into the update-operand storage G (free once the
// factorisation is done), indexed by the envelope's tile order e(a, b) =
// eoff_a + b - env_a:
//   forward   G[e(i, j)]      = L_ii^-1 L_ij       (j < i),  L_ii^-1    (j = i)
//   backward  G[E + e(j, i)]  = (L_ji L_ii^-1)^T   (j > i),  L_ii^-T    (j = i)
// (E = the envelope's tile count), so that a solved row block is
//   u_i = L_ii^-1 b_i - sum_j (L_ii^-1 L_ij) u_j,
//   w_i = L_ii^-T c_i - sum_j (L_ji L_ii^-1)^T w_j.
__global__ void __launch_bounds__(LG_THREADS) k_lg_chainmat(const LgProb* __restrict__ probs, const int* status) {
  __shared__ __align__(16) float gx[NB * LDS];
  __shared__ __align__(16) float gy[NB * LDS];
  if (dpv_status(status)) return;
  const LgProb& P = probs[blockIdx.y];
  const int E = __ldg(P.eoff + P.T);
  const bool bwd = (int)blockIdx.x >= E;
  const int t = bwd ? (int)blockIdx.x - E : (int)blockIdx.x;
  if (t >= E) return;
  int a, b;
  env_tile(P, t, a, b);  // tile (a, b) of the envelope, b <= a
  float* out = P.G + (size_t)blockIdx.x * TILE;
  if (a == b) {  // L_aa^-1, or its transpose
    const float* li = P.Linv + (size_t)a * TILE;
    for (int q = threadIdx.x; q < TILE; q += LG_THREADS) {
      const int r = q >> 6, c = q & 63;
      out[q] = bwd ? __ldcg(li + c * NB + r) : __ldcg(li + q);
    }
  } else if (!bwd) {
    chain_matrix4(P.Linv + (size_t)a * TILE, P.A + (size_t)(tri2(a) + b) * TILE, out, false, gx, gy);
  } else {
    chain_matrix4(P.A + (size_t)(tri2(a) + b) * TILE, P.Linv + (size_t)b * TILE, out, true, gx, gy);
  }
}

// Wait (bounded) until the tagged word p of this CTA's shared memory carries
// tag; its value in v.
__device__ __forceinline__ bool wait_local(const unsigned long long* p, unsigned tag, float& v, int* status,
                                           long long timeout) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    const unsigned long long w = *reinterpret_cast<const volatile unsigned long long*>(p);
    if ((unsigned)(w >> 32) == tag) {
      v = __uint_as_float((unsigned)w);
      return true;
    }
    if ((it & 255u) == 255u) {
      if (dpv_status(status)) return false;
      if (clock64() - t0 > timeout) {
        dpv_set_status(status, DST_TIMEOUT);
        return false;
      }
    }
    if (it > 64) __nanosleep(16);
  }
}

// This lane's slice of a chain matrix: rows 8w .. 8w+7, columns 2l, 2l+1.
struct ChainSlice {
  float2 m[8];
};
__device__ __forceinline__ ChainSlice load_slice(const float* M) {
  const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) & 7;  // (the warp within its group of 8)
  ChainSlice c;
#pragma unroll
  for (int r = 0; r < 8; ++r) c.m[r] = __ldcg(reinterpret_cast<const float2*>(M + (8 * w + r) * NB) + lane);
  return c;
}
// the sum over the warp of the eight row partials (see chain_product): lane
// l ends with row 8w + (l >> 2)
__device__ __forceinline__ float reduce_rows8(const float (&s)[8]) {
  const int lane = threadIdx.x & 31;
  float t4[4];
  {
    const bool up = lane & 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float send = up ? s[q] : s[q + 4], keep = up ? s[q + 4] : s[q];
      t4[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  float t2[2];
  {
    const bool up = lane & 8;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float send = up ? t4[q] : t4[q + 2], keep = up ? t4[q + 2] : t4[q];
      t2[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  const bool up = lane & 4;
  float t1 = (up ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, up ? t2[0] : t2[1], 4);
  t1 += __shfl_xor_sync(0xffffffffu, t1, 2);
  t1 += __shfl_xor_sync(0xffffffffu, t1, 1);
  return t1;
}

constexpr int CH_MAX_T = 128;  // tile rows of a system whose chains run in a cluster (2 x 64 KB of tagged words)
constexpr int CH_GROUPS = 3;                 // groups of 8 warps: consecutive row blocks of one CTA
constexpr int CH_THREADS = 256 * CH_GROUPS;
// The cluster form costs two launches per CG sweep instead of one kernel for
// all sweeps; it pays where the chains are long (measured: 1000 keyframes,
// 94 tile rows, 180 -> 130 us per sweep), not for the 64-problem batch
// (at most 38 tile rows: 8.55k -> 8.14k problem GN it/s).
constexpr int CH_MIN_T = 64;
constexpr unsigned CH_TAG = 1;  // tag of a solved value (the copies are cleared to tag 0 by each launch)

// One sweep's chains: cluster b solves system b (forward L u = rhs, then
// backward L^T w = D^-1 u), writing u to xf and w to xb, and adds its rows'
// shares of rho = r.w (sweeps > 0).  Systems already converged are skipped.
// Row block i belongs to cluster rank i mod C; within it warp w takes rows
// 8w .. 8w+7 and works on its own (no block barrier): per tile of the
// envelope its lanes read the two solved values they need from their
// shared memory and multiply them into the slice of the chain matrix that
// was loaded meanwhile.
__global__ void __launch_bounds__(CH_THREADS) k_lg_chain(const LgProb* __restrict__ probs, int nsys, int sweep,
                                                         const int* conv, double* red, float tol, int* status,
                                                         long long timeout) {
  // this CTA's copies of the forward and the backward vectors, tagged; each
  // word is written once per launch (a word written twice by one thread
  // through the cluster could be observed in either order)
  extern __shared__ __align__(16) unsigned long long xs[];  // [2][T * NB]
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int sy = blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, wid = (tid >> 5) & 7, grp = tid >> 8;
  // (the same decision in every CTA of the cluster: the convergence words
  // are final; an error reported meanwhile ends the waits below)
  if (sy >= nsys || sys_finished(conv, nsys, sy, sweep - 1, tol)) return;
  const LgProb& P = probs[sy];
  const int T = P.T, E = __ldg(P.eoff + T);
  unsigned long long* xf = xs;           // forward values u
  unsigned long long* xb = xs + T * NB;  // backward values w
  for (int q = tid; q < 2 * T * NB; q += CH_THREADS) xs[q] = 0ull;
  cl.sync();  // every copy is cleared before any CTA stores into it
  const int row = 8 * wid + (lane >> 2);  // the row this lane reports after the reduction
  // (remote stores go to every CTA of the cluster, this one included: lanes
  // l, l+1, l+2, l+3 hold the same row value and share the destinations)
  auto publish = [&](unsigned long long* vec, int i, float v) {
    const unsigned long long w = ((unsigned long long)CH_TAG << 32) | __float_as_uint(v);
    for (int d = lane & 3; d < C; d += 4) {
      unsigned long long* rx = d == rank ? vec : cl.map_shared_rank(vec, (unsigned)d);
      reinterpret_cast<volatile unsigned long long*>(rx)[i * NB + row] = w;
    }
  };
  // the row blocks come in runs of CH_GROUPS consecutive blocks (run p on
  // cluster rank p mod C), one per group of 8 warps: the dependencies inside
  // a run stay in this CTA's shared memory
  const int nruns = (T + CH_GROUPS - 1) / CH_GROUPS;
  bool good = true;
  // ---- forward: the runs rank, rank + C, ...
  for (int pp = rank; pp < nruns && good; pp += C) {
    const int i = CH_GROUPS * pp + grp;
    if (i >= T) break;
    const int j0 = __ldg(P.env + i);
    const float* Nr = P.G + (size_t)(__ldg(P.eoff + i) - j0) * TILE;  // N_ij at Nr + j * TILE
    float s[8];
    {
      const ChainSlice li = load_slice(Nr + (size_t)i * TILE);
      const float2 b = __ldcg(reinterpret_cast<const float2*>(P.rhs + i * NB) + lane);
#pragma unroll
      for (int r = 0; r < 8; ++r) s[r] = fmaf(li.m[r].x, b.x, li.m[r].y * b.y);
    }
    // the tiles j0 .. i-1, their slices loaded two tiles ahead
    const int jc = i;  // (the end of the list)
    ChainSlice b[2];
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (j0 + q < jc) b[q] = load_slice(Nr + (size_t)(j0 + q) * TILE);
    for (int j = j0; j < jc && good; j += 2) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int jj = j + q;
        if (jj < jc && good) {
          float x0 = 0.f, x1 = 0.f;
          if (!wait_local(xf + jj * NB + 2 * lane, CH_TAG, x0, status, timeout) ||
              !wait_local(xf + jj * NB + 2 * lane + 1, CH_TAG, x1, status, timeout)) {
            good = false;
          } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) s[r] = fmaf(-b[q].m[r].x, x0, fmaf(-b[q].m[r].y, x1, s[r]));
            if (jj + 2 < jc) b[q] = load_slice(Nr + (size_t)(jj + 2) * TILE);
          }
        }
      }
    }
    good = __all_sync(0xffffffffu, good);
    if (!good) break;
    const float v = reduce_rows8(s);
    publish(xf, i, v);
    if ((lane & 3) == 0) P.xf[i * NB + row] = v;
  }
  // ---- backward: the runs of this rank, descending
  for (int pp = rank + C * ((nruns - 1 - rank) / C); pp >= 0 && rank < nruns && good; pp -= C) {
    const int i = CH_GROUPS * pp + grp;
    if (i >= T) continue;
    float s[8];
    {
      const ChainSlice lt = load_slice(P.G + (size_t)(E + __ldg(P.eoff + i) + i - __ldg(P.env + i)) * TILE);
      float u0 = 0.f, u1 = 0.f;
      if (!wait_local(xf + i * NB + 2 * lane, CH_TAG, u0, status, timeout) ||
          !wait_local(xf + i * NB + 2 * lane + 1, CH_TAG, u1, status, timeout))
        good = false;
      const float2 dv = __ldcg(reinterpret_cast<const float2*>(P.invD + i * NB) + lane);
      u0 *= dv.x;
      u1 *= dv.y;
#pragma unroll
      for (int r = 0; r < 8; ++r) s[r] = fmaf(lt.m[r].x, u0, lt.m[r].y * u1);
    }
    // the rows j > i whose envelope reaches column i, bottom up, their
    // slices loaded two rows ahead (next_row: the next such row below j)
    const int lo = i;  // the ring takes the rows above lo
    auto next_row = [&](int j) {
      do { --j; } while (j > lo && __ldg(P.env + j) > i);
      return j;
    };
    auto bslice = [&](int j) { return P.G + (size_t)(E + __ldg(P.eoff + j) + i - __ldg(P.env + j)) * TILE; };
    int jr[2];  // the rows whose slices sit in b[0..1] (lo: none)
    ChainSlice b[2];
    {
      int j = T;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        j = j > lo ? next_row(j) : lo;
        jr[q] = j;
        if (j > lo) b[q] = load_slice(bslice(j));
      }
    }
    while (good && jr[0] > lo) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int j = jr[q];
        if (j > lo && good) {
          float x0 = 0.f, x1 = 0.f;
          if (!wait_local(xb + j * NB + 2 * lane, CH_TAG, x0, status, timeout) ||
              !wait_local(xb + j * NB + 2 * lane + 1, CH_TAG, x1, status, timeout)) {
            good = false;
          } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) s[r] = fmaf(-b[q].m[r].x, x0, fmaf(-b[q].m[r].y, x1, s[r]));
            // the row two places further down the list
            const int last = jr[q ^ 1];
            const int jn = last > lo ? next_row(last) : lo;
            jr[q] = jn;
            if (jn > lo) b[q] = load_slice(bslice(jn));
          }
        } else {
          jr[q] = lo;
        }
      }
    }
    good = __all_sync(0xffffffffu, good);
    if (!good) break;
    const float v = reduce_rows8(s);
    publish(xb, i, v);
    if ((lane & 3) == 0) P.xb[i * NB + row] = v;
    if (sweep > 0) {  // this warp's share of rho = r.w
      double rw = (lane & 3) == 0 ? __ldcg(P.r + i * NB + row) * dpv_f2d_bits(v) : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rw += __shfl_xor_sync(0xffffffffu, rw, o);
      if (lane == 0) dpv_red_add(red + 2 * (sweep * nsys + sy), rw);
    }
  }
  cl.sync();  // no CTA leaves while another may still store into its copy
}

// Task list of several systems, in dependency order within each system and
// interleaved by step across systems, so that every critical chain advances
// together.  Per system: step k's update of columns k+1, k+2 and the panels
// of column k+1 come before the bulk of step k's trailing update, whose
// column pairs run left to right; the critical CTA does DIAG(k),
// PANEL(k, k-1) and UPDATE(k, k, k-1).
std::vector<unsigned long long> build_tasks(const std::vector<int>& Ts) {
  std::vector<unsigned long long> v;
  auto put = [&](int p, int type, int k, int i, int j) {
    v.push_back(((unsigned long long)p << 32) | pack_task(type, k, i, j));
  };
  int maxT = 0;
  for (int T : Ts) maxT = std::max(maxT, T);
  for (int p = 0; p < (int)Ts.size(); ++p)
    for (int i = 2; i < Ts[p]; ++i) put(p, TASK_PANEL, 0, i, 0);
  // updates cover 2 x 2 tiles: rows (i, i+1), columns (j, j+1)
  for (int k = 0; k + 1 < maxT; ++k)
    for (int p = 0; p < (int)Ts.size(); ++p) {
      const int T = Ts[p];
      if (k + 1 >= T) continue;
      // columns k+1, k+2 first (tile (k+1, k+1) is the critical CTA's)
      for (int i = k + 2; i < T; i += 2) put(p, TASK_UPDATE, k, i, k + 1);
      for (int i = k + 3; i < T; ++i) put(p, TASK_PANEL, k + 1, i, k + 1);
      for (int j = k + 3; j < T; j += 2)
        for (int i = j; i < T; i += 2) put(p, TASK_UPDATE, k, i, j);
    }
  return v;
}

struct TaskCache {
  std::mutex mu;
  std::map<std::pair<int, std::vector<int>>, std::pair<unsigned long long*, int>> lists;  // (device, Ts)
};
TaskCache& task_cache() {
  static TaskCache c;
  return c;
}

// every CTA resident at once (the kernels wait on one another's tiles); the
// launch attribute form is also what a CUDA-graph capture records
cudaError_t launch_cooperative(const void* fn, int grid, size_t smem, cudaStream_t st, void** args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(LG_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

int co_resident(ba_handle_t h, const void* fn, size_t smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LG_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * h->num_sms;
}

}  // namespace

long long dpv_large_scratch_floats(int n_pad) {
  const long long T = n_pad / NB;
  // tiles of A, inverses of the diagonal factors, D, D^-1, rhs, xf, xb,
  // equilibration scale, the pre-split update operands, S as float pairs,
  // the conjugate-gradient vectors r, p0, p1, u (FP64), the tagged solved rows
  return (long long)tri2((int)T) * TILE + T * TILE + 6LL * n_pad + 2LL * tri2((int)T) * TILE +
         2LL * tri2((int)T) * TILE + 8LL * n_pad + 4LL * n_pad;
}

namespace {

constexpr int MAX_SWEEPS = 16;

// The cluster size of k_lg_chain on this device: 16 CTAs (a non-portable
// size) where one such cluster fits, else 8; 0 when neither does (the chains
// then run in k_lg_solve).  Found once.
int chain_cluster(ba_handle_t h) {
  static int C = -1;
  if (C >= 0) return C;
  C = 0;
  const int smem = (int)(2 * sizeof(unsigned long long) * CH_MAX_T * NB);
  if (cudaFuncSetAttribute(k_lg_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_lg_chain, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return C;
  }
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3(CH_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = h->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_lg_chain, &cfg) == cudaSuccess && n > 0) {
      C = c;
      break;
    }
    cudaGetLastError();
  }
  return C;
}

// The large systems' descriptors, row-block table, task list and sync-word
// layout for the current pose-system layout; grows the solver's buffers.
struct LgPlan {
  std::vector<int> Ts;
  std::vector<LgProb> pr;
  std::vector<int> rb_sys;
  long long soff_sync = 0, nsync = 0;
  unsigned long long* tasks = nullptr;
  int ntasks = 0;
};

ba_status_t lg_plan(ba_handle_t h, LgPlan& L) {
  Workspace* ws = h->ws;
  const int nsys = (int)h->large_sys.size();
  L.Ts.assign(nsys, 0);
  L.pr.assign(nsys, LgProb{});
  L.rb_sys.clear();
  long long foff = 0;
  L.soff_sync = 0;
  for (int p = 0; p < nsys; ++p) {
    const SysDesc& sd = h->sys[h->large_sys[p]];
    if (sd.TS != NB || sd.n_pad % NB) return dpv_fail(h, BA_ERR_UNSUPPORTED, "large solver needs 64-row tiles");
    const int T = sd.n_pad / NB;
    if (T > LG_MAX_T) return dpv_fail(h, BA_ERR_UNSUPPORTED, "pose system above 65472 unknowns");
    L.Ts[p] = T;
    LgProb& P = L.pr[p];
    float* base = ws->L.p + foff;
    P.A = base;
    P.Linv = P.A + (size_t)tri2(T) * TILE;
    P.D = P.Linv + (size_t)T * TILE;
    P.invD = P.D + sd.n_pad;
    P.rhs = P.invD + sd.n_pad;
    P.xf = P.rhs + sd.n_pad;
    P.xb = P.xf + sd.n_pad;
    P.sc = P.xb + sd.n_pad;
    P.G = P.sc + sd.n_pad;  // 256-byte aligned: every piece above is a multiple of 64 floats
    P.Sdf = reinterpret_cast<float2*>(P.G + 2LL * tri2(T) * TILE);
    P.r = reinterpret_cast<double*>(P.G + 4LL * tri2(T) * TILE);
    P.p0 = P.r + sd.n_pad;
    P.p1 = P.p0 + sd.n_pad;
    P.u = P.p1 + sd.n_pad;
    P.tf = reinterpret_cast<unsigned long long*>(P.u + sd.n_pad);
    P.tb = P.tf + sd.n_pad;
    foff += dpv_large_scratch_floats(sd.n_pad);
    P.S = ws->S.p + sd.soff;
    P.y = ws->y.p + sd.voff;
    P.xacc = ws->r64.p + sd.voff;
    P.dx = ws->dx.p + sd.voff;
    P.dxf = ws->tmpv.p + sd.voff;
    P.T = T;
    P.n = sd.n;
    P.n_pad = sd.n_pad;
    P.rb0 = (int)L.rb_sys.size();
    for (int i = 0; i < T; ++i) L.rb_sys.push_back(p);
    L.soff_sync += tri2(T) + 2 * T + 1;  // versions, envelope, envelope offsets
  }
  {
    // the chain orders of the triangular solves: by position in the chain,
    // then by system
    const int R = (int)L.rb_sys.size();
    std::vector<int> fw(R), bw(R);
    for (int r = 0; r < R; ++r) fw[r] = bw[r] = r;
    auto pos = [&](int r) { return r - L.pr[L.rb_sys[r]].rb0; };
    std::stable_sort(fw.begin(), fw.end(), [&](int a, int b) { return pos(a) < pos(b); });
    std::stable_sort(bw.begin(), bw.end(), [&](int a, int b) {
      return L.pr[L.rb_sys[a]].T - 1 - pos(a) < L.pr[L.rb_sys[b]].T - 1 - pos(b);
    });
    L.rb_sys.insert(L.rb_sys.end(), fw.begin(), fw.end());
    L.rb_sys.insert(L.rb_sys.end(), bw.begin(), bw.end());
  }
  if (foff > ws->L.cap) return dpv_fail(h, BA_ERR_STATE, "large solver scratch");
  // the task list of this set of sizes, built once per device
  {
    TaskCache& tc = task_cache();
    std::lock_guard<std::mutex> lk(tc.mu);
    auto key = std::make_pair(h->device, L.Ts);
    auto it = tc.lists.find(key);
    if (it == tc.lists.end()) {
      if (h->capturing) return dpv_fail(h, BA_ERR_STATE, "large solver task list built during graph capture");
      std::vector<unsigned long long> v = build_tasks(L.Ts);
      unsigned long long* d = nullptr;
      if (cudaMalloc(&d, sizeof(unsigned long long) * std::max<size_t>(v.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        return dpv_fail(h, BA_ERR_OOM, "large solver task list");
      }
      if (!v.empty()) DPV_CUDA(h, cudaMemcpy(d, v.data(), sizeof(unsigned long long) * v.size(), cudaMemcpyHostToDevice));
      it = tc.lists.emplace(key, std::make_pair(d, (int)v.size())).first;
    }
    L.tasks = it->second.first;
    L.ntasks = it->second.second;
  }
  // sync words: per system tile versions, envelope and its offsets; task
  // counter, barrier, critical SMs, convergence maxima per (sweep, system),
  // the envelope compaction's counts
  L.nsync = L.soff_sync + 4 + nsys + 2LL * MAX_SWEEPS * nsys + ENV_MAX_CTAS;
  ba_status_t s;
  if ((s = dpv_grow(h, ws->lg_sync, L.nsync, "large solver sync")) ||
      (s = dpv_grow(h, ws->lg_red, 2LL * MAX_SWEEPS * nsys, "large solver reductions")) ||
      (s = dpv_grow(h, ws->lg_prob, (long long)nsys * sizeof(LgProb) / sizeof(long long) + 1, "large systems")) ||
      (s = dpv_grow(h, ws->lg_rb, (long long)L.rb_sys.size(), "row blocks")) ||
      (s = dpv_grow(h, ws->lg_live, (long long)L.ntasks + 1, "live factorisation tasks")))
    return s;
  return BA_OK;
}

}  // namespace

// The row envelopes of the large systems as the last factorisation found
// them: out[0] = systems, then per system its tile count T and env[0..T-1].
ba_status_t dpv_large_envelope(ba_handle_t h, int* out, long long cap, long long* count) {
  const int nsys = (int)h->large_sys.size();
  std::vector<int> Ts(nsys);
  long long need = 1, words = 0;
  for (int p = 0; p < nsys; ++p) {
    Ts[p] = h->sys[h->large_sys[p]].n_pad / NB;
    need += 1 + Ts[p];
    words += tri2(Ts[p]) + 2 * Ts[p] + 1;
  }
  *count = need;
  if (cap < need) return dpv_fail(h, BA_ERR_INVALID_ARG, "envelope buffer too small");
  out[0] = nsys;
  if (nsys == 0) return BA_OK;
  if (!h->ws->lg_sync.p || h->ws->lg_sync.cap < words)
    return dpv_fail(h, BA_ERR_STATE, "no factorisation of the bound systems yet");
  DPV_CUDA(h, cudaStreamSynchronize(h->stream));
  long long o = 0, w = 1;
  for (int p = 0; p < nsys; ++p) {
    out[w] = Ts[p];
    DPV_CUDA(h, cudaMemcpy(out + w + 1, h->ws->lg_sync.p + o + tri2(Ts[p]), sizeof(int) * Ts[p],
                           cudaMemcpyDeviceToHost));
    w += 1 + Ts[p];
    o += tri2(Ts[p]) + 2 * Ts[p] + 1;
  }
  return BA_OK;
}

// Size the large solver's buffers and build its task list for the current
// layout (ahead of the steps, so that a step allocates nothing).
ba_status_t dpv_large_reserve(ba_handle_t h) {
  if (h->large_sys.empty()) return BA_OK;
  LgPlan L;
  return lg_plan(h, L);
}

// Solve every large system (h->large_sys) with one factorisation launch and
// one solve launch.  refine: the most refinement sweeps allowed.
ba_status_t dpv_solve_large(ba_handle_t h, int refine) {
  Workspace* ws = h->ws;
  const int nsys = (int)h->large_sys.size();
  if (nsys == 0) return BA_OK;
  refine = std::min(refine, MAX_SWEEPS - 1);
  LgPlan L;
  ba_status_t s;
  if ((s = lg_plan(h, L))) return s;
  std::vector<int>& Ts = L.Ts;
  std::vector<LgProb>& pr = L.pr;
  std::vector<int>& rb_sys = L.rb_sys;
  const long long soff_sync = L.soff_sync, nsync = L.nsync;
  unsigned long long* tasks = L.tasks;
  int ntasks = L.ntasks;
  const int R = (int)rb_sys.size() / 3;  // systems of the row blocks, then the two chain orders
  int* sync = ws->lg_sync.p;
  for (int p = 0, o = 0; p < nsys; ++p) {
    pr[p].ver = sync + o;
    pr[p].env = pr[p].ver + tri2(Ts[p]);
    pr[p].eoff = pr[p].env + Ts[p];
    o += tri2(Ts[p]) + 2 * Ts[p] + 1;
  }
  int* ctr = sync + soff_sync;
  int* bar = ctr + 1;   // two ints
  int* dsm = bar + 3;   // [nsys]
  int* conv = dsm + nsys;  // [2 MAX_SWEEPS nsys]
  int* status = ws->status;
  cudaStream_t st = h->stream;
  const LgProb* dprobs = reinterpret_cast<const LgProb*>(ws->lg_prob.p);
  DPV_CUDA(h, cudaMemsetAsync(sync, 0, sizeof(int) * nsync, st));
  DPV_CUDA(h, cudaMemsetAsync(ws->lg_red.p, 0, sizeof(double) * 2 * MAX_SWEEPS * nsys, st));
  double* red = ws->lg_red.p;
  {
    // the descriptors change only with the systems' layout or the workspace:
    // upload them when they differ from what the device holds (never while a
    // step is captured into a graph)
    // (the workspace generation too: a reallocated lg_prob holds nothing)
    std::vector<unsigned char> up;
    auto put = [&up](const void* p, size_t n) {
      const unsigned char* c = static_cast<const unsigned char*>(p);
      up.insert(up.end(), c, c + n);
    };
    put(pr.data(), sizeof(LgProb) * nsys);
    put(rb_sys.data(), sizeof(int) * 3 * R);
    put(&h->ws_gen, sizeof(long long));
    if (up != ws->lg_uploaded) {
      if (h->capturing) return dpv_fail(h, BA_ERR_STATE, "large solver tables changed during graph capture");
      DPV_CUDA(h, cudaMemcpyAsync(ws->lg_prob.p, pr.data(), sizeof(LgProb) * nsys, cudaMemcpyHostToDevice, st));
      DPV_CUDA(h, cudaMemcpyAsync(ws->lg_rb.p, rb_sys.data(), sizeof(int) * 3 * R, cudaMemcpyHostToDevice, st));
      ws->lg_uploaded.swap(up);  // (pageable-source copies are staged before they return)
    }
  }
  int maxpad = 0, maxtiles = 0;
  for (int T : Ts) {
    maxpad = std::max(maxpad, T * NB);
    maxtiles = std::max(maxtiles, tri2(T));
  }
  k_lg_scale<<<dim3((maxpad + 255) / 256, nsys), 256, 0, st>>>(dprobs, status);
  ++h->launches;
  k_lg_convert<<<dim3(std::min(maxtiles, 8 * h->num_sms), nsys), 256, 0, st>>>(dprobs, status);
  ++h->launches;
  // the factorisation's live tasks and initial versions, the envelope offsets
  unsigned long long* live = ws->lg_live.p;
  {
    int* counts = sync + nsync - ENV_MAX_CTAS;
    const int g = std::max(1, std::min({ENV_MAX_CTAS, h->num_sms, (ntasks + ENV_THREADS - 1) / ENV_THREADS}));
    k_lg_envelope<<<g, ENV_THREADS, 0, st>>>(dprobs, nsys, ws->lg_rb.p, R, tasks, ntasks, counts, status);
    ++h->launches;
    k_lg_compact<<<g, ENV_THREADS, 0, st>>>(dprobs, tasks, ntasks, counts, live, status);
    ++h->launches;
  }
  long long timeout = h->opt.timeout_cycles;
  {
    // at most two CTAs per SM; the critical CTAs get their SMs to themselves
    // while at least half the SMs remain for the workers
    const size_t smem = TC_OFF + (size_t)TC_SMEM;  // CUDA-core tasks' storage, then the tensor-core operands
    static bool attr = false;
    if (!attr) {
      DPV_CUDA(h, cudaFuncSetAttribute(k_lg_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      // all of the unified L1 / shared storage as shared memory: two CTAs per SM
      DPV_CUDA(h, cudaFuncSetAttribute(k_lg_factor, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      attr = true;
    }
    const int grid = std::min(co_resident(h, (const void*)k_lg_factor, smem), 2 * h->num_sms);
    if (grid <= nsys) return dpv_fail(h, BA_ERR_UNSUPPORTED, "more large systems than the solver's resident CTAs");
    int isolate = 2 * nsys <= h->num_sms ? 1 : 0;
    int nsys_ = nsys;
    void* args[] = {(void*)&dprobs, (void*)&nsys_, (void*)&live,   (void*)&ntasks,
                    (void*)&ctr,    (void*)&dsm,   (void*)&isolate, (void*)&status, (void*)&timeout};
    // timed as its own class (inside the solve class's region)
    dpv_prof_end(h);
    dpv_prof_begin(h, BA_KERNEL_FACTOR);
    DPV_CUDA(h, launch_cooperative((const void*)k_lg_factor, grid, smem, st, args));
    ++h->launches;
    dpv_prof_end(h);
    dpv_prof_begin(h, BA_KERNEL_SOLVE);
  }
  {
    // every resident CTA: the row-block chains use R of them, the products
    // with S all of them
    const int grid = co_resident(h, (const void*)k_lg_solve);
    if (grid <= 0) return dpv_fail(h, BA_ERR_CUDA, "large solver occupancy");
    int sweeps = refine + 1;
    int nsys_ = nsys, R_ = R;
    const int* rb = ws->lg_rb.p;
    float tol = dpv_solve_tol(h);
    int maxT = 0, maxE = 0;
    for (int T : Ts) {
      maxT = std::max(maxT, T);
      maxE = std::max(maxE, tri2(T));  // (the envelope has at most tri(T) tiles; the rest of the grid returns)
    }
    const int C = maxT >= CH_MIN_T && maxT <= CH_MAX_T ? chain_cluster(h) : 0;
    if (C > 0) {
      // the chains in clusters, the rest of each sweep in the cooperative kernel
      k_lg_chainmat<<<dim3(2 * maxE, nsys), LG_THREADS, 0, st>>>(dprobs, status);
      ++h->launches;
      for (int sw = 0; sw < sweeps; ++sw) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(nsys * C));
        cfg.blockDim = dim3(CH_THREADS);
        cfg.dynamicSmemBytes = 2 * sizeof(unsigned long long) * (size_t)maxT * NB;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        DPV_CUDA(h, cudaLaunchKernelEx(&cfg, k_lg_chain, dprobs, nsys, sw, (const int*)conv, red, tol, status,
                                       timeout));
        ++h->launches;
        int s0 = sw, s1 = sw + 1, ext = 1;
        void* args[] = {(void*)&dprobs, (void*)&nsys_, (void*)&rb,  (void*)&R_,  (void*)&s0,
                        (void*)&s1,     (void*)&sweeps, (void*)&ext, (void*)&bar, (void*)&conv,
                        (void*)&red,    (void*)&tol,    (void*)&status, (void*)&timeout};
        DPV_CUDA(h, launch_cooperative((const void*)k_lg_solve, grid, 0, st, args));
        ++h->launches;
      }
    } else {
      int s0 = 0, ext = 0;
      void* args[] = {(void*)&dprobs, (void*)&nsys_,  (void*)&rb,  (void*)&R_,  (void*)&s0,
                      (void*)&sweeps, (void*)&sweeps, (void*)&ext, (void*)&bar, (void*)&conv,
                      (void*)&red,    (void*)&tol,    (void*)&status, (void*)&timeout};
      DPV_CUDA(h, launch_cooperative((const void*)k_lg_solve, grid, 0, st, args));
      ++h->launches;
    }
  }
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
