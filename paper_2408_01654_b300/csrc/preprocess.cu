// Graph preprocessing for ba_set_graph (runs once per bound graph).
//
// Builds, on the GPU and without host round trips:
//   * validation of every index and of "one source frame per patch"
//     (the patch graph of Sec. 3.1: patch k belongs to frame i; edges (i,k,j)),
//     and whether kk is already non-decreasing;
//   * the patch-major order: a stable sort of the edges by kk (skipped on the
//     device when the input is already kk-sorted, the usual case);
//   * the group and patch CSR (gptr, pptr) from the patch-major order;
//   * per group of G consecutive patches: its window (sorted frames touched by
//     its edges, at most DPV_WMAX), and a counting sort of its edges by
//     (source slot, target slot) in shared memory, so that every
//     (source frame, target frame) pair is one contiguous "run"; the run
//     table is per group (at most DPV_RMAX runs), so no global scan is needed.
// The resulting edge order is the stable sort by (group, ii, jj, kk).
// A graph whose groups and 256-edge blocks fit in one co-resident wave (an
// odometry window) is bound by two launches: k_bind_init, then k_bind with
// the steps above as phases between grid barriers; larger graphs take one
// launch per step at full occupancy.
#include "internal.cuh"

#include <algorithm>
#include <map>
#include <mutex>

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int RS_SCAN_ITEMS = 4;  // the sort's own scan: 256 threads x 4 items per tile
constexpr int RS_SCAN_TILE = RS_THREADS * RS_SCAN_ITEMS;

// ---------------------------------------------------------------------------
// exclusive scan of int32 (tile sums, scan of the sums, down-sweep)
// ---------------------------------------------------------------------------
__device__ int block_exclusive_scan(int v, int* sh, int& total) {
  const int t = threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (w == 0) {
    int s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;
  }
  __syncthreads();
  const int wpre = w ? sh[w - 1] : 0;
  total = sh[nw - 1];
  __syncthreads();
  return wpre + x - v;
}

__global__ void k_scan_tiles(const int* __restrict__ in, int n, int* __restrict__ sums, const int* run_if) {
  __shared__ int sh[32];
  if (run_if && !*run_if) return;
  const int base = blockIdx.x * SCAN_TILE;
  int s = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    const int idx = base + r * SCAN_THREADS + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  int total;
  block_exclusive_scan(s, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int* sums, int nb, const int* run_if) {
  __shared__ int sh[32];
  if (run_if && !*run_if) return;
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += sums[i];
  int total;
  int run = block_exclusive_scan(s, sh, total);
  for (int i = lo; i < hi; ++i) {
    const int v = sums[i];
    sums[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) sums[nb] = total;
}

__global__ void k_scan_down(const int* __restrict__ in, int n, const int* __restrict__ sums,
                            int* __restrict__ out, const int* run_if) {
  __shared__ int sh[32];
  if (run_if && !*run_if) return;
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    v[r] = (base + r < n) ? in[base + r] : 0;
    s += v[r];
  }
  int total;
  int run = block_exclusive_scan(s, sh, total) + sums[blockIdx.x];
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    if (base + r < n) out[base + r] = run;
    run += v[r];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

// ---------------------------------------------------------------------------
// validation and sort keys
// ---------------------------------------------------------------------------
// Edge e: its sort key (kk) and value (e), the "kk not non-decreasing" flag,
// index checks, and the patch's source frame (every edge of patch k must
// leave the same frame i; src[] holds -1 on entry).
__device__ void validate_edge(int e, int E, int N, int P, const int* __restrict__ ii, const int* __restrict__ jj,
                              const int* __restrict__ kk, int* __restrict__ src, unsigned long long* __restrict__ keys,
                              int* __restrict__ vals, int* __restrict__ unsorted, int* status) {
  const int i = ii[e], j = jj[e], k = kk[e];
  vals[e] = e;
  keys[e] = (unsigned)k;
  if (e + 1 < E && k > kk[e + 1]) atomicOr(unsorted, 1);
  if (i < 0 || i >= N || j < 0 || j >= N || k < 0 || k >= P) {
    dpv_set_status(status, DST_BAD_INDEX);
    keys[e] = 0ull;
    return;
  }
  const int old = atomicCAS(&src[k], -1, i);
  if (old != -1 && old != i) dpv_set_status(status, DST_BAD_INDEX);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits.  Inside a tile, items are ranked in
// rounds of 256 consecutive keys; a warp ranks equal digits with
// __match_any_sync, warps are ordered through a per-digit prefix, so equal
// keys keep their input order.
// ---------------------------------------------------------------------------
// one tile's digit counts: hist[digit * nblocks + tile]
__device__ void rs_hist_tile(const unsigned long long* __restrict__ keys, int M, int shift, int* __restrict__ hist,
                             int nblocks, int tile, int* cnt) {
  const int t = threadIdx.x;
  cnt[t] = 0;
  __syncthreads();
  const int base = tile * RS_TILE;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int idx = base + r * RS_THREADS + t;
    if (idx < M) atomicAdd(&cnt[(unsigned)(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(size_t)t * nblocks + tile] = cnt[t];
  __syncthreads();
}

// one tile's stable scatter to its digits' offsets
__device__ void rs_scatter_tile(const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
                                unsigned long long* __restrict__ kout, int* __restrict__ vout, int M, int shift,
                                const int* __restrict__ offs, int nblocks, int tile, int* base_off,
                                int (*wcnt)[256]) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  base_off[t] = offs[(size_t)t * nblocks + tile];
  const unsigned lt = (1u << lane) - 1u;
  const int base = tile * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
#pragma unroll
    for (int q = 0; q < RS_THREADS / 32; ++q) wcnt[q][t] = 0;
    __syncthreads();
    const int idx = base + r * RS_THREADS + t;
    const bool valid = idx < M;
    unsigned long long key = 0;
    int val = 0;
    unsigned digit = 256u;
    if (valid) {
      key = kin[idx];
      val = vin[idx];
      digit = (unsigned)(key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int lrank = __popc(peers & lt);
    if (valid && lrank == 0) wcnt[w][digit] = __popc(peers);
    __syncthreads();
    int run = 0;
#pragma unroll
    for (int q = 0; q < RS_THREADS / 32; ++q) {
      const int c = wcnt[q][t];
      wcnt[q][t] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      const int pos = base_off[digit] + wcnt[w][digit] + lrank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    base_off[t] += run;
  }
  __syncthreads();
}

// Grid-wide barrier of a cooperative launch (count / generation in bar[0..1],
// count 0 on entry).  Gives up after `timeout` cycles or when another CTA
// reported an error.  Returns success.
__device__ bool rs_grid_barrier(int* bar, int* status, long long timeout) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile int* gen = bar + 1;
    const int g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1) == (int)gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1);
    } else {
      const long long t0 = clock64();
      for (unsigned it = 0; *gen == g0; ++it) {
        if ((it & 63u) == 63u && (dpv_status(status) || clock64() - t0 > timeout)) {
          if (!dpv_status(status)) dpv_set_status(status, DST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
    }
  }
  __syncthreads();
  return ok != 0;
}

// The passes of the stable LSD radix sort (8-bit digits, the low `bits` bits)
// inside a cooperative launch: per pass the tiles' histograms, the exclusive
// scan of the histogram (tile sums, the sums' scan in CTA 0, down-sweep) and
// the stable scatter, separated by grid barriers; CTAs stride over tiles.
// scratch: hist [256 nb], offs [256 nb + 1], sums [ns + 1].  Returns false
// when a barrier gave up (status set).
struct RsShared {
  int cnt[256];
  int wcnt[RS_THREADS / 32][256];
};

__device__ bool rs_passes(unsigned long long* k0, int* v0, unsigned long long* k1, int* v1, int M, int bits,
                          int* scratch, int* bar, int* status, long long timeout, RsShared& rs, int* sh) {
  const int nb = (M + RS_TILE - 1) / RS_TILE;
  const int nh = 256 * nb;
  const int ns = (nh + RS_SCAN_TILE - 1) / RS_SCAN_TILE;
  int* hist = scratch;
  int* offs = hist + nh;
  int* sums = offs + nh + 1;
  unsigned long long *kin = k0, *kout = k1;
  int *vin = v0, *vout = v1;
  for (int shift = 0; shift < bits; shift += 8) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) rs_hist_tile(kin, M, shift, hist, nb, t, rs.cnt);
    if (!rs_grid_barrier(bar, status, timeout)) return false;
    // tile sums of the histogram
    for (int t = blockIdx.x; t < ns; t += gridDim.x) {
      int v = 0;
#pragma unroll
      for (int r = 0; r < RS_SCAN_ITEMS; ++r) {
        const int idx = t * RS_SCAN_TILE + threadIdx.x * RS_SCAN_ITEMS + r;
        if (idx < nh) v += hist[idx];
      }
      int total;
      block_exclusive_scan(v, sh, total);
      if (threadIdx.x == 0) sums[t] = total;
    }
    if (!rs_grid_barrier(bar, status, timeout)) return false;
    if (blockIdx.x == 0) {
      const int per = (ns + RS_THREADS - 1) / RS_THREADS;
      const int lo = threadIdx.x * per, hi = min(ns, lo + per);
      int v = 0;
      for (int q = lo; q < hi; ++q) v += sums[q];
      int total;
      int run = block_exclusive_scan(v, sh, total);
      for (int q = lo; q < hi; ++q) {
        const int x = sums[q];
        sums[q] = run;
        run += x;
      }
    }
    if (!rs_grid_barrier(bar, status, timeout)) return false;
    // down-sweep: offs = exclusive scan of hist
    for (int t = blockIdx.x; t < ns; t += gridDim.x) {
      const int base = t * RS_SCAN_TILE + threadIdx.x * RS_SCAN_ITEMS;
      int v[RS_SCAN_ITEMS], sum = 0;
#pragma unroll
      for (int r = 0; r < RS_SCAN_ITEMS; ++r) {
        v[r] = (base + r < nh) ? hist[base + r] : 0;
        sum += v[r];
      }
      int total;
      int run = block_exclusive_scan(sum, sh, total) + sums[t];
#pragma unroll
      for (int r = 0; r < RS_SCAN_ITEMS; ++r) {
        if (base + r < nh) offs[base + r] = run;
        run += v[r];
      }
    }
    if (!rs_grid_barrier(bar, status, timeout)) return false;
    for (int t = blockIdx.x; t < nb; t += gridDim.x)
      rs_scatter_tile(kin, vin, kout, vout, M, shift, offs, nb, t, rs.cnt, rs.wcnt);
    if (!rs_grid_barrier(bar, status, timeout)) return false;
    unsigned long long* tk = kin;
    kin = kout;
    kout = tk;
    int* tv = vin;
    vin = vout;
    vout = tv;
  }
  return true;
}

// The whole sort in one cooperative launch.  Exits at once when run_if is
// given and *run_if is 0 (an input already in order), so that a sorted input
// costs one launch.
__global__ void __launch_bounds__(RS_THREADS) k_radix_sort(unsigned long long* k0, int* v0, unsigned long long* k1,
                                                           int* v1, int M, int bits, int* scratch, int* bar,
                                                           const int* run_if, int* status, long long timeout) {
  __shared__ RsShared rs;
  __shared__ int sh[32];
  if (run_if && !*run_if) return;
  if (dpv_status(status)) return;
  rs_passes(k0, v0, k1, v1, M, bits, scratch, bar, status, timeout, rs, sh);
}

// ---------------------------------------------------------------------------
// group and patch CSR over the patch-major (kk-sorted) order
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pm_edge(int s, const int* perm0, int unsorted) { return unsorted ? perm0[s] : s; }

// Position s of the patch-major order: the patches (kp, k] and the groups
// that start there begin at s (kp = the previous position's patch).
__device__ void bounds_edge(int s, int E, int P, int G, int ngroups, const int* __restrict__ kk,
                            const int* __restrict__ perm0, int uns, int* __restrict__ gptr, int* __restrict__ pptr) {
  const int k = kk[pm_edge(s, perm0, uns)];
  const int kp = s ? kk[pm_edge(s - 1, perm0, uns)] : -1;
  for (int q = kp + 1; q <= k; ++q) pptr[q] = s;
  for (int q = (kp < 0 ? 0 : kp / G + 1); q <= k / G; ++q)
    if (kp < 0 || q * G > kp) gptr[q] = s;
  if (s == E - 1) {
    for (int q = k + 1; q <= P; ++q) pptr[q] = E;
    for (int q = k / G + 1; q <= ngroups; ++q) gptr[q] = E;
  }
}

// bounds_edge on the input order, before it is known whether the input needs
// the kk sort: for a kk-sorted input it writes exactly what bounds_edge
// writes.  It skips positions with an invalid patch index (validation reports
// it) or a descending one (an unsorted input: bounds_edge runs again after
// the sort), and flags with bit 2 of *flag the positions that would write
// more than BOUNDS_SPAN entries (long runs of patches without edges), for
// the exact pass.
constexpr int BOUNDS_SPAN = 256;
__device__ void spec_bounds_edge(int s, int E, int P, int G, int ngroups, const int* __restrict__ kk,
                                 int* __restrict__ gptr, int* __restrict__ pptr, int* flag) {
  const int k = kk[s];
  const int kp = s ? kk[s - 1] : -1;
  if (k < 0 || k >= P || kp < -1 || kp >= P || kp > k) return;
  const int tail = s == E - 1 ? P - k : 0;
  if (k - kp > BOUNDS_SPAN || tail > BOUNDS_SPAN) {
    atomicOr(flag, 2);
    return;
  }
  bounds_edge(s, E, P, G, ngroups, kk, nullptr, 0, gptr, pptr);
}

// ---------------------------------------------------------------------------
// per group: window, slots, counting sort into (source, target) runs
// ---------------------------------------------------------------------------
constexpr int NBUCKET = DPV_WMAX * DPV_WMAX;
constexpr int GB_EDGES = 2048;  // a group of at most this many edges keeps them in shared memory
constexpr int GB_CNT_BITS = 18;  // the packed bucket scan: edge counts below, non-empty buckets above

struct GbShared {
  int bk[NBUCKET];          // bucket counts, then (scanned in place) each bucket's next position
  unsigned slot[GB_EDGES];  // per edge (group order): its frames (16 bits each), then its packed slot
  unsigned char kl[GB_EDGES];  // per edge: its patch within the group
};

// Group g by one CTA of 256 threads: the window (frames touched, as a bitmap
// over N frames and its prefix counts in smw), the (source slot, target slot)
// bucket counts over the window's W x W buckets, the run table and the stable
// placement of the group's edges into bucket order.  A group of at most
// GB_EDGES edges over at most 65,536 frames keeps its edges' frames and
// slots in shared memory, so that the edges are read from global memory once
// and the serial placement reads none.  Returns false (status set) when the
// window or the run count is too large; the result is uniform over the CTA.
__device__ bool group_build_one(int g, int N, int G, const int* __restrict__ gptr, const int* __restrict__ perm0,
                                int uns, const int* __restrict__ ii, const int* __restrict__ jj,
                                const int* __restrict__ kk, int* __restrict__ win, int* __restrict__ wlen,
                                int* __restrict__ perm, unsigned* __restrict__ eslot, int* __restrict__ pmpos,
                                int* __restrict__ grun, int* __restrict__ gnr, int* status, unsigned* smw,
                                GbShared& gb, int* sh) {
  const int nwords = (N + 31) >> 5;
  unsigned* bm = smw;
  int* wpre = (int*)(smw + nwords);
  const int s0 = gptr[g], s1 = gptr[g + 1];
  const bool keep = s1 - s0 <= GB_EDGES && N <= 65536;
  for (int q = threadIdx.x; q < nwords; q += blockDim.x) bm[q] = 0u;
  __syncthreads();
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const int e = pm_edge(s, perm0, uns);
    const int i = ii[e], j = jj[e];
    atomicOr(&bm[i >> 5], 1u << (i & 31));
    atomicOr(&bm[j >> 5], 1u << (j & 31));
    if (keep) {
      gb.slot[s - s0] = ((unsigned)i << 16) | (unsigned)j;
      gb.kl[s - s0] = (unsigned char)(kk[e] % G);
    }
  }
  __syncthreads();
  // the window: prefix counts of the bitmap words (one warp when they fit)
  int total;
  if (nwords <= 32) {
    if (threadIdx.x < 32) {
      const int c = threadIdx.x < nwords ? __popc(bm[threadIdx.x]) : 0;
      int x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)threadIdx.x >= o) x += y;
      }
      if ((int)threadIdx.x < nwords) wpre[threadIdx.x] = x - c;
      if (threadIdx.x == 31) sh[0] = x;
    }
    __syncthreads();
    total = sh[0];
  } else {
    const int per = (nwords + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(nwords, lo + per);
    int c = 0;
    for (int q = lo; q < hi; ++q) c += __popc(bm[q]);
    int run = block_exclusive_scan(c, sh, total);
    for (int q = lo; q < hi; ++q) {
      wpre[q] = run;
      run += __popc(bm[q]);
    }
  }
  if (total > DPV_WMAX) {
    if (threadIdx.x == 0) {
      wlen[g] = total;
      dpv_set_status(status, DST_WIDE);
    }
    return false;
  }
  const int W = total, W2 = W * W;
  for (int q = threadIdx.x; q < W2; q += blockDim.x) gb.bk[q] = 0;
  __syncthreads();  // wpre complete, the buckets cleared, sh free again
  for (int q = threadIdx.x; q < nwords; q += blockDim.x) {
    unsigned word = bm[q];
    int slot = wpre[q];
    while (word) {
      const int b = __ffs(word) - 1;
      win[g * DPV_WMAX + slot++] = (q << 5) + b;
      word &= word - 1;
    }
  }
  for (int q = W + threadIdx.x; q < DPV_WMAX; q += blockDim.x) win[g * DPV_WMAX + q] = -1;
  if (threadIdx.x == 0) wlen[g] = W;
  // bucket counts by (source slot, target slot); the packed slots kept
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    int i, j, k;
    if (keep) {
      const unsigned f = gb.slot[s - s0];
      i = (int)(f >> 16);
      j = (int)(f & 0xffffu);
      k = gb.kl[s - s0];
    } else {
      const int e = pm_edge(s, perm0, uns);
      i = ii[e];
      j = jj[e];
      k = kk[e] % G;
    }
    const int si = wpre[i >> 5] + __popc(bm[i >> 5] & ((1u << (i & 31)) - 1u));
    const int sj = wpre[j >> 5] + __popc(bm[j >> 5] & ((1u << (j & 31)) - 1u));
    atomicAdd(&gb.bk[si * W + sj], 1);
    if (keep) gb.slot[s - s0] = dpv_pack_slot(si, sj, k);
  }
  __syncthreads();
  // positions of the buckets (in place) and the run table (non-empty
  // buckets, in order): thread t owns buckets 16t .. 16t + 15 of the W^2
  {
    constexpr int PER = NBUCKET / 256;
    int v[PER], cnt = 0, nz = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int q = PER * threadIdx.x + r;
      v[r] = q < W2 ? gb.bk[q] : 0;
      cnt += v[r];
      nz += v[r] > 0;
    }
    int off, rid, tot, rtot;
    if (s1 - s0 < (1 << GB_CNT_BITS)) {  // one scan of (runs, edges) packed
      int t2;
      const int x = block_exclusive_scan((nz << GB_CNT_BITS) | cnt, sh, t2);
      off = x & ((1 << GB_CNT_BITS) - 1);
      rid = x >> GB_CNT_BITS;
      tot = t2 & ((1 << GB_CNT_BITS) - 1);
      rtot = t2 >> GB_CNT_BITS;
    } else {
      off = block_exclusive_scan(cnt, sh, tot);
      rid = block_exclusive_scan(nz, sh, rtot);
    }
    if (rtot > DPV_RMAX) {
      if (threadIdx.x == 0) dpv_set_status(status, DST_WIDE);
      return false;
    }
    int* gr = grun + (size_t)g * (DPV_RMAX + 1);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int q = PER * threadIdx.x + r;
      if (q < W2) gb.bk[q] = off;
      if (v[r] > 0) gr[rid++] = off;
      off += v[r];
    }
    if (threadIdx.x == 0) {
      gr[rtot] = tot;
      gnr[g] = rtot;
    }
  }
  __syncthreads();
  // stable placement (one warp walks the group in patch-major order; from
  // the kept slots when there are, so the serial walk reads no global memory
  // for a kk-sorted input)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    for (int b = s0; b < s1; b += 32) {
      const int s = b + lane;
      const bool valid = s < s1;
      int bucket = NBUCKET, e = 0;
      unsigned slot = 0u;
      if (valid) {
        e = pm_edge(s, perm0, uns);
        if (keep) {
          slot = gb.slot[s - s0];
        } else {
          const int i = ii[e], j = jj[e];
          const int si = wpre[i >> 5] + __popc(bm[i >> 5] & ((1u << (i & 31)) - 1u));
          const int sj = wpre[j >> 5] + __popc(bm[j >> 5] & ((1u << (j & 31)) - 1u));
          slot = dpv_pack_slot(si, sj, kk[e] % G);
        }
        bucket = dpv_slot_i(slot) * W + dpv_slot_j(slot);
      }
      const unsigned peers = __match_any_sync(0xffffffffu, bucket);
      const int rank = __popc(peers & lt);
      const int base = valid ? gb.bk[bucket] : 0;
      if (valid) {
        const int pos = s0 + base + rank;
        perm[pos] = e;
        eslot[pos] = slot;
        pmpos[pos] = s;
      }
      __syncwarp();
      if (valid && rank == 0) gb.bk[bucket] = base + __popc(peers);
      __syncwarp();
    }
  }
  __syncthreads();  // the next group of this CTA reuses the shared arrays
  return true;
}

// The binding as separate launches (graphs too large for one co-resident
// wave of the fused kernel): validation, the sort (k_radix_sort), the CSR
// bounds, then one CTA per group.
__global__ void k_validate(int E, int N, int P, const int* __restrict__ ii, const int* __restrict__ jj,
                           const int* __restrict__ kk, int* __restrict__ src, unsigned long long* __restrict__ keys,
                           int* __restrict__ vals, int* __restrict__ unsorted, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E) validate_edge(e, E, N, P, ii, jj, kk, src, keys, vals, unsorted, status);
}

__global__ void k_bounds(int E, int P, int G, int ngroups, const int* __restrict__ kk, const int* __restrict__ perm0,
                         const int* __restrict__ unsorted_p, int* __restrict__ gptr, int* __restrict__ pptr,
                         const int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= E || dpv_status(status)) return;
  bounds_edge(s, E, P, G, ngroups, kk, perm0, *unsorted_p, gptr, pptr);
}

__global__ void __launch_bounds__(256) k_group_build(
    int N, int G, const int* __restrict__ gptr, const int* __restrict__ perm0, const int* __restrict__ unsorted_p,
    const int* __restrict__ ii, const int* __restrict__ jj, const int* __restrict__ kk, int* __restrict__ win,
    int* __restrict__ wlen, int* __restrict__ perm, unsigned* __restrict__ eslot, int* __restrict__ pmpos,
    int* __restrict__ grun, int* __restrict__ gnr, int* status) {
  extern __shared__ unsigned smw[];
  __shared__ GbShared gb;
  __shared__ int sh[32];
  __shared__ int flag;
  if (threadIdx.x == 0) flag = dpv_status(status);
  __syncthreads();
  if (flag) return;
  group_build_one(blockIdx.x, N, G, gptr, perm0, *unsorted_p, ii, jj, kk, win, wlen, perm, eslot, pmpos, grun, gnr,
                  status, smw, gb, sh);
}

// The device status as one value for the whole CTA.
__device__ int cta_status(const int* status, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) *flag = dpv_status(status);
  __syncthreads();
  return *flag;
}

// What the binding's fused kernel accumulates into, cleared: the patch
// source table (-1), the "kk unsorted" flag and the grid barrier's words; for
// one bound problem also the frame and group problem tables (every frame and
// group in problem 0, the frame offsets {0, N} after the per-frame entries)
// and the device status, and the four intrinsics when intr_src (device
// memory) is given.
__global__ void k_bind_init(int P, int* __restrict__ src, int* __restrict__ unsorted, int* __restrict__ bar,
                            int single, int N, int* __restrict__ fprob, int Gn, int* __restrict__ gprob, int* status,
                            const float* __restrict__ intr_src, float* __restrict__ intr) {
  const int stride = gridDim.x * blockDim.x;
  const int q0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (intr_src && q0 < 4) intr[q0] = intr_src[q0];
  for (int q = q0; q < P; q += stride) src[q] = -1;
  if (q0 == 0) {
    *unsorted = 0;
    bar[0] = 0;
    bar[1] = 0;
  }
  if (!single) return;
  for (int q = q0; q <= N + 1; q += stride) fprob[q] = q <= N ? 0 : N;
  for (int q = q0; q < Gn; q += stride) gprob[q] = 0;
  if (q0 == 0) *status = 0;
}

// The whole binding of E > 0 edges in one cooperative launch of 256-thread
// CTAs, its phases separated by bounded grid barriers: validation and sort
// keys, with the group and patch CSR (gptr, pptr) written speculatively in
// input order; the stable sort by kk (only when the input is not kk-sorted;
// its result is in (k1, v1) after an odd number of 8-bit passes) and the
// exact CSR (only for an unsorted input or a flagged long gap); then every
// group's window, runs and edge order (CTAs stride over the groups).  k_bind_init runs first.  A failed phase leaves
// its code in the status and the later phases undone.  The sort's barriers
// take the handle's budget; the two between the phases stand where kernel
// boundaries stood, so they keep a floor of ~0.05 s (BIND_WAIT_MIN cycles):
// a short budget meant for the solvers' waits does not fail a binding.
constexpr long long BIND_WAIT_MIN = 100000000LL;

__global__ void __launch_bounds__(256) k_bind(int E, int N, int P, int G, int ngroups, const int* __restrict__ ii,
                                              const int* __restrict__ jj, const int* __restrict__ kk, int* src,
                                              unsigned long long* k0, int* v0, unsigned long long* k1, int* v1,
                                              int bits, int* scratch, int* bar, int* unsorted, int* gptr, int* pptr,
                                              int* win, int* wlen, int* perm, unsigned* eslot, int* pmpos, int* grun,
                                              int* gnr, int* status, long long timeout) {
  extern __shared__ unsigned smw[];
  __shared__ union {
    RsShared rs;
    GbShared gb;
  } u;
  __shared__ int sh[32];
  __shared__ int flag;
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
    validate_edge(e, E, N, P, ii, jj, kk, src, k0, v0, unsorted, status);
    spec_bounds_edge(e, E, P, G, ngroups, kk, gptr, pptr, unsorted);
  }
  const long long phase_timeout = timeout > BIND_WAIT_MIN ? timeout : BIND_WAIT_MIN;
  if (!rs_grid_barrier(bar, status, phase_timeout) || cta_status(status, &flag)) return;
  const int fl = *(volatile int*)unsorted;  // final after the barrier
  const int uns = fl & 1;
  if (uns && E > 1) {
    if (!rs_passes(k0, v0, k1, v1, E, bits, scratch, bar, status, timeout, u.rs, sh)) return;
  }
  const int* perm0 = ((bits + 7) / 8) & 1 ? v1 : v0;
  if (fl) {  // unsorted, or a long run of patches without edges: the exact bounds
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < E; s += stride)
      bounds_edge(s, E, P, G, ngroups, kk, perm0, uns, gptr, pptr);
    if (!rs_grid_barrier(bar, status, phase_timeout) || cta_status(status, &flag)) return;
  }
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x)
    if (!group_build_one(g, N, G, gptr, perm0, uns, ii, jj, kk, win, wlen, perm, eslot, pmpos, grun, gnr, status,
                         smw, u.gb, sh))
      return;
}

// block keys (inspection): three candidate keys per sorted edge, invalid ->
// ~0.  The edge's frames are read back from its group window and slots.
__global__ void k_key_candidates(int N, int fixed, const int* __restrict__ gptr, const unsigned* __restrict__ eslot,
                                 const int* __restrict__ win, unsigned long long* __restrict__ keys,
                                 int* __restrict__ vals) {
  const int g = blockIdx.x;
  for (int s = gptr[g] + threadIdx.x; s < gptr[g + 1]; s += blockDim.x) {
    const unsigned w = eslot[s];
    const int i = win[g * DPV_WMAX + dpv_slot_i(w)], j = win[g * DPV_WMAX + dpv_slot_j(w)];
    const int a[3] = {i, j, min(i, j)}, b[3] = {i, j, max(i, j)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const bool ok = (i != j) && a[q] >= fixed && b[q] >= fixed;
      keys[3 * (size_t)s + q] = ok ? (unsigned long long)a[q] * (unsigned)N + (unsigned)b[q] : ~0ull;
      vals[3 * (size_t)s + q] = 3 * s + q;
    }
  }
}

__global__ void k_key_unique_flags(int M, const unsigned long long* __restrict__ keys, int* __restrict__ flag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const unsigned long long k = keys[s];
  flag[s] = (k != ~0ull) && (s == 0 || keys[s - 1] != k);
}

__global__ void k_key_emit(int M, int N, const unsigned long long* __restrict__ keys, const int* __restrict__ flag,
                           const int* __restrict__ pos, int* __restrict__ out, int cap) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M || !flag[s]) return;
  const int p = pos[s];
  if (p < cap) {
    out[2 * p] = (int)(keys[s] / (unsigned)N);
    out[2 * p + 1] = (int)(keys[s] % (unsigned)N);
  }
}

// Sorts (k0, v0) by the low `bits` bits of the keys; `which` tells whether
// the result ended in (k0, v0) or (k1, v1).  scratch needs dpv_hist_entries(M)
// ints (its last two are the grid barrier's words).  One cooperative launch.
ba_status_t radix_sort(ba_handle_t h, unsigned long long* k0, int* v0, unsigned long long* k1, int* v1, int M,
                       int bits, int* scratch, int& which, const int* run_if = nullptr) {
  which = 0;
  if (M <= 1) return BA_OK;
  which = ((bits + 7) / 8) & 1;
  const int nb = (M + RS_TILE - 1) / RS_TILE;
  int* bar = scratch + dpv_hist_entries(M) - 2;
  static int per_sm = 0;  // co-resident CTAs per SM (queried by an eager run, never inside a graph capture)
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radix_sort, RS_THREADS, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 0;
      return dpv_fail(h, BA_ERR_CUDA, "radix sort occupancy");
    }
  }
  int grid = std::min(nb, per_sm * h->num_sms);
  DPV_CUDA(h, cudaMemsetAsync(bar, 0, 2 * sizeof(int), h->stream));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(RS_THREADS);
  cfg.stream = h->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  long long timeout = h->opt.timeout_cycles;
  int* status = h->ws->status;
  void* args[] = {(void*)&k0,      (void*)&v0,  (void*)&k1,     (void*)&v1,     (void*)&M,      (void*)&bits,
                  (void*)&scratch, (void*)&bar, (void*)&run_if, (void*)&status, (void*)&timeout};
  DPV_CUDA(h, cudaLaunchKernelExC(&cfg, (const void*)k_radix_sort, args));
  ++h->launches;
  return BA_OK;
}

// Co-resident k_bind CTAs per SM for `smem` bytes of dynamic shared memory,
// cached per size (the kernel's limit only ever rises): queried by the eager
// first run of a binding, so a later capture of the same binding finds it.
int bind_ctas_per_sm(size_t smem) {
  static std::mutex mu;  // handles may be bound from several host threads
  static std::map<size_t, int> cache;
  static size_t raised = 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(smem);
  if (it != cache.end()) return it->second;
  if (smem > raised) {
    if (cudaFuncSetAttribute(k_bind, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    raised = smem;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bind, 256, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cache[smem] = per_sm;
  return per_sm;
}

}  // namespace

long long dpv_scan_scratch(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 2; }
long long dpv_hist_entries(long long m) {
  const long long nh = 256 * ((m + RS_TILE - 1) / RS_TILE);
  // histogram, its exclusive scan (+ total), the scan's tile sums, two barrier words
  return 2 * nh + 1 + (nh + RS_SCAN_TILE - 1) / RS_SCAN_TILE + 1 + 2;
}

ba_status_t dpv_exclusive_scan(ba_handle_t h, const int* in, int* out, int n, const int* run_if) {
  Workspace* ws = h->ws;
  if (n <= 0) {
    DPV_CUDA(h, cudaMemsetAsync(out, 0, sizeof(int), h->stream));
    return BA_OK;
  }
  const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb + 1 > ws->scan.cap) return dpv_fail(h, BA_ERR_UNSUPPORTED, "scan larger than its scratch");
  k_scan_tiles<<<nb, SCAN_THREADS, 0, h->stream>>>(in, n, ws->scan.p, run_if);
  ++h->launches;
  k_scan_sums<<<1, SCAN_THREADS, 0, h->stream>>>(ws->scan.p, nb, run_if);
  ++h->launches;
  k_scan_down<<<nb, SCAN_THREADS, 0, h->stream>>>(in, n, ws->scan.p, out, run_if);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

ba_status_t dpv_preprocess(ba_handle_t h, const int* ii, const int* jj, const int* kk, int single,
                           const float* intr_src) {
  Workspace* ws = h->ws;
  const int E = h->E, N = h->N, P = h->P, G = h->G;
  cudaStream_t st = h->stream;
  const long long En = std::max(E, 1);
  int* bar = ws->hist.p + dpv_hist_entries(En) - 2;
  const int Gn = h->ngroups + 1;
  const int M = std::max(std::max(P, N + 2), Gn);
  k_bind_init<<<std::min((M + 255) / 256, 4 * h->num_sms), 256, 0, st>>>(P, ws->src.p, ws->unsorted, bar, single, N,
                                                                         ws->fprob.p, Gn, ws->gprob.p, ws->status,
                                                                         intr_src, ws->intr);
  ++h->launches;
  if (E == 0) {
    DPV_CUDA(h, cudaMemsetAsync(ws->gptr.p, 0, sizeof(int) * (h->ngroups + 1), st));
    DPV_CUDA(h, cudaMemsetAsync(ws->pptr.p, 0, sizeof(int) * (P + 1), st));
    DPV_CUDA(h, cudaMemsetAsync(ws->gnr.p, 0, sizeof(int) * h->ngroups, st));
    DPV_CUDA(h, cudaMemsetAsync(ws->wlen.p, 0, sizeof(int) * h->ngroups, st));
    DPV_CUDA(h, cudaGetLastError());
    return BA_OK;
  }
  const int nwords = (N + 31) / 32;
  const size_t smem = sizeof(unsigned) * nwords + sizeof(int) * nwords;
  if (smem > 160 * 1024) return dpv_fail(h, BA_ERR_UNSUPPORTED, "too many frames for the window kernel");
  const int per_sm = bind_ctas_per_sm(smem);
  if (per_sm < 1) return dpv_fail(h, BA_ERR_CUDA, "binding kernel occupancy");
  const int want = std::max(std::max((E + 255) / 256, h->ngroups), (E + RS_TILE - 1) / RS_TILE);
  if (want > per_sm * h->num_sms) {
    // more groups or edge blocks than one co-resident wave: separate launches
    // at full occupancy (the fused kernel would loop at a quarter of it)
    k_validate<<<(E + 255) / 256, 256, 0, st>>>(E, N, P, ii, jj, kk, ws->src.p, ws->keys0.p, ws->vals0.p,
                                                 ws->unsorted, ws->status);
    ++h->launches;
    int which = 0;
    ba_status_t s = radix_sort(h, ws->keys0.p, ws->vals0.p, ws->keys1.p, ws->vals1.p, E, h->kk_bits, ws->hist.p,
                               which, ws->unsorted);
    if (s) return s;
    const int* perm0 = which ? ws->vals1.p : ws->vals0.p;
    k_bounds<<<(E + 255) / 256, 256, 0, st>>>(E, P, G, h->ngroups, kk, perm0, ws->unsorted, ws->gptr.p, ws->pptr.p,
                                               ws->status);
    ++h->launches;
    static size_t smem_set = 0;  // raised once (not inside a graph capture of a later binding)
    if (smem > smem_set) {
      DPV_CUDA(h, cudaFuncSetAttribute(k_group_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      smem_set = smem;
    }
    k_group_build<<<h->ngroups, 256, smem, st>>>(N, G, ws->gptr.p, perm0, ws->unsorted, ii, jj, kk, ws->win.p,
                                                 ws->wlen.p, ws->perm.p, ws->eslot.p, ws->pmpos.p, ws->grun.p,
                                                 ws->gnr.p, ws->status);
    ++h->launches;
    DPV_CUDA(h, cudaGetLastError());
    return BA_OK;
  }
  const int grid = want;  // one wave: every group and edge block has its own CTA
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int bits = h->kk_bits, ngroups = h->ngroups;
  long long timeout = h->opt.timeout_cycles;
  int* scratch = ws->hist.p;
  void* args[] = {(void*)&E,          (void*)&N,          (void*)&P,          (void*)&G,
                  (void*)&ngroups,    (void*)&ii,         (void*)&jj,         (void*)&kk,
                  (void*)&ws->src.p,  (void*)&ws->keys0.p, (void*)&ws->vals0.p, (void*)&ws->keys1.p,
                  (void*)&ws->vals1.p, (void*)&bits,      (void*)&scratch,    (void*)&bar,
                  (void*)&ws->unsorted, (void*)&ws->gptr.p, (void*)&ws->pptr.p, (void*)&ws->win.p,
                  (void*)&ws->wlen.p, (void*)&ws->perm.p, (void*)&ws->eslot.p, (void*)&ws->pmpos.p,
                  (void*)&ws->grun.p, (void*)&ws->gnr.p,  (void*)&ws->status, (void*)&timeout};
  DPV_CUDA(h, cudaLaunchKernelExC(&cfg, (const void*)k_bind, args));
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}

ba_status_t dpv_block_keys(ba_handle_t h, int fixed, int* keys_out, int cap, int* n_out) {
  const int E = h->E, N = h->N;
  const long long M = 3LL * E;
  *n_out = 0;
  if (E == 0) return BA_OK;
  if (M > (1LL << 30)) return dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_debug_keys: graph too large");
  unsigned long long* kb[2] = {nullptr, nullptr};
  int* vb[2] = {nullptr, nullptr};
  int *flag = nullptr, *pos = nullptr, *scan = nullptr, *hist = nullptr;
  int* saved_scan = h->ws->scan.p;
  const long long saved_cap = h->ws->scan.cap;
  auto cleanup = [&]() {
    cudaFree(kb[0]); cudaFree(kb[1]); cudaFree(vb[0]); cudaFree(vb[1]);
    cudaFree(flag); cudaFree(pos); cudaFree(scan); cudaFree(hist);
    h->ws->scan.p = saved_scan;
    h->ws->scan.cap = saved_cap;
  };
  const long long hist_n = dpv_hist_entries(M);
  const long long scan_n = std::max(dpv_scan_scratch(M), dpv_scan_scratch(hist_n));
  if (cudaMalloc(&kb[0], 8 * M) || cudaMalloc(&kb[1], 8 * M) || cudaMalloc(&vb[0], 4 * M) ||
      cudaMalloc(&vb[1], 4 * M) || cudaMalloc(&flag, 4 * M) || cudaMalloc(&pos, 4 * (M + 1)) ||
      cudaMalloc(&scan, 4 * scan_n) || cudaMalloc(&hist, 4 * hist_n)) {
    cleanup();
    return dpv_fail(h, BA_ERR_OOM, "ba_debug_keys: allocation failed");
  }
  h->ws->scan.p = scan;
  h->ws->scan.cap = scan_n;
  k_key_candidates<<<h->ngroups, 256, 0, h->stream>>>(N, fixed, h->ws->gptr.p, h->ws->eslot.p, h->ws->win.p, kb[0],
                                                      vb[0]);
  ++h->launches;
  int which = 0;
  ba_status_t rc = radix_sort(h, kb[0], vb[0], kb[1], vb[1], (int)M, 64, hist, which);
  if (!rc) {
    k_key_unique_flags<<<(unsigned)((M + 255) / 256), 256, 0, h->stream>>>((int)M, kb[which], flag);
    ++h->launches;
    rc = dpv_exclusive_scan(h, flag, pos, (int)M);
  }
  if (!rc) {
    k_key_emit<<<(unsigned)((M + 255) / 256), 256, 0, h->stream>>>((int)M, N, kb[which], flag, pos, keys_out, cap);
    ++h->launches;
    int cnt = 0;
    if (cudaMemcpyAsync(&cnt, pos + M, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      rc = dpv_fail(h, BA_ERR_CUDA, "ba_debug_keys: copy failed");
    *n_out = cnt;
    if (!rc && cnt > cap) rc = dpv_fail(h, BA_ERR_INVALID_ARG, "ba_debug_keys: cap too small");
  }
  cleanup();
  return rc;
}
