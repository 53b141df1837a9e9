// Internal declarations of the dpvba library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/dpvba.h"

// ---------------------------------------------------------------------------
// limits of the kernels
// ---------------------------------------------------------------------------
#define DPV_WMAX 64          // frames in one group window (slots fit in 8 bits)
#define DPV_GMAX 64          // patches per group
#define DPV_GMAX_DD 32       // patches per group of the double-float (BA_MIXED) assembly
#define DPV_DENSE_MAX_ENTRIES (8LL << 20)  // dense pose-depth matrix of the dense form: n_pad x P entries at most
// BA_DENSE_AUTO takes the dense form up to this many edges: the measured
// crossover on B300 is below the smallest graph measured (8 keyframes, 5,376
// edges: 237 us dense vs 172 us block-sparse per two-iteration step, the
// block-sparse form ahead at every size up to 44 keyframes), so automatic
// selection keeps the block-sparse form
#define DPV_DENSE_AUTO_EDGES 0
#define DPV_SMALL_N 256      // pose systems up to this size use the one-CTA solver
#define DPV_TILE 64          // tile edge of the blocked pose system (large n)
#define DPV_RMAX 64          // (source, target) runs in one group

// device status codes (mirror ba_status_t)
#define DST_OK 0
#define DST_BAD_INDEX 1
#define DST_NOT_SPD 4
#define DST_TIMEOUT 5
#define DST_WIDE 7

struct Workspace;

// One independent pose system: its dense FP64 lower triangle at S + soff
// (tiles of TS x TS, T per dimension), its vectors (y, dx, ...) at voff with
// n_pad entries of which the first n are unknowns.
struct SysDesc {
  long long soff;
  int voff;
  int n;
  int n_pad;
  int TS;
  int T;
  int problem;
};

struct ba_handle_s {
  ba_options_t opt;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 148;
  std::string last_error;

  // bound graph (borrowed user buffers)
  int have_graph = 0;
  int N = 0, P = 0, E = 0;
  double* poses = nullptr;
  float* patches = nullptr;
  const float* targets = nullptr;
  const float* weights = nullptr;

  // grouping
  int G = 32;            // patches per group
  int ngroups = 0;
  int kk_bits = 0;      // bits of the patch index (width of the kk sort)

  // independent problems bound together (1 for ba_set_graph)
  int nprob = 1;
  std::vector<int> frame_off;   // [nprob + 1] first frame of each problem
  std::vector<int> patch_moff;  // [nprob + 1] first patch of each problem in the library's numbering
  std::vector<long long> user_patch_off;  // [nprob + 1] the caller's patch offsets
  int min_frames = 0;           // smallest problem (bound on fixed_poses)
  float* user_patches = nullptr;  // caller's patches when the library works on a padded copy
  int patches_padded = 0;

  // solver geometry for the last fixed value
  int fixed = -1;
  int n = 0;             // unknowns over all systems: sum of 6 (N_b - fixed)
  int TS = 0;            // tile edge (of system 0)
  int T = 0;             // tiles per dimension (of system 0)
  int n_pad = 0;         // length of the concatenated system vectors (sum of the padded sizes)
  long long nS = 0;      // FP64 entries of all system matrices
  std::vector<SysDesc> sys;       // per system
  std::vector<int> small_nq[9];   // systems solved by the one-CTA solver, by 32-row blocks
  std::vector<int> large_sys;     // systems solved by the persistent tiled solver
  int last_iters = 0;
  int last_dense = 0;   // the last ba_step ran the dense form

  Workspace* ws = nullptr;

  // event timing of kernel classes (ba_profile_enable, ba_profile_classes):
  // bit k set = launches of class k are bracketed by an event pair; 0 = off
  int prof_on = 0;
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  int prof_open = -1;
  // the records go on a side stream forked at each record point, so that the
  // kernels keep their programmatic dependencies on one another
  cudaStream_t prof_side = nullptr;
  cudaEvent_t prof_fork = nullptr;
  int prof_side_used = 0;  // a capture forked the side stream: join it before the capture ends

  long long launches = 0;  // kernels launched by this handle so far
  // side streams: the one-CTA solver launches of different block counts run
  // concurrently (fork from and join back to the handle's stream)
  cudaStream_t side[8] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[8] = {};

  // CUDA-graph replay of ba_step and of ba_set_graph's device work (ba_set_capture)
  int capture_on = 0;       // replay from captured graphs
  int capturing = 0;        // a capture is in progress: allocations and uploads are errors
  long long bind_gen = 0;   // bumped when the binding (pointers, sizes, offsets, group size) changes
  long long ws_gen = 0;     // bumped when a workspace buffer is reallocated
  std::vector<long long> bind_sig;
  struct GraphKey {
    long long bind_gen, ws_gen;
    int iters, fixed, prof;
    cudaStream_t stream;
  };
  struct CapGraph {
    GraphKey key{};
    int valid = 0;          // key describes this graph (or the eager run that precedes its capture)
    int failed = 0;         // capturing this key failed: run it eagerly
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;  // kernels in one replay
    std::vector<ProfRec> prof;  // event pairs recorded by every replay (profiling on)
    int pending = 0;            // a replay's events wait to be read
    long long captures = 0, replays = 0;
  };
  CapGraph step_graph, bind_graph;
  std::vector<ProfRec>* cap_prof = nullptr;  // where event records go while capturing
  cudaStream_t cap_stream = nullptr;         // private stream the captures run on
  double prof_ms[BA_KERNEL_CLASSES] = {};
  long long prof_n[BA_KERNEL_CLASSES] = {};

  // the arguments of the last binding (ba_autotune re-binds with other group sizes)
  struct Bind {
    int batched = 0;
    int B = 1, N = 0, P = 0, E = 0;
    std::vector<long long> frame_off, patch_off, edge_off;
    double* poses = nullptr;
    float* patches = nullptr;
    const int *ii = nullptr, *jj = nullptr, *kk = nullptr;
    const float *targets = nullptr, *weights = nullptr, *intrinsics = nullptr;
  } bind;

  // tape of the last recorded ba_step (ba_set_record / ba_backward)
  int record = 0;
  int tape_valid = 0;
  int tape_iters = 0;
  int tape_fixed = 0;
  int tape_iters_pending = 0;
};

// A device buffer owned by the handle, grown on demand (never shrunk).
template <class T>
struct DBuf {
  T* p = nullptr;
  long long cap = 0;
};

// device buffers, all owned by the handle
struct Workspace {
  int* status = nullptr;          // [1] first device-detected error
  float* intr = nullptr;          // [4 * intr_cap] intrinsics per problem
  int intr_cap = 1;
  double* cost = nullptr;         // [cost_cap] cost at each iteration's linearisation point
  int* unsorted = nullptr;        // [1] input kk not non-decreasing
  long long cost_cap = 0;
  // preprocessing
  DBuf<int> src;                  // [P] source frame of each patch, -1 none
  DBuf<unsigned long long> keys0, keys1;  // [E] sort keys
  DBuf<int> vals0, vals1;         // [E] sort values
  DBuf<int> hist;                 // radix histograms + their scan
  DBuf<int> perm;                 // [E] sorted position -> input edge
  DBuf<unsigned> eslot;           // [E] packed slots
  DBuf<int> gptr;                 // [groups+1] edge range of each group
  DBuf<int> grun;                 // [groups][RMAX+1] run starts relative to the group, then the group size
  DBuf<int> gnr;                  // [groups] runs per group
  DBuf<int> win;                  // [groups * DPV_WMAX] window frames
  DBuf<int> wlen;                 // [groups]
  DBuf<int> scan;                 // block sums of the scan
  DBuf<int> pmpos;                // [E] sorted position -> patch-major position
  DBuf<int> pptr;                 // [P+1] patch-major edge range of each patch
  DBuf<int> fprob;                // [N] problem of each frame
  DBuf<int> gprob;                // [groups] problem of each patch group
  DBuf<int> fdx;                  // [N] offset of the frame's 6 unknowns in the system vectors, -1 fixed
  DBuf<SysDesc> sysd;             // [systems]
  DBuf<int> syslist;              // system indices of the solver launches
  DBuf<int> mii, mjj, mkk;        // [E] edge indices in the library's numbering (bound problems)
  DBuf<long long> offs;           // [3 (nprob + 1)] frame, patch and edge offsets of the bound problems
  DBuf<float> pcopy;              // [P][27] padded patch copy (bound problems whose patch counts need padding)
  // per iteration
  DBuf<double> S;                 // tiled lower triangle of the pose system (FP64 accumulation)
  DBuf<double> y;                 // [n_pad]
  DBuf<double> dx;                // [n_pad]
  DBuf<float2> dx2;               // [n_pad] the step as double-float pairs (BA_MIXED back-substitution)
  DBuf<float> Ct, wk, dd;         // [P]
  DBuf<float2> Ct2, wk2;          // [P] Ct and w as double-float pairs (BA_MIXED)
  DBuf<double> dE;                // [P][n_pad] the dense form's pose-depth columns
  DBuf<double> dCw;               // [P][2] the dense form's C and w
  DBuf<float> posef;              // [N][16] R (9), camera centre hi (3), lo (3)
  DBuf<float4> pterm;             // [E][4] per-edge depth terms, patch-major (see assemble.cu);
                                  // [E][8] as double-float pairs with BA_MIXED (assemble_df.cu)
  // blocked solver
  DBuf<float> L;                  // factor (large n)
  DBuf<int> lg_sync;              // large solver: tile versions, row flags, task counter, grid barrier
  DBuf<long long> lg_prob;        // large solver: per-system descriptors
  DBuf<double> lg_red;            // large solver: conjugate-gradient dot products per (iteration, system)
  std::vector<unsigned char> lg_uploaded;  // host copy of what lg_prob and lg_rb hold
  DBuf<int> lg_rb;                // large solver: system of each global row block
  DBuf<unsigned long long> lg_live;  // large solver: the factorisation tasks inside the envelope (+ count)
  DBuf<double> r64;               // [n_pad]
  DBuf<float> tmpv;               // [n_pad]
  // tape of a recorded ba_step: states before each iteration (+ the final poses) and the steps
  DBuf<double> tp_poses;          // [iters+1][N][7]
  DBuf<float> tp_patches;         // [iters][P][27]
  DBuf<double> tp_dx;             // [iters][n]
  DBuf<float> tp_dd;              // [iters][P]
  // adjoint pass
  DBuf<double> ad_xb;             // [2][N][6] pose cotangents (tangent space), double-buffered
  DBuf<float> ad_w;               // [2][P] depth cotangents that pass the clamp, double-buffered
  DBuf<float> ad_gd;              // [E] per-edge depth cotangents, patch-major
  DBuf<unsigned char> prox;       // ba_proximity_edges scratch (counters, CTA flags, centres, transforms)
  long long prox_blocks = 0, prox_frames = 0;  // what its layout holds
  DBuf<int> corr;                 // ba_patch_correlation: frame histogram, cursors, edge order
  DBuf<double> pgo;               // ba_pgo_lm: LM state (3), candidate similarities [N][8], factor costs [F]
  DBuf<float> ad_lamd;            // [P] depth part of the adjoint solve
  DBuf<double> ad_v;              // [n_pad] pose part of the adjoint right-hand side
  DBuf<float> ad_gt, ad_gw;       // [E][2] scratch when the caller passes no output
};

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
ba_status_t dpv_fail(ba_handle_t h, ba_status_t s, const std::string& msg);

// grow a handle-owned device buffer to at least `need` elements (contents not kept)
template <class T>
ba_status_t dpv_grow(ba_handle_t h, DBuf<T>& b, long long need, const char* what) {
  need = need < 1 ? 1 : need;
  if (need <= b.cap && b.p) return BA_OK;
  if (h->capturing) return dpv_fail(h, BA_ERR_STATE, std::string("allocating ") + what + " during graph capture");
  ++h->ws_gen;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  cudaError_t e = cudaMalloc((void**)&b.p, sizeof(T) * (size_t)need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return dpv_fail(h, BA_ERR_OOM, std::string("allocating ") + what + ": " + cudaGetErrorString(e));
  }
  b.cap = need;
  return BA_OK;
}
#define DPV_CUDA(h, call)                                                              \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess)                                                             \
      return dpv_fail((h), _e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, \
                      std::string(#call) + ": " + cudaGetErrorString(_e));             \
  } while (0)

// group size recorded by ba_autotune for this shape class (0: none)
int dpv_tuned_group(ba_handle_t h, long long P, long long E, int batched);

// event timing around a kernel class (no-ops unless profiling is enabled)
void dpv_prof_begin(ba_handle_t h, int kind);
void dpv_prof_end(ba_handle_t h);
void dpv_prof_join(ba_handle_t h);

// preprocessing (preprocess.cu)
ba_status_t dpv_preprocess(ba_handle_t h, const int* ii, const int* jj, const int* kk, int single,
                           const float* intr_src);
ba_status_t dpv_block_keys(ba_handle_t h, int fixed, int* keys_out, int cap, int* n_out);
// out has n+1 entries; when run_if is given the kernels do nothing unless *run_if != 0
ba_status_t dpv_exclusive_scan(ba_handle_t h, const int* in, int* out, int n, const int* run_if = nullptr);
long long dpv_scan_scratch(long long n);
long long dpv_hist_entries(long long m);
// one GN iteration (assemble.cu, solve_*.cu, update.cu)
// skip_init: S, y and the pose table are already prepared (the one-CTA solver
// of the previous iteration re-zeroed S and y, the retraction refreshed the table)
ba_status_t dpv_assemble(ba_handle_t h, int it, int skip_init);
ba_status_t dpv_assemble_ext(ba_handle_t h, int it, const double* v_ext, const float* w_ext);
ba_status_t dpv_assemble_dd(ba_handle_t h, double* cost, const float* w_ext);  // assemble_df.cu
bool dpv_use_dense(ba_handle_t h);                       // dense.cu: the dense form for the next iterations
ba_status_t dpv_dense_assemble(ba_handle_t h, double* cost);
ba_status_t dpv_dense_backsub(ba_handle_t h);
// largest patches-per-group the handle's assembly kernel supports
inline int dpv_max_group(ba_handle_t h) { return h->opt.precision == BA_MIXED ? DPV_GMAX_DD : DPV_GMAX; }
// The solvers stop once the estimated error left in the pose step is below
// this fraction of it: 1e-7 with the FP32 linearisation, 1e-10 with the
// double-float one (BA_MIXED), whose steps are compared with an FP64
// solution on ill-conditioned loop-closure systems (a 1e-7 error of the step
// there moves near-clamp inverse depths by ~2e-5, relative).
inline float dpv_solve_tol(ba_handle_t h) { return h->opt.precision == BA_MIXED ? 1e-10f : 1e-7f; }
// pterm float4 per edge for the handle's precision
inline int dpv_pterm_width(ba_handle_t h) { return h->opt.precision == BA_MIXED ? 8 : 4; }
ba_status_t dpv_ensure_system(ba_handle_t h, int fixed);
ba_status_t dpv_ensure_generic_system(ba_handle_t h, int n);  // one dense system of n unknowns
ba_status_t dpv_tape_reserve(ba_handle_t h, int iters);
ba_status_t dpv_tape_state(ba_handle_t h, int it);
ba_status_t dpv_tape_step(ba_handle_t h, int it);
ba_status_t dpv_backsub_ext(ba_handle_t h, const float* w_ext, float* out);
ba_status_t dpv_solve(ba_handle_t h, int* retracted, int reset_system = 0);
ba_status_t dpv_backsub(ba_handle_t h, int retract);  // retract: also update the poses
ba_status_t dpv_export_S(ba_handle_t h, double* dst);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dpv_set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Programmatic dependent launch between the kernels of a step: a kernel
// launched by dpv_launch_pdl may become resident while its predecessor in the
// stream still runs; its first statement, dpv_pdl_enter(), waits until the
// predecessor has completed and its writes are visible (a no-op when the
// kernel was launched without the attribute), then lets its own successor
// launch.  Only the launch latency overlaps; no data is read early.
__device__ __forceinline__ void dpv_pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t dpv_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
__device__ __forceinline__ int dpv_status(const int* status) { return *(volatile const int*)status; }

// Tiled lower-triangular storage of the pose system: tile (ti, tj), ti >= tj,
// is a TS x TS row-major block at offset (ti (ti+1)/2 + tj) TS^2.
__host__ __device__ __forceinline__ size_t dpv_tile_base(int ti, int tj, int TS) {
  return ((size_t)ti * (ti + 1) / 2 + tj) * (size_t)TS * TS;
}
__host__ __device__ __forceinline__ size_t dpv_s_index(int r, int c, int TS) {
  const int ti = r / TS, tj = c / TS;
  return dpv_tile_base(ti, tj, TS) + (size_t)(r - ti * TS) * TS + (c - tj * TS);
}

__device__ __forceinline__ void dpv_red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void dpv_red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// The float as an FP64 value, built with integer operations: B300 runs FP64
// arithmetic (conversions included) at ~1/64 of the FP32 rate, and the
// assembly converts several values per thread for its FP64 reductions.  Exact for normal
// floats; subnormals (|v| < 1.2e-38) become signed zero; inf/NaN stay inf/NaN.
__device__ __forceinline__ double dpv_f2d_bits(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned long long d = (unsigned long long)(u >> 31) << 63;
  if (e != 0) {
    const unsigned long long E = e == 255u ? 2047ull : (unsigned long long)(e + 896u);
    d |= (E << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  }
  return __longlong_as_double((long long)d);
}

// The double rounded to the nearest float (ties to even) with integer
// operations, for the same reason.  |v| below 2^-126 gives signed zero,
// above the float range infinity; NaN stays NaN.
__device__ __forceinline__ float dpv_d2f_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ed = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  const int e = ed - 1023 + 127;
  if (ed == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned mant = (unsigned)(m >> 29);
  const unsigned long long rest = m & 0x1fffffffull;
  unsigned r = ((unsigned)e << 23) | mant;
  if (rest > 0x10000000ull || (rest == 0x10000000ull && (mant & 1u))) r += 1u;  // may carry to infinity
  return __uint_as_float(sign | r);
}

// The double as a pair of floats, v = hi + lo up to 2^-48 |v|: hi is v
// rounded to float, lo the rest rounded to float, with integer operations
// (lo is 0 when v is out of the float range or the rest would underflow).
__device__ __forceinline__ float2 dpv_d2df_bits(double v) {
  const float hi = dpv_d2f_bits(v);
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ed = (int)((b >> 52) & 0x7ff);
  const int e = ed - 1023 + 127;
  // the rest is a multiple of 2^(ed - 1075): a normal float scale needs
  // 1 <= ed - 948 <= 254
  if (ed == 0x7ff || e <= 0 || e >= 255 || ed < 949 || ed > 1202) return make_float2(hi, 0.f);
  const unsigned long long m = b & 0xfffffffffffffull;
  const unsigned mant = (unsigned)(m >> 29);
  const long long rest = (long long)(m & 0x1fffffffull);
  const bool up = rest > 0x10000000ll || (rest == 0x10000000ll && (mant & 1u));
  const long long d = up ? rest - 0x20000000ll : rest;  // |v| - |hi| in units of 2^(ed - 1075), |d| <= 2^28
  float lo = __ll2float_rn(d) * __int_as_float((ed - 948) << 23);
  if (b >> 63) lo = -lo;
  return make_float2(hi, lo);
}

// rotation matrix of a unit quaternion (x, y, z, w), FP64
__device__ __forceinline__ void dpv_quat_rot64(const double* q, double* R) {
  const double x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - z * w); R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w); R[7] = 2.0 * (y * z + x * w); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// One row of the per-pose table used by the linearisation (DPV_POSE_ROW
// floats): R as double-float pairs (hi 9, lo 9) and the camera centre
// c = -R^T t as pairs (hi 3, lo 3), formed in FP64 from the FP64 pose (t, q).
#define DPV_POSE_ROW 32
__device__ __forceinline__ void dpv_pose_table_row(const double* __restrict__ p, float* __restrict__ o) {
  double R[9];
  dpv_quat_rot64(p + 3, R);
#pragma unroll
  for (int m = 0; m < 9; ++m) {
    const float hi = dpv_d2f_bits(R[m]);
    o[m] = hi;
    o[9 + m] = dpv_d2f_bits(R[m] - dpv_f2d_bits(hi));
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double c = -(R[m] * p[0] + R[3 + m] * p[1] + R[6 + m] * p[2]);
    const float hi = dpv_d2f_bits(c);
    o[18 + m] = hi;
    o[21 + m] = dpv_d2f_bits(c - dpv_f2d_bits(hi));
  }
}

struct RelPose {
  float R[9], t[3], txR[9];  // rotation, translation, [t]x R (translation-rotation block of Ad)
};


// Per-edge linearisation of Eq. 3 at the patch centre (FP32).
//   X = R xb + t d  (xb = ((u-cx)/fx, (v-cy)/fy, 1), homogeneous 4th entry d)
//   proj = (fx X/Z + cx, fy Y/Z + cy),  r = target - proj
//   Jj = dproj/dX [ d I | -[X]x ],  Ji = -Jj Ad(T_ij),  Jd = dproj/dX t
struct EdgeLin {
  float r[2];
  float Ji[2][6], Jj[2][6], Jd[2];
  bool valid;
};

__device__ __forceinline__ void dpv_edge_linearize(const RelPose& T, float xb0, float xb1, float d, float tu,
                                                   float tv, const float* K, float z_min, bool self_edge,
                                                   EdgeLin& o) {
  const float X = fmaf(T.R[0], xb0, fmaf(T.R[1], xb1, fmaf(T.t[0], d, T.R[2])));
  const float Y = fmaf(T.R[3], xb0, fmaf(T.R[4], xb1, fmaf(T.t[1], d, T.R[5])));
  const float Z = fmaf(T.R[6], xb0, fmaf(T.R[7], xb1, fmaf(T.t[2], d, T.R[8])));
  o.valid = !self_edge && (Z > z_min * d);
  const float iz = 1.0f / Z;
  const float fx = K[0], fy = K[1];
  o.r[0] = tu - fmaf(fx * X, iz, K[2]);
  o.r[1] = tv - fmaf(fy * Y, iz, K[3]);
  const float a0 = fx * iz, a2 = -fx * X * iz * iz;
  const float b1 = fy * iz, b2 = -fy * Y * iz * iz;
  o.Jj[0][0] = a0 * d; o.Jj[0][1] = 0.f; o.Jj[0][2] = a2 * d;
  o.Jj[0][3] = a2 * Y; o.Jj[0][4] = a0 * Z - a2 * X; o.Jj[0][5] = -a0 * Y;
  o.Jj[1][0] = 0.f; o.Jj[1][1] = b1 * d; o.Jj[1][2] = b2 * d;
  o.Jj[1][3] = -b1 * Z + b2 * Y; o.Jj[1][4] = -b2 * X; o.Jj[1][5] = b1 * X;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float jr = o.Jj[a][0] * T.R[c] + o.Jj[a][1] * T.R[3 + c] + o.Jj[a][2] * T.R[6 + c];
      const float jt = o.Jj[a][0] * T.txR[c] + o.Jj[a][1] * T.txR[3 + c] + o.Jj[a][2] * T.txR[6 + c] +
                       o.Jj[a][3] * T.R[c] + o.Jj[a][4] * T.R[3 + c] + o.Jj[a][5] * T.R[6 + c];
      o.Ji[a][c] = -jr;
      o.Ji[a][3 + c] = -jt;
    }
  }
  o.Jd[0] = a0 * T.t[0] + a2 * T.t[2];
  o.Jd[1] = b1 * T.t[1] + b2 * T.t[2];
}

// ---------------------------------------------------------------------------
// compensated FP32 accumulation ("double-float"): value = hi + lo.
// TwoSum gives the exact rounding error of a sum; fma(a, b, -p) gives the
// exact rounding error of a product, so acc += a*b keeps ~44 bits.
// ---------------------------------------------------------------------------
struct DF {
  float hi, lo;
};
// The explicit _rn intrinsics keep the compiler from contracting a product
// into the following sum, which would break the error terms.
__device__ __forceinline__ void df_add(DF& a, float b) {
  const float s = __fadd_rn(a.hi, b);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}
__device__ __forceinline__ void df_fma(DF& a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);
  df_add(a, p);
  a.lo = __fadd_rn(a.lo, pe);
}
__device__ __forceinline__ void df_add_df(DF& a, const DF& b) {
  df_add(a, b.hi);
  a.lo = __fadd_rn(a.lo, b.lo);
}
__device__ __forceinline__ float df_val(const DF& a) { return a.hi + a.lo; }

// Kahan-compensated FP32 accumulation of products: value = s - c.  The
// product is fused into the compensation step (one rounding), so one term
// costs 4 operations instead of the 10 of df_fma; the error stays
// 2u sum|x| + O(n u^2) sum|x| (Kahan's bound), independent of the term count.
struct KS {
  float s, c;
};
__device__ __forceinline__ void ks_fma(KS& a, float x, float y) {
  const float yv = __fmaf_rn(x, y, -a.c);
  const float t = __fadd_rn(a.s, yv);
  a.c = __fsub_rn(__fsub_rn(t, a.s), yv);
  a.s = t;
}
__device__ __forceinline__ DF ks_df(const KS& a) { return DF{a.s, -a.c}; }

// Relative pose T_ij = T_j T_i^-1 from two rows of the pose table, in
// double-float arithmetic on the FP32 pipe and rounded once to FP32 (as
// accurate as forming it in FP64 from the FP64 poses, at a fraction of the
// cost; FP32 products of FP32-rounded rotations cost ~1e-5 of the step on
// ill-conditioned systems):  R = R_j R_i^T,  t = R_j (c_i - c_j).
__device__ __forceinline__ float dpv_dot3_df(const float* ah, const float* al, int as, const float* bh,
                                             const float* bl, int bs) {
  DF acc = {0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a = ah[k * as], b = bh[k * bs];
    df_fma(acc, a, b);
    acc.lo = __fmaf_rn(a, bl[k * bs], __fmaf_rn(al[k * as], b, acc.lo));
  }
  return acc.hi + acc.lo;
}
__device__ __forceinline__ void dpv_relative_pose_df(const float* Pi, const float* Pj, RelPose& o) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      o.R[3 * r + c] = dpv_dot3_df(Pj + 3 * r, Pj + 9 + 3 * r, 1, Pi + 3 * c, Pi + 9 + 3 * c, 1);
  float dh[3], dl[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {  // c_i - c_j as a pair
    DF d = {Pi[18 + m], 0.f};
    df_add(d, -Pj[18 + m]);
    d.lo = __fadd_rn(d.lo, __fsub_rn(Pi[21 + m], Pj[21 + m]));
    dh[m] = d.hi;
    dl[m] = d.lo;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) o.t[r] = dpv_dot3_df(Pj + 3 * r, Pj + 9 + 3 * r, 1, dh, dl, 1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.txR[0 + c] = -o.t[2] * o.R[3 + c] + o.t[1] * o.R[6 + c];
    o.txR[3 + c] = o.t[2] * o.R[0 + c] - o.t[0] * o.R[6 + c];
    o.txR[6 + c] = -o.t[1] * o.R[0 + c] + o.t[0] * o.R[3 + c];
  }
}

// packed per-edge slot word
__host__ __device__ __forceinline__ unsigned dpv_pack_slot(int si, int sj, int kl) {
  return (unsigned)si | ((unsigned)sj << 8) | ((unsigned)kl << 16);
}
__host__ __device__ __forceinline__ int dpv_slot_i(unsigned w) { return (int)(w & 0xff); }
__host__ __device__ __forceinline__ int dpv_slot_j(unsigned w) { return (int)((w >> 8) & 0xff); }
__host__ __device__ __forceinline__ int dpv_slot_k(unsigned w) { return (int)(w >> 16); }
