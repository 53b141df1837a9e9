// C ABI of the library (declared in include/dpvba.h).
#include "internal.cuh"

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

size_t dpv_assemble_smem(int G);

ba_status_t dpv_fail(ba_handle_t h, ba_status_t s, const std::string& msg) {
  if (h) h->last_error = std::string(ba_status_string(s)) + ": " + msg;
  return s;
}

static cudaEvent_t pool_event(ba_handle_t h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Record e once the work enqueued so far on the handle's stream is done, on
// the profiling side stream forked at this point: the next kernel on the
// handle's stream keeps its programmatic dependency on the previous one (an
// event record between them would serialise the pair).  While a step is
// captured the record is an event-record node on a side branch of the graph
// (every replay records it again; see prof_harvest).
static void prof_record(ba_handle_t h, cudaEvent_t e) {
  const unsigned flags = h->capturing ? cudaEventRecordExternal : 0u;
  if (!h->prof_side || !h->prof_fork) {
    cudaEventRecordWithFlags(e, h->stream, flags);
    return;
  }
  cudaEventRecord(h->prof_fork, h->stream);
  cudaStreamWaitEvent(h->prof_side, h->prof_fork, 0);
  cudaEventRecordWithFlags(e, h->prof_side, flags);
  if (h->capturing) h->prof_side_used = 1;
}

void dpv_prof_begin(ba_handle_t h, int kind) {
  if (!((h->prof_on >> kind) & 1)) return;
  cudaEvent_t a = pool_event(h), b = pool_event(h);
  if (!a || !b) return;
  std::vector<ba_handle_s::ProfRec>& list = h->capturing ? *h->cap_prof : h->prof;
  prof_record(h, a);
  list.push_back({kind, a, b});
  h->prof_open = (int)list.size() - 1;
}

void dpv_prof_end(ba_handle_t h) {
  if (!h->prof_on || h->prof_open < 0) return;
  prof_record(h, h->capturing ? (*h->cap_prof)[h->prof_open].b : h->prof[h->prof_open].b);
  h->prof_open = -1;
}

// A capture that forked the profiling side stream joins it back into the
// captured stream (a capture must end with every forked stream joined).
void dpv_prof_join(ba_handle_t h) {
  if (!h->prof_side_used) return;
  cudaEventRecord(h->prof_fork, h->prof_side);
  cudaStreamWaitEvent(h->stream, h->prof_fork, 0);
  h->prof_side_used = 0;
}

static void prof_release(ba_handle_t h, std::vector<ba_handle_s::ProfRec>& list) {
  for (auto& r : list) {
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  list.clear();
}

// Add the event times of a graph's last replay to the totals (waits for that replay).
static ba_status_t prof_harvest(ba_handle_t h, ba_handle_s::CapGraph& g) {
  if (!g.pending) return BA_OK;
  g.pending = 0;
  if (g.prof.empty()) return BA_OK;
  DPV_CUDA(h, cudaEventSynchronize(g.prof.back().b));
  for (auto& r : g.prof) {
    float ms = 0.f;
    DPV_CUDA(h, cudaEventElapsedTime(&ms, r.a, r.b));
    h->prof_ms[r.kind] += ms;
    ++h->prof_n[r.kind];
  }
  return BA_OK;
}

static ba_status_t prof_harvest_all(ba_handle_t h) {
  ba_status_t s = prof_harvest(h, h->bind_graph);
  if (!s) s = prof_harvest(h, h->step_graph);
  return s;
}

static void prof_clear(ba_handle_t h) {
  prof_release(h, h->prof);
  h->prof_open = -1;
  h->step_graph.pending = 0;
  h->bind_graph.pending = 0;
  for (int k = 0; k < BA_KERNEL_CLASSES; ++k) {
    h->prof_ms[k] = 0.0;
    h->prof_n[k] = 0;
  }
}

static void graph_drop(ba_handle_t h, ba_handle_s::CapGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.pending = 0;
  prof_release(h, g.prof);
  g.valid = 0;
  g.failed = 0;
}

static bool same_key(const ba_handle_s::GraphKey& a, const ba_handle_s::GraphKey& b) {
  return a.bind_gen == b.bind_gen && a.ws_gen == b.ws_gen && a.iters == b.iters && a.fixed == b.fixed &&
         a.prof == b.prof && a.stream == b.stream;
}

// Run `body` (work enqueued on h->stream) through the captured graph g.  The
// graph holds pointers and sizes, so it is keyed (binding, workspace
// allocation, iteration count, fixed poses, profiling, stream).  The first
// call of a key runs eagerly (it sizes the workspace and uploads tables,
// which a capture may not do); the second captures the body on a private
// stream; later calls launch the graph on the handle's stream.  A body that
// cannot be captured keeps running eagerly for that key.
template <class Body>
static ba_status_t graph_run(ba_handle_t h, ba_handle_s::CapGraph& g, const ba_handle_s::GraphKey& key, Body body) {
  ba_status_t s;
  if (!g.valid || !same_key(g.key, key)) {
    if (g.exec || g.pending) {  // the old graph may still run: finish it first
      DPV_CUDA(h, cudaStreamSynchronize(h->stream));
      if ((s = prof_harvest(h, g))) return s;
    }
    graph_drop(h, g);
    g.key = key;
    g.valid = 1;
    return body();
  }
  if (!g.exec) {
    if (g.failed) return body();
    if (!h->cap_stream) DPV_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t user = h->stream;
    const long long l0 = h->launches;
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    s = BA_OK;
    h->stream = h->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      h->capturing = 1;
      h->cap_prof = &g.prof;
      h->prof_side_used = 0;
      s = body();
      dpv_prof_join(h);
      h->capturing = 0;
      h->cap_prof = nullptr;
      e = cudaStreamEndCapture(h->cap_stream, &gr);
    }
    h->stream = user;
    if (e == cudaSuccess && s == BA_OK && gr) e = cudaGraphInstantiate(&ex, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess || s != BA_OK || !ex) {
      cudaGetLastError();
      prof_release(h, g.prof);
      h->prof_open = -1;
      h->launches = l0;
      g.failed = 1;
      return body();
    }
    g.exec = ex;
    g.kernels = h->launches - l0;
    h->launches = l0;
    ++g.captures;
  }
  // the previous replay's event times are read before the events are recorded again
  if ((s = prof_harvest(h, g))) return s;
  DPV_CUDA(h, cudaGraphLaunch(g.exec, h->stream));
  h->launches += g.kernels;
  ++g.replays;
  g.pending = g.prof.empty() ? 0 : 1;
  return BA_OK;
}

// Record the binding's signature; a change invalidates the captured step.
static void bind_signature(ba_handle_t h, std::vector<long long> sig) {
  if (sig != h->bind_sig) {
    h->bind_sig = std::move(sig);
    ++h->bind_gen;
  }
}

long long dpv_large_scratch_floats(int n_pad);
ba_status_t dpv_large_reserve(ba_handle_t h);
ba_status_t dpv_large_envelope(ba_handle_t h, int* out, long long cap, long long* count);

namespace {

template <class T>
void release(DBuf<T>& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

int bits_for(unsigned long long x) {
  int b = 0;
  while (b < 64 && (x >> b)) ++b;
  return b;
}

// pose-system geometry for a given number of free poses
void system_geometry(int n, int& TS, int& T, int& n_pad) {
  if (n <= DPV_SMALL_N) {
    n_pad = std::max(32, (n + 31) / 32 * 32);
    TS = n_pad;
    T = 1;
  } else {
    TS = DPV_TILE;
    T = (n + TS - 1) / TS;
    n_pad = T * TS;
  }
}

int auto_group(ba_handle_t h, long long P, long long E, int batched) {
  // a size measured by ba_autotune for this shape class
  const int tuned = dpv_tuned_group(h, P, E, batched);
  if (tuned > 0) return std::min(tuned, dpv_max_group(h));
  // large graphs: 32 patches per group; small ones: keep about one group
  // per SM or more (measured on the 22-frame odometry window: 16 best)
  if ((long long)P >= 32LL * 2 * h->num_sms) return 32;
  if ((long long)P >= 8LL * h->num_sms) return 16;
  return 8;
}

// problem of index x for non-decreasing offsets off[0..B] (largest b with off[b] <= x)
__device__ __forceinline__ int find_problem(const long long* off, int B, long long x) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Edge indices of bound problems -> the library's numbering: frames offset by
// the problem's first frame, patches by its (group-aligned) first patch.  Local
// indices out of range become -1, which validation reports.
__global__ void k_remap_edges(int E, int B, const long long* __restrict__ offs, const int* __restrict__ ii,
                              const int* __restrict__ jj, const int* __restrict__ kk, int* __restrict__ mii,
                              int* __restrict__ mjj, int* __restrict__ mkk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const long long* foff = offs;
  const long long* moff = offs + (B + 1);
  const long long* eoff = offs + 2 * (B + 1);
  const long long* poff = offs + 3 * (B + 1);
  const int b = find_problem(eoff, B, e);
  const int nf = (int)(foff[b + 1] - foff[b]), np = (int)(poff[b + 1] - poff[b]);
  const int i = ii[e], j = jj[e], k = kk[e];
  mii[e] = (i >= 0 && i < nf) ? (int)foff[b] + i : -1;
  mjj[e] = (j >= 0 && j < nf) ? (int)foff[b] + j : -1;
  mkk[e] = (k >= 0 && k < np) ? (int)moff[b] + k : -1;
}

__global__ void k_frame_problems(int N, int B, const long long* __restrict__ offs, int* __restrict__ fprob) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < N) fprob[f] = find_problem(offs, B, f);
}

// padded copy <-> caller's patches (to_copy: caller -> copy, zero padding)
__global__ void k_patch_copy(int Ppad, int B, const long long* __restrict__ offs, float* __restrict__ user,
                             float* __restrict__ copy, int to_copy) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 27LL * Ppad) return;
  const int km = (int)(q / 27), c = (int)(q % 27);
  const long long* moff = offs + (B + 1);
  const long long* poff = offs + 3 * (B + 1);
  const int b = find_problem(moff, B, km);
  const long long k = km - moff[b];
  const bool real = k < poff[b + 1] - poff[b];
  if (to_copy) copy[q] = real ? user[27 * (poff[b] + k) + c] : 0.f;
  else if (real) user[27 * (poff[b] + k) + c] = copy[q];
}

// fdx[f]: offset of frame f's six unknowns in the concatenated system vectors,
// -1 for the first `fixed` frames of each problem
__global__ void k_build_fdx(int N, int fixed, const int* __restrict__ fprob, const int* __restrict__ frame_off,
                            const SysDesc* __restrict__ sysd, int* __restrict__ fdx) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= N) return;
  const int b = fprob[f];
  const int lf = f - frame_off[b];
  fdx[f] = lf < fixed ? -1 : sysd[b].voff + 6 * (lf - fixed);
}

// Per-problem pose systems for a fixed-pose count: geometry, storage and the
// frame -> unknown map.
ba_status_t ensure_system(ba_handle_t h, int fixed) {
  Workspace* ws = h->ws;
  if (fixed == h->fixed) return BA_OK;
  h->fixed = fixed;
  const int B = h->nprob;
  h->sys.assign(B, SysDesc{});
  for (auto& v : h->small_nq) v.clear();
  h->large_sys.clear();
  long long soff = 0, voff = 0, nsum = 0, large_scratch = 0;
  for (int b = 0; b < B; ++b) {
    SysDesc& d = h->sys[b];
    d.problem = b;
    d.n = 6 * (h->frame_off[b + 1] - h->frame_off[b] - fixed);
    system_geometry(d.n, d.TS, d.T, d.n_pad);
    d.soff = soff;
    d.voff = (int)voff;
    soff += (long long)d.T * (d.T + 1) / 2 * d.TS * d.TS;
    voff += d.n_pad;
    nsum += d.n;
    if (d.n == 0) continue;
    if (d.n <= DPV_SMALL_N) {
      h->small_nq[d.n_pad / 32].push_back(b);
    } else {
      h->large_sys.push_back(b);
      large_scratch += dpv_large_scratch_floats(d.n_pad);  // all large systems are factored together
    }
  }
  if (voff > (1LL << 30) || soff > (1LL << 40)) return dpv_fail(h, BA_ERR_UNSUPPORTED, "pose systems too large");
  h->n = (int)nsum;
  h->n_pad = (int)voff;
  h->nS = soff;
  h->TS = h->sys[0].TS;
  h->T = h->sys[0].T;
  ba_status_t s;
  if ((s = dpv_grow(h, ws->S, soff, "pose system")) || (s = dpv_grow(h, ws->y, voff, "rhs")) ||
      (s = dpv_grow(h, ws->dx, voff, "step")) || (s = dpv_grow(h, ws->r64, voff, "residual")) ||
      (s = dpv_grow(h, ws->tmpv, voff, "vector")) || (s = dpv_grow(h, ws->dx2, voff, "step pairs")) ||
      (s = dpv_grow(h, ws->sysd, B, "system table")) ||
      (s = dpv_grow(h, ws->syslist, B, "system lists")) || (s = dpv_grow(h, ws->fdx, h->N, "frame map")))
    return s;
  if (large_scratch > 0 && (s = dpv_grow(h, ws->L, large_scratch, "factor"))) return s;
  DPV_CUDA(h, cudaMemcpyAsync(ws->sysd.p, h->sys.data(), sizeof(SysDesc) * B, cudaMemcpyHostToDevice, h->stream));
  // the solver launches read their system indices from syslist: small systems
  // grouped by block count, then the large ones
  std::vector<int> lists;
  for (auto& v : h->small_nq) lists.insert(lists.end(), v.begin(), v.end());
  lists.insert(lists.end(), h->large_sys.begin(), h->large_sys.end());
  if (!lists.empty())
    DPV_CUDA(h, cudaMemcpyAsync(ws->syslist.p, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice,
                                h->stream));
  k_build_fdx<<<(h->N + 255) / 256, 256, 0, h->stream>>>(h->N, fixed, ws->fprob.p, ws->fprob.p + h->N,
                                                          ws->sysd.p, ws->fdx.p);
  ++h->launches;
  DPV_CUDA(h, cudaGetLastError());
  if ((s = dpv_large_reserve(h))) return s;
  return BA_OK;  // (pageable-source async copies are staged before they return)
}

}  // namespace

ba_status_t dpv_ensure_system(ba_handle_t h, int fixed) { return ensure_system(h, fixed); }

// Lay out one dense system of n unknowns that is not a bundle-adjustment pose
// system (the pose-graph optimisation's), in the same buffers and with the
// same solver selection.  The next ba_step lays out its own system again.
ba_status_t dpv_ensure_generic_system(ba_handle_t h, int n) {
  Workspace* ws = h->ws;
  h->fixed = -1;
  h->sys.assign(1, SysDesc{});
  for (auto& v : h->small_nq) v.clear();
  h->large_sys.clear();
  SysDesc& d = h->sys[0];
  d.problem = 0;
  d.n = n;
  system_geometry(n, d.TS, d.T, d.n_pad);
  d.soff = 0;
  d.voff = 0;
  const long long soff = (long long)d.T * (d.T + 1) / 2 * d.TS * d.TS;
  long long large_scratch = 0;
  if (n > 0 && n <= DPV_SMALL_N) {
    h->small_nq[d.n_pad / 32].push_back(0);
  } else if (n > 0) {
    h->large_sys.push_back(0);
    large_scratch = dpv_large_scratch_floats(d.n_pad);
  }
  h->n = n;
  h->n_pad = d.n_pad;
  h->nS = soff;
  h->TS = d.TS;
  h->T = d.T;
  ba_status_t s;
  if ((s = dpv_grow(h, ws->S, soff, "pose system")) || (s = dpv_grow(h, ws->y, d.n_pad, "rhs")) ||
      (s = dpv_grow(h, ws->dx, d.n_pad, "step")) || (s = dpv_grow(h, ws->r64, d.n_pad, "residual")) ||
      (s = dpv_grow(h, ws->tmpv, d.n_pad, "vector")) || (s = dpv_grow(h, ws->dx2, d.n_pad, "step pairs")) ||
      (s = dpv_grow(h, ws->sysd, 1, "system table")) ||
      (s = dpv_grow(h, ws->syslist, 1, "system lists")))
    return s;
  if (large_scratch > 0 && (s = dpv_grow(h, ws->L, large_scratch, "factor"))) return s;
  const int zero = 0;
  DPV_CUDA(h, cudaMemcpyAsync(ws->sysd.p, h->sys.data(), sizeof(SysDesc), cudaMemcpyHostToDevice, h->stream));
  DPV_CUDA(h, cudaMemcpyAsync(ws->syslist.p, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  return dpv_large_reserve(h);
}

extern "C" {

const char* ba_status_string(ba_status_t s) {
  switch (s) {
    case BA_OK: return "BA_OK";
    case BA_ERR_INVALID_ARG: return "BA_ERR_INVALID_ARG";
    case BA_ERR_CUDA: return "BA_ERR_CUDA";
    case BA_ERR_OOM: return "BA_ERR_OOM";
    case BA_ERR_NOT_SPD: return "BA_ERR_NOT_SPD";
    case BA_ERR_TIMEOUT: return "BA_ERR_TIMEOUT";
    case BA_ERR_STATE: return "BA_ERR_STATE";
    case BA_ERR_UNSUPPORTED: return "BA_ERR_UNSUPPORTED";
  }
  return "BA_ERR_UNKNOWN";
}

ba_status_t ba_default_options(ba_options_t* opt) {
  if (!opt) return BA_ERR_INVALID_ARG;
  opt->precision = BA_FP32;
  opt->lambda_pose = 1e-4f;
  opt->lambda_depth = 1e-4f;
  opt->z_min = 0.1f;
  opt->d_min = 1e-3f;
  opt->patches_per_group = 0;
  opt->max_refine = 3;
  opt->timeout_cycles = 2000000000LL;
  opt->stream = nullptr;
  opt->residual_pixels = 1;
  opt->dense_policy = BA_DENSE_AUTO;
  return BA_OK;
}

ba_status_t ba_create(ba_handle_t* out, const ba_options_t* opt) {
  if (!out) return BA_ERR_INVALID_ARG;
  *out = nullptr;
  ba_handle_t h = new (std::nothrow) ba_handle_s();
  if (!h) return BA_ERR_OOM;
  if (opt) h->opt = *opt;
  else ba_default_options(&h->opt);
  if (h->opt.patches_per_group < 0 || h->opt.patches_per_group > dpv_max_group(h) ||
      (h->opt.precision != BA_FP32 && h->opt.precision != BA_MIXED) || h->opt.max_refine < 0 ||
      (h->opt.residual_pixels != 1 && h->opt.residual_pixels != 9) || h->opt.dense_policy < 0 ||
      h->opt.dense_policy > BA_DENSE_NEVER ||
      h->opt.max_refine > 16) {
    delete h;
    return BA_ERR_INVALID_ARG;
  }
  h->stream = (cudaStream_t)h->opt.stream;
  h->ws = new (std::nothrow) Workspace();
  if (!h->ws || cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      cudaMalloc(&h->ws->status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->ws->intr, 4 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&h->ws->cost, 256 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->ws->unsorted, sizeof(int)) != cudaSuccess ||
      cudaMemset(h->ws->status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    ba_destroy(h);
    return BA_ERR_CUDA;
  }
  h->ws->cost_cap = 256;
  *out = h;
  return BA_OK;
}

ba_status_t ba_destroy(ba_handle_t h) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (h->stream || h->ws) cudaStreamSynchronize(h->stream);
  if (Workspace* ws = h->ws) {
    void* raw[] = {ws->status, ws->intr, ws->cost, ws->unsorted};
    for (void* b : raw)
      if (b) cudaFree(b);
    release(ws->src); release(ws->keys0); release(ws->keys1); release(ws->vals0); release(ws->vals1);
    release(ws->hist); release(ws->perm); release(ws->eslot); release(ws->grun); release(ws->gnr);
    release(ws->gptr); release(ws->win); release(ws->wlen);
    release(ws->scan); release(ws->S); release(ws->y); release(ws->dx); release(ws->Ct); release(ws->wk);
    release(ws->dd); release(ws->L); release(ws->r64); release(ws->tmpv); release(ws->pmpos); release(ws->pptr);
    release(ws->pterm); release(ws->posef); release(ws->Ct2); release(ws->wk2); release(ws->dx2);
    release(ws->dE); release(ws->dCw);
    release(ws->tp_poses); release(ws->tp_patches); release(ws->tp_dx); release(ws->tp_dd);
    release(ws->ad_xb); release(ws->ad_w); release(ws->ad_gd); release(ws->ad_lamd); release(ws->ad_v);
    release(ws->ad_gt); release(ws->ad_gw); release(ws->lg_sync); release(ws->lg_red); release(ws->lg_prob); release(ws->lg_rb); release(ws->lg_live); release(ws->fprob); release(ws->gprob);
    release(ws->fdx); release(ws->sysd); release(ws->syslist); release(ws->mii); release(ws->mjj); release(ws->mkk);
    release(ws->offs); release(ws->pcopy); release(ws->prox); release(ws->corr); release(ws->pgo);
    delete ws;
  }
  graph_drop(h, h->step_graph);
  graph_drop(h, h->bind_graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->prof_side) cudaStreamDestroy(h->prof_side);
  if (h->prof_fork) cudaEventDestroy(h->prof_fork);
  for (int q = 0; q < 8; ++q) {
    if (h->side[q]) cudaStreamDestroy(h->side[q]);
    if (h->ev_join[q]) cudaEventDestroy(h->ev_join[q]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  prof_clear(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return BA_OK;
}

ba_status_t ba_profile_classes(ba_handle_t h, unsigned mask) {
  if (!h || (mask >> BA_KERNEL_CLASSES)) return BA_ERR_INVALID_ARG;
  if (mask) {
    DPV_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->prof_side) DPV_CUDA(h, cudaStreamSynchronize(h->prof_side));
    prof_clear(h);
    if (!h->prof_side) DPV_CUDA(h, cudaStreamCreateWithFlags(&h->prof_side, cudaStreamNonBlocking));
    if (!h->prof_fork) DPV_CUDA(h, cudaEventCreateWithFlags(&h->prof_fork, cudaEventDisableTiming));
  }
  h->prof_on = (int)mask;
  return BA_OK;
}

ba_status_t ba_profile_enable(ba_handle_t h, int on) {
  return ba_profile_classes(h, on ? (1u << BA_KERNEL_CLASSES) - 1u : 0u);
}

ba_status_t ba_set_capture(ba_handle_t h, int on) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!on && (h->step_graph.exec || h->bind_graph.exec)) {
    DPV_CUDA(h, cudaStreamSynchronize(h->stream));
    ba_status_t s = prof_harvest_all(h);
    graph_drop(h, h->step_graph);
    graph_drop(h, h->bind_graph);
    if (s) return s;
  }
  h->capture_on = on ? 1 : 0;
  return BA_OK;
}

ba_status_t ba_profile_read(ba_handle_t h, int kind, double* total_ms, long long* launches) {
  if (!h || !total_ms || !launches || kind < 0 || kind >= BA_KERNEL_CLASSES) return BA_ERR_INVALID_ARG;
  DPV_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->prof_side) DPV_CUDA(h, cudaStreamSynchronize(h->prof_side));  // the eager records
  ba_status_t s = prof_harvest_all(h);
  if (s) return s;
  double t = h->prof_ms[kind];
  long long c = h->prof_n[kind];
  for (auto& r : h->prof) {
    if (r.kind != kind) continue;
    float ms = 0.f;
    DPV_CUDA(h, cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms;
    ++c;
  }
  *total_ms = t;
  *launches = c;
  return BA_OK;
}

ba_status_t ba_set_stream(ba_handle_t h, void* stream) {
  if (!h) return BA_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  h->opt.stream = stream;
  return BA_OK;
}

ba_status_t ba_set_graph(ba_handle_t h, int N, int P, int E, double* poses, float* patches, const int* ii,
                         const int* jj, const int* kk, const float* targets, const float* weights,
                         const float* intrinsics) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (N < 1 || P < 1 || E < 0) return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph: need N >= 1, P >= 1, E >= 0");
  if (!poses || !patches || !intrinsics || (E > 0 && (!ii || !jj || !kk || !targets || !weights)))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph: null pointer");
  if (N > (1 << 20)) return dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_set_graph: more than 2^20 frames");
  if ((reinterpret_cast<uintptr_t>(targets) | reinterpret_cast<uintptr_t>(weights)) & 7)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph: targets/weights must be 8-byte aligned");
  Workspace* ws = h->ws;
  h->bind = ba_handle_s::Bind{};
  h->bind.N = N;
  h->bind.P = P;
  h->bind.E = E;
  h->bind.poses = poses;
  h->bind.patches = patches;
  h->bind.ii = ii;
  h->bind.jj = jj;
  h->bind.kk = kk;
  h->bind.targets = targets;
  h->bind.weights = weights;
  h->bind.intrinsics = intrinsics;
  h->have_graph = 0;
  // the frame -> unknown map survives a rebinding with the same frame count
  const bool same_frames = h->nprob == 1 && h->N == N && h->fixed >= 0;
  h->nprob = 1;
  h->user_patches = nullptr;
  h->patches_padded = 0;
  h->frame_off.assign({0, N});
  h->min_frames = N;
  h->N = N;
  h->P = P;
  h->E = E;
  h->poses = poses;
  h->patches = patches;
  h->targets = targets;
  h->weights = weights;
  h->G = h->opt.patches_per_group > 0 ? h->opt.patches_per_group : auto_group(h, P, E, 0);
  h->ngroups = (P + h->G - 1) / h->G;
  if (!same_frames) h->fixed = -1;
  // intrinsics in device memory are copied by the binding's first kernel (so
  // the pointer joins the signature); host memory is copied outside any graph
  cudaPointerAttributes pa = {};
  const bool intr_dev = cudaPointerGetAttributes(&pa, intrinsics) == cudaSuccess &&
                        (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  bind_signature(h, {1, N, P, E, (long long)(uintptr_t)poses, (long long)(uintptr_t)patches,
                     (long long)(uintptr_t)targets, (long long)(uintptr_t)weights, (long long)(uintptr_t)ii,
                     (long long)(uintptr_t)jj, (long long)(uintptr_t)kk, h->G,
                     intr_dev ? (long long)(uintptr_t)intrinsics : 0LL});
  h->tape_valid = 0;
  h->kk_bits = bits_for((unsigned long long)P);
  ba_status_t s;
  const long long En = std::max(E, 1);
  const long long Gn = h->ngroups + 1;
  const long long scan_need = std::max(dpv_scan_scratch(En + 1), dpv_scan_scratch(dpv_hist_entries(En)));
  if ((s = dpv_grow(h, ws->src, P, "patch table")) || (s = dpv_grow(h, ws->Ct, P, "Ct")) || (s = dpv_grow(h, ws->wk, P, "w")) ||
      (s = dpv_grow(h, ws->Ct2, P, "Ct pairs")) || (s = dpv_grow(h, ws->wk2, P, "w pairs")) ||
      (s = dpv_grow(h, ws->dd, P, "dd")) || (s = dpv_grow(h, ws->keys0, En, "sort keys")) ||
      (s = dpv_grow(h, ws->keys1, En, "sort keys")) || (s = dpv_grow(h, ws->vals0, En, "sort values")) ||
      (s = dpv_grow(h, ws->vals1, En, "sort values")) || (s = dpv_grow(h, ws->perm, En, "permutation")) ||
      (s = dpv_grow(h, ws->eslot, En, "slots")) || (s = dpv_grow(h, ws->grun, Gn * (DPV_RMAX + 1), "run tables")) ||
      (s = dpv_grow(h, ws->gnr, Gn, "run counts")) ||
      (s = dpv_grow(h, ws->hist, dpv_hist_entries(En), "histograms")) || (s = dpv_grow(h, ws->scan, scan_need, "scan")) ||
      (s = dpv_grow(h, ws->gptr, Gn, "groups")) ||
      (s = dpv_grow(h, ws->win, Gn * DPV_WMAX, "windows")) || (s = dpv_grow(h, ws->wlen, Gn, "windows")) ||
      (s = dpv_grow(h, ws->pmpos, En, "patch-major positions")) || (s = dpv_grow(h, ws->pptr, (long long)P + 1, "patch CSR")) ||
      (s = dpv_grow(h, ws->pterm, dpv_pterm_width(h) * En, "edge depth terms")) || (s = dpv_grow(h, ws->posef, (long long)DPV_POSE_ROW * N, "pose table")) ||
      (s = dpv_grow(h, ws->fprob, (long long)N + 2, "frame problems")) || (s = dpv_grow(h, ws->gprob, Gn, "group problems")))
    return s;
  if (!intr_dev)
    DPV_CUDA(h, cudaMemcpyAsync(ws->intr, intrinsics, 4 * sizeof(float), cudaMemcpyDefault, h->stream));
  auto device_work = [&]() -> ba_status_t {
    // one problem: every frame and group belongs to problem 0 (written by the
    // preprocessing's first kernel, which also clears the device status)
    dpv_prof_begin(h, BA_KERNEL_PREPROCESS);
    ba_status_t r = dpv_preprocess(h, ii, jj, kk, 1, intr_dev ? intrinsics : nullptr);
    dpv_prof_end(h);
    return r;
  };
  if (h->capture_on) {
    const ba_handle_s::GraphKey key{h->bind_gen, h->ws_gen, -1, -1, h->prof_on, h->stream};
    s = graph_run(h, h->bind_graph, key, device_work);
  } else {
    s = device_work();
  }
  if (s) return s;
  h->have_graph = 1;
  return BA_OK;
}

ba_status_t ba_set_graph_batched(ba_handle_t h, int B, const long long* frame_off, const long long* patch_off,
                                 const long long* edge_off, double* poses, float* patches, const int* ii,
                                 const int* jj, const int* kk, const float* targets, const float* weights,
                                 const float* intrinsics) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (B < 1 || !frame_off || !patch_off || !edge_off)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph_batched: need B >= 1 and host offset arrays");
  if (frame_off[0] || patch_off[0] || edge_off[0])
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph_batched: offsets must start at 0");
  int min_frames = INT32_MAX;
  for (int b = 0; b < B; ++b) {
    if (frame_off[b + 1] - frame_off[b] < 1 || patch_off[b + 1] - patch_off[b] < 1 ||
        edge_off[b + 1] < edge_off[b])
      return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph_batched: each problem needs a frame and a patch");
    min_frames = std::min<long long>(min_frames, frame_off[b + 1] - frame_off[b]);
  }
  const long long Nl = frame_off[B], Pl = patch_off[B], El = edge_off[B];
  if (Nl > (1 << 20) || Pl > (1LL << 30) || El > (1LL << 30))
    return dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_set_graph_batched: problem sizes");
  if (!poses || !patches || !intrinsics || (El > 0 && (!ii || !jj || !kk || !targets || !weights)))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph_batched: null pointer");
  if ((reinterpret_cast<uintptr_t>(targets) | reinterpret_cast<uintptr_t>(weights)) & 7)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_set_graph_batched: targets/weights must be 8-byte aligned");
  Workspace* ws = h->ws;
  const int N = (int)Nl, E = (int)El;
  const int G = h->opt.patches_per_group > 0 ? h->opt.patches_per_group : auto_group(h, Pl, El, 1);
  h->bind = ba_handle_s::Bind{};
  h->bind.batched = 1;
  h->bind.B = B;
  h->bind.frame_off.assign(frame_off, frame_off + B + 1);
  h->bind.patch_off.assign(patch_off, patch_off + B + 1);
  h->bind.edge_off.assign(edge_off, edge_off + B + 1);
  h->bind.poses = poses;
  h->bind.patches = patches;
  h->bind.ii = ii;
  h->bind.jj = jj;
  h->bind.kk = kk;
  h->bind.targets = targets;
  h->bind.weights = weights;
  h->bind.intrinsics = intrinsics;
  // group-aligned patch numbering: every reduction group lies inside one problem
  std::vector<long long> offs(4 * (B + 1));
  long long* foff = offs.data();
  long long* moff = foff + (B + 1);
  long long* eoff = moff + (B + 1);
  long long* poff = eoff + (B + 1);
  bool padded = false;
  moff[0] = 0;
  for (int b = 0; b <= B; ++b) {
    foff[b] = frame_off[b];
    eoff[b] = edge_off[b];
    poff[b] = patch_off[b];
    if (b < B) {
      const long long np = patch_off[b + 1] - patch_off[b];
      moff[b + 1] = moff[b] + (np + G - 1) / G * G;
      padded = padded || (np % G != 0);
    }
  }
  const long long Ppad = padded ? moff[B] : Pl;
  if (!padded)
    for (int b = 0; b <= B; ++b) moff[b] = poff[b];
  if (Ppad > (1LL << 30)) return dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_set_graph_batched: problem sizes");
  const int P = (int)Ppad;
  h->have_graph = 0;
  h->tape_valid = 0;
  h->fixed = -1;
  h->nprob = B;
  h->frame_off.assign(frame_off, frame_off + B + 1);
  h->patch_moff.assign(moff, moff + B + 1);
  h->user_patch_off.assign(patch_off, patch_off + B + 1);
  h->min_frames = min_frames;
  h->N = N;
  h->P = P;
  h->E = E;
  h->poses = poses;
  h->user_patches = padded ? patches : nullptr;
  h->patches_padded = padded ? 1 : 0;
  h->targets = targets;
  h->weights = weights;
  h->G = G;
  h->ngroups = (P + G - 1) / G;
  h->kk_bits = bits_for((unsigned long long)P);
  {
    std::vector<long long> sig = {2, B, N, P, E, (long long)(uintptr_t)poses, (long long)(uintptr_t)patches,
                                  (long long)(uintptr_t)targets, (long long)(uintptr_t)weights,
                                  (long long)(uintptr_t)ii, (long long)(uintptr_t)jj, (long long)(uintptr_t)kk, G};
    sig.insert(sig.end(), offs.begin(), offs.end());
    bind_signature(h, std::move(sig));
  }
  ba_status_t s;
  const long long En = std::max(E, 1);
  const long long Gn = h->ngroups + 1;
  const long long scan_need = std::max(dpv_scan_scratch(En + 1), dpv_scan_scratch(dpv_hist_entries(En)));
  if ((s = dpv_grow(h, ws->src, P, "patch table")) || (s = dpv_grow(h, ws->Ct, P, "Ct")) ||
      (s = dpv_grow(h, ws->Ct2, P, "Ct pairs")) || (s = dpv_grow(h, ws->wk2, P, "w pairs")) ||
      (s = dpv_grow(h, ws->wk, P, "w")) || (s = dpv_grow(h, ws->dd, P, "dd")) ||
      (s = dpv_grow(h, ws->keys0, En, "sort keys")) || (s = dpv_grow(h, ws->keys1, En, "sort keys")) ||
      (s = dpv_grow(h, ws->vals0, En, "sort values")) || (s = dpv_grow(h, ws->vals1, En, "sort values")) ||
      (s = dpv_grow(h, ws->perm, En, "permutation")) || (s = dpv_grow(h, ws->eslot, En, "slots")) ||
      (s = dpv_grow(h, ws->grun, Gn * (DPV_RMAX + 1), "run tables")) || (s = dpv_grow(h, ws->gnr, Gn, "run counts")) ||
      (s = dpv_grow(h, ws->hist, dpv_hist_entries(En), "histograms")) || (s = dpv_grow(h, ws->scan, scan_need, "scan")) ||
      (s = dpv_grow(h, ws->gptr, Gn, "groups")) || (s = dpv_grow(h, ws->win, Gn * DPV_WMAX, "windows")) ||
      (s = dpv_grow(h, ws->wlen, Gn, "windows")) || (s = dpv_grow(h, ws->pmpos, En, "patch-major positions")) ||
      (s = dpv_grow(h, ws->pptr, (long long)P + 1, "patch CSR")) || (s = dpv_grow(h, ws->pterm, dpv_pterm_width(h) * En, "edge depth terms")) ||
      (s = dpv_grow(h, ws->posef, (long long)DPV_POSE_ROW * N, "pose table")) ||
      (s = dpv_grow(h, ws->fprob, (long long)N + B + 1, "frame problems")) ||
      (s = dpv_grow(h, ws->gprob, Gn, "group problems")) || (s = dpv_grow(h, ws->mii, En, "edge frames")) ||
      (s = dpv_grow(h, ws->mjj, En, "edge frames")) || (s = dpv_grow(h, ws->mkk, En, "edge patches")) ||
      (s = dpv_grow(h, ws->offs, 4LL * (B + 1), "problem offsets")) ||
      (padded && (s = dpv_grow(h, ws->pcopy, 27LL * P, "padded patches"))))
    return s;
  if (B > ws->intr_cap) {
    float* p = nullptr;
    if (cudaMalloc(&p, sizeof(float) * 4 * B) != cudaSuccess) {
      cudaGetLastError();
      return dpv_fail(h, BA_ERR_OOM, "allocating intrinsics");
    }
    DPV_CUDA(h, cudaStreamSynchronize(h->stream));
    cudaFree(ws->intr);
    ws->intr = p;
    ws->intr_cap = B;
    ++h->ws_gen;
  }
  h->patches = padded ? ws->pcopy.p : patches;
  // the intrinsics may live in host memory: copied outside any graph
  DPV_CUDA(h, cudaMemcpyAsync(ws->intr, intrinsics, sizeof(float) * 4 * B, cudaMemcpyDefault, h->stream));
  std::vector<int> gp(h->ngroups);
  for (int g = 0, b = 0; g < h->ngroups; ++g) {
    while (b + 1 < B && (long long)g * G >= h->patch_moff[b + 1]) ++b;
    gp[g] = b;
  }
  auto device_work = [&]() -> ba_status_t {
    cudaStream_t st = h->stream;
    if (!h->capturing) {
      // offsets, frame offsets and group problems: fixed by the binding's
      // signature, so a captured binding finds them in place
      DPV_CUDA(h, cudaMemcpyAsync(ws->offs.p, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice, st));
      DPV_CUDA(h, cudaMemcpyAsync(ws->fprob.p + N, h->frame_off.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice,
                                  st));
      if (h->ngroups > 0)
        DPV_CUDA(h, cudaMemcpyAsync(ws->gprob.p, gp.data(), sizeof(int) * h->ngroups, cudaMemcpyHostToDevice, st));
    }
    DPV_CUDA(h, cudaMemsetAsync(ws->status, 0, sizeof(int), st));
    // per-frame problem (the frame offsets follow it)
    k_frame_problems<<<(N + 255) / 256, 256, 0, st>>>(N, B, ws->offs.p, ws->fprob.p);
    ++h->launches;
    if (padded) {
      k_patch_copy<<<(unsigned)((27LL * P + 255) / 256), 256, 0, st>>>(P, B, ws->offs.p, patches, ws->pcopy.p, 1);
      ++h->launches;
    }
    if (E > 0) {
      k_remap_edges<<<(E + 255) / 256, 256, 0, st>>>(E, B, ws->offs.p, ii, jj, kk, ws->mii.p, ws->mjj.p, ws->mkk.p);
      ++h->launches;
    }
    dpv_prof_begin(h, BA_KERNEL_PREPROCESS);
    ba_status_t r = dpv_preprocess(h, ws->mii.p, ws->mjj.p, ws->mkk.p, 0, nullptr);
    dpv_prof_end(h);
    return r;
  };
  if (h->capture_on) {
    const ba_handle_s::GraphKey key{h->bind_gen, h->ws_gen, -1, -1, h->prof_on, h->stream};
    s = graph_run(h, h->bind_graph, key, device_work);
  } else {
    s = device_work();
  }
  if (s) return s;
  h->have_graph = 1;
  return BA_OK;
}

static ba_status_t check_step_args(ba_handle_t h, int fixed_poses) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (!h->have_graph) return dpv_fail(h, BA_ERR_STATE, "no graph bound (call ba_set_graph first)");
  if (fixed_poses < 0 || fixed_poses > h->min_frames)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "fixed_poses out of range");
  return BA_OK;
}

// The work of one ba_step after its checks, enqueued on h->stream.
static ba_status_t step_body(ba_handle_t h, int run, int fixed_poses) {
  ba_status_t s;
  if (h->patches_padded) {  // the padded working copy follows the caller's patches
    k_patch_copy<<<(unsigned)((27LL * h->P + 255) / 256), 256, 0, h->stream>>>(h->P, h->nprob, h->ws->offs.p,
                                                                               h->user_patches, h->ws->pcopy.p, 1);
    ++h->launches;
  }
  // the cost slots are cleared by the first iteration's k_init_system
  int prepared = 0;  // S, y and the pose table already set up by the previous iteration
  for (int it = 0; it < run; ++it) {
    if (h->record && (s = dpv_tape_state(h, it))) return s;
    if ((s = dpv_assemble(h, it, prepared))) return s;
    int retracted = 0;
    // the one-CTA solver re-zeroes S and y for the next iteration's assembly
    const int reset = it + 1 < run && h->large_sys.empty();
    dpv_prof_begin(h, BA_KERNEL_SOLVE);
    s = dpv_solve(h, &retracted, reset);
    dpv_prof_end(h);
    if (s) return s;
    // back-substitution of the depths, with the pose retraction in the same launch
    dpv_prof_begin(h, BA_KERNEL_BACKSUB);
    s = dpv_backsub(h, !retracted);
    dpv_prof_end(h);
    if (s) return s;
    if (h->record && (s = dpv_tape_step(h, it))) return s;
    prepared = reset;
  }
  if (h->record) {
    if ((s = dpv_tape_state(h, run))) return s;
    h->tape_iters = run;
    h->tape_fixed = fixed_poses;
    h->tape_valid = 1;
  }
  if (h->patches_padded && run > 0) {
    k_patch_copy<<<(unsigned)((27LL * h->P + 255) / 256), 256, 0, h->stream>>>(h->P, h->nprob, h->ws->offs.p,
                                                                               h->user_patches, h->ws->pcopy.p, 0);
    ++h->launches;
    DPV_CUDA(h, cudaGetLastError());
  }
  return BA_OK;
}

ba_status_t ba_step(ba_handle_t h, int iters, int fixed_poses) {
  ba_status_t s = check_step_args(h, fixed_poses);
  if (s) return s;
  if (iters < 0) return dpv_fail(h, BA_ERR_INVALID_ARG, "iters < 0");
  if ((s = ensure_system(h, fixed_poses))) return s;
  h->last_iters = iters;
  h->last_dense = dpv_use_dense(h) ? 1 : 0;
  // fixed_poses = N leaves no pose unknowns: the iterations then update the
  // inverse depths only (structure-only bundle adjustment)
  const int run = iters > 0 ? iters : 0;
  if (h->record) {
    // this call becomes the tape of ba_backward
    h->tape_valid = 0;
    h->tape_iters_pending = run;
    if ((s = dpv_tape_reserve(h, run))) return s;
  }
  if (h->capture_on && !h->record && run > 0) {
    const ba_handle_s::GraphKey key{h->bind_gen, h->ws_gen, run, fixed_poses, h->prof_on, h->stream};
    return graph_run(h, h->step_graph, key, [&]() { return step_body(h, run, fixed_poses); });
  }
  return step_body(h, run, fixed_poses);
}

ba_status_t ba_linearize(ba_handle_t h, int fixed_poses) {
  ba_status_t s = check_step_args(h, fixed_poses);
  if (s) return s;
  if ((s = ensure_system(h, fixed_poses))) return s;
  if (h->n == 0) return BA_OK;
  DPV_CUDA(h, cudaMemsetAsync(h->ws->cost, 0, sizeof(double), h->stream));
  return dpv_assemble(h, 0, 0);
}

ba_status_t ba_sync(ba_handle_t h) {
  if (!h) return BA_ERR_INVALID_ARG;
  DPV_CUDA(h, cudaStreamSynchronize(h->stream));
  int st = 0;
  DPV_CUDA(h, cudaMemcpy(&st, h->ws->status, sizeof(int), cudaMemcpyDeviceToHost));
  switch (st) {
    case DST_OK: return BA_OK;
    case DST_BAD_INDEX:
      return dpv_fail(h, BA_ERR_INVALID_ARG, "edge index out of range, or a patch with two source frames");
    case DST_NOT_SPD: return dpv_fail(h, BA_ERR_NOT_SPD, "reduced pose system is not positive definite");
    case DST_TIMEOUT: return dpv_fail(h, BA_ERR_TIMEOUT, "a device-side wait ran out");
    case DST_WIDE:
      return dpv_fail(h, BA_ERR_UNSUPPORTED,
                      "a patch group touches more than 64 frames or has more than 64 (source, target) runs");
  }
  return dpv_fail(h, BA_ERR_CUDA, "unknown device status");
}

const char* ba_last_error(ba_handle_t h) {
  if (!h) return "invalid handle";
  return h->last_error.c_str();
}

ba_status_t ba_debug_info(ba_handle_t h, long long* info, int cap) {
  if (!h || !info) return BA_ERR_INVALID_ARG;
  long long nr = 0;
  if (h->have_graph && h->ngroups > 0) {
    DPV_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<int> gnr(h->ngroups);
    DPV_CUDA(h, cudaMemcpy(gnr.data(), h->ws->gnr.p, sizeof(int) * h->ngroups, cudaMemcpyDeviceToHost));
    for (int v : gnr) nr += v;
  }
  const ba_handle_s::CapGraph &sg = h->step_graph, &bg = h->bind_graph;
  const long long v[16] = {h->N,        h->P,       h->E,        h->G,        h->ngroups,
                           h->n,        h->TS,      nr,          h->launches, sg.captures,
                           sg.replays,  sg.kernels, bg.captures, bg.replays,  bg.kernels,
                           h->last_dense};
  for (int q = 0; q < cap && q < 16; ++q) info[q] = v[q];
  return BA_OK;
}

ba_status_t ba_debug_export(ba_handle_t h, int what, void* dst, long long bytes) {
  if (!h || !dst) return BA_ERR_INVALID_ARG;
  if (!h->have_graph) return dpv_fail(h, BA_ERR_STATE, "no graph bound");
  Workspace* ws = h->ws;
  const void* src = nullptr;
  long long need = 0;
  switch (what) {
    case BA_EXPORT_S:
      if (h->nprob != 1) return dpv_fail(h, BA_ERR_UNSUPPORTED, "the S export is single-problem only");
      need = 8LL * h->n * h->n;
      break;
    case BA_EXPORT_Y: src = ws->y.p; need = 8LL * h->n; break;
    case BA_EXPORT_DX: src = ws->dx.p; need = 8LL * h->n; break;
    case BA_EXPORT_DD: src = ws->dd.p; need = 4LL * h->P; break;
    case BA_EXPORT_CT: src = ws->Ct.p; need = 4LL * h->P; break;
    case BA_EXPORT_W: src = ws->wk.p; need = 4LL * h->P; break;
    case BA_EXPORT_PERM: src = ws->perm.p; need = 4LL * h->E; break;
    case BA_EXPORT_SLOTS: src = ws->eslot.p; need = 4LL * h->E; break;
    case BA_EXPORT_GPTR: src = ws->gptr.p; need = 4LL * (h->ngroups + 1); break;
    case BA_EXPORT_WIN: src = ws->win.p; need = 4LL * h->ngroups * DPV_WMAX; break;
    case BA_EXPORT_PMPOS: src = ws->pmpos.p; need = 4LL * h->E; break;
    case BA_EXPORT_PPTR: src = ws->pptr.p; need = 4LL * (h->P + 1); break;
    case BA_EXPORT_COST: src = ws->cost; need = 8LL * std::max(1, std::min<int>(h->last_iters, (int)ws->cost_cap)); break;
    default: return dpv_fail(h, BA_ERR_INVALID_ARG, "unknown export");
  }
  if (bytes < need) return dpv_fail(h, BA_ERR_INVALID_ARG, "export buffer too small");
  ba_status_t s;
  if (what == BA_EXPORT_S) {
    if ((s = dpv_export_S(h, (double*)dst))) return s;
  } else if (need > 0) {
    DPV_CUDA(h, cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, h->stream));
  }
  DPV_CUDA(h, cudaStreamSynchronize(h->stream));
  return BA_OK;
}

ba_status_t ba_debug_envelope(ba_handle_t h, int* out, long long cap, long long* count) {
  if (!h || !count || (cap > 0 && !out)) return BA_ERR_INVALID_ARG;
  return dpv_large_envelope(h, out, cap, count);  // (also the pose graph of ba_pgo_lm)
}

ba_status_t ba_debug_keys(ba_handle_t h, int fixed_poses, int* keys_out, int cap, int* n_out) {
  if (!h || !n_out || (cap > 0 && !keys_out)) return BA_ERR_INVALID_ARG;
  if (!h->have_graph) return dpv_fail(h, BA_ERR_STATE, "no graph bound");
  if (h->nprob != 1) return dpv_fail(h, BA_ERR_UNSUPPORTED, "block keys are single-problem only");
  return dpv_block_keys(h, fixed_poses, keys_out, cap, n_out);
}

}  // extern "C"
