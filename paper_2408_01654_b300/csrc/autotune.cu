// Autotuner of the patch-group size (the assembly's tile: patches reduced by
// one CTA) and the process-wide table of tuned sizes that the automatic
// choice consults.
//
// ba_autotune times whole ba_step calls of the bound graph for every
// candidate group size, restoring the caller's poses and patches before each
// step, keeps the fastest feasible size (a group whose window exceeds the
// kernel's limits reports BA_ERR_UNSUPPORTED on the device and is skipped)
// and records it under the binding's shape class.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace {

// shape class: device, batched or not, half-octave buckets of the patch and
// edge counts, precision
using TuneKey = std::tuple<int, int, int, int, int>;

struct TuneTable {
  std::mutex mu;
  std::map<TuneKey, int> best;
};
TuneTable& table() {
  static TuneTable t;
  return t;
}

int half_octave(long long x) { return x < 1 ? 0 : (int)std::floor(2.0 * std::log2((double)x)); }

TuneKey key_of(ba_handle_t h, long long P, long long E, int batched) {
  return TuneKey{h->device, batched, half_octave(P), half_octave(E), (int)h->opt.precision};
}

constexpr int CANDIDATES[] = {8, 16, 24, 32, 48, 64};

}  // namespace

int dpv_tuned_group(ba_handle_t h, long long P, long long E, int batched) {
  TuneTable& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  auto it = t.best.find(key_of(h, P, E, batched));
  return it == t.best.end() ? 0 : it->second;
}

extern "C" {

ba_status_t ba_autotune_clear(void) {
  TuneTable& t = table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.best.clear();
  return BA_OK;
}

ba_status_t ba_autotune(ba_handle_t h, int iters, int fixed_poses, int reps, int max_cand, int* cand_group,
                        float* cand_ms, int* n_cand, int* best_group) {
  if (!h || !best_group || iters < 1 || reps < 1 || max_cand < 0 || (max_cand > 0 && (!cand_group || !cand_ms)))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_autotune: bad arguments");
  if (!h->have_graph) return dpv_fail(h, BA_ERR_STATE, "ba_autotune: no graph bound");
  if (fixed_poses < 0 || fixed_poses > h->min_frames)
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_autotune: fixed_poses out of range");
  const ba_handle_s::Bind b = h->bind;  // the binding is redone for every candidate
  const long long Nu = b.batched ? b.frame_off[b.B] : b.N;
  const long long Pu = b.batched ? b.patch_off[b.B] : b.P;
  const long long Eu = b.batched ? b.edge_off[b.B] : b.E;
  const int saved_group = h->opt.patches_per_group, saved_prof = h->prof_on, saved_record = h->record;
  ba_status_t s = BA_OK;
  double* keep_poses = nullptr;
  float* keep_patches = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&keep_poses, sizeof(double) * 7 * Nu) != cudaSuccess ||
      cudaMalloc(&keep_patches, sizeof(float) * 27 * Pu) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(keep_poses);
    cudaFree(keep_patches);
    if (e0) cudaEventDestroy(e0);
    return dpv_fail(h, BA_ERR_OOM, "ba_autotune: temporaries");
  }
  cudaStream_t st = h->stream;
  auto restore = [&]() {
    cudaMemcpyAsync(b.poses, keep_poses, sizeof(double) * 7 * Nu, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(b.patches, keep_patches, sizeof(float) * 27 * Pu, cudaMemcpyDeviceToDevice, st);
  };
  auto rebind = [&](int G) {
    h->opt.patches_per_group = G;
    return b.batched ? ba_set_graph_batched(h, b.B, b.frame_off.data(), b.patch_off.data(), b.edge_off.data(),
                                            b.poses, b.patches, b.ii, b.jj, b.kk, b.targets, b.weights,
                                            b.intrinsics)
                     : ba_set_graph(h, b.N, b.P, b.E, b.poses, b.patches, b.ii, b.jj, b.kk, b.targets, b.weights,
                                    b.intrinsics);
  };
  cudaMemcpyAsync(keep_poses, b.poses, sizeof(double) * 7 * Nu, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(keep_patches, b.patches, sizeof(float) * 27 * Pu, cudaMemcpyDeviceToDevice, st);
  h->prof_on = 0;
  h->record = 0;
  int best = 0, nc = 0;
  float best_ms = 0.f;
  for (int G : CANDIDATES) {
    if (G > dpv_max_group(h)) continue;
    float ms = -1.f;  // infeasible
    ba_status_t c = rebind(G);
    // warm-up: one eager step, and with graph replay on also the capture
    for (int w = 0; w < (h->capture_on ? 2 : 1) && c == BA_OK; ++w) {
      restore();
      c = ba_step(h, iters, fixed_poses);
    }
    if (c == BA_OK) c = ba_sync(h);
    if (c == BA_OK) {
      std::vector<float> t;
      for (int r = 0; r < reps && c == BA_OK; ++r) {
        restore();
        cudaEventRecord(e0, st);
        c = ba_step(h, iters, fixed_poses);
        cudaEventRecord(e1, st);
        if (c == BA_OK && cudaEventSynchronize(e1) != cudaSuccess) c = BA_ERR_CUDA;
        float x = 0.f;
        if (c == BA_OK && cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) c = BA_ERR_CUDA;
        t.push_back(x);
      }
      if (c == BA_OK) c = ba_sync(h);
      if (c == BA_OK) {
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
      }
    }
    if (c == BA_ERR_CUDA) {  // not a property of the candidate
      s = c;
      break;
    }
    if (nc < max_cand) {
      cand_group[nc] = G;
      cand_ms[nc] = ms;
    }
    ++nc;
    if (ms >= 0.f && (best == 0 || ms < best_ms)) {
      best = G;
      best_ms = ms;
    }
  }
  if (s == BA_OK && best == 0) s = dpv_fail(h, BA_ERR_UNSUPPORTED, "ba_autotune: no feasible group size");
  // the handle keeps the best size (an automatic choice through the table)
  const int final_group = s == BA_OK ? best : saved_group;
  if (s == BA_OK) {
    TuneTable& tt = table();
    std::lock_guard<std::mutex> lk(tt.mu);
    tt.best[key_of(h, Pu, Eu, b.batched)] = best;
  }
  ba_status_t r = rebind(saved_group == 0 && s == BA_OK ? 0 : final_group);
  if (saved_group != 0) h->opt.patches_per_group = final_group;
  restore();
  cudaStreamSynchronize(st);
  h->prof_on = saved_prof;
  h->record = saved_record;
  cudaFree(keep_poses);
  cudaFree(keep_patches);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_cand) *n_cand = nc;
  *best_group = best;
  if (s == BA_OK && r != BA_OK) s = r;
  return s;
}

}  // extern "C"
