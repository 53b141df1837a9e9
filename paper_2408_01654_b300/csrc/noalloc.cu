// Allocation-free solve of a reduced pose system (ba_solve_pose_system_noalloc).
//
// Some callers cannot allocate device memory at the time they need a solve:
// a tracking loop that has to keep a fixed frame budget (cudaMalloc can
// synchronise the device and stall the camera pipeline), or a host framework
// that owns every device allocation and forbids libraries from making their
// own.  For them this entry point solves S x = y for a dense pose system of up
// to DPV_NOALLOC_MAX_N unknowns with the same one-CTA LDL^T kernel that
// ba_step uses, and keeps its working copy in a fixed device array compiled
// into the library instead of in handle workspace.
//
// That array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 0.5 MB) until the process exits.  Host code cannot
// use its name as a device address, so every call looks the address up with
// cudaGetSymbolAddress on the current device (a lookup in the loaded module,
// no allocation; not cached, because cudaDeviceReset reloads the module and
// may move the array).  All calls on a
// device share the array and it keeps the previous call's contents, so the
// staging kernel rewrites every entry the solver reads (and clears the status
// word) on each call, and calls whose GPU work overlaps race on it.
#include "internal.cuh"

#define DPV_NOALLOC_MAX_N 256  // largest n accepted (= the one-CTA solver's limit)

namespace {
constexpr int NPMAX = DPV_NOALLOC_MAX_N;
// padded system (NPMAX^2), padded rhs (NPMAX), FP32 solution copy (NPMAX floats
// = NPMAX/2 doubles), status word (one double slot)
constexpr size_t SCR_S = 0;
constexpr size_t SCR_Y = SCR_S + (size_t)NPMAX * NPMAX;
constexpr size_t SCR_XF = SCR_Y + NPMAX;
constexpr size_t SCR_STATUS = SCR_XF + NPMAX / 2;
constexpr size_t SCR_TOTAL = SCR_STATUS + 1;
}  // namespace

static __device__ __align__(256) double dpv_noalloc_scratch[SCR_TOTAL];

ba_status_t dpv_launch_small_solver(cudaStream_t st, int n, int n_pad, const double* S, const double* y, double* dx,
                                    float* dxf, int refine, int* status);

namespace {

// Copy the caller's dense n x n system (lower triangle of a row-major array)
// into the padded tile the solver reads: identity on the padding, zeros above
// the diagonal; pad the right-hand side with zeros; clear the status word.
__global__ void k_noalloc_stage(int n, int n_pad, const double* __restrict__ S_in, const double* __restrict__ y_in,
                                double* __restrict__ scr) {
  const int stride = gridDim.x * blockDim.x;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  double* S = scr + SCR_S;
  double* y = scr + SCR_Y;
  for (int q = gid; q < n_pad * n_pad; q += stride) {
    const int r = q / n_pad, c = q % n_pad;
    double v = 0.0;
    if (r < n && c < n) {
      if (c <= r) v = S_in[(size_t)r * n + c];
    } else if (r == c) {
      v = 1.0;
    }
    S[q] = v;
  }
  for (int q = gid; q < n_pad; q += stride) y[q] = q < n ? y_in[q] : 0.0;
  if (gid == 0) *reinterpret_cast<int*>(scr + SCR_STATUS) = 0;
}

// The array's device address on the current device (looked up on every call).
ba_status_t scratch_for_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, dpv_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return BA_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return BA_OK;
}

}  // namespace

extern "C" ba_status_t ba_solve_pose_system_noalloc(int n, const double* S, const double* y, double* x, int refine,
                                                    void* stream) {
  if (!S || !y || !x || n < 1 || refine < 0 || refine > 16) return BA_ERR_INVALID_ARG;
  if (n > DPV_NOALLOC_MAX_N) return BA_ERR_UNSUPPORTED;
  double* scr = nullptr;
  ba_status_t s = scratch_for_current_device(&scr);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n_pad = (n + 31) / 32 * 32;
  k_noalloc_stage<<<32, 256, 0, st>>>(n, n_pad, S, y, scr);
  if (cudaGetLastError() != cudaSuccess) return BA_ERR_CUDA;
  int* status = reinterpret_cast<int*>(scr + SCR_STATUS);
  s = dpv_launch_small_solver(st, n, n_pad, scr + SCR_S, scr + SCR_Y, x, reinterpret_cast<float*>(scr + SCR_XF),
                              refine, status);
  if (s) return s;
  int st_host = 0;
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(&st_host, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BA_ERR_CUDA;
  return st_host == DST_NOT_SPD ? BA_ERR_NOT_SPD : (st_host ? BA_ERR_CUDA : BA_OK);
}
