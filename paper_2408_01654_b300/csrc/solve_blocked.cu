// Blocked solver for pose systems larger than one CTA can hold (see below).
#include "internal.cuh"

ba_status_t dpv_solve_blocked(ba_handle_t h, int refine) {
  (void)refine;
  return dpv_fail(h, BA_ERR_UNSUPPORTED, "pose systems above 256 unknowns are not built yet");
}
