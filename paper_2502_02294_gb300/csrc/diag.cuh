// Per-step diagnostics of a run (launcher used by the handle).
#pragma once

#include "common.cuh"

namespace dh {

// sums of one record (per instance), in this order
enum {
  DG_S_MASS = 0, DG_S_MX, DG_S_MY, DG_S_MZ, DG_S_ENERGY, DG_S_PX, DG_S_PY, DG_S_PZ,
  DG_S_STARS, DG_S_EVENTS, DG_S_NONFINITE, DG_NSUM
};

// Record of the current state: sums[b][DG_NSUM] (doubles) and mins[b][2] (the smallest
// density and pressure as order-preserving ints; ordered_to_float decodes them). p: particle
// momenta (B x 3 n^3); zhat (B n^3) and events (B x ceil(n^3/32) words) may be NULL. The
// record is cleared by the same call.
sim_status launch_diag(const float* gas, const float* p, const float* zhat,
                       const uint32_t* events, long long N3, float gamma, SArg cm, int B,
                       double* sums, int* mins, cudaStream_t st);
float ordered_to_float(int i);

}  // namespace dh
