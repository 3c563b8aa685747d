// Learned closure (Sec. 4, solver-in-the-loop refinement): the hooks the simulation uses.
#pragma once

#include "common.cuh"

struct sim_closure_s;

namespace dh {

// Workspace for B instances of an n^3 grid (allocates; never call inside a graph capture).
sim_status closure_prepare(sim_closure_s* c, int n, int B, bool training);
// Changes whenever closure_prepare moves the workspace: graphs that captured
// closure_apply before must be captured again.
uint64_t closure_generation(const sim_closure_s* c);
// gas (B x 5 n^3) += s * NN((gas - mu) / sigma), stream-ordered on st.
sim_status closure_apply(sim_closure_s* c, float* gas, int n, int B, cudaStream_t st);

}  // namespace dh
