// Field-level inference launchers (Sec. 3.2 of arXiv 2502.02294) used by the handle.
#pragma once

#include <cmath>

#include "common.cuh"

namespace dh {

// Adam update of B instances of `count` floats (instance stride count) with the gradient
// g + prior_w x: x, m, v in place; grad_out (may be NULL) <- g + prior_w x; prior (may be
// NULL, B doubles) += prior_w / 2 sum x^2 at the input x.
sim_status launch_fli_adam(float* x, const float* g, float* m, float* v, long long count,
                           int B, double lr, double beta1, double beta2, double eps, int t,
                           double prior_w, float* grad_out, double* prior, cudaStream_t st);

// grad = g + prior_w x; prior (may be NULL, B doubles) += prior_w / 2 sum x^2
sim_status launch_prior_grad(const float* x, const float* g, float* grad, long long count,
                             int B, double prior_w, double* prior, cudaStream_t st);

}  // namespace dh
