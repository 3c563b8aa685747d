// Initial conditions (Sec. 2.1 of arXiv 2502.02294): launchers.
#pragma once

#include "pm.cuh"

namespace dh {

// Philox (tag 0) Box-Muller white noise, n^3 floats.
sim_status launch_noise(uint64_t seed, int instance, float* w, long long N3, cudaStream_t st);
// delta and Zel'dovich psi (4 n^3) from white noise; ck needs 5 n^2(n/2+1) complex.
sim_status launch_linear_field(const float* w, float* f4, cufftComplex* ck, int n, double box,
                               double kc_frac, double C, FFTPlans& plans, cudaStream_t st);
// DM and gas state from (delta, psi).
sim_status launch_place(const float* f4, float* gas, float* s, float* p, double rp, double fb,
                        double a2e0, long long N3, cudaStream_t st);
// Adjoint: lam4 (4 n^3 scratch) <- d/d(delta, psi); lam_w (n^3, may be NULL) <- d/dw;
// drp, dfb accumulated. lgas / ls / lp may be NULL (zero).
sim_status launch_ic_adjoint(const float* f4, const float* lgas, const float* ls,
                             const float* lp, float* lam4, float* lam_w, cufftComplex* ck,
                             int n, double box, double kc_frac, double C, double rp, double fb,
                             double a2e0, double* drp, double* dfb, FFTPlans& plans,
                             cudaStream_t st);

}  // namespace dh
