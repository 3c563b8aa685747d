// Subgrid star formation (Sec. 2.4 of arXiv 2502.02294): launchers.
#pragma once

#include "common.cuh"

namespace dh {

// Per-run constants of the subgrid step, in float for the kernels.
struct SubgridConst {
  float a2;        // a^2 at the update
  float inv_a2;    // 1 / a^2
  float inv_fb;    // 1 / f_b
  float fb;
  float tpe;       // temperature per unit specific energy
  float delta_c, inv_wd, T_c, inv_wT, lnPi0, Pi0, E0, inv_tau;
  float ef0;       // T0_uv / tpe (0: floor off)
  float gexp;      // gamma_uv - 1
  float T0;
  float inv_T0, inv_Pi0, mgexp_fb;  // 1 / T0_uv (0 when off), 1 / Pi0, -(gamma_uv - 1) / f_b
  uint32_t k0, k1, step, instance;
};

SubgridConst make_subgrid_const(const sim_params& p, double a, int step);

// Constants of a batched launch: one set for all instances, or a device array per instance.
struct SubArg {
  SubgridConst v;
  const SubgridConst* p;
  __device__ __forceinline__ SubgridConst at(int b) const { return p ? p[b] : v; }
};
inline SubArg subarg(const SubgridConst& v) { return SubArg{v, nullptr}; }
inline SubArg subarg(const SubgridConst* p) { return SubArg{SubgridConst{}, p}; }
double temperature_per_energy(double gamma, double mu);

// B instances one after another (as the PM launchers).
// out = subgrid(in) (may alias); zhat (n^3) and events (ceil(n^3/32) words) may be NULL
// gd (may be NULL): receives g0 - g1 of every cell ([B][n^3]) for the adjoint of this step;
// star (may be NULL, with zhat): the star mesh, += zhat
sim_status launch_subgrid(const float* in, float* out, SubArg c, float* zhat,
                          uint32_t* events, long long N3, int B, cudaStream_t st,
                          float* gd = nullptr, float* star = nullptr);
// lam (5 n^3) in/out through the update at `in`; dpar[SIM_P_*] and dfb accumulated.
// gd (may be NULL): the forward's g0 - g1 (else the pair is drawn again from Philox)
sim_status launch_subgrid_adjoint(const float* in, float* lam, SubArg c, DPart dpar, DPart dfb,
                                  long long N3, int B, cudaStream_t st,
                                  const float* gd = nullptr);
// max over cells and directions of |v_d| + c_s  (float bits in out_bits[b], atomicMax)
sim_status launch_signal_speed(const float* gas, float gamma, long long N3,
                               unsigned int* out_bits, int B, cudaStream_t st);

}  // namespace dh
