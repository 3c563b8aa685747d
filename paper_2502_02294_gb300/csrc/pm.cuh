// Particle-mesh gravity kernels (Sec. 2.2 of arXiv 2502.02294) and their adjoints.
#pragma once

#include <cufft.h>

#include "common.cuh"

namespace dh {

// Fixed-point scale of the deterministic CIC accumulation: weights * 2^31 in int64.
constexpr float kFix = 2147483648.0f;
constexpr float kInvFix = 4.656612873077393e-10f;

// cuFFT plans for one grid size and a batch of B instances: r2c over 1/3/4 fields per
// instance (batch B, 3B, 4B), c2r likewise (n^3 real <-> n^2(n/2+1) complex each).
struct FFTPlans {
  int n = 0, B = 0;
  cufftHandle r2c1 = 0, r2c3 = 0, r2c4 = 0, c2r1 = 0, c2r3 = 0, c2r4 = 0;
  sim_status create(int n, int B);
  void destroy();
  sim_status set_stream(cudaStream_t st);
};

// Plans (batch 1) shared by the standalone entry points, keyed by n (created on first use).
FFTPlans* shared_plans(int n);

// ------------------------------------------------------------------ launchers
// Every launcher below runs B instances of one grid size at once; array arguments hold the
// instances one after another (see SArg / DPart in common.cuh).
//
// grid (int64 fixed point, n^3) += sum_p value_p W(x_p - node); values may be NULL (= 1)
sim_status launch_deposit(const float* s, const float* values, int n, float inv_dx,
                          unsigned long long* acc, int B, cudaStream_t st);
// out = scale * fixed_to_float(acc) + add (add may be NULL; instance stride add_stride)
// + offset; acc is zeroed when zero_acc (else left for the caller to clear)
sim_status launch_fix_to_float(unsigned long long* acc, SArg scale, const float* add,
                               int add_stride, float offset, float* out, int n, int B,
                               cudaStream_t st, bool zero_acc = true);
// pref / n^3 in float, the normalisation the Green's function kernels take
float gravity_pref_norm(double pref, int n);
// g (3 n^3) from delta (n^3): r2c, Green's function * i k * pref / n^3, c2r x3
sim_status launch_gravity(const float* delta, float* g, cufftComplex* dk, cufftComplex* gk,
                          int n, double box, SArg pref_norm, int B, FFTPlans& plans,
                          cudaStream_t st);
// lam_delta (n^3) = (d g / d delta)^T lam_g (3 n^3)
sim_status launch_gravity_adjoint(const float* lam_g, float* lam_delta, cufftComplex* gk,
                                  cufftComplex* dk, int n, double box, SArg pref_norm, int B,
                                  FFTPlans& plans, cudaStream_t st);
// out[f][p] = CIC readout of grid f at particle p, nf fields
sim_status launch_interp(const float* grid, int nf, int n, float inv_dx, const float* s,
                         float* out, int B, cudaStream_t st);
// p_out = p + K interp(g, s); s_out = s + dtau p_out (s_out / p_out may be s / p: in place,
// where s is left as it is when dtau = 0). If zhat != NULL also aux += interp(zhat, s) at
// the position before the drift.
sim_status launch_kick_drift(const float* s, float* s_out, const float* p, float* p_out,
                             const float* g, SArg K, SArg dtau, const float* zhat, float* aux,
                             int n, float inv_dx, int B, cudaStream_t st);
// out = in with m += rho g K, eps += K m.g + K^2 rho |g|^2 / 2 (gas 5 n^3, g 3 n^3; out may
// be in)
sim_status launch_gas_kick(const float* in, float* out, const float* g, SArg K, int n, int B,
                           cudaStream_t st);

// ---- adjoints
// The adjoint of the force field is accumulated node-interleaved: lam_g4[b][i] = (lam_gx,
// lam_gy, lam_gz, 0) for node i of instance b (16-byte aligned), so that a particle adds
// its three components at a CIC corner with one vector atomic.
// Particle kick (+ preceding drift if dtau != 0), reverse order:
//   forward: p1 = p0 + K interp(g, s0); s1 = s0 + dtau p1
//   given lam_s (= lam_s1), lam_p (= lam_p1 from later use), both in/out:
//   lam_p1 += dtau lam_s1; d_dtau += lam_s1 . p1; lam_p0 = lam_p1;
//   lam_s0 = lam_s1 + K grad(interp g)(s0) . lam_p1; lam_g4 += interp^T(K lam_p1) (float4
//   atomics); dK += lam_p1 . interp(g)(s0).
// If lam_gas != NULL, in the same launch the gas kick's adjoint at the pre-kick gas state
// gas_u: lam_gas (5 n^3, in/out, cell-owned), lam_g4 += its partial (float4 atomic),
// dK += lam_gas . d/dK.
sim_status launch_kick_drift_adjoint(const float* s0, const float* p0, const float* g, SArg K,
                                     SArg dtau, float* lam_s, float* lam_p, float4* lam_g4,
                                     DPart dK, DPart ddtau, const float* gas_u, float* lam_gas,
                                     int n, float inv_dx, int B, cudaStream_t st);
// Deposit adjoint for delta = cm * count + rho_gas - 1:
//   lam_s += cm grad(interp lam_delta)(s) / dx ; d_cm += sum_p interp(lam_delta)(s_p);
//   lam_rho (may be NULL; instance stride rho_stride) += lam_delta cell by cell
sim_status launch_deposit_adjoint(const float* s, const float* lam_delta, SArg cm,
                                  float* lam_s, DPart dcm, int n, float inv_dx, int B,
                                  cudaStream_t st, float* lam_rho = nullptr,
                                  long long rho_stride = 0);
// lam_g[b][j][i] = lam_g4[b][i].j (j = x, y, z) and out.at(b) += sum_{i,j} lam_g4 g (the
// force-field dot product), per instance
sim_status launch_unpack_dot(const float4* lam_g4, const float* g, float* lam_g, DPart out,
                             int n, int B, cudaStream_t st);
// per instance: sum_i a_i b_i over `count` floats into out.at(b) (device double, accumulated)
sim_status launch_dot(const float* a, const float* b, long long count, DPart out, int B,
                      cudaStream_t st);
// y += alpha x over count floats
sim_status launch_axpy(float alpha, const float* x, float* y, long long count, cudaStream_t st);
// per instance b: y[b * ystride + i] += x[b * count + i], i < count
sim_status launch_add_strided(const float* x, float* y, long long count, long long ystride,
                              int B, cudaStream_t st);
// per instance: grad[0][i] = 2 c (rho_i - t_i) with rho the first field of the gas state
// (instance stride 5 n^3, as grad); loss[b] += c sum (rho - t)^2
sim_status launch_density_loss(const float* gas, const float* target, float c, float* grad,
                               double* loss, long long N3, int B, cudaStream_t st);
// per instance: u = eps - |m|^2/(2 rho); grad (5 n^3, all fields written) = 2 c (u - t) du/dU;
// loss[b] += c sum (u - t)^2
sim_status launch_thermal_loss(const float* gas, const float* target, float c, float* grad,
                               double* loss, long long N3, int B, cudaStream_t st);

}  // namespace dh
