// Stochastic star formation with Gumbel-softmax relaxation (Sec. 2.4 of arXiv 2502.02294).
//
// Per cell, with e = (eps - |m|^2/(2 rho)) / (a^2 rho), T = t_per_e e, delta = rho/f_b - 1:
//   ln pi_0 = ln Pi_0 + log sigma((delta - delta_c)/w_delta) + log sigma((T_c - T)/w_T)
//   l       = ln pi_0 - ln(1 - pi_0) + (g_0 - g_1),  g_i = -ln(-ln u_i), u from Philox
//   zhat    = sigma(l / tau)                          (Eq. gumbelsoftmax, rewritten stably)
//   event   = l > 0                                   (hard Gumbel-max draw)
//   e      <- max(e + E_0 zhat, (T_0/t_per_e) (rho/f_b)^(gamma_uv - 1))   (floor if T_0 > 0)
// Only eps changes. The adjoint holds the Gumbel draws fixed (Eq. reparam).
#include "subgrid.cuh"

namespace dh {

double temperature_per_energy(double gamma, double mu) {
  const double kB = 1.380649e-23, mp = 1.67262192595e-27, v = 1.0e5;
  return (gamma - 1.0) * mu * mp * v * v / kB;
}

SubgridConst make_subgrid_const(const sim_params& p, double a, int step) {
  SubgridConst c;
  const double fb = p.omega_b / p.omega_m;
  const double tpe = temperature_per_energy(p.gamma, p.mu);
  c.a2 = (float)(a * a);
  c.inv_a2 = (float)(1.0 / (a * a));
  c.fb = (float)fb;
  c.inv_fb = (float)(1.0 / fb);
  c.tpe = (float)tpe;
  c.delta_c = (float)p.delta_c;
  c.inv_wd = (float)(1.0 / p.w_delta);
  c.T_c = (float)p.T_c;
  c.inv_wT = (float)(1.0 / p.w_T);
  c.Pi0 = (float)p.Pi0;
  c.lnPi0 = (float)log(p.Pi0);
  c.E0 = (float)p.E0;
  c.inv_tau = (float)(1.0 / p.tau);
  c.T0 = (float)p.T0_uv;
  c.ef0 = (float)(p.T0_uv > 0 ? p.T0_uv / tpe : 0.0);
  c.gexp = (float)(p.gamma_uv - 1.0);
  c.inv_T0 = (float)(p.T0_uv > 0 ? 1.0 / p.T0_uv : 0.0);
  c.inv_Pi0 = (float)(1.0 / p.Pi0);
  c.mgexp_fb = (float)(-(p.gamma_uv - 1.0) / fb);
  c.k0 = (uint32_t)(p.seed & 0xffffffffull);
  c.k1 = (uint32_t)(p.seed >> 32);
  c.step = (uint32_t)step;
  c.instance = (uint32_t)p.instance;
  return c;
}

__device__ __forceinline__ float log_sigmoid(float x) {
  // -softplus(-x) = -(max(-x, 0) + log1p(exp(-|x|)))
  return -(fmaxf(-x, 0.0f) + log1pf(__expf(-fabsf(x))));
}

__device__ __forceinline__ float sigmoidf_(float x) { return __frcp_rn(1.0f + __expf(-x)); }

// One reciprocal of rho serves every division by it (the forward's and the adjoint's).
struct SgFwd {
  float inv_rho, ke, e, T, delta, x1, x2, lnpi, pi, logit, zhat, e1, lnr, ef, e2;
  bool floor_on, use_floor;
};

// gd = g0 - g1, the only way the Gumbel pair enters (the forward and the adjoint use the
// same float, drawn once or read back from the tape)
__device__ __forceinline__ void subgrid_cell(const float u[5], const SubgridConst& c, float gd,
                                             SgFwd& r) {
  const float rho = u[0];
  r.inv_rho = __frcp_rn(rho);
  r.ke = 0.5f * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * r.inv_rho;
  r.e = (u[4] - r.ke) * r.inv_rho * c.inv_a2;
  r.T = c.tpe * r.e;
  r.delta = rho * c.inv_fb - 1.0f;
  r.x1 = (r.delta - c.delta_c) * c.inv_wd;
  r.x2 = (c.T_c - r.T) * c.inv_wT;
  r.lnpi = c.lnPi0 + log_sigmoid(r.x1) + log_sigmoid(r.x2);
  r.pi = expf(r.lnpi);
  r.logit = (r.lnpi - log1pf(-r.pi)) + gd;
  r.zhat = sigmoidf_(r.logit * c.inv_tau);
  r.e1 = r.e + c.E0 * r.zhat;
  r.floor_on = c.ef0 > 0.0f;
  // (rho / f_b)^(gamma_uv - 1) through its logarithm, which the adjoint reuses
  r.lnr = r.floor_on ? logf(rho * c.inv_fb) : 0.0f;
  r.ef = r.floor_on ? c.ef0 * expf(c.gexp * r.lnr) : 0.0f;
  r.use_floor = r.floor_on && !(r.e1 >= r.ef);
  r.e2 = r.use_floor ? r.ef : r.e1;
}

__device__ __forceinline__ float gumbel_diff(const SubgridConst& c, long long i) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)i, c.step, c.instance, TAG_SUBGRID), c.k0, c.k1);
  const float g0 = -logf(-logf(uniform_from_word(w.x)));
  const float g1 = -logf(-logf(uniform_from_word(w.y)));
  return g0 - g1;
}

// grid (cdiv(N3, 256), B); instance b uses constants ca.at(b)
// gd_out (may be NULL): g0 - g1 of every cell, for the adjoint of the same step; star (may
// be NULL, used with zhat): the star mesh, += zhat
__global__ void subgrid_kernel(const float* __restrict__ in, float* __restrict__ out,
                               SubArg ca, float* __restrict__ zhat,
                               uint32_t* __restrict__ events, float* __restrict__ gd_out,
                               float* __restrict__ star, long long N3) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  in += (size_t)b * 5 * N3;
  out += (size_t)b * 5 * N3;
  if (zhat) zhat += (size_t)b * N3;
  if (events) events += (size_t)b * ((N3 + 31) / 32);
  const SubgridConst c = ca.at(b);
  bool ev = false;
  if (i < N3) {
    float u[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) u[k] = in[k * N3 + i];
    const float gd = gumbel_diff(c, i);
    if (gd_out) gd_out[(size_t)b * N3 + i] = gd;
    SgFwd r;
    subgrid_cell(u, c, gd, r);
    ev = r.logit > 0.0f;
    if (out != in) {
#pragma unroll
      for (int k = 0; k < 4; ++k) out[k * N3 + i] = u[k];
    }
    out[4 * N3 + i] = r.ke + c.a2 * u[0] * r.e2;
    if (zhat) {
      zhat[i] = r.zhat;
      if (star) star[(size_t)b * N3 + i] += r.zhat;
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, ev);
  if (events && (threadIdx.x & 31) == 0) {
    const long long word = i >> 5;
    if (word * 32 < N3) events[word] = mask;
  }
}

// gd_in (may be NULL): the g0 - g1 the forward drew (else drawn again from Philox)
__global__ void subgrid_adj_kernel(const float* __restrict__ in, float* __restrict__ lam,
                                   SubArg ca, DPart dpar_b, DPart dfb_b,
                                   const float* __restrict__ gd_in, long long N3) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  in += (size_t)b * 5 * N3;
  lam += (size_t)b * 5 * N3;
  const SubgridConst c = ca.at(b);
  double* dpar = dpar_b.at(b);
  double* dfb = dfb_b.at(b);
  float a_dc = 0, a_pi = 0, a_e0 = 0, a_t0 = 0, a_g = 0, a_fb = 0;
  if (i < N3) {
    float u[5], l[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      u[k] = in[k * N3 + i];
      l[k] = lam[k * N3 + i];
    }
    const float gd = gd_in ? __ldg(gd_in + (size_t)b * N3 + i) : gumbel_diff(c, i);
    SgFwd r;
    subgrid_cell(u, c, gd, r);
    const float rho = u[0];
    // eps' = ke + a^2 rho e2
    const float leps = l[4];
    float lke = leps;
    float lrho = l[0] + leps * c.a2 * r.e2;
    const float le2 = leps * c.a2 * rho;
    float le1 = 0.0f;
    const float irho = r.inv_rho;
    if (r.use_floor) {
      const float lef = le2;
      lrho += lef * r.ef * c.gexp * irho;
      a_t0 = lef * r.ef * c.inv_T0;
      a_g = lef * r.ef * r.lnr;
      a_fb += lef * r.ef * c.mgexp_fb;
    } else {
      le1 = le2;
    }
    float le = le1;
    a_e0 = le1 * r.zhat;
    const float lz = le1 * c.E0;
    const float ll = lz * r.zhat * (1.0f - r.zhat) * c.inv_tau;
    const float llnpi = __fdividef(ll, 1.0f - r.pi);
    a_pi = llnpi * c.inv_Pi0;
    const float lx1 = llnpi * sigmoidf_(-r.x1);
    const float lx2 = llnpi * sigmoidf_(-r.x2);
    const float ldelta = lx1 * c.inv_wd;
    a_dc = -ldelta;
    const float lT = -lx2 * c.inv_wT;
    le += lT * c.tpe;
    lrho += ldelta * c.inv_fb;
    a_fb += -(ldelta * rho * c.inv_fb * c.inv_fb);
    // e = (eps - ke) / (a^2 rho)
    const float inv_a2r = irho * c.inv_a2;
    const float leps_in = le * inv_a2r;
    lke -= le * inv_a2r;
    lrho -= le * r.e * irho;
    // ke = |m|^2 / (2 rho)
#pragma unroll
    for (int k = 1; k <= 3; ++k) lam[k * N3 + i] = l[k] + lke * u[k] * irho;
    lrho -= lke * r.ke * irho;
    lam[i] = lrho;
    lam[4 * N3 + i] = leps_in;
  }
  if (dpar) {
    block_sum_atomic(a_dc, dpar + SIM_P_DELTA_C);
    block_sum_atomic(a_pi, dpar + SIM_P_PI0);
    block_sum_atomic(a_e0, dpar + SIM_P_E0);
    block_sum_atomic(a_t0, dpar + SIM_P_T0_UV);
    block_sum_atomic(a_g, dpar + SIM_P_GAMMA_UV);
  }
  if (dfb) block_sum_atomic(a_fb, dfb);
}

sim_status launch_subgrid(const float* in, float* out, SubArg c, float* zhat,
                          uint32_t* events, long long N3, int B, cudaStream_t st, float* gd,
                          float* star) {
  DH_CUDA_TRY((launch_pdl(subgrid_kernel, dim3(cdiv(N3, 256), B), 256, 0, st, in, out, c, zhat, events, gd, star, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

sim_status launch_subgrid_adjoint(const float* in, float* lam, SubArg c, DPart dpar, DPart dfb,
                                  long long N3, int B, cudaStream_t st, const float* gd) {
  DH_CUDA_TRY((launch_pdl(subgrid_adj_kernel, dim3(cdiv(N3, 256), B), 256, 0, st, in, lam, c, dpar, dfb, gd, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// grid (blocks, B): out[b] = float bits of instance b's maximum signal speed
// max that keeps a NaN from either operand
__device__ __forceinline__ float max_keep_nan(float a, float b) {
  return (a != a || b != b) ? __int_as_float(0x7fc00000) : fmaxf(a, b);
}

__global__ void signal_speed_kernel(const float* __restrict__ u, float gam, long long N3,
                                    unsigned int* __restrict__ out) {
  pdl_enter();
  const int b = blockIdx.y;
  u += (size_t)b * 5 * N3;
  out += b;
  float vmax = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x) {
    const float rho = u[i], inv = 1.0f / rho;
    const float mx = u[N3 + i], my = u[2 * N3 + i], mz = u[3 * N3 + i];
    const float P = (gam - 1.0f) * (u[4 * N3 + i] - 0.5f * (mx * mx + my * my + mz * mz) * inv);
    const float cs2 = gam * P * inv;
    const float cs = cs2 > 0.0f ? sqrtf(cs2) : 0.0f;
    const float v = fmaxf(fabsf(mx), fmaxf(fabsf(my), fabsf(mz))) * inv;
    vmax = max_keep_nan(vmax, v + cs);
    // fmaxf drops NaN operands: a non-finite energy or momentum must still reach the host
    if (!isfinite(rho) || !isfinite(mx) || !isfinite(my) || !isfinite(mz) ||
        !isfinite(u[4 * N3 + i]))
      vmax = __int_as_float(0x7fc00000);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = max_keep_nan(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  // speeds are >= 0 and a quiet NaN (0x7fc00000) orders above every finite float's bits
  if ((threadIdx.x & 31) == 0) atomicMax(out, vmax != vmax ? 0x7fc00000u : __float_as_uint(vmax));
}

sim_status launch_signal_speed(const float* gas, float gamma, long long N3,
                               unsigned int* out_bits, int B, cudaStream_t st) {
  int blocks = cdiv(N3, 256);
  const int cap = cdiv(152 * 8, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(signal_speed_kernel, dim3(blocks, B), 256, 0, st, gas, gamma, N3, out_bits)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

}  // namespace dh

using namespace dh;

extern "C" sim_status sim_max_signal_speed(const float* gas, int32_t n, double gamma,
                                           float* out, void* stream) {
  if (!gas || !out || n < 1 || !(gamma > 1)) {
    set_error("sim_max_signal_speed: invalid arguments");
    return SIM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DH_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(float), st));
  // speeds are >= 0, so the largest float is the largest bit pattern (a NaN above all)
  return launch_signal_speed(gas, (float)gamma, (long long)n * n * n,
                             reinterpret_cast<unsigned int*>(out), 1, st);
}

extern "C" sim_status sim_subgrid(float* gas, int32_t n, double a, const sim_params* p,
                                  int32_t step, float* zhat, uint32_t* events, void* stream) {
  if (!gas || !p || n < 1 || !(a > 0) || !(p->Pi0 > 0 && p->Pi0 < 1) || !(p->tau > 0) ||
      !(p->w_delta > 0) || !(p->w_T > 0) || !(p->omega_b > 0) || !(p->omega_m > 0)) {
    set_error("sim_subgrid: invalid arguments (need 0 < Pi0 < 1, tau, widths, omegas > 0)");
    return SIM_EINVAL;
  }
  const long long N3 = (long long)n * n * n;
  return launch_subgrid(gas, gas, subarg(make_subgrid_const(*p, a, step)), zhat, events, N3, 1,
                        (cudaStream_t)stream);
}

extern "C" sim_status sim_subgrid_adjoint(const float* gas_in, float* lam, int32_t n, double a,
                                          const sim_params* p, int32_t step, double* dparams,
                                          double* dfb, void* stream) {
  if (!gas_in || !lam || !p || n < 1 || !(a > 0) || !(p->Pi0 > 0 && p->Pi0 < 1) ||
      !(p->tau > 0) || !(p->w_delta > 0) || !(p->w_T > 0)) {
    set_error("sim_subgrid_adjoint: invalid arguments");
    return SIM_EINVAL;
  }
  const long long N3 = (long long)n * n * n;
  return launch_subgrid_adjoint(gas_in, lam, subarg(make_subgrid_const(*p, a, step)),
                                dpart(dparams), dpart(dfb), N3, 1, (cudaStream_t)stream);
}

__global__ void philox_kernel(uint32_t k0, uint32_t k1, uint32_t step, uint32_t inst,
                              uint32_t tag, long long count, uint32_t* out) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)i, step, inst, tag), k0, k1);
  reinterpret_cast<uint4*>(out)[i] = w;
}

extern "C" sim_status sim_philox(uint64_t seed, uint32_t step, uint32_t instance, uint32_t tag,
                                 int64_t count, uint32_t* out, void* stream) {
  if (!out || count < 0 || count > 0xffffffffll || ((uintptr_t)out & 15)) {
    set_error("sim_philox: invalid arguments (out must be 16-byte aligned, count < 2^32)");
    return SIM_EINVAL;
  }
  if (count == 0) return SIM_OK;
  DH_CUDA_TRY((launch_pdl(philox_kernel, cdiv(count, 256), 256, 0, (cudaStream_t)stream, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32), step, instance, tag, count, out)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}
