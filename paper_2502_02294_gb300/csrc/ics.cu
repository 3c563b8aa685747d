// Initial conditions (Sec. 2.1 of arXiv 2502.02294) and their adjoint.
//
// white noise w -> W = fft(w) -> D_k = (C/n^3) sqrt(P(k)) W_k, Psi_j,k = i kgrad_j / k^2 D_k
// -> (delta, psi_x, psi_y, psi_z) by one batched c2r -> DM s = psi, p = r_p psi; gas
// rho = f_b (1 + delta), m = rho p, eps = a^2 rho e_0 + |m|^2 / (2 rho).
// P(k) = k^-2 exp(-(k/k_c)^2); C normalises the expected cell rms of delta (host, FP64).
#include "ics.cuh"

namespace dh {

__global__ void noise_kernel(uint32_t k0, uint32_t k1, uint32_t inst, float* __restrict__ w,
                             long long N3) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N3) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0u, inst, TAG_IC_NOISE), k0, k1);
  const float u1 = uniform_from_word(r.x), u2 = uniform_from_word(r.y);
  w[i] = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__device__ __forceinline__ void kvec(long long i, int n, int nh, float kf, float kc,
                                     float& sqrtP, float& ix, float& iy, float& iz) {
  int kx = (int)(i % nh);
  const long long r = i / nh;
  int ky = (int)(r % n), kz = (int)(r / n);
  const bool even = (n % 2 == 0);
  const bool nx = even && kx == n / 2, ny = even && ky == n / 2, nz = even && kz == n / 2;
  if (ky > n / 2) ky -= n;
  if (kz > n / 2) kz -= n;
  const float fx = kf * kx, fy = kf * ky, fz = kf * kz;
  const float k2 = fx * fx + fy * fy + fz * fz;
  if (k2 > 0.0f) {
    const float k = sqrtf(k2);
    const float q = k / kc;
    sqrtP = expf(-0.5f * q * q) / k;
    const float inv = 1.0f / k2;
    ix = nx ? 0.0f : fx * inv;
    iy = ny ? 0.0f : fy * inv;
    iz = nz ? 0.0f : fz * inv;
  } else {
    sqrtP = ix = iy = iz = 0.0f;
  }
}

// out[0] = Cn sqrtP W ; out[1+j] = i kgrad_j / k^2 * out[0]
__global__ void shape_kernel(const cufftComplex* __restrict__ W, cufftComplex* __restrict__ out,
                             int n, float kf, float kc, float Cn) {
  pdl_enter();
  const int nh = n / 2 + 1;
  const long long NC = (long long)n * n * nh;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NC) return;
  float sp, ix, iy, iz;
  kvec(i, n, nh, kf, kc, sp, ix, iy, iz);
  const cufftComplex w = W[i];
  const float dr = Cn * sp * w.x, di = Cn * sp * w.y;
  out[i] = make_cuFloatComplex(dr, di);
  out[NC + i] = make_cuFloatComplex(-ix * di, ix * dr);
  out[2 * NC + i] = make_cuFloatComplex(-iy * di, iy * dr);
  out[3 * NC + i] = make_cuFloatComplex(-iz * di, iz * dr);
}

// adjoint of shape + c2r: Y = Cn sqrtP (L0 - i sum_j kgrad_j/k^2 L_j)
__global__ void unshape_kernel(const cufftComplex* __restrict__ L, cufftComplex* __restrict__ Y,
                               int n, float kf, float kc, float Cn) {
  pdl_enter();
  const int nh = n / 2 + 1;
  const long long NC = (long long)n * n * nh;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NC) return;
  float sp, ix, iy, iz;
  kvec(i, n, nh, kf, kc, sp, ix, iy, iz);
  const cufftComplex a = L[i], bx = L[NC + i], by = L[2 * NC + i], bz = L[3 * NC + i];
  // -i c (re + i im) = c im - i c re
  const float re = a.x + ix * bx.y + iy * by.y + iz * bz.y;
  const float im = a.y - (ix * bx.x + iy * by.x + iz * bz.x);
  Y[i] = make_cuFloatComplex(Cn * sp * re, Cn * sp * im);
}

__global__ void place_kernel(const float* __restrict__ f4, float* __restrict__ gas,
                             float* __restrict__ s, float* __restrict__ p, float rp, float fb,
                             float a2e0, long long N3) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N3) return;
  const float delta = f4[i];
  const float rho = fb * (1.0f + delta);
  float m2 = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float psi = f4[(1 + j) * N3 + i];
    const float pj = rp * psi;
    s[j * N3 + i] = psi;
    p[j * N3 + i] = pj;
    const float mj = rho * pj;
    gas[(1 + j) * N3 + i] = mj;
    m2 += mj * mj;
  }
  gas[i] = rho;
  gas[4 * N3 + i] = a2e0 * rho + 0.5f * m2 / rho;
}

// Reverse of place_kernel: lam4 = (lam_delta, lam_psi_x, lam_psi_y, lam_psi_z);
// d_rp += sum (lam_p . psi + lam_m . rho psi), d_fb += sum lam_rho (1 + delta)
__global__ void unplace_kernel(const float* __restrict__ f4, const float* __restrict__ lgas,
                               const float* __restrict__ ls, const float* __restrict__ lp,
                               float* __restrict__ lam4, float rp, float fb, float a2e0,
                               double* __restrict__ drp, double* __restrict__ dfb, long long N3) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float arp = 0.0f, afb = 0.0f;
  if (i < N3) {
    const float delta = f4[i];
    const float rho = fb * (1.0f + delta);
    float psi[3], m[3], m2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      psi[j] = f4[(1 + j) * N3 + i];
      m[j] = rho * rp * psi[j];
      m2 += m[j] * m[j];
    }
    const float le = lgas ? lgas[4 * N3 + i] : 0.0f;
    float lrho = (lgas ? lgas[i] : 0.0f) + le * (a2e0 - 0.5f * m2 / (rho * rho));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float lm = (lgas ? lgas[(1 + j) * N3 + i] : 0.0f) + le * m[j] / rho;
      lrho += lm * rp * psi[j];
      const float lpj = lp ? lp[j * N3 + i] : 0.0f;
      const float lsj = ls ? ls[j * N3 + i] : 0.0f;
      lam4[(1 + j) * N3 + i] = lsj + rp * lpj + lm * rho * rp;
      arp += lpj * psi[j] + lm * rho * psi[j];
    }
    lam4[i] = fb * lrho;
    afb = lrho * (1.0f + delta);
  }
  block_sum_atomic(arp, drp);
  block_sum_atomic(afb, dfb);
}

sim_status launch_noise(uint64_t seed, int instance, float* w, long long N3, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(noise_kernel, cdiv(N3, 256), 256, 0, st, (uint32_t)(seed & 0xffffffffull),
                                               (uint32_t)(seed >> 32), (uint32_t)instance, w, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// f4 (4 n^3): delta, psi_x, psi_y, psi_z from noise w (n^3). ck: 5 NC complex scratch.
sim_status launch_linear_field(const float* w, float* f4, cufftComplex* ck, int n, double box,
                               double kc_frac, double C, FFTPlans& plans, cudaStream_t st) {
  const long long NC = (long long)n * n * (n / 2 + 1);
  DH_TRY(plans.set_stream(st));
  if (cufftExecR2C(plans.r2c1, const_cast<float*>(w), ck) != CUFFT_SUCCESS) {
    set_error("cufftExecR2C (ICs) failed");
    return SIM_ECUDA;
  }
  const float kf = (float)(2.0 * M_PI / box);
  const float kc = (float)(kc_frac * M_PI * n / box);
  const float Cn = (float)(C / ((double)n * n * n));
  DH_CUDA_TRY((launch_pdl(shape_kernel, cdiv(NC, 256), 256, 0, st, ck, ck + NC, n, kf, kc, Cn)));
  DH_LAUNCH_CHECK();
  if (cufftExecC2R(plans.c2r4, ck + NC, f4) != CUFFT_SUCCESS) {
    set_error("cufftExecC2R (ICs) failed");
    return SIM_ECUDA;
  }
  return SIM_OK;
}

sim_status launch_place(const float* f4, float* gas, float* s, float* p, double rp, double fb,
                        double a2e0, long long N3, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(place_kernel, cdiv(N3, 256), 256, 0, st, f4, gas, s, p, (float)rp, (float)fb,
                                               (float)a2e0, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

sim_status launch_ic_adjoint(const float* f4, const float* lgas, const float* ls,
                             const float* lp, float* lam4, float* lam_w, cufftComplex* ck,
                             int n, double box, double kc_frac, double C, double rp, double fb,
                             double a2e0, double* drp, double* dfb, FFTPlans& plans,
                             cudaStream_t st) {
  const long long N3 = (long long)n * n * n;
  const long long NC = (long long)n * n * (n / 2 + 1);
  DH_CUDA_TRY((launch_pdl(unplace_kernel, cdiv(N3, 256), 256, 0, st, f4, lgas, ls, lp, lam4, (float)rp, (float)fb,
                                                 (float)a2e0, drp, dfb, N3)));
  DH_LAUNCH_CHECK();
  if (!lam_w) return SIM_OK;
  DH_TRY(plans.set_stream(st));
  if (cufftExecR2C(plans.r2c4, lam4, ck) != CUFFT_SUCCESS) {
    set_error("cufftExecR2C (IC adjoint) failed");
    return SIM_ECUDA;
  }
  const float kf = (float)(2.0 * M_PI / box);
  const float kc = (float)(kc_frac * M_PI * n / box);
  const float Cn = (float)(C / ((double)n * n * n));
  DH_CUDA_TRY((launch_pdl(unshape_kernel, cdiv(NC, 256), 256, 0, st, ck, ck + 4 * NC, n, kf, kc, Cn)));
  DH_LAUNCH_CHECK();
  if (cufftExecC2R(plans.c2r1, ck + 4 * NC, lam_w) != CUFFT_SUCCESS) {
    set_error("cufftExecC2R (IC adjoint) failed");
    return SIM_ECUDA;
  }
  return SIM_OK;
}

}  // namespace dh
