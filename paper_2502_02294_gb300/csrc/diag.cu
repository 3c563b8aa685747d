// Per-step diagnostics of a run (the time-step control of Sec. 2.3.3 and the conservation
// properties of the finite-volume scheme, Sec. 2.3): totals of the gas mass, momentum and
// energy, of the dark-matter momentum, of the step's relaxed star field and hard events,
// the smallest density and pressure, and a count of non-finite cells. One launch per
// recorded state reads the gas (20 B per cell), the particle momenta (12 B per particle),
// the step's zhat (4 B) and event words; it writes one record per instance.
#include <climits>
#include <cstring>

#include "diag.cuh"

namespace dh {

// order-preserving map of a float onto an int (atomicMin on ints orders the floats)
__device__ __forceinline__ int float_to_ordered(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}

float ordered_to_float(int i) {
  if (i == INT_MAX) return NAN;  // no finite value was recorded
  if (i < 0) i ^= 0x7FFFFFFF;
  float f;
  memcpy(&f, &i, sizeof(f));
  return f;
}

__global__ void __launch_bounds__(256) diag_kernel(const float* __restrict__ gas,
                                                   const float* __restrict__ p,
                                                   const float* __restrict__ zhat,
                                                   const uint32_t* __restrict__ events,
                                                   long long N3, float gam, SArg cm,
                                                   double* __restrict__ sums,
                                                   int* __restrict__ mins) {
  pdl_enter();
  const int b = blockIdx.y;
  gas += (size_t)b * 5 * N3;
  p += (size_t)b * 3 * N3;
  if (zhat) zhat += (size_t)b * N3;
  const long long nw = (N3 + 31) / 32;
  if (events) events += (size_t)b * nw;
  sums += (size_t)b * DG_NSUM;
  mins += (size_t)b * 2;
  float acc[DG_NSUM];
#pragma unroll
  for (int k = 0; k < DG_NSUM; ++k) acc[k] = 0.0f;
  float rmin = __int_as_float(0x7f800000), pmin = rmin;  // +inf
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3; i += stride) {
    const float rho = gas[i], mx = gas[N3 + i], my = gas[2 * N3 + i], mz = gas[3 * N3 + i];
    const float e = gas[4 * N3 + i];
    const float P = (gam - 1.0f) * (e - 0.5f * (mx * mx + my * my + mz * mz) / rho);
    const bool fin = isfinite(rho) && isfinite(mx) && isfinite(my) && isfinite(mz) &&
                     isfinite(e) && isfinite(P);
    if (fin) {
      acc[DG_S_MASS] += rho;
      acc[DG_S_MX] += mx;
      acc[DG_S_MY] += my;
      acc[DG_S_MZ] += mz;
      acc[DG_S_ENERGY] += e;
      rmin = fminf(rmin, rho);
      pmin = fminf(pmin, P);
    } else {
      acc[DG_S_NONFINITE] += 1.0f;
    }
    acc[DG_S_PX] += p[i];
    acc[DG_S_PY] += p[N3 + i];
    acc[DG_S_PZ] += p[2 * N3 + i];
    if (zhat) acc[DG_S_STARS] += zhat[i];
  }
  if (events)
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += stride)
      acc[DG_S_EVENTS] += (float)__popc(events[w]);
  const float cmb = cm.at(b);
  acc[DG_S_PX] *= cmb;
  acc[DG_S_PY] *= cmb;
  acc[DG_S_PZ] *= cmb;
#pragma unroll
  for (int k = 0; k < DG_NSUM; ++k) block_sum_atomic(acc[k], sums + k);
  // minima: warp, then one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    pmin = fminf(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (rmin < __int_as_float(0x7f800000)) atomicMin(mins, float_to_ordered(rmin));
    if (pmin < __int_as_float(0x7f800000)) atomicMin(mins + 1, float_to_ordered(pmin));
  }
}

__global__ void diag_clear_kernel(double* __restrict__ sums, int* __restrict__ mins, int B) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * DG_NSUM) sums[i] = 0.0;
  if (i < B * 2) mins[i] = INT_MAX;
}

sim_status launch_diag(const float* gas, const float* p, const float* zhat,
                       const uint32_t* events, long long N3, float gamma, SArg cm, int B,
                       double* sums, int* mins, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(diag_clear_kernel, cdiv((long long)B * DG_NSUM, 128), 128, 0, st, sums, mins, B)));
  DH_LAUNCH_CHECK();
  int blocks = cdiv(N3, 256);
  const int cap = cdiv(152 * 4, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(diag_kernel, dim3(blocks, B), 256, 0, st, gas, p, zhat, events, N3, gamma, cm, sums, mins)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

}  // namespace dh
