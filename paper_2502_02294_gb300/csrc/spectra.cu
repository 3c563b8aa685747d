// Binned power spectrum (Sec. 3.1 of arXiv 2502.02294; cross spectrum for r_c, Sec. 3.2).
// Bins of width k_f = 2 pi / L, index round(|k| / k_f); the half spectrum counts twice for
// 0 < k_x < n/2. Each CTA histograms its modes in shared memory (FP64) and adds its bins
// to the global sums once.
#include "pm.cuh"

namespace dh {

__global__ void pk_bin_kernel(const cufftComplex* __restrict__ a, const cufftComplex* __restrict__ b,
                              int n, int nbins, double* __restrict__ sums) {
  pdl_enter();
  extern __shared__ double hist[];  // 3 * nbins: weight, weight*|k|, weight*power
  for (int j = threadIdx.x; j < 3 * nbins; j += blockDim.x) hist[j] = 0.0;
  __syncthreads();
  const int nh = n / 2 + 1;
  const long long NC = (long long)n * n * nh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < NC;
       i += (long long)gridDim.x * blockDim.x) {
    int kx = (int)(i % nh);
    const long long r = i / nh;
    int ky = (int)(r % n), kz = (int)(r / n);
    if (ky > n / 2) ky -= n;
    if (kz > n / 2) kz -= n;
    const double kk = sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz);
    const int bin = (int)rint(kk);
    if (bin < 1 || bin > nbins) continue;
    const double w = (kx == 0 || (n % 2 == 0 && kx == n / 2)) ? 1.0 : 2.0;
    const cufftComplex x = a[i], y = b[i];
    const double pw = (double)x.x * y.x + (double)x.y * y.y;
    atomicAdd(&hist[bin - 1], w);
    atomicAdd(&hist[nbins + bin - 1], w * kk);
    atomicAdd(&hist[2 * nbins + bin - 1], w * pw);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 3 * nbins; j += blockDim.x)
    if (hist[j] != 0.0) atomicAdd(&sums[j], hist[j]);
}

__global__ void pk_finish_kernel(const double* __restrict__ sums, int nbins, double kf,
                                 double norm, double* __restrict__ k, double* __restrict__ pk,
                                 double* __restrict__ nm) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nbins) return;
  const double w = sums[j];
  nm[j] = w;
  k[j] = w > 0 ? kf * sums[nbins + j] / w : 0.0;
  pk[j] = w > 0 ? norm * sums[2 * nbins + j] / w : 0.0;
}

// Adjoint of the binned spectrum: for the half-complex mode k of bin b,
//   ak <- ak * 2 norm dL/dP_b / W_b   (W_b the bin's mode weight, from sums[0..nbins)),
// modes outside bins 1..nbins <- 0. The unnormalised c2r of the result is dL/da: each P_b is
// norm / W_b sum_half w |a_k|^2, and the half-complex weights w make sum_half w Re(conj(a_k)
// e^{-ikx}) the full-grid sum that c2r evaluates.
__global__ void pk_adj_scale_kernel(cufftComplex* __restrict__ ak, int n, int nbins,
                                    const double* __restrict__ dL_dpk,
                                    const double* __restrict__ sums, double norm) {
  pdl_enter();
  const int nh = n / 2 + 1;
  const long long NC = (long long)n * n * nh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < NC;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nh);
    const long long r = i / nh;
    int ky = (int)(r % n), kz = (int)(r / n);
    if (ky > n / 2) ky -= n;
    if (kz > n / 2) kz -= n;
    const int bin = (int)rint(sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz));
    float c = 0.0f;
    if (bin >= 1 && bin <= nbins && sums[bin - 1] > 0)
      c = (float)(2.0 * norm * dL_dpk[bin - 1] / sums[bin - 1]);
    ak[i].x *= c;
    ak[i].y *= c;
  }
}

}  // namespace dh

using namespace dh;

extern "C" sim_status sim_power_spectrum_adjoint(const float* a, int32_t n, double box,
                                                 int32_t nbins, const double* dL_dpk,
                                                 float* dL_da, void* stream) {
  if (!a || !dL_dpk || !dL_da || n < 2 || !(box > 0) || nbins < 1 || nbins > 2048) {
    set_error("sim_power_spectrum_adjoint: invalid arguments (1 <= nbins <= 2048)");
    return SIM_EINVAL;
  }
  FFTPlans* plans = shared_plans(n);
  if (!plans) return SIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long NC = (long long)n * n * (n / 2 + 1);
  cufftComplex* ak = nullptr;
  double* sums = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&ak, NC * sizeof(cufftComplex), st));
  if (cudaMallocAsync((void**)&sums, 3 * nbins * sizeof(double), st) != cudaSuccess) {
    cudaFreeAsync(ak, st);
    set_error("cudaMallocAsync failed");
    return SIM_ENOMEM;
  }
  sim_status r = plans->set_stream(st);
  if (r == SIM_OK && cudaMemsetAsync(sums, 0, 3 * nbins * sizeof(double), st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK && cufftExecR2C(plans->r2c1, const_cast<float*>(a), ak) != CUFFT_SUCCESS) {
    set_error("cufftExecR2C failed");
    r = SIM_ECUDA;
  }
  int blocks = cdiv(NC, 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (r == SIM_OK) {  // mode weights per bin (the power sums are not needed)
    DH_CUDA_TRY((launch_pdl(pk_bin_kernel, blocks, 256, 3 * nbins * sizeof(double), st, ak, ak, n, nbins, sums)));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("pk_bin_kernel launch failed");
      r = SIM_ECUDA;
    }
  }
  if (r == SIM_OK) {
    const double norm = box * box * box / ((double)n * n * n * (double)n * n * n);
    DH_CUDA_TRY((launch_pdl(pk_adj_scale_kernel, blocks, 256, 0, st, ak, n, nbins, dL_dpk, sums, norm)));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("pk_adj_scale_kernel launch failed");
      r = SIM_ECUDA;
    }
  }
  if (r == SIM_OK && cufftExecC2R(plans->c2r1, ak, dL_da) != CUFFT_SUCCESS) {
    set_error("cufftExecC2R failed");
    r = SIM_ECUDA;
  }
  cudaFreeAsync(ak, st);
  cudaFreeAsync(sums, st);
  return r;
}

extern "C" sim_status sim_power_spectrum(const float* a, const float* b, int32_t n, double box,
                                         int32_t nbins, double* k, double* pk, double* nmodes,
                                         void* stream) {
  if (!a || !k || !pk || !nmodes || n < 2 || !(box > 0) || nbins < 1 || nbins > 2048) {
    set_error("sim_power_spectrum: invalid arguments (1 <= nbins <= 2048)");
    return SIM_EINVAL;
  }
  FFTPlans* plans = shared_plans(n);
  if (!plans) return SIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long NC = (long long)n * n * (n / 2 + 1);
  cufftComplex* buf = nullptr;
  double* sums = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&buf, 2 * NC * sizeof(cufftComplex), st));
  sim_status r = SIM_OK;
  if (cudaMallocAsync((void**)&sums, 3 * nbins * sizeof(double), st) != cudaSuccess) {
    cudaFreeAsync(buf, st);
    set_error("cudaMallocAsync failed");
    return SIM_ENOMEM;
  }
  cufftComplex* ak = buf;
  cufftComplex* bk = b ? buf + NC : buf;
  if (plans->set_stream(st) != SIM_OK) r = SIM_ECUDA;
  if (r == SIM_OK && cudaMemsetAsync(sums, 0, 3 * nbins * sizeof(double), st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK && cufftExecR2C(plans->r2c1, const_cast<float*>(a), ak) != CUFFT_SUCCESS) {
    set_error("cufftExecR2C failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK && b && cufftExecR2C(plans->r2c1, const_cast<float*>(b), bk) != CUFFT_SUCCESS) {
    set_error("cufftExecR2C failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK) {
    int blocks = cdiv(NC, 256);
    if (blocks > 152 * 4) blocks = 152 * 4;
    DH_CUDA_TRY((launch_pdl(pk_bin_kernel, blocks, 256, 3 * nbins * sizeof(double), st, ak, bk, n, nbins, sums)));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("pk_bin_kernel launch failed");
      r = SIM_ECUDA;
    }
  }
  if (r == SIM_OK) {
    const double norm = box * box * box / ((double)n * n * n * (double)n * n * n);
    DH_CUDA_TRY((launch_pdl(pk_finish_kernel, cdiv(nbins, 128), 128, 0, st, sums, nbins, 2.0 * M_PI / box, norm, k,
                                                        pk, nmodes)));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("pk_finish_kernel launch failed");
      r = SIM_ECUDA;
    }
  }
  cudaFreeAsync(buf, st);
  cudaFreeAsync(sums, st);
  return r;
}
