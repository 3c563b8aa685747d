// Field-level inference of the initial conditions (Sec. 3.2 of arXiv 2502.02294): the
// posterior of the white-noise amplitudes s given a final gas density d,
//
//   L(s) = 1/2 [ sum_cells (d - F(s))^2 / sigma_n^2 + sum_modes |s|^2 ],
//
// minimised with Adam (Kingma & Ba 2015, Algorithm 1) on the 2,097,152 amplitudes of a
// 128^3 box, and the cross-correlation coefficient r_c(k) = P_XY / sqrt(P_XX P_YY) that
// judges the reconstruction.
//
// fli_adam_kernel fuses what follows the simulator's reverse pass: the prior's value and
// gradient (1/2 |s|^2, s), the gradient sum, and the Adam update of s, m, v in place. It is
// a pure streaming kernel (16 B read + 12 B written per amplitude, +4 B when the gradient is
// also stored): grid-stride over float4 groups, a block partial of the prior per instance.
#include <vector>

#include "fli.cuh"
#include "pm.cuh"

namespace dh {

// 1 - beta is formed in double on the host: in float32, 1 - fl(0.999) is 1.3e-5 off 0.001.
// At step t = 1 the moments start from zero (Adam's initialisation): m and v are not read.
struct AdamConst {
  float lr, b1, b2, omb1, omb2, eps, inv_bc1, inv_bc2, prior_w;
  int first;
};

__device__ __forceinline__ float adam_one(float x, float g, float& m, float& v, const AdamConst& c) {
  m = c.first ? c.omb1 * g : c.b1 * m + c.omb1 * g;
  v = c.first ? c.omb2 * g * g : c.b2 * v + c.omb2 * g * g;
  const float mh = m * c.inv_bc1, vh = v * c.inv_bc2;
  return x - c.lr * mh / (sqrtf(vh) + c.eps);
}

// x, g, m, v: B instances of `count` floats each (instance stride `count`); g is the
// gradient of the data term; the update uses g + prior_w x. grad_out (may be NULL) receives
// g + prior_w x; prior (may be NULL) accumulates prior_w / 2 sum x^2 per instance.
template <bool VEC>
__global__ void __launch_bounds__(256) fli_adam_kernel(float* __restrict__ x, const float* __restrict__ g,
                                                       float* __restrict__ m, float* __restrict__ v,
                                                       long long count, AdamConst c,
                                                       float* __restrict__ grad_out,
                                                       double* __restrict__ prior) {
  pdl_enter();
  const int b = blockIdx.y;
  const size_t off = (size_t)b * count;
  x += off;
  g += off;
  m += off;
  v += off;
  if (grad_out) grad_out += off;
  float acc = 0.0f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (VEC) {
    const long long nq = count >> 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
      float4 xv = reinterpret_cast<float4*>(x)[q];
      const float4 gv = __ldg(reinterpret_cast<const float4*>(g) + q);
      float4 mv = c.first ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<float4*>(m)[q];
      float4 vv = c.first ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<float4*>(v)[q];
      float4 gt;
      gt.x = gv.x + c.prior_w * xv.x;
      gt.y = gv.y + c.prior_w * xv.y;
      gt.z = gv.z + c.prior_w * xv.z;
      gt.w = gv.w + c.prior_w * xv.w;
      acc += xv.x * xv.x + xv.y * xv.y + xv.z * xv.z + xv.w * xv.w;
      if (grad_out) reinterpret_cast<float4*>(grad_out)[q] = gt;
      xv.x = adam_one(xv.x, gt.x, mv.x, vv.x, c);
      xv.y = adam_one(xv.y, gt.y, mv.y, vv.y, c);
      xv.z = adam_one(xv.z, gt.z, mv.z, vv.z, c);
      xv.w = adam_one(xv.w, gt.w, mv.w, vv.w, c);
      reinterpret_cast<float4*>(x)[q] = xv;
      reinterpret_cast<float4*>(m)[q] = mv;
      reinterpret_cast<float4*>(v)[q] = vv;
    }
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
      const float xi = x[i];
      const float gt = __ldg(g + i) + c.prior_w * xi;
      acc += xi * xi;
      if (grad_out) grad_out[i] = gt;
      float mi = c.first ? 0.0f : m[i], vi = c.first ? 0.0f : v[i];
      x[i] = adam_one(xi, gt, mi, vi, c);
      m[i] = mi;
      v[i] = vi;
    }
  }
  if (prior) block_sum_atomic(0.5f * c.prior_w * acc, prior + b);
}

sim_status launch_fli_adam(float* x, const float* g, float* m, float* v, long long count,
                           int B, double lr, double beta1, double beta2, double eps, int t,
                           double prior_w, float* grad_out, double* prior, cudaStream_t st) {
  if (t < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) ||
      !(eps > 0) || count < 1 || B < 1) {
    set_error("adam: need t >= 1, lr > 0, 0 <= beta < 1, eps > 0, count >= 1");
    return SIM_EINVAL;
  }
  AdamConst c;
  c.lr = (float)lr;
  c.b1 = (float)beta1;
  c.b2 = (float)beta2;
  c.omb1 = (float)(1.0 - beta1);
  c.omb2 = (float)(1.0 - beta2);
  c.eps = (float)eps;
  c.inv_bc1 = (float)(1.0 / (1.0 - std::pow(beta1, t)));
  c.inv_bc2 = (float)(1.0 / (1.0 - std::pow(beta2, t)));
  c.prior_w = (float)prior_w;
  c.first = t == 1;
  const uintptr_t align = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(g) |
                          reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v) |
                          reinterpret_cast<uintptr_t>(grad_out);
  const bool vec = (count % 4 == 0) && (align % 16 == 0);
  const long long items = vec ? count / 4 : count;
  int blocks = cdiv(items, 256);
  const int cap = cdiv(152 * 8, B);  // a few waves of 256-thread blocks over all SMs
  if (blocks > cap) blocks = cap;
  const dim3 grid(blocks, B);
  if (vec)
    DH_CUDA_TRY((launch_pdl(fli_adam_kernel<true>, grid, 256, 0, st, x, g, m, v, count, c, grad_out, prior)));
  else
    DH_CUDA_TRY((launch_pdl(fli_adam_kernel<false>, grid, 256, 0, st, x, g, m, v, count, c, grad_out, prior)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// grad = g + prior_w x and prior[b] += prior_w / 2 sum x^2 (the posterior's gradient and
// prior term without an update)
__global__ void __launch_bounds__(256) prior_grad_kernel(const float* __restrict__ x,
                                                         const float* __restrict__ g,
                                                         float* __restrict__ grad, long long count,
                                                         float prior_w, double* __restrict__ prior) {
  pdl_enter();
  const int b = blockIdx.y;
  const size_t off = (size_t)b * count;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float xi = x[off + i];
    grad[off + i] = g[off + i] + prior_w * xi;
    acc += xi * xi;
  }
  if (prior) block_sum_atomic(0.5f * prior_w * acc, prior + b);
}

sim_status launch_prior_grad(const float* x, const float* g, float* grad, long long count,
                             int B, double prior_w, double* prior, cudaStream_t st) {
  int blocks = cdiv(count, 256);
  const int cap = cdiv(152 * 8, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(prior_grad_kernel, dim3(blocks, B), 256, 0, st, x, g, grad, count, (float)prior_w, prior)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// y = alpha x + beta y over count floats
__global__ void axpby_kernel(float alpha, const float* __restrict__ x, float beta,
                             float* __restrict__ y, long long count) {
  pdl_enter();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = alpha * x[i] + beta * y[i];
}

// ------------------------------------------------------------------ r_c(k)
// One pass over the half spectra of X and Y: per bin the mode weight, weight * |k| and the
// three weighted powers |X|^2, |Y|^2, Re(X conj Y) (FP64 histograms in shared memory).
__global__ void xc_bin_kernel(const cufftComplex* __restrict__ a, const cufftComplex* __restrict__ b,
                              int n, int nbins, double* __restrict__ sums) {
  pdl_enter();
  extern __shared__ double hist[];  // 5 * nbins
  for (int j = threadIdx.x; j < 5 * nbins; j += blockDim.x) hist[j] = 0.0;
  __syncthreads();
  const int nh = n / 2 + 1;
  const long long NC = (long long)n * n * nh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < NC;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nh);
    const long long r = i / nh;
    int ky = (int)(r % n), kz = (int)(r / n);
    if (ky > n / 2) ky -= n;
    if (kz > n / 2) kz -= n;
    const double kk = sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz);
    const int bin = (int)rint(kk);
    if (bin < 1 || bin > nbins) continue;
    const double w = (kx == 0 || (n % 2 == 0 && kx == n / 2)) ? 1.0 : 2.0;
    const cufftComplex x = a[i], y = b[i];
    atomicAdd(&hist[bin - 1], w);
    atomicAdd(&hist[nbins + bin - 1], w * kk);
    atomicAdd(&hist[2 * nbins + bin - 1], w * ((double)x.x * x.x + (double)x.y * x.y));
    atomicAdd(&hist[3 * nbins + bin - 1], w * ((double)y.x * y.x + (double)y.y * y.y));
    atomicAdd(&hist[4 * nbins + bin - 1], w * ((double)x.x * y.x + (double)x.y * y.y));
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 5 * nbins; j += blockDim.x)
    if (hist[j] != 0.0) atomicAdd(&sums[j], hist[j]);
}

__global__ void xc_finish_kernel(const double* __restrict__ sums, int nbins, double kf,
                                 double* __restrict__ k, double* __restrict__ rc,
                                 double* __restrict__ nm) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nbins) return;
  const double w = sums[j], pxx = sums[2 * nbins + j], pyy = sums[3 * nbins + j];
  nm[j] = w;
  k[j] = w > 0 ? kf * sums[nbins + j] / w : 0.0;
  rc[j] = (pxx > 0 && pyy > 0) ? sums[4 * nbins + j] / sqrt(pxx * pyy) : 0.0;
}

}  // namespace dh

using namespace dh;

extern "C" sim_status sim_adam(float* x, const float* g, float* m, float* v, int64_t count,
                               double lr, double beta1, double beta2, double eps, int32_t t,
                               double prior_w, float* grad_out, double* prior, void* stream) {
  if (!x || !g || !m || !v || count < 1) {
    set_error("sim_adam: null arrays or count < 1");
    return SIM_EINVAL;
  }
  return launch_fli_adam(x, g, m, v, count, 1, lr, beta1, beta2, eps, t, prior_w, grad_out,
                         prior, (cudaStream_t)stream);
}

extern "C" sim_status sim_dot(const float* a, const float* b, int64_t count, double* out,
                              void* stream) {
  if (!a || !b || !out || count < 1) {
    set_error("sim_dot: null arrays or count < 1");
    return SIM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DH_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), st));
  return launch_dot(a, b, count, dpart(out), 1, st);
}

extern "C" sim_status sim_axpby(double alpha, const float* x, double beta, float* y,
                                int64_t count, void* stream) {
  if (!x || !y || count < 1) {
    set_error("sim_axpby: null arrays or count < 1");
    return SIM_EINVAL;
  }
  int blocks = cdiv(count, 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  DH_CUDA_TRY((launch_pdl(axpby_kernel, blocks, 256, 0, (cudaStream_t)stream, (float)alpha, x, (float)beta, y, count)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

extern "C" sim_status sim_cross_correlation(const float* a, const float* b, int32_t n,
                                            double box, int32_t nbins, double* k, double* rc,
                                            double* nmodes, void* stream) {
  if (!a || !b || !k || !rc || !nmodes || n < 2 || !(box > 0) || nbins < 1 || nbins > 1024) {
    set_error("sim_cross_correlation: invalid arguments (1 <= nbins <= 1024)");
    return SIM_EINVAL;
  }
  FFTPlans* plans = shared_plans(n);
  if (!plans) return SIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long NC = (long long)n * n * (n / 2 + 1);
  cufftComplex* buf = nullptr;
  double* sums = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&buf, 2 * NC * sizeof(cufftComplex), st));
  if (cudaMallocAsync((void**)&sums, 5 * nbins * sizeof(double), st) != cudaSuccess) {
    cudaFreeAsync(buf, st);
    set_error("cudaMallocAsync failed");
    return SIM_ENOMEM;
  }
  sim_status r = plans->set_stream(st);
  if (r == SIM_OK && cudaMemsetAsync(sums, 0, 5 * nbins * sizeof(double), st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK && (cufftExecR2C(plans->r2c1, const_cast<float*>(a), buf) != CUFFT_SUCCESS ||
                      cufftExecR2C(plans->r2c1, const_cast<float*>(b), buf + NC) != CUFFT_SUCCESS)) {
    set_error("cufftExecR2C failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK) {
    int blocks = cdiv(NC, 256);
    if (blocks > 152 * 4) blocks = 152 * 4;
    DH_CUDA_TRY((launch_pdl(xc_bin_kernel, blocks, 256, 5 * nbins * sizeof(double), st, buf, buf + NC, n, nbins, sums)));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("xc_bin_kernel launch failed");
      r = SIM_ECUDA;
    }
  }
  if (r == SIM_OK) {
    DH_CUDA_TRY((launch_pdl(xc_finish_kernel, cdiv(nbins, 128), 128, 0, st, sums, nbins, 2.0 * M_PI / box, k, rc, nmodes)));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("xc_finish_kernel launch failed");
      r = SIM_ECUDA;
    }
  }
  cudaFreeAsync(buf, st);
  cudaFreeAsync(sums, st);
  return r;
}
