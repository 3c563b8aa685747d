// Shared device helpers for the diffHydro GB300 library: error plumbing, the Philox
// counter-based generator, and the per-cell relaxing-TVD flux split and its adjoint.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "diffhydro.h"

namespace dh {

// ------------------------------------------------------------------ error plumbing
// The last error message of the calling host thread (calls without a handle) is kept in a
// thread-local buffer; handle calls also copy it into the handle.
void set_error(const char* fmt, ...);
const char* get_error();

#define DH_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::dh::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                      __LINE__);                                                       \
      return SIM_ECUDA;                                                                \
    }                                                                                  \
  } while (0)

// Every kernel launch of the library is followed by DH_LAUNCH_CHECK, which also counts it
// (sim_kernel_launches() reports the process-wide total).
void count_launch();
#define DH_LAUNCH_CHECK()            \
  do {                               \
    ::dh::count_launch();            \
    DH_CUDA_TRY(cudaGetLastError()); \
  } while (0)

#define DH_TRY(expr)                    \
  do {                                  \
    sim_status _s = (expr);             \
    if (_s != SIM_OK) return _s;        \
  } while (0)

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ dependent launches
// Kernels of the step follow one another on one stream. Each is launched with programmatic
// stream serialisation (launch_pdl) and opens with pdl_enter(): it waits there until the
// grid before it has completed and its writes are visible, then lets the grid after it be
// scheduled. So the next kernel's blocks are launched while this one's last wave drains,
// and nothing is read before its producer has finished. (Launched without the attribute,
// both instructions return at once.)
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// ------------------------------------------------------------------ batched launches
// Every kernel of the step takes B instances of one grid size stored one after another
// (instance b of a field with F components of n^3 cells starts at b * F * n^3). A scalar
// that differs between instances is an SArg: one value for all instances, or a device
// array indexed by the instance. Partial sums of instance b go to base + b * stride.
struct SArg {
  float v;
  const float* p;
  __device__ __forceinline__ float at(int b) const { return p ? __ldg(p + b) : v; }
};
inline SArg sarg(float v) { return SArg{v, nullptr}; }
inline SArg sarg(const float* p) { return SArg{0.0f, p}; }

struct DPart {
  double* p;
  int stride;
  __device__ __forceinline__ double* at(int b) const { return p ? p + (size_t)b * stride : nullptr; }
};
inline DPart dpart(double* p, int stride = 0) { return DPart{p, stride}; }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al. (SC'11): 10 rounds of two 32x32->64 multiplies whose halves are mixed
// with the other counter words and the key; Weyl key bumps between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// u = ((x >> 9) + 0.5) * 2^-23: an odd multiple of 2^-24 in (0,1), exact in float.
__device__ __forceinline__ float uniform_from_word(uint32_t x) {
  return (__uint2float_rn(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

enum { TAG_IC_NOISE = 0, TAG_SUBGRID = 1 };

// ------------------------------------------------------------------ relaxing TVD cell
// Flux split of one cell for a sweep whose momentum component is u[f] (f = 1 + axis):
//   v = m_f / rho, P = (gamma-1)(eps - |m|^2/(2 rho)), c = |v| + sqrt(max(gamma P/rho, 0))
//   F = (m_f, m_x v, m_y v, m_z v, (eps+P) v) + P e_f,  F^R = (cU + F)/2, F^L = (cU - F)/2.
// Reciprocal and square root use the SFU approximations (about 1 ulp), far below the
// float32 round-off that accumulates over a sweep.
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }

__device__ __forceinline__ void split_flux(const float u[5], int f, float gam, float FR[5],
                                           float FL[5]) {
  const float inv = fast_rcp(u[0]);
  const float md = u[f];
  const float v = md * inv;
  const float m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const float P = (gam - 1.0f) * (u[4] - 0.5f * m2 * inv);
  const float cs2 = gam * P * inv;
  const float c = fabsf(v) + (cs2 > 0.0f ? cs2 * rsqrtf(cs2) : 0.0f);
  float F[5];
  F[0] = md;
  F[1] = u[1] * v;
  F[2] = u[2] * v;
  F[3] = u[3] * v;
  F[f] += P;
  F[4] = (u[4] + P) * v;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float cu = c * u[k];
    FR[k] = 0.5f * (cu + F[k]);
    FL[k] = 0.5f * (cu - F[k]);
  }
}

// Vector-Jacobian product of split_flux: lu += (dF^R/dU)^T lR + (dF^L/dU)^T lL.
// Conventions at kinks match the oracle: d|v|/dv = 0 at v = 0, dc_s = 0 where c_s = 0.
__device__ __forceinline__ void split_flux_vjp(const float u[5], int f, float gam,
                                               const float lR[5], const float lL[5],
                                               float lu[5]) {
  const float inv = fast_rcp(u[0]);
  const float md = u[f];
  const float v = md * inv;
  const float m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const float P = (gam - 1.0f) * (u[4] - 0.5f * m2 * inv);
  const float cs2 = gam * P * inv;
  const float rcs = cs2 > 0.0f ? rsqrtf(cs2) : 0.0f;
  const float cs = cs2 * rcs;
  const float c = fabsf(v) + cs;
  float sig[5], del[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    sig[k] = 0.5f * (lR[k] + lL[k]);
    del[k] = 0.5f * (lR[k] - lL[k]);
  }
  // c U term
  float lc = 0.0f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    lu[k] += c * sig[k];
    lc += sig[k] * u[k];
  }
  // flux term with del
  float lv = 0.0f, lP = del[f], lrho = 0.0f;
  lu[f] += del[0];  // F0 = m_f
#pragma unroll
  for (int k = 1; k <= 3; ++k) {  // F_k = m_k v (+P)
    lu[k] += del[k] * v;
    lv += del[k] * u[k];
  }
  lu[4] += del[4] * v;  // F4 = (eps + P) v
  lP += del[4] * v;
  lv += del[4] * (u[4] + P);
  // c = |v| + cs, cs = sqrt(gam P / rho): dcs/dP = gam/(2 cs rho), dcs/drho = -cs/(2 rho)
  lv += lc * (float)((v > 0.0f) - (v < 0.0f));
  if (cs2 > 0.0f) {
    lP += lc * 0.5f * gam * rcs * inv;
    lrho -= lc * 0.5f * cs * inv;
  }
  // P = (gam-1)(eps - m2/(2 rho))
  const float gP = (gam - 1.0f) * lP;
  lu[4] += gP;
#pragma unroll
  for (int k = 1; k <= 3; ++k) lu[k] -= gP * u[k] * inv;
  lrho += gP * 0.5f * m2 * inv * inv;
  // v = m_f / rho
  lu[f] += lv * inv;
  lrho -= lv * v * inv;
  lu[0] += lrho;
}

// Gravity half kick of one gas cell (Sec. 2.2): m += rho g K, eps += K m.g + K^2 rho |g|^2 / 2,
// g the three force components at offsets 0, N3, 2 N3 from g. Every product and sum is
// rounded on its own (no FMA contraction), so that the kick kernel and the sweeps that kick
// their cells as they load them give the same bits.
__device__ __forceinline__ void gas_kick_cell(float u[5], const float* g, long long N3, float K) {
  const float rho = u[0];
  float mg = 0.0f, g2 = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float gj = __ldg(g + j * N3);
    const float mj = u[1 + j];
    mg = __fadd_rn(mg, __fmul_rn(mj, gj));
    g2 = __fadd_rn(g2, __fmul_rn(gj, gj));
    u[1 + j] = __fadd_rn(mj, __fmul_rn(__fmul_rn(rho, gj), K));
  }
  const float de = __fadd_rn(__fmul_rn(K, mg), __fmul_rn(__fmul_rn(__fmul_rn(0.5f, K), K), __fmul_rn(rho, g2)));
  u[4] = __fadd_rn(u[4], de);
}

// Gated harmonic-mean (van Leer) limiter 2 max(ab,0) / (a + b + copysign(eps, a+b)).
__device__ __forceinline__ float vanleer(float a, float b, float eps) {
  const float ab = a * b;
  const float s = a + b;
  return ab > 0.0f ? __fdividef(2.0f * ab, s + copysignf(eps, s)) : 0.0f;
}

__device__ __forceinline__ void vanleer_grad(float a, float b, float eps, float& da,
                                             float& db) {
  const float ab = a * b;
  if (ab > 0.0f) {
    const float s = a + b;
    const float D = s + copysignf(eps, s);
    const float iD = fast_rcp(D);
    const float i2 = iD * iD;
    da = 2.0f * b * (D - a) * i2;
    db = 2.0f * a * (D - b) * i2;
  } else {
    da = 0.0f;
    db = 0.0f;
  }
}

// Limiter value and both partials in one pass (the adjoint needs the face flux for d/dnu):
// phi as vanleer() up to the rounding of the reciprocal, da = dphi/da, db = dphi/db.
__device__ __forceinline__ void vanleer_vg(float a, float b, float eps, float& phi, float& da,
                                           float& db) {
  const float ab = a * b;
  if (ab > 0.0f) {
    const float s = a + b;
    const float D = s + copysignf(eps, s);
    const float q = 2.0f * fast_rcp(D);  // 2 / D
    const float q2 = 0.5f * q * q;       // 2 / D^2
    phi = ab * q;
    da = b * (D - a) * q2;
    db = a * (D - b) * q2;
  } else {
    phi = 0.0f;
    da = 0.0f;
    db = 0.0f;
  }
}

// ------------------------------------------------------------------ reductions
// Per-thread partial sums stay in float32 (GB300's FP64 rate is a small fraction of FP32);
// each block converts its float32 total once and adds it to a double accumulator.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one float per thread, added atomically (as double) to *out by one
// thread. All threads of the block must call it; blockDim a multiple of 32, <= 1024.
__device__ __forceinline__ void block_sum_atomic(float v, double* out) {
  __shared__ float red[32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    float w = (tid < (nt >> 5)) ? red[tid] : 0.0f;
    w = warp_sum(w);
    if (tid == 0 && w != 0.0f) atomicAdd(out, (double)w);
  }
}

// periodic wrap of an index known to lie within a few periods of [0, n)
__device__ __forceinline__ int wrap_periodic(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

}  // namespace dh
