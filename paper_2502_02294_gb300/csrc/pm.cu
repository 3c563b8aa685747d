// Particle-mesh gravity (Sec. 2.2 of arXiv 2502.02294): CIC deposit with deterministic
// 64-bit fixed-point accumulation, spectral Poisson solve (cuFFT + a fused Green's
// function / gradient kernel), CIC readout with kick and drift, and the adjoints.
//
// Cell decision: t = s * (n / box) in float32 with a single rounded multiply; the base node
// is q + floor(t) (mod n) and the weight fraction f = t - floor(t) is exact in float32.
#include <map>
#include <mutex>

#include "pm.cuh"

namespace dh {

// ------------------------------------------------------------------ FFT plans
static sim_status make_plan(cufftHandle* h, int n, cufftType type, int batch) {
  int dims[3] = {n, n, n};
  int real_emb[3] = {n, n, n};
  int cplx_emb[3] = {n, n, n / 2 + 1};
  const long long nr = (long long)n * n * n, nc = (long long)n * n * (n / 2 + 1);
  cufftResult r;
  if (type == CUFFT_R2C)
    r = cufftPlanMany(h, 3, dims, real_emb, 1, (int)nr, cplx_emb, 1, (int)nc, type, batch);
  else
    r = cufftPlanMany(h, 3, dims, cplx_emb, 1, (int)nc, real_emb, 1, (int)nr, type, batch);
  if (r != CUFFT_SUCCESS) {
    set_error("cufftPlanMany(n=%d, batch=%d) failed with code %d", n, batch, (int)r);
    return r == CUFFT_ALLOC_FAILED ? SIM_ENOMEM : SIM_ECUDA;
  }
  return SIM_OK;
}

sim_status FFTPlans::create(int n_, int B_) {
  n = n_;
  B = B_;
  DH_TRY(make_plan(&r2c1, n, CUFFT_R2C, B));
  DH_TRY(make_plan(&r2c3, n, CUFFT_R2C, 3 * B));
  DH_TRY(make_plan(&r2c4, n, CUFFT_R2C, 4 * B));
  DH_TRY(make_plan(&c2r1, n, CUFFT_C2R, B));
  DH_TRY(make_plan(&c2r3, n, CUFFT_C2R, 3 * B));
  DH_TRY(make_plan(&c2r4, n, CUFFT_C2R, 4 * B));
  return SIM_OK;
}

void FFTPlans::destroy() {
  for (cufftHandle* h : {&r2c1, &r2c3, &r2c4, &c2r1, &c2r3, &c2r4})
    if (*h) {
      cufftDestroy(*h);
      *h = 0;
    }
}

sim_status FFTPlans::set_stream(cudaStream_t st) {
  for (cufftHandle h : {r2c1, r2c3, r2c4, c2r1, c2r3, c2r4})
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) {
      set_error("cufftSetStream failed");
      return SIM_ECUDA;
    }
  return SIM_OK;
}

FFTPlans* shared_plans(int n) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, FFTPlans*> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, n});
  if (it != cache.end()) return it->second;
  FFTPlans* p = new FFTPlans();
  if (p->create(n, 1) != SIM_OK) {
    p->destroy();
    delete p;
    return nullptr;
  }
  cache[{dev, n}] = p;
  return p;
}

static sim_status fft_exec_r2c(cufftHandle h, const float* in, cufftComplex* out) {
  cufftResult r = cufftExecR2C(h, const_cast<float*>(in), out);
  if (r != CUFFT_SUCCESS) {
    set_error("cufftExecR2C failed with code %d", (int)r);
    return SIM_ECUDA;
  }
  return SIM_OK;
}

static sim_status fft_exec_c2r(cufftHandle h, cufftComplex* in, float* out) {
  cufftResult r = cufftExecC2R(h, in, out);
  if (r != CUFFT_SUCCESS) {
    set_error("cufftExecC2R failed with code %d", (int)r);
    return SIM_ECUDA;
  }
  return SIM_OK;
}

// ------------------------------------------------------------------ CIC geometry
// Particle kernels run on a 2-D grid: x over the n^3 particles of an instance in Lagrangian
// order (lattice x fastest), y = the instance, so every thread of a block has a particle
// for any n (a grid of one block per lattice row left 3/4 of the threads idle at n = 32) and
// the blocks of one instance run before the next instance's (its force field stays in L2).
// Node and particle indices are 32-bit (n <= 1024).
struct Cic {
  int ix[2], iy[2], iz[2];
  float wx[2], wy[2], wz[2];
};

__device__ __forceinline__ void cic_axis(float s, int q, int n, float inv_dx, int* idx,
                                         float* w) {
  const float t = __fmul_rn(s, inv_dx);
  const float fl = floorf(t);
  const float f = t - fl;
  // the clamp (a no-op for displacements within 64 boxes) bounds the periodic wrap for any
  // input, a non-finite one included (fminf/fmaxf return the other operand for a NaN)
  const float flc = fminf(fmaxf(fl, -64.0f * n), 64.0f * n);
  const int b = wrap_periodic(q + (int)flc, n);
  idx[0] = b;
  idx[1] = (b + 1 == n) ? 0 : b + 1;
  w[0] = 1.0f - f;
  w[1] = f;
}

struct PIdx {
  int qx, qy, qz, p, b;
  bool ok;
};

// grid (cdiv(n^3, threads), B); lanes past the last particle get ok = false (and a lattice
// site past the end, never used)
__device__ __forceinline__ PIdx particle_index(int n) {
  PIdx r;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nn = (unsigned)n * (unsigned)n;
  r.b = blockIdx.y;
  r.p = (int)t;
  r.ok = t < nn * (unsigned)n;
  if ((n & (n - 1)) == 0) {
    // n a power of two (the usual grid): shifts and masks instead of two divisions
    const int lg = __ffs(n) - 1;
    const unsigned m = (unsigned)n - 1u;
    r.qx = (int)(t & m);
    r.qy = (int)((t >> lg) & m);
    r.qz = (int)(t >> (2 * lg));
  } else {
    r.qz = (int)(t / nn);
    const unsigned rem = t - (unsigned)r.qz * nn;
    r.qy = (int)(rem / (unsigned)n);
    r.qx = (int)(rem - (unsigned)r.qy * (unsigned)n);
  }
  return r;
}

static inline dim3 particle_grid(int n, int threads, int B) {
  return dim3((unsigned)cdiv((long long)n * n * n, threads), B);
}
constexpr int kPT = 128;  // threads per particle block

__device__ __forceinline__ void cic_setup(const float* s, const PIdx& q, int N3, int n,
                                          float inv_dx, Cic& c) {
  cic_axis(s[q.p], q.qx, n, inv_dx, c.ix, c.wx);
  cic_axis(s[N3 + q.p], q.qy, n, inv_dx, c.iy, c.wy);
  cic_axis(s[2 * N3 + q.p], q.qz, n, inv_dx, c.iz, c.wz);
}

__device__ __forceinline__ int node(const Cic& c, int oz, int oy, int ox, int n) {
  return (c.iz[oz] * n + c.iy[oy]) * n + c.ix[ox];
}

// ------------------------------------------------------------------ deposit
// Fixed point: 2^31 units per unit weight, accumulated in 64-bit integers (deterministic).
// Values below 2^31 units convert through 32-bit integers (the 64-bit conversions run on
// the FP64 pipe, which is slow on this part).
__device__ __forceinline__ unsigned long long to_fix(float x) {
  const float y = x * kFix;
  if (fabsf(y) < 2147483520.0f) return (unsigned long long)(long long)__float2int_rn(y);
  return (unsigned long long)__float2ll_rn(y);
}

__device__ __forceinline__ float from_fix(unsigned long long a) {
  const int hi = (int)(a >> 32);
  const unsigned lo = (unsigned)(a & 0xffffffffull);
  return 2.0f * __int2float_rn(hi) + __uint2float_rn(lo) * kInvFix;
}

// Warp-aggregated CIC scatter. The lanes of a warp hold consecutive lattice x sites of one
// (y, z) row (particle order is Lagrangian), so where the flow has not crossed, a lane's
// upper x corner is its right neighbour's lower x corner. Per (z, y) corner pair each lane
// adds its neighbour's upper-corner value into its own lower corner when the nodes agree
// and skips the upper corner its neighbour has taken: about four atomics per particle
// instead of eight, with the same sums. All lanes of the warp must call it (ok = false for
// lanes without a particle).
struct XPair {
  bool take;   // this lane adds the left lane's upper value into its lower node
  bool given;  // the right lane took this lane's upper value
};

__device__ __forceinline__ XPair xpair(int a0, int a1, bool ok) {
  const int lane = threadIdx.x & 31;
  const int pa1 = __shfl_up_sync(0xffffffffu, ok ? a1 : -1, 1);
  const bool take = ok && lane > 0 && pa1 == a0;
  const unsigned tk = __ballot_sync(0xffffffffu, take);
  return XPair{take, lane < 31 && ((tk >> (lane + 1)) & 1u)};
}

__global__ void deposit_kernel(const float* __restrict__ s, const float* __restrict__ vals,
                               int n, float inv_dx, unsigned long long* __restrict__ acc) {
  pdl_enter();
  const int N3 = n * n * n;
  const PIdx q = particle_index(n);  // lanes past the last particle stay for the warp exchange
  s += (size_t)q.b * 3 * N3;
  acc += (size_t)q.b * N3;
  Cic c;
  float v = 0.0f;
  if (q.ok) {
    cic_setup(s, q, N3, n, inv_dx, c);
    v = vals ? vals[(size_t)q.b * N3 + q.p] : 1.0f;
  } else {
    c = Cic{{0, 0}, {0, 0}, {0, 0}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  }
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const int a0 = node(c, oz, oy, 0, n), a1 = node(c, oz, oy, 1, n);
      const float wyz = c.wz[oz] * c.wy[oy];
      unsigned long long f0 = to_fix(wyz * c.wx[0] * v);
      const unsigned long long f1 = to_fix(wyz * c.wx[1] * v);
      const XPair x = xpair(a0, a1, q.ok);
      const unsigned long long fl = __shfl_up_sync(0xffffffffu, f1, 1);
      if (x.take) f0 += fl;
      if (q.ok) {
        if (f0) atomicAdd(acc + a0, f0);
        if (!x.given && f1) atomicAdd(acc + a1, f1);
      }
    }
}

// grid (cdiv(N3, 1024), B): four cells per thread, 16-byte vector accesses where N3 and the
// instance's pointers allow (add may alias out: each cell is read before it is written).
// ZERO: the accumulator is cleared behind the read (else the caller clears it before the
// next deposit with a memset, which streams at the copy rate: the clearing stores here cost
// more than the conversion itself)
template <bool ZERO>
__global__ void fix_to_float_kernel(unsigned long long* __restrict__ acc, SArg scale,
                                    const float* add, int add_stride, float offset, float* out,
                                    int N3) {
  pdl_enter();
  const int b = blockIdx.y;
  const float sc = scale.at(b);
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= N3) return;
  unsigned long long* a = acc + (size_t)b * N3;
  float* o = out + (size_t)b * N3;
  const float* ad = add ? add + (size_t)b * add_stride : nullptr;
  const uintptr_t al = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(o) |
                       reinterpret_cast<uintptr_t>(ad);
  if ((N3 & 3) == 0 && (al & 15) == 0) {
    const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(a + i0);
    const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(a + i0 + 2);
    const float4 r = ad ? *reinterpret_cast<const float4*>(ad + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (ZERO) {
      const ulonglong2 z = make_ulonglong2(0ull, 0ull);
      *reinterpret_cast<ulonglong2*>(a + i0) = z;
      *reinterpret_cast<ulonglong2*>(a + i0 + 2) = z;
    }
    float4 w;
    w.x = sc * from_fix(v0.x) + r.x + offset;
    w.y = sc * from_fix(v0.y) + r.y + offset;
    w.z = sc * from_fix(v1.x) + r.z + offset;
    w.w = sc * from_fix(v1.y) + r.w + offset;
    *reinterpret_cast<float4*>(o + i0) = w;
  } else {
    const int i1 = i0 + 4 < N3 ? i0 + 4 : N3;
    for (int i = i0; i < i1; ++i) {
      const float cnt = from_fix(a[i]);
      if (ZERO) a[i] = 0ull;
      o[i] = sc * cnt + (ad ? ad[i] : 0.0f) + offset;
    }
  }
}

sim_status launch_deposit(const float* s, const float* values, int n, float inv_dx,
                          unsigned long long* acc, int B, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(deposit_kernel, particle_grid(n, kPT, B), kPT, 0, st, s, values, n, inv_dx, acc)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

sim_status launch_fix_to_float(unsigned long long* acc, SArg scale, const float* add,
                               int add_stride, float offset, float* out, int n, int B,
                               cudaStream_t st, bool zero_acc) {
  const int N3 = n * n * n;
  const dim3 grid(cdiv(N3, 1024), B);
  if (zero_acc)
    DH_CUDA_TRY((launch_pdl(fix_to_float_kernel<true>, grid, 256, 0, st, acc, scale, add, add_stride, offset, out, N3)));
  else
    DH_CUDA_TRY((launch_pdl(fix_to_float_kernel<false>, grid, 256, 0, st, acc, scale, add, add_stride, offset, out, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// ------------------------------------------------------------------ Green's function
// half-complex index -> signed integer wavenumbers and Nyquist flags
__device__ __forceinline__ void kindex(int i, int n, int nh, int& kx, int& ky, int& kz,
                                       bool& nx, bool& ny, bool& nz) {
  kx = i % nh;
  const int r = i / nh;
  ky = r % n;
  kz = r / n;
  const bool even = (n % 2 == 0);
  nx = even && kx == n / 2;
  ny = even && ky == n / 2;
  nz = even && kz == n / 2;
  if (ky > n / 2) ky -= n;
  if (kz > n / 2) kz -= n;
}

// gk[j] = i kgrad_j (pref / k^2) dk / n^3   (j = x, y, z); grid (cdiv(NC, 256), B)
__global__ void green_kernel(const cufftComplex* __restrict__ dk, cufftComplex* __restrict__ gk,
                             int n, float kf, SArg pref_norm) {
  pdl_enter();
  const int nh = n / 2 + 1;
  const int NC = n * n * nh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= NC) return;
  dk += (size_t)b * NC;
  gk += (size_t)b * 3 * NC;
  int kx, ky, kz;
  bool nx, ny, nz;
  kindex(i, n, nh, kx, ky, kz, nx, ny, nz);
  const float fx = kf * kx, fy = kf * ky, fz = kf * kz;
  const float k2 = fx * fx + fy * fy + fz * fz;
  const float G = (k2 > 0.0f) ? pref_norm.at(b) / k2 : 0.0f;
  const cufftComplex d = dk[i];
  const float gxs = nx ? 0.0f : fx * G, gys = ny ? 0.0f : fy * G, gzs = nz ? 0.0f : fz * G;
  // i * c * (a + ib) = -c b + i c a
  gk[i] = make_cuFloatComplex(-gxs * d.y, gxs * d.x);
  gk[NC + i] = make_cuFloatComplex(-gys * d.y, gys * d.x);
  gk[2 * NC + i] = make_cuFloatComplex(-gzs * d.y, gzs * d.x);
}

// Adjoint: Y = sum_j (-i kgrad_j)(pref / k^2) L_j / n^3 (the operator with the sign of the
// gradient flipped; the Hermitian weights of the half spectrum cancel, see sim_gravity_adjoint)
__global__ void green_adj_kernel(const cufftComplex* __restrict__ lk, cufftComplex* __restrict__ yk,
                                 int n, float kf, SArg pref_norm) {
  pdl_enter();
  const int nh = n / 2 + 1;
  const int NC = n * n * nh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= NC) return;
  lk += (size_t)b * 3 * NC;
  yk += (size_t)b * NC;
  int kx, ky, kz;
  bool nx, ny, nz;
  kindex(i, n, nh, kx, ky, kz, nx, ny, nz);
  const float fx = kf * kx, fy = kf * ky, fz = kf * kz;
  const float k2 = fx * fx + fy * fy + fz * fz;
  const float G = (k2 > 0.0f) ? pref_norm.at(b) / k2 : 0.0f;
  const float cx = nx ? 0.0f : fx * G, cy = ny ? 0.0f : fy * G, cz = nz ? 0.0f : fz * G;
  const cufftComplex a = lk[i], bb = lk[NC + i], c = lk[2 * NC + i];
  // -i c (re + i im) = c im - i c re
  const float re = cx * a.y + cy * bb.y + cz * c.y;
  const float im = -(cx * a.x + cy * bb.x + cz * c.x);
  yk[i] = make_cuFloatComplex(re, im);
}

float gravity_pref_norm(double pref, int n) { return (float)(pref / ((double)n * n * n)); }

sim_status launch_gravity(const float* delta, float* g, cufftComplex* dk, cufftComplex* gk,
                          int n, double box, SArg pref_norm, int B, FFTPlans& plans,
                          cudaStream_t st) {
  if (plans.B != B) {
    set_error("internal: FFT plans for batch %d used with batch %d", plans.B, B);
    return SIM_EINVAL;
  }
  const int NC = n * n * (n / 2 + 1);
  DH_TRY(plans.set_stream(st));
  DH_TRY(fft_exec_r2c(plans.r2c1, delta, dk));
  const float kf = (float)(2.0 * M_PI / box);
  DH_CUDA_TRY((launch_pdl(green_kernel, dim3(cdiv(NC, 256), B), 256, 0, st, dk, gk, n, kf, pref_norm)));
  DH_LAUNCH_CHECK();
  DH_TRY(fft_exec_c2r(plans.c2r3, gk, g));
  return SIM_OK;
}

sim_status launch_gravity_adjoint(const float* lam_g, float* lam_delta, cufftComplex* gk,
                                  cufftComplex* dk, int n, double box, SArg pref_norm, int B,
                                  FFTPlans& plans, cudaStream_t st) {
  if (plans.B != B) {
    set_error("internal: FFT plans for batch %d used with batch %d", plans.B, B);
    return SIM_EINVAL;
  }
  const int NC = n * n * (n / 2 + 1);
  DH_TRY(plans.set_stream(st));
  DH_TRY(fft_exec_r2c(plans.r2c3, lam_g, gk));
  const float kf = (float)(2.0 * M_PI / box);
  DH_CUDA_TRY((launch_pdl(green_adj_kernel, dim3(cdiv(NC, 256), B), 256, 0, st, gk, dk, n, kf, pref_norm)));
  DH_LAUNCH_CHECK();
  DH_TRY(fft_exec_c2r(plans.c2r1, dk, lam_delta));
  return SIM_OK;
}

// ------------------------------------------------------------------ readout, kick, drift
__global__ void interp_kernel(const float* __restrict__ grid, int nf, int n, float inv_dx,
                              const float* __restrict__ s, float* __restrict__ out) {
  pdl_enter();
  const int N3 = n * n * n;
  const PIdx q = particle_index(n);
  if (!q.ok) return;
  grid += (size_t)q.b * nf * N3;
  s += (size_t)q.b * 3 * N3;
  out += (size_t)q.b * nf * N3;
  Cic c;
  cic_setup(s, q, N3, n, inv_dx, c);
  for (int f = 0; f < nf; ++f) {
    const float* gf = grid + (size_t)f * N3;
    float acc = 0.0f;
#pragma unroll
    for (int oz = 0; oz < 2; ++oz)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox)
          acc += c.wz[oz] * c.wy[oy] * c.wx[ox] * __ldg(gf + node(c, oz, oy, ox, n));
    out[(size_t)f * N3 + q.p] = acc;
  }
}

sim_status launch_interp(const float* grid, int nf, int n, float inv_dx, const float* s,
                         float* out, int B, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(interp_kernel, particle_grid(n, kPT, B), kPT, 0, st, grid, nf, n, inv_dx, s, out)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

__device__ __forceinline__ void interp3(const float* __restrict__ g, const Cic& c, int n,
                                        int N3, float out[3]) {
  out[0] = out[1] = out[2] = 0.0f;
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        const float w = c.wz[oz] * c.wy[oy] * c.wx[ox];
        const int o = node(c, oz, oy, ox, n);
        out[0] += w * __ldg(g + o);
        out[1] += w * __ldg(g + N3 + o);
        out[2] += w * __ldg(g + 2 * N3 + o);
      }
}

// 32 registers (16 resident blocks per SM instead of 9 at 56, a few words spilled): more
// warps in flight for the CIC gathers (kick class 44.7 -> 43.2 us per launch at 128^3 with
// 40 registers, 44.3 -> 43.5 us with 32).
// s_out / p_out may be s / p (in place); out of place the positions are written even when
// dtau = 0
__global__ void __launch_bounds__(128, 16) kick_drift_kernel(const float* s, float* s_out,
                                  const float* p, float* p_out,
                                  const float* __restrict__ g, SArg Ka, SArg dtaua,
                                  const float* __restrict__ zhat, float* __restrict__ aux,
                                  int n, float inv_dx) {
  pdl_enter();
  const int N3 = n * n * n;
  const PIdx q = particle_index(n);
  if (!q.ok) return;
  const int i = q.p;
  const size_t o3 = (size_t)q.b * 3 * N3;
  s += o3;
  s_out += o3;
  p += o3;
  p_out += o3;
  g += o3;
  const float K = Ka.at(q.b), dtau = dtaua.at(q.b);
  Cic c;
  cic_setup(s, q, N3, n, inv_dx, c);
  float gi[3];
  interp3(g, c, n, N3, gi);
  const bool moved = s_out != s;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float pj = p[j * N3 + i] + K * gi[j];
    p_out[j * N3 + i] = pj;
    if (dtau != 0.0f || moved) s_out[j * N3 + i] = s[j * N3 + i] + dtau * pj;
  }
  // star readout at the position the kick saw (before this launch's drift)
  if (zhat) {
    zhat += (size_t)q.b * N3;
    float acc = 0.0f;
#pragma unroll
    for (int oz = 0; oz < 2; ++oz)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox)
          acc += c.wz[oz] * c.wy[oy] * c.wx[ox] * __ldg(zhat + node(c, oz, oy, ox, n));
    aux[(size_t)q.b * N3 + i] += acc;
  }
}

sim_status launch_kick_drift(const float* s, float* s_out, const float* p, float* p_out,
                             const float* g, SArg K, SArg dtau, const float* zhat, float* aux,
                             int n, float inv_dx, int B, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(kick_drift_kernel, particle_grid(n, kPT, B), kPT, 0, st, s, s_out, p,
                          p_out, g, K, dtau, zhat, aux, n, inv_dx)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// grid (cdiv(N3, 256), B)
// out may be in (in place); out of place the density is copied along
__global__ void gas_kick_kernel(const float* in, float* out, const float* __restrict__ g,
                                SArg Ka, int N3) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= N3) return;
  in += (size_t)b * 5 * N3;
  out += (size_t)b * 5 * N3;
  g += (size_t)b * 3 * N3;
  const float K = Ka.at(b);
  float u[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) u[k] = in[k * N3 + i];
  gas_kick_cell(u, g + i, N3, K);
  if (out != in) out[i] = u[0];
#pragma unroll
  for (int k = 1; k < 5; ++k) out[k * N3 + i] = u[k];
}

sim_status launch_gas_kick(const float* in, float* out, const float* g, SArg K, int n, int B,
                           cudaStream_t st) {
  const int N3 = n * n * n;
  DH_CUDA_TRY((launch_pdl(gas_kick_kernel, dim3(cdiv(N3, 256), B), 256, 0, st, in, out, g, K, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// ------------------------------------------------------------------ adjoints
// Adjoint of kick_drift_kernel: the particle part and, when lam_gas is not NULL, the gas
// kick of the cell with the same index at the pre-kick gas state gas_u (its force adjoint
// goes to lam_g4 with a float4 atomic: other particles scatter into the node concurrently).
__global__ void kick_drift_adj_kernel(const float* __restrict__ s0, const float* __restrict__ p0,
                                      const float* __restrict__ g, SArg Ka, SArg dtaua,
                                      float* __restrict__ lam_s, float* __restrict__ lam_p,
                                      float4* __restrict__ lam_g4, DPart dK, DPart ddtau,
                                      const float* __restrict__ gas_u, float* __restrict__ lam_gas,
                                      int n, float inv_dx) {
  pdl_enter();
  const int N3 = n * n * n;
  const PIdx q = particle_index(n);
  const size_t o3 = (size_t)q.b * 3 * N3;
  s0 += o3;
  if (p0) p0 += o3;
  g += o3;
  lam_s += o3;
  lam_p += o3;
  lam_g4 += (size_t)q.b * N3;
  const float K = Ka.at(q.b), dtau = dtaua.at(q.b);
  float dk = 0.0f, dd = 0.0f;
  Cic c = Cic{{0, 0}, {0, 0}, {0, 0}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  float lp[3] = {0.0f, 0.0f, 0.0f};
  if (q.ok) {
    const int i = q.p;
    cic_setup(s0, q, N3, n, inv_dx, c);
    float ls[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ls[j] = lam_s[j * N3 + i];
      lp[j] = lam_p[j * N3 + i] + dtau * ls[j];
    }
    // one pass over the 8 corners gathers g once for both uses: gi = interp(g) (summed in
    // the order of interp3) and lam_s0 += K d/ds (sum_j lp_j interp(g_j))
    float gi[3] = {0.0f, 0.0f, 0.0f};
    float gs[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int oz = 0; oz < 2; ++oz)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
          const int o = node(c, oz, oy, ox, n);
          const float w = c.wz[oz] * c.wy[oy] * c.wx[ox];
          const float dwx = (ox ? inv_dx : -inv_dx) * c.wy[oy] * c.wz[oz];
          const float dwy = (oy ? inv_dx : -inv_dx) * c.wx[ox] * c.wz[oz];
          const float dwz = (oz ? inv_dx : -inv_dx) * c.wx[ox] * c.wy[oy];
          float gv[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            gv[j] = __ldg(g + j * N3 + o);
            gi[j] += w * gv[j];
          }
          float lg = 0.0f;
#pragma unroll
          for (int j = 0; j < 3; ++j) lg += lp[j] * gv[j];
          gs[0] += dwx * lg;
          gs[1] += dwy * lg;
          gs[2] += dwz * lg;
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (p0) dd += ls[j] * (p0[j * N3 + i] + K * gi[j]);
      dk += lp[j] * gi[j];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lam_s[j * N3 + i] = ls[j] + K * gs[j];
      lam_p[j * N3 + i] = lp[j];
    }
    if (lam_gas) {
      // gas kick of cell i: m' = m + rho g K, eps' = eps + K m.g + K^2 rho |g|^2 / 2
      const float* u = gas_u + (size_t)q.b * 5 * N3;
      float* lam = lam_gas + (size_t)q.b * 5 * N3;
      const float rho = u[i];
      const float le = lam[4 * N3 + i];
      float lrho = lam[i];
      float mg = 0.0f, g2 = 0.0f;
      float m[3], gg[3], lm[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        gg[j] = g[j * N3 + i];
        m[j] = u[(1 + j) * N3 + i];
        lm[j] = lam[(1 + j) * N3 + i];
        mg += m[j] * gg[j];
        g2 += gg[j] * gg[j];
      }
      dk += le * (mg + K * rho * g2);
      float lg[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        lrho += K * lm[j] * gg[j];
        dk += lm[j] * rho * gg[j];
        lg[j] = lm[j] * rho * K + le * (K * m[j] + K * K * rho * gg[j]);
        lam[(1 + j) * N3 + i] = lm[j] + le * K * gg[j];
      }
      lrho += 0.5f * K * K * g2 * le;
      lam[i] = lrho;
      atomicAdd(lam_g4 + i, make_float4(lg[0], lg[1], lg[2], 0.0f));
    }
  }
  // lam_g += interp^T(K lp): warp-aggregated float4 atomics (all lanes take part)
  float lpl[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) lpl[j] = __shfl_up_sync(0xffffffffu, lp[j], 1);
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const int a0 = node(c, oz, oy, 0, n), a1 = node(c, oz, oy, 1, n);
      const float kyz = K * c.wz[oz] * c.wy[oy];
      const float w0 = kyz * c.wx[0], w1 = kyz * c.wx[1];
      const XPair x = xpair(a0, a1, q.ok);
      const float wl = __shfl_up_sync(0xffffffffu, w1, 1);
      if (q.ok) {
        float4 v0 = make_float4(w0 * lp[0], w0 * lp[1], w0 * lp[2], 0.0f);
        if (x.take) {
          v0.x += wl * lpl[0];
          v0.y += wl * lpl[1];
          v0.z += wl * lpl[2];
        }
        atomicAdd(lam_g4 + a0, v0);
        if (!x.given) atomicAdd(lam_g4 + a1, make_float4(w1 * lp[0], w1 * lp[1], w1 * lp[2], 0.0f));
      }
    }
  // a block never spans two instances (blockIdx.y carries the instance)
  if (dK.p) block_sum_atomic(dk, dK.at(q.b));
  if (ddtau.p) block_sum_atomic(dd, ddtau.at(q.b));
}

sim_status launch_kick_drift_adjoint(const float* s0, const float* p0, const float* g, SArg K,
                                     SArg dtau, float* lam_s, float* lam_p, float4* lam_g4,
                                     DPart dK, DPart ddtau, const float* gas_u, float* lam_gas,
                                     int n, float inv_dx, int B, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(kick_drift_adj_kernel, particle_grid(n, kPT, B), kPT, 0, st, s0, p0, g, K, dtau, lam_s, lam_p, lam_g4, dK, ddtau, gas_u, lam_gas, n, inv_dx)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

__global__ void deposit_adj_kernel(const float* __restrict__ s, const float* __restrict__ ld,
                                   SArg cma, float* __restrict__ lam_s, DPart dcm, int n,
                                   float inv_dx, float* __restrict__ lam_rho,
                                   long long rho_stride) {
  pdl_enter();
  const int N3 = n * n * n;
  const PIdx q = particle_index(n);
  s += (size_t)q.b * 3 * N3;
  lam_s += (size_t)q.b * 3 * N3;
  ld += (size_t)q.b * N3;
  const float cm = cma.at(q.b);
  float itp = 0.0f;
  if (q.ok) {
    const int i = q.p;
    Cic c;
    cic_setup(s, q, N3, n, inv_dx, c);
    float gs[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int oz = 0; oz < 2; ++oz)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
          const float v = __ldg(ld + node(c, oz, oy, ox, n));
          itp += c.wz[oz] * c.wy[oy] * c.wx[ox] * v;
          gs[0] += (ox ? inv_dx : -inv_dx) * c.wy[oy] * c.wz[oz] * v;
          gs[1] += (oy ? inv_dx : -inv_dx) * c.wx[ox] * c.wz[oz] * v;
          gs[2] += (oz ? inv_dx : -inv_dx) * c.wx[ox] * c.wy[oy] * v;
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) lam_s[j * N3 + i] += cm * gs[j];
    // the cell of this particle's lattice site: one particle per cell
    if (lam_rho) lam_rho[(size_t)q.b * rho_stride + i] += __ldg(ld + i);
  }
  if (dcm.p) block_sum_atomic(itp, dcm.at(q.b));
}

sim_status launch_deposit_adjoint(const float* s, const float* lam_delta, SArg cm,
                                  float* lam_s, DPart dcm, int n, float inv_dx, int B,
                                  cudaStream_t st, float* lam_rho, long long rho_stride) {
  DH_CUDA_TRY((launch_pdl(deposit_adj_kernel, particle_grid(n, kPT, B), kPT, 0, st, s, lam_delta,
                          cm, lam_s, dcm, n, inv_dx, lam_rho, rho_stride)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// grid (blocks, B): lam_g[b][j][i] = lam_g4[b][i].j, out.at(b) += sum lam_g4[b][i].j g[b][j][i]
__global__ void unpack_dot_kernel(const float4* __restrict__ lam_g4, const float* __restrict__ g,
                                  float* __restrict__ lam_g, DPart out, long long N3) {
  pdl_enter();
  const int b = blockIdx.y;
  lam_g4 += (size_t)b * N3;
  g += (size_t)b * 3 * N3;
  lam_g += (size_t)b * 3 * N3;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 v = lam_g4[i];
    lam_g[i] = v.x;
    lam_g[N3 + i] = v.y;
    lam_g[2 * N3 + i] = v.z;
    acc += v.x * __ldg(g + i) + v.y * __ldg(g + N3 + i) + v.z * __ldg(g + 2 * N3 + i);
  }
  if (out.p) block_sum_atomic(acc, out.at(b));
}

sim_status launch_unpack_dot(const float4* lam_g4, const float* g, float* lam_g, DPart out,
                             int n, int B, cudaStream_t st) {
  const long long N3 = (long long)n * n * n;
  int blocks = cdiv(N3, 256);
  const int cap = cdiv(152 * 16, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(unpack_dot_kernel, dim3(blocks, B), 256, 0, st, lam_g4, g, lam_g, out, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// grid (blocks, B): instance b sums a[b count + i] b[b count + i]
__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ bv,
                           long long count, DPart out) {
  pdl_enter();
  const int b = blockIdx.y;
  a += (size_t)b * count;
  bv += (size_t)b * count;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    acc += a[i] * bv[i];
  block_sum_atomic(acc, out.at(b));
}

sim_status launch_dot(const float* a, const float* b, long long count, DPart out, int B,
                      cudaStream_t st) {
  int blocks = cdiv(count, 256);
  const int cap = cdiv(152 * 16, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(dot_kernel, dim3(blocks, B), 256, 0, st, a, b, count, out)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

__global__ void axpy_kernel(float alpha, const float* __restrict__ x, float* __restrict__ y,
                            long long count) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] += alpha * x[i];
}

sim_status launch_axpy(float alpha, const float* x, float* y, long long count, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(axpy_kernel, cdiv(count, 256), 256, 0, st, alpha, x, y, count)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// y[b][ystride] += x[b][count] over B instances (first `count` floats of each y block)
__global__ void axpy_strided_kernel(const float* __restrict__ x, float* __restrict__ y,
                                    long long count, long long ystride) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i < count) y[(size_t)b * ystride + i] += x[(size_t)b * count + i];
}

sim_status launch_add_strided(const float* x, float* y, long long count, long long ystride,
                              int B, cudaStream_t st) {
  DH_CUDA_TRY((launch_pdl(axpy_strided_kernel, dim3(cdiv(count, 256), B), 256, 0, st, x, y, count, ystride)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// instance b: grad[b][0][i] = 2 c (rho_i - t_i) for rho = gas[b][0]; loss[b] += c sum (rho - t)^2
__global__ void density_loss_kernel(const float* __restrict__ gas, const float* __restrict__ t,
                                    float c, float* __restrict__ grad, double* __restrict__ loss,
                                    long long N3) {
  pdl_enter();
  const int b = blockIdx.y;
  const float* rho = gas + (size_t)b * 5 * N3;
  t += (size_t)b * N3;
  grad += (size_t)b * 5 * N3;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = rho[i] - t[i];
    grad[i] = 2.0f * c * d;
    acc += c * d * d;
  }
  block_sum_atomic(acc, loss + b);
}

// instance b: u = eps - |m|^2 / (2 rho), the internal energy density a^2 rho e (proportional
// to the gas-mass-weighted temperature rho T, the delta_b T observable of Sec. 3.2);
// loss[b] += c sum (u - t)^2, grad[b] = 2 c (u - t) du/d(rho, m, eps) (all five fields)
__global__ void thermal_loss_kernel(const float* __restrict__ gas, const float* __restrict__ t,
                                    float c, float* __restrict__ grad, double* __restrict__ loss,
                                    long long N3) {
  pdl_enter();
  const int b = blockIdx.y;
  const float* g = gas + (size_t)b * 5 * N3;
  t += (size_t)b * N3;
  grad += (size_t)b * 5 * N3;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x) {
    const float rho = g[i], mx = g[N3 + i], my = g[2 * N3 + i], mz = g[3 * N3 + i];
    const float inv = 1.0f / rho;
    const float ke = 0.5f * (mx * mx + my * my + mz * mz) * inv;
    const float d = (g[4 * N3 + i] - ke) - t[i];
    const float w = 2.0f * c * d;
    grad[i] = w * ke * inv;  // du/drho = |m|^2 / (2 rho^2)
    grad[N3 + i] = -w * mx * inv;
    grad[2 * N3 + i] = -w * my * inv;
    grad[3 * N3 + i] = -w * mz * inv;
    grad[4 * N3 + i] = w;
    acc += c * d * d;
  }
  block_sum_atomic(acc, loss + b);
}

sim_status launch_thermal_loss(const float* gas, const float* target, float c, float* grad,
                               double* loss, long long N3, int B, cudaStream_t st) {
  int blocks = cdiv(N3, 256);
  const int cap = cdiv(152 * 16, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(thermal_loss_kernel, dim3(blocks, B), 256, 0, st, gas, target, c, grad, loss, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

sim_status launch_density_loss(const float* gas, const float* target, float c, float* grad,
                               double* loss, long long N3, int B, cudaStream_t st) {
  int blocks = cdiv(N3, 256);
  const int cap = cdiv(152 * 16, B);
  if (blocks > cap) blocks = cap;
  DH_CUDA_TRY((launch_pdl(density_loss_kernel, dim3(blocks, B), 256, 0, st, gas, target, c, grad, loss, N3)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

}  // namespace dh

// ------------------------------------------------------------------ C ABI
using namespace dh;

extern "C" sim_status sim_deposit_cic(const float* s, const float* values, int32_t n, double box,
                                      float* grid, void* stream) {
  if (!s || !grid || n < 1 || !(box > 0)) {
    set_error("sim_deposit_cic: invalid arguments");
    return SIM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long N3 = (long long)n * n * n;
  unsigned long long* acc = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&acc, N3 * sizeof(unsigned long long), st));
  sim_status r = SIM_OK;
  if (cudaMemsetAsync(acc, 0, N3 * sizeof(unsigned long long), st) != cudaSuccess) {
    set_error("cudaMemsetAsync failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK) r = launch_deposit(s, values, n, (float)(n / box), acc, 1, st);
  if (r == SIM_OK) r = launch_fix_to_float(acc, sarg(1.0f), grid, (int)N3, 0.0f, grid, n, 1, st);
  cudaFreeAsync(acc, st);
  return r;
}

extern "C" sim_status sim_interp_cic(const float* grid, int32_t nf, int32_t n, double box,
                                     const float* s, float* out, void* stream) {
  if (!grid || !s || !out || n < 1 || nf < 1 || !(box > 0)) {
    set_error("sim_interp_cic: invalid arguments");
    return SIM_EINVAL;
  }
  return launch_interp(grid, nf, n, (float)(n / box), s, out, 1, (cudaStream_t)stream);
}

extern "C" sim_status sim_gravity(const float* delta, int32_t n, double box, double pref,
                                  float* g, void* stream) {
  if (!delta || !g || n < 2 || !(box > 0)) {
    set_error("sim_gravity: invalid arguments");
    return SIM_EINVAL;
  }
  FFTPlans* plans = shared_plans(n);
  if (!plans) return SIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long NC = (long long)n * n * (n / 2 + 1);
  cufftComplex* buf = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&buf, 4 * NC * sizeof(cufftComplex), st));
  sim_status r = launch_gravity(delta, g, buf, buf + NC, n, box,
                                sarg(gravity_pref_norm(pref, n)), 1, *plans, st);
  cudaFreeAsync(buf, st);
  return r;
}

extern "C" sim_status sim_gravity_adjoint(const float* lam_g, int32_t n, double box, double pref,
                                          float* lam_delta, void* stream) {
  if (!lam_g || !lam_delta || n < 2 || !(box > 0)) {
    set_error("sim_gravity_adjoint: invalid arguments");
    return SIM_EINVAL;
  }
  FFTPlans* plans = shared_plans(n);
  if (!plans) return SIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long NC = (long long)n * n * (n / 2 + 1);
  cufftComplex* buf = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&buf, 4 * NC * sizeof(cufftComplex), st));
  sim_status r = launch_gravity_adjoint(lam_g, lam_delta, buf, buf + 3 * NC, n, box,
                                        sarg(gravity_pref_norm(pref, n)), 1, *plans, st);
  cudaFreeAsync(buf, st);
  return r;
}
