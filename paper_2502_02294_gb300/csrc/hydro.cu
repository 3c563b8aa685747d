// Relaxing TVD sweep (Sec. 2.3.1-2.3.2 of arXiv 2502.02294) and its adjoint.
//
// One CTA owns a tile of S output cells along the sweep axis times W lines. It reads the
// tile plus a halo (3 cells per side forward, 5 adjoint) once from global memory into
// registers, keeps the per-cell flux splits and the per-face fluxes in shared memory, and
// evaluates every flux split and every limited face flux exactly once per tile cell. For
// the y and z sweeps the W lines are W consecutive x cells (128-byte rows per warp load);
// for the x sweep the lines are W consecutive y rows read as contiguous segments.
//
//   half step  (Eq. TVD_halfstep):  Uh_i = U_i - nu/2 (F_{i+1/2} - F_{i-1/2}),
//              F_{i+1/2} = F^R_i - F^L_{i+1}  (first-order upwind of the relaxed fluxes)
//   full step  (Eq. TVD_fullstep):  U'_i = U_i - nu (F2_{i+1/2} - F2_{i-1/2}),
//              F2_{i+1/2} = [Fh^R_i + phi(dL, dR)] - [Fh^L_{i+1} - phi(dL', dR')]
//              with the gated van Leer limiter phi and half differences of Fh^R / Fh^L.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace dh {

// global offset of (sweep coordinate sg, line coordinate wg, third coordinate t)
template <int AXIS>
__device__ __forceinline__ long long goff(int sg, int wg, int t, int n) {
  if (AXIS == 0) return ((long long)t * n + wg) * n + sg;  // x sweep: lines are y rows
  if (AXIS == 1) return ((long long)t * n + sg) * n + wg;  // y sweep: lines are x cells
  return ((long long)sg * n + t) * n + wg;                 // z sweep: lines are x cells
}

template <int AXIS, int S, int W, int H>
struct TileGeom {
  static constexpr int SP = S + 2 * H;  // cells along the sweep including the halo
  static constexpr int NC = SP * W;
  static constexpr int DS = (AXIS == 0) ? 1 : W;  // shared-memory stride along the sweep
  __device__ static __forceinline__ int s_of(int c) { return AXIS == 0 ? c % SP : c / W; }
  __device__ static __forceinline__ int w_of(int c) { return AXIS == 0 ? c / SP : c % W; }
};

// Line of a thread of the marching and per-cell kernels: blocks of blockDim.x lanes along
// x (each lane `wmul` adjacent x columns) times blockDim.y rows of the third coordinate, so
// that grids with n below the block width keep their threads busy (one row per block left
// 3/4 of them idle at n = 32); blockIdx.y = instance x row blocks. Rows past n are not live.
struct LineIdx {
  int w, t, b;
  bool live;
};
__device__ __forceinline__ LineIdx line_index(int n, int wmul) {
  const int nry = (n + (int)blockDim.y - 1) / (int)blockDim.y;
  LineIdx r;
  r.b = blockIdx.y / nry;
  r.t = (blockIdx.y - r.b * nry) * blockDim.y + threadIdx.y;
  r.w = wmul * (blockIdx.x * blockDim.x + threadIdx.x);
  r.live = r.w < n && r.t < n;
  return r;
}

// tile shapes (forward / adjoint): x sweep 64 x 4 lines, y/z sweeps 32 x 32 and 16 x 32
template <int AXIS> struct SweepCfg;
template <> struct SweepCfg<0> { static constexpr int S = 64, W = 4, NT = 128, SA = 64, WA = 4, NTA = 128; };
#ifndef DH_TILE_S
#define DH_TILE_S 16
#endif
template <> struct SweepCfg<1> { static constexpr int S = DH_TILE_S, W = 32, NT = 256, SA = 16, WA = 32, NTA = 256; };
template <> struct SweepCfg<2> { static constexpr int S = DH_TILE_S, W = 32, NT = 256, SA = 16, WA = 32, NTA = 256; };

// packed FP32x2 arithmetic of sm_100+ (FADD2 / FMUL2 / FFMA2: one issue slot for two lanes)
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, pk(-1.0f), a); }

// gated van Leer limiter of two lanes, as vanleer
__device__ __forceinline__ float2 vanleer2(float2 a, float2 b, float eps) {
  const float2 ab = mul2(a, b);
  const float2 s = add2(a, b);
  const float2 D = add2(s, make_float2(copysignf(eps, s.x), copysignf(eps, s.y)));
  const float2 t = mul2(add2(ab, ab), make_float2(fast_rcp(D.x), fast_rcp(D.y)));
  return make_float2(ab.x > 0.0f ? t.x : 0.0f, ab.y > 0.0f ? t.y : 0.0f);
}

// limited second-order face flux at face c+1/2 from the half-step splits R = Fh^R, L = Fh^L
__device__ __forceinline__ float face_flux(const float* R, const float* L, int DS, float eps) {
  const float Rm1 = R[-DS], R0 = R[0], Rp1 = R[DS];
  const float L0 = L[0], Lp1 = L[DS], Lp2 = L[2 * DS];
  const float fr = R0 + vanleer(0.5f * (R0 - Rm1), 0.5f * (Rp1 - R0), eps);
  const float fl = Lp1 - vanleer(0.5f * (Lp1 - L0), 0.5f * (Lp2 - Lp1), eps);
  return fr - fl;
}

// the same face flux for components (k, k + 1) as one FP32x2 pair
__device__ __forceinline__ float2 face_flux2(const float2* R, const float2* L, int DS, float eps) {
  const float2 Rm1 = R[-DS], R0 = R[0], Rp1 = R[DS];
  const float2 L0 = L[0], Lp1 = L[DS], Lp2 = L[2 * DS];
  const float2 fr = add2(R0, vanleer2(mul2(pk(0.5f), sub2(R0, Rm1)), mul2(pk(0.5f), sub2(Rp1, R0)), eps));
  const float2 fl = sub2(Lp1, vanleer2(mul2(pk(0.5f), sub2(Lp1, L0)), mul2(pk(0.5f), sub2(Lp2, Lp1)), eps));
  return sub2(fr, fl);
}

// Shared memory holds the flux splits and face fluxes with components (0, 1) and (2, 3) as
// interleaved float pairs (one 8-byte access and one FP32x2 instruction for two components)
// and component 4 alone: per array [pair 0: NC float2][pair 1: NC float2][component 4: NC].
template <int AXIS>
__global__ void __launch_bounds__(SweepCfg<AXIS>::NT, 2)
sweep_fwd_kernel(const float* __restrict__ uin, float* __restrict__ uout, int n, SArg nua,
                 float gam, float eps, const float* __restrict__ kick_g, SArg kick_K) {
  pdl_enter();
  constexpr int S = SweepCfg<AXIS>::S, W = SweepCfg<AXIS>::W, NT = SweepCfg<AXIS>::NT;
  using G = TileGeom<AXIS, S, W, 3>;
  constexpr int NC = G::NC, DS = G::DS, SP = G::SP, CPT = (NC + NT - 1) / NT;
  constexpr int F = 1 + AXIS;
  static_assert(NC % 2 == 0, "float2 regions need an even cell count");
  extern __shared__ float sm[];
  float2* rp = reinterpret_cast<float2*>(sm);            // F^R pairs  [2][NC]
  float* r4 = sm + 4 * NC;                                // F^R_4      [NC]
  float2* lp = reinterpret_cast<float2*>(sm + 5 * NC);   // F^L pairs
  float* l4 = sm + 9 * NC;
  float2* gp = reinterpret_cast<float2*>(sm + 10 * NC);  // face fluxes (face c+1/2 at c)
  float* g4 = sm + 14 * NC;
  const long long N3 = (long long)n * n * n;
  const int b = blockIdx.z / n;  // instance; blockIdx.z = b n + third coordinate
  const int s0 = blockIdx.x * S, w0 = blockIdx.y * W, t = blockIdx.z - b * n;
  uin += (size_t)b * 5 * N3;
  uout += (size_t)b * 5 * N3;
  if (kick_g) kick_g += (size_t)b * 3 * N3;
  const float nu = nua.at(b), kK = kick_K.at(b);
  const float2 hnu = pk(0.5f * nu), mnu = pk(-nu);

  float ureg[CPT][5];
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    if (c < NC) {
      const int s = G::s_of(c), w = G::w_of(c), wg = w0 + w;
      const int sgl = wrap_periodic(s0 + s - 3, n);
      float u[5] = {1.f, 0.f, 0.f, 0.f, 1.f};
      if (wg < n) {
        const long long o = goff<AXIS>(sgl, wg, t, n);
#pragma unroll
        for (int k = 0; k < 5; ++k) u[k] = __ldg(uin + k * N3 + o);
        if (kick_g) gas_kick_cell(u, kick_g + o, N3, kK);  // the step's opening gas kick
      }
      float FR[5], FL[5];
      split_flux(u, F, gam, FR, FL);
#pragma unroll
      for (int k = 0; k < 5; ++k) ureg[i][k] = u[k];
      rp[c] = make_float2(FR[0], FR[1]);
      rp[NC + c] = make_float2(FR[2], FR[3]);
      r4[c] = FR[4];
      lp[c] = make_float2(FL[0], FL[1]);
      lp[NC + c] = make_float2(FL[2], FL[3]);
      l4[c] = FL[4];
    }
  }
  __syncthreads();
  float uh[CPT][5];
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c);
    if (c < NC && s >= 1 && s < SP - 1) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2* R = rp + j * NC;
        const float2* Lq = lp + j * NC;
        const float2 fp = sub2(R[c], Lq[c + DS]);
        const float2 fm = sub2(R[c - DS], Lq[c]);
        const float2 h = fma2(hnu, sub2(fm, fp), make_float2(ureg[i][2 * j], ureg[i][2 * j + 1]));
        uh[i][2 * j] = h.x;
        uh[i][2 * j + 1] = h.y;
      }
      const float fp = r4[c] - l4[c + DS];
      const float fm = r4[c - DS] - l4[c];
      uh[i][4] = ureg[i][4] - 0.5f * nu * (fp - fm);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c);
    if (c < NC && s >= 1 && s < SP - 1) {
      float FR[5], FL[5];
      split_flux(uh[i], F, gam, FR, FL);
      rp[c] = make_float2(FR[0], FR[1]);
      rp[NC + c] = make_float2(FR[2], FR[3]);
      r4[c] = FR[4];
      lp[c] = make_float2(FL[0], FL[1]);
      lp[NC + c] = make_float2(FL[2], FL[3]);
      l4[c] = FL[4];
    }
  }
  __syncthreads();
  // faces c+1/2 for s in [2, S+3): each computed once
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c);
    if (c < NC && s >= 2 && s < S + 3) {
      gp[c] = face_flux2(rp + c, lp + c, DS, eps);
      gp[NC + c] = face_flux2(rp + NC + c, lp + NC + c, DS, eps);
      g4[c] = face_flux(r4 + c, l4 + c, DS, eps);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c), w = G::w_of(c);
    const int sgl = s0 + s - 3, wg = w0 + w;
    if (c < NC && s >= 3 && s < S + 3 && sgl < n && wg < n) {
      const long long o = goff<AXIS>(sgl, wg, t, n);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2 v = fma2(mnu, sub2(gp[j * NC + c], gp[j * NC + c - DS]),
                              make_float2(ureg[i][2 * j], ureg[i][2 * j + 1]));
        uout[2 * j * N3 + o] = v.x;
        uout[(2 * j + 1) * N3 + o] = v.y;
      }
      uout[4 * N3 + o] = ureg[i][4] - nu * (g4[c] - g4[c - DS]);
    }
  }
}

// ------------------------------------------------------------- forward, marching form
// Each thread owns one line and a segment of L output cells along the sweep axis. It loads
// the segment plus 3 halo cells per side in order and keeps a sliding window in registers:
// at load j it forms the first-order face j-1/2, the half-step state Uh_{j-1} and its
// splits, the limited face (j-3)+1/2 and the output U'_{j-3}. No shared memory, no
// barriers; adjacent threads own adjacent lines (x for the y/z sweeps, y for x).
template <int AXIS>
__global__ void __launch_bounds__(128)
sweep_march_kernel(const float* __restrict__ uin, float* __restrict__ uout, int n, SArg nua,
                   float gam, float eps, int L) {
  pdl_enter();
  constexpr int F = 1 + AXIS;
  const LineIdx li = line_index(n, 1);
  const int w = li.w, t = li.t, b = li.b;  // line coordinate, third coordinate, instance
  const int s0 = blockIdx.z * L;
  if (!li.live) return;
  const long long N3 = (long long)n * n * n;
  uin += (size_t)b * 5 * N3;
  uout += (size_t)b * 5 * N3;
  const float nu = nua.at(b);
  const float hnu = 0.5f * nu;
  float Ua[5], Ub[5], Uc[5];      // U_{j-3}, U_{j-2}, U_{j-1}
  float FRp[5], f1m[5];           // F^R_{j-1}, first-order face (j-3/2)
  float R0[5], R1[5], R2[5];      // Fh^R_{j-4..j-2}
  float L0[5], L1[5];             // Fh^L_{j-3..j-2}
  float F2m[5];                   // limited face (j-4)+1/2
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float init = (k == 0 || k == 4) ? 1.0f : 0.0f;
    Ua[k] = Ub[k] = Uc[k] = init;
    FRp[k] = f1m[k] = R0[k] = R1[k] = R2[k] = L0[k] = L1[k] = F2m[k] = 0.0f;
  }
  int j = wrap_periodic(s0 - 3, n);
  // software pipelining: the next cell's state is requested one iteration ahead
  float un[5];
  {
    const long long o = goff<AXIS>(j, w, t, n);
#pragma unroll
    for (int k = 0; k < 5; ++k) un[k] = __ldg(uin + k * N3 + o);
  }
#pragma unroll 1
  for (int it = 0; it < L + 6; ++it) {
    float u[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) u[k] = un[k];
    const int jn = (j + 1 == n) ? 0 : j + 1;
    if (it + 1 < L + 6) {
      const long long on = goff<AXIS>(jn, w, t, n);
#pragma unroll
      for (int k = 0; k < 5; ++k) un[k] = __ldg(uin + k * N3 + on);
    }
    float FR[5], FL[5];
    split_flux(u, F, gam, FR, FL);
    float f1[5], uh[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      f1[k] = FRp[k] - FL[k];                 // face j-1/2
      uh[k] = Uc[k] - hnu * (f1[k] - f1m[k]);  // Uh_{j-1}
    }
    float FRh[5], FLh[5];
    split_flux(uh, F, gam, FRh, FLh);
    const int jo = s0 + it - 6;  // output cell j-3 (unwrapped)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float fr = R1[k] + vanleer(0.5f * (R1[k] - R0[k]), 0.5f * (R2[k] - R1[k]), eps);
      const float fl = L1[k] - vanleer(0.5f * (L1[k] - L0[k]), 0.5f * (FLh[k] - L1[k]), eps);
      const float F2 = fr - fl;               // face (j-3)+1/2
      if (it >= 6 && jo < n) uout[k * N3 + goff<AXIS>(jo, w, t, n)] = Ua[k] - nu * (F2 - F2m[k]);
      F2m[k] = F2;
      Ua[k] = Ub[k];
      Ub[k] = Uc[k];
      Uc[k] = u[k];
      FRp[k] = FR[k];
      f1m[k] = f1[k];
      R0[k] = R1[k];
      R1[k] = R2[k];
      R2[k] = FRh[k];
      L0[k] = L1[k];
      L1[k] = FLh[k];
    }
    j = jn;
  }
}

// ------------------------------------------------------------- forward, paired marching form
// The marching form above for two adjacent lines per thread (x columns w, w + 1 of a y or z
// sweep): each field is one 8-byte load per cell, and every per-cell operation runs on the
// pair with the packed FP32x2 instructions of sm_100+ (FADD2 / FMUL2 / FFMA2: one issue slot
// for two lanes), so the instruction count per cell roughly halves; reciprocals, square
// roots, sign tests and selects stay per lane. The half differences of the limiter inputs
// are formed once per cell and kept in the window (face j uses those of cells j and j + 1).
// flux splits of two cells (F^R = (cU + F)/2, F^L = (cU - F)/2), as split_flux
__device__ __forceinline__ void split_flux2(const float2 u[5], int f, float gam, float2 FR[5],
                                            float2 FL[5]) {
  const float2 inv = make_float2(fast_rcp(u[0].x), fast_rcp(u[0].y));
  const float2 hinv = mul2(inv, pk(0.5f));
  const float2 hv = mul2(u[f], hinv);  // v / 2
  const float2 m2 = fma2(u[1], u[1], fma2(u[2], u[2], mul2(u[3], u[3])));
  const float2 P = mul2(pk(gam - 1.0f), fma2(mul2(m2, hinv), pk(-1.0f), u[4]));
  const float2 cs2 = mul2(mul2(P, inv), pk(gam));
  const float csx = cs2.x > 0.0f ? cs2.x * rsqrtf(cs2.x) : 0.0f;
  const float csy = cs2.y > 0.0f ? cs2.y * rsqrtf(cs2.y) : 0.0f;
  const float2 hc = fma2(make_float2(csx, csy), pk(0.5f), make_float2(fabsf(hv.x), fabsf(hv.y)));
  float2 hF[5];
  hF[0] = mul2(u[f], pk(0.5f));
  hF[1] = mul2(u[1], hv);
  hF[2] = mul2(u[2], hv);
  hF[3] = mul2(u[3], hv);
  hF[f] = fma2(P, pk(0.5f), hF[f]);
  hF[4] = mul2(add2(u[4], P), hv);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    FR[k] = fma2(hc, u[k], hF[k]);
    FL[k] = fma2(hF[k], pk(-2.0f), FR[k]);
  }
}

// AXIS 1 or 2; n even (8-byte aligned pairs). Thread: lines w, w + 1 (adjacent x columns,
// w even), a segment of L output cells from s0 along the sweep axis. (An x sweep on pairs of
// y rows measured 2.2x slower than the tile at 128^3 and 6.7x at 256^3: its loads touch 64
// rows per warp and thrash L1.)
template <int AXIS, int MINB>
__global__ void __launch_bounds__(128, MINB)
sweep_march2_kernel(const float* __restrict__ uin, float* __restrict__ uout, int n, SArg nua,
                    float gam, float eps, int L, const float* __restrict__ kick_g, SArg kick_K) {
  pdl_enter();
  constexpr int F = 1 + AXIS;
  const LineIdx li = line_index(n, 2);
  const int w = li.w, t = li.t, b = li.b;
  const int s0 = blockIdx.z * L;
  if (!li.live) return;
  const long long N3 = (long long)n * n * n;
  uin += (size_t)b * 5 * N3;
  uout += (size_t)b * 5 * N3;
  if (kick_g) kick_g += (size_t)b * 3 * N3;
  const float nu = nua.at(b), kK = kick_K.at(b);
  const float2 hnu = pk(0.5f * nu), mnu = pk(-nu);
  float2 Ua[5], Ub[5], Uc[5];  // U_{j-3}, U_{j-2}, U_{j-1}
  float2 FRp[5], f1m[5];       // F^R_{j-1}, first-order face j-3/2
  float2 R1[5], R2[5];         // Fh^R_{j-3}, Fh^R_{j-2}
  float2 dRa[5], dRb[5];       // (Fh^R_{j-3} - Fh^R_{j-4}) / 2, (Fh^R_{j-2} - Fh^R_{j-3}) / 2
  float2 L1[5], dLa[5];        // Fh^L_{j-2}, (Fh^L_{j-2} - Fh^L_{j-3}) / 2
  float2 F2m[5];               // limited face (j-4)+1/2
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float init = (k == 0 || k == 4) ? 1.0f : 0.0f;
    Ua[k] = Ub[k] = Uc[k] = pk(init);
    FRp[k] = f1m[k] = R1[k] = R2[k] = dRa[k] = dRb[k] = L1[k] = dLa[k] = F2m[k] = pk(0.0f);
  }
  int j = wrap_periodic(s0 - 3, n);
#pragma unroll 1
  for (int it = 0; it < L + 6; ++it) {
    float2 u[5];
    const long long o = goff<AXIS>(j, w, t, n);
#pragma unroll
    for (int k = 0; k < 5; ++k) u[k] = __ldg(reinterpret_cast<const float2*>(uin + k * N3 + o));
    if (kick_g) {
      // the step's opening gas kick of both columns, as the kick kernel does it
      float a[5], c[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        a[k] = u[k].x;
        c[k] = u[k].y;
      }
      gas_kick_cell(a, kick_g + o, N3, kK);
      gas_kick_cell(c, kick_g + o + 1, N3, kK);
#pragma unroll
      for (int k = 0; k < 5; ++k) u[k] = make_float2(a[k], c[k]);
    }
    float2 FR[5], FL[5];
    split_flux2(u, F, gam, FR, FL);
    float2 f1[5], uh[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      f1[k] = sub2(FRp[k], FL[k]);                       // face j-1/2
      uh[k] = fma2(hnu, sub2(f1m[k], f1[k]), Uc[k]);     // Uh_{j-1}
    }
    float2 FRh[5], FLh[5];
    split_flux2(uh, F, gam, FRh, FLh);
    const int jo = s0 + it - 6;  // output cell j-3 (unwrapped)
    const bool store = it >= 6 && jo < n;
    const long long oo = goff<AXIS>(jo < n ? jo : 0, w, t, n);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float2 dLb = mul2(sub2(FLh[k], L1[k]), pk(0.5f));
      const float2 fr = add2(R1[k], vanleer2(dRa[k], dRb[k], eps));
      const float2 fl = sub2(L1[k], vanleer2(dLa[k], dLb, eps));
      const float2 F2 = sub2(fr, fl);                    // face (j-3)+1/2
      if (store)
        *reinterpret_cast<float2*>(uout + k * N3 + oo) = fma2(mnu, sub2(F2, F2m[k]), Ua[k]);
      F2m[k] = F2;
      dRa[k] = dRb[k];
      dRb[k] = mul2(sub2(FRh[k], R2[k]), pk(0.5f));
      R1[k] = R2[k];
      R2[k] = FRh[k];
      dLa[k] = dLb;
      L1[k] = FLh[k];
      Ua[k] = Ub[k];
      Ub[k] = Uc[k];
      Uc[k] = u[k];
      FRp[k] = FR[k];
      f1m[k] = f1[k];
    }
    j = (j + 1 == n) ? 0 : j + 1;
  }
}

// Limiter value and both partials of two lanes, as vanleer_vg (branch-free: the gate selects
// per lane after the arithmetic of both).
__device__ __forceinline__ void vanleer_vg2(float2 a, float2 b, float eps, float2& phi, float2& da,
                                            float2& db) {
  const float2 ab = mul2(a, b);
  const float2 s = add2(a, b);
  const float2 D = add2(s, make_float2(copysignf(eps, s.x), copysignf(eps, s.y)));
  const float2 q = mul2(pk(2.0f), make_float2(fast_rcp(D.x), fast_rcp(D.y)));  // 2 / D
  const float2 q2 = mul2(mul2(q, q), pk(0.5f));                                  // 2 / D^2
  const float2 p = mul2(ab, q);
  const float2 dA = mul2(mul2(b, sub2(D, a)), q2);
  const float2 dB = mul2(mul2(a, sub2(D, b)), q2);
  const bool gx = ab.x > 0.0f, gy = ab.y > 0.0f;
  phi = make_float2(gx ? p.x : 0.0f, gy ? p.y : 0.0f);
  da = make_float2(gx ? dA.x : 0.0f, gy ? dA.y : 0.0f);
  db = make_float2(gx ? dB.x : 0.0f, gy ? dB.y : 0.0f);
}

// ------------------------------------------------------------- adjoint, marching form
// Pass 1: each thread streams one line segment [s0, s0 + L) plus a halo and produces
// lamUh_j for its own cells. At load i it recomputes the forward stages for cell i-1
// (first-order face, Uh, half-step splits), evaluates the limited face t = i-3 once (its
// flux for d/dnu and its limiter derivatives), and adds the face's contributions to the
// running adjoints of the half-step splits of cells t-1 .. t+2:
//   lamFh^R_{t-1} -= A_t, lamFh^R_t += lf_t + A_t - B_t, lamFh^R_{t+1} += B_t,
//   lamFh^L_t -= C_t, lamFh^L_{t+1} += -lf_t + C_t - D_t, lamFh^L_{t+2} += D_t,
// with lf_t = nu (lam_out_{t+1} - lam_out_t), A = lf daR/2, B = lf dbR/2, C = lf daL/2,
// D = lf dbL/2 (daR, dbR the limiter partials of the right-moving face flux, daL, dbL of
// the left-moving one). Cell i-4 is then complete and lamUh_{i-4} = VJP(Uh_{i-4}).
// d/dnu gathers sum_t F2_t lf_t / nu - sum_j lamUh_j dF1_j / 2.
template <int AXIS, int FC = 1 + AXIS>
__global__ void __launch_bounds__(128, 3)
sweep_adj_march_kernel(const float* __restrict__ uin, const float* __restrict__ lout,
                       float* __restrict__ luh_out, int n, SArg nua, float gam, float eps,
                       DPart dnub, int L) {
  pdl_enter();
  constexpr int F = FC;  // momentum component along the sweep
  const LineIdx li = line_index(n, 1);
  const int w = li.w, b = li.b;  // line coordinate, instance
  const int t3 = li.t < n ? li.t : 0;  // third coordinate (rows past n load row 0, store nothing)
  const int s0 = blockIdx.z * L;
  const bool live = li.live;
  const long long N3 = (long long)n * n * n;
  uin += (size_t)b * 5 * N3;
  lout += (size_t)b * 5 * N3;
  luh_out += (size_t)b * 5 * N3;
  const float nu = nua.at(b);
  double* dnu = dnub.at(b);
  const float hnu = 0.5f * nu, inv_nu = 1.0f / nu;
  float Uc[5], FRp[5], f1m[5];          // U_{i-1}, F^R_{i-1}, face (i-3/2)
  float R0[5], R1[5], R2[5];            // Fh^R_{i-4}, Fh^R_{i-3}, Fh^R_{i-2}
  float L0[5], L1[5];                   // Fh^L_{i-3}, Fh^L_{i-2}
  float H0[5], H1[5], H2[5];            // Uh_{i-4}, Uh_{i-3}, Uh_{i-2}
  float D0[5], D1[5], D2[5];            // dF1_{i-4}, dF1_{i-3}, dF1_{i-2}
  float M0[5], M1[5], M2[5];            // lam_out_{i-3}, lam_out_{i-2}, lam_out_{i-1}
  float aR0[5], aR1[5], aR2[5];         // lamFh^R accumulators of cells i-4, i-3, i-2
  float aL0[5], aL1[5], aL2[5], aL3[5]; // lamFh^L accumulators of cells i-4 .. i-1
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float init = (k == 0 || k == 4) ? 1.0f : 0.0f;
    Uc[k] = H0[k] = H1[k] = H2[k] = init;
    FRp[k] = f1m[k] = R0[k] = R1[k] = R2[k] = L0[k] = L1[k] = 0.0f;
    D0[k] = D1[k] = D2[k] = M0[k] = M1[k] = M2[k] = 0.0f;
    aR0[k] = aR1[k] = aR2[k] = aL0[k] = aL1[k] = aL2[k] = aL3[k] = 0.0f;
  }
  float dnu_acc = 0.0f;
  // loads run from s0 - 5 to s0 + L + 3: cells s0 .. s0 + L - 1 complete at i = j + 4
  const int ww = live ? w : 0;
  int j = wrap_periodic(s0 - 5, n);
  float un[5], ln[5];
  {
    const long long o = goff<AXIS>(j, ww, t3, n);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      un[k] = __ldg(uin + k * N3 + o);
      ln[k] = __ldg(lout + k * N3 + o);
    }
  }
  // unrolled by the windows' period: the three-deep register windows rotate by renaming
  // instead of moves (measured 119 -> 114 us per call at 128^3 despite a few spilled words)
#pragma unroll 3
  for (int it = 0; it < L + 9; ++it) {
    float u[5], lo[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      u[k] = un[k];
      lo[k] = ln[k];
    }
    const int jn = (j + 1 == n) ? 0 : j + 1;
    if (it + 1 < L + 9) {
      const long long on = goff<AXIS>(jn, ww, t3, n);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        un[k] = __ldg(uin + k * N3 + on);
        ln[k] = __ldg(lout + k * N3 + on);
      }
    }
    // forward stages for cell i-1
    float FR[5], FL[5];
    split_flux(u, F, gam, FR, FL);
    float f1[5], dF[5], uh[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      f1[k] = FRp[k] - FL[k];  // face i-1/2
      dF[k] = f1[k] - f1m[k];  // dF1_{i-1}
      uh[k] = Uc[k] - hnu * dF[k];
    }
    float FRh[5], FLh[5];
    split_flux(uh, F, gam, FRh, FLh);
    // face t = i-3: R from Fh^R_{i-4..i-2}, L from Fh^L_{i-3..i-1}; lf_t from lam_out
    // face t = i-3 belongs to this segment's d/dnu sum when t is one of its cells: over a
    // periodic line sum_k -lam_out_k (F2_k - F2_{k-1}) = sum_t F2_t lf_t / nu
    const int jt = s0 + it - 8;  // unwrapped index of face cell t (face t + 1/2)
    const bool face_in = (jt >= s0) && (jt < s0 + L) && (jt < n);
    // components (0, 1) and (2, 3) as FP32x2 pairs, component 4 alone: the same operations
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const float2 lf = mul2(pk(nu), sub2(make_float2(M1[k], M1[k + 1]), make_float2(M0[k], M0[k + 1])));
      const float2 r0 = make_float2(R0[k], R0[k + 1]), r1 = make_float2(R1[k], R1[k + 1]);
      const float2 r2 = make_float2(R2[k], R2[k + 1]);
      const float2 l0 = make_float2(L0[k], L0[k + 1]), l1 = make_float2(L1[k], L1[k + 1]);
      const float2 aR = mul2(pk(0.5f), sub2(r1, r0)), bR = mul2(pk(0.5f), sub2(r2, r1));
      const float2 aL = mul2(pk(0.5f), sub2(l1, l0));
      const float2 bL = mul2(pk(0.5f), sub2(make_float2(FLh[k], FLh[k + 1]), l1));
      float2 pR, daR, dbR, pL, daL, dbL;
      vanleer_vg2(aR, bR, eps, pR, daR, dbR);
      vanleer_vg2(aL, bL, eps, pL, daL, dbL);
      const float2 hl = mul2(pk(0.5f), lf);
      const float2 A = mul2(hl, daR), B = mul2(hl, dbR), C = mul2(hl, daL), D = mul2(hl, dbL);
      const float2 a0 = sub2(make_float2(aR0[k], aR0[k + 1]), A);
      const float2 a1 = add2(make_float2(aR1[k], aR1[k + 1]), sub2(add2(lf, A), B));
      const float2 a2 = add2(make_float2(aR2[k], aR2[k + 1]), B);
      const float2 b1 = sub2(make_float2(aL1[k], aL1[k + 1]), C);
      const float2 b2 = add2(make_float2(aL2[k], aL2[k + 1]), sub2(sub2(C, lf), D));
      const float2 b3 = add2(make_float2(aL3[k], aL3[k + 1]), D);
      aR0[k] = a0.x; aR0[k + 1] = a0.y;
      aR1[k] = a1.x; aR1[k + 1] = a1.y;
      aR2[k] = a2.x; aR2[k + 1] = a2.y;
      aL1[k] = b1.x; aL1[k + 1] = b1.y;
      aL2[k] = b2.x; aL2[k + 1] = b2.y;
      aL3[k] = b3.x; aL3[k + 1] = b3.y;
      // d/dnu part 1: faces of the segment's output cells (t in [s0-1, s0+L))
      if (face_in) {
        const float2 f2 = mul2(sub2(add2(r1, pR), sub2(l1, pL)), lf);
        dnu_acc += (f2.x + f2.y) * inv_nu;
      }
    }
    {
      const int k = 4;
      const float lf = nu * (M1[k] - M0[k]);  // nu (lam_out_{t+1} - lam_out_t), t = i-3
      const float aR = 0.5f * (R1[k] - R0[k]), bR = 0.5f * (R2[k] - R1[k]);
      const float aL = 0.5f * (L1[k] - L0[k]), bL = 0.5f * (FLh[k] - L1[k]);
      float pR, daR, dbR, pL, daL, dbL;
      vanleer_vg(aR, bR, eps, pR, daR, dbR);
      vanleer_vg(aL, bL, eps, pL, daL, dbL);
      const float A = 0.5f * lf * daR, B = 0.5f * lf * dbR;
      const float C = 0.5f * lf * daL, D = 0.5f * lf * dbL;
      aR0[k] -= A;
      aR1[k] += lf + A - B;
      aR2[k] += B;
      aL1[k] -= C;
      aL2[k] += -lf + C - D;
      aL3[k] += D;
      if (face_in) dnu_acc += ((R1[k] + pR) - (L1[k] - pL)) * lf * inv_nu;
    }
    // cell i-4 is complete
    const int jc = s0 + it - 9;  // unwrapped index of cell i-4
    if (it >= 9 && live && jc < n) {
      float luh[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      split_flux_vjp(H0, F, gam, aR0, aL0, luh);
      const long long oc = goff<AXIS>(jc, w, t3, n);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        luh_out[k * N3 + oc] = luh[k];
        dnu_acc -= 0.5f * luh[k] * D0[k];
      }
    }
    // shift the windows
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      aR0[k] = aR1[k];
      aR1[k] = aR2[k];
      aR2[k] = 0.0f;
      aL0[k] = aL1[k];
      aL1[k] = aL2[k];
      aL2[k] = aL3[k];
      aL3[k] = 0.0f;
      H0[k] = H1[k];
      H1[k] = H2[k];
      H2[k] = uh[k];
      D0[k] = D1[k];
      D1[k] = D2[k];
      D2[k] = dF[k];
      R0[k] = R1[k];
      R1[k] = R2[k];
      R2[k] = FRh[k];
      L0[k] = L1[k];
      L1[k] = FLh[k];
      M0[k] = M1[k];
      M1[k] = M2[k];
      M2[k] = lo[k];
      Uc[k] = u[k];
      FRp[k] = FR[k];
      f1m[k] = f1[k];
    }
    j = jn;
  }
  if (dnu) {
    if (!live) dnu_acc = 0.0f;
    block_sum_atomic(dnu_acc, dnu);
  }
}

// Pass 2: lam_in_k = lam_out_k + lamUh_k + VJP(U_k; nu/2 (lamUh_{k+1} - lamUh_k),
// -nu/2 (lamUh_k - lamUh_{k-1})), one thread per cell.
template <int AXIS, int FC = 1 + AXIS>
__global__ void __launch_bounds__(256)
sweep_adj_final_kernel(const float* __restrict__ uin, const float* __restrict__ lout,
                       const float* __restrict__ luh, float* __restrict__ lin, int n,
                       SArg nua, float gam) {
  pdl_enter();
  constexpr int F = FC;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.z / n;  // instance
  const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z - b * n;
  if (x >= n || y >= n) return;
  const long long N3 = (long long)n * n * n;
  uin += (size_t)b * 5 * N3;
  lout += (size_t)b * 5 * N3;
  luh += (size_t)b * 5 * N3;
  lin += (size_t)b * 5 * N3;
  const float nu = nua.at(b);
  const long long o = ((long long)z * n + y) * n + x;
  int cm, cp;  // neighbour offsets along the sweep axis (periodic)
  long long om, op;
  if (AXIS == 0) {
    cm = x == 0 ? n - 1 : x - 1;
    cp = x + 1 == n ? 0 : x + 1;
    om = o - x + cm;
    op = o - x + cp;
  } else if (AXIS == 1) {
    cm = y == 0 ? n - 1 : y - 1;
    cp = y + 1 == n ? 0 : y + 1;
    om = o + (long long)(cm - y) * n;
    op = o + (long long)(cp - y) * n;
  } else {
    cm = z == 0 ? n - 1 : z - 1;
    cp = z + 1 == n ? 0 : z + 1;
    om = o + (long long)(cm - z) * n * n;
    op = o + (long long)(cp - z) * n * n;
  }
  float u[5], lR[5], lL[5], lu[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    u[k] = __ldg(uin + k * N3 + o);
    const float h0 = __ldg(luh + k * N3 + o);
    const float hm = __ldg(luh + k * N3 + om);
    const float hp = __ldg(luh + k * N3 + op);
    lR[k] = 0.5f * nu * (hp - h0);
    lL[k] = -0.5f * nu * (h0 - hm);
    lu[k] = __ldg(lout + k * N3 + o) + h0;
  }
  split_flux_vjp(u, F, gam, lR, lL, lu);
#pragma unroll
  for (int k = 0; k < 5; ++k) lin[k * N3 + o] = lu[k];
}

// Pass 2 on two adjacent x cells per thread (n even), in packed FP32x2 arithmetic: the same
// operations as split_flux_vjp and sweep_adj_final_kernel, for the pair.
__device__ __forceinline__ void split_flux_vjp2(const float2 u[5], int f, float gam,
                                                const float2 lR[5], const float2 lL[5],
                                                float2 lu[5]) {
  const float2 inv = make_float2(fast_rcp(u[0].x), fast_rcp(u[0].y));
  const float2 v = mul2(u[f], inv);
  const float2 m2 = fma2(u[1], u[1], fma2(u[2], u[2], mul2(u[3], u[3])));
  const float2 hm2inv = mul2(mul2(m2, inv), pk(0.5f));
  const float2 P = mul2(pk(gam - 1.0f), sub2(u[4], hm2inv));
  const float2 cs2 = mul2(mul2(P, inv), pk(gam));
  const float rx = cs2.x > 0.0f ? rsqrtf(cs2.x) : 0.0f;
  const float ry = cs2.y > 0.0f ? rsqrtf(cs2.y) : 0.0f;
  const float2 rcs = make_float2(rx, ry);
  const float2 cs = mul2(cs2, rcs);
  const float2 c = add2(make_float2(fabsf(v.x), fabsf(v.y)), cs);
  float2 sig[5], del[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    sig[k] = mul2(add2(lR[k], lL[k]), pk(0.5f));
    del[k] = mul2(sub2(lR[k], lL[k]), pk(0.5f));
  }
  float2 lc = pk(0.0f);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    lu[k] = fma2(c, sig[k], lu[k]);
    lc = fma2(sig[k], u[k], lc);
  }
  float2 lv = pk(0.0f), lP = del[f], lrho = pk(0.0f);
  lu[f] = add2(lu[f], del[0]);
#pragma unroll
  for (int k = 1; k <= 3; ++k) {
    lu[k] = fma2(del[k], v, lu[k]);
    lv = fma2(del[k], u[k], lv);
  }
  lu[4] = fma2(del[4], v, lu[4]);
  lP = fma2(del[4], v, lP);
  lv = fma2(del[4], add2(u[4], P), lv);
  const float2 sgn = make_float2((float)((v.x > 0.0f) - (v.x < 0.0f)), (float)((v.y > 0.0f) - (v.y < 0.0f)));
  lv = fma2(lc, sgn, lv);
  // where cs2 <= 0: rcs = 0 and cs = 0, so both terms below vanish, as in split_flux_vjp
  lP = fma2(mul2(lc, pk(0.5f * gam)), mul2(rcs, inv), lP);
  lrho = fma2(mul2(lc, pk(-0.5f)), mul2(cs, inv), lrho);
  const float2 gP = mul2(pk(gam - 1.0f), lP);
  lu[4] = add2(lu[4], gP);
  const float2 gPinv = mul2(gP, inv);
#pragma unroll
  for (int k = 1; k <= 3; ++k) lu[k] = fma2(mul2(gPinv, pk(-1.0f)), u[k], lu[k]);
  lrho = fma2(gPinv, hm2inv, lrho);
  lu[f] = fma2(lv, inv, lu[f]);
  lrho = fma2(mul2(lv, pk(-1.0f)), mul2(v, inv), lrho);
  lu[0] = add2(lu[0], lrho);
}

// lam_in of cells x, x + 1 of row (y, z) (one instance's arrays): lam_out + lamUh + the
// flux-split VJP of U with the face adjoints from lamUh of the neighbours along the axis
template <int AXIS, int F>
__device__ __forceinline__ void adj_final2_cells(const float* __restrict__ uin,
                                                 const float* __restrict__ lout,
                                                 const float* __restrict__ luh, int n, int x,
                                                 int y, int z, float nu, float gam,
                                                 float2 lu[5]) {
  const long long N3 = (long long)n * n * n;
  const long long o = ((long long)z * n + y) * n + x;
  long long om, op;  // neighbours along the sweep axis (y or z), periodic
  if (AXIS == 1) {
    om = o + (long long)((y == 0 ? n - 1 : y - 1) - y) * n;
    op = o + (long long)((y + 1 == n ? 0 : y + 1) - y) * n;
  } else {
    om = o + (long long)((z == 0 ? n - 1 : z - 1) - z) * n * n;
    op = o + (long long)((z + 1 == n ? 0 : z + 1) - z) * n * n;
  }
  const float2 hnu = pk(0.5f * nu), mhnu = pk(-0.5f * nu);
  float2 u[5], lR[5], lL[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    u[k] = __ldg(reinterpret_cast<const float2*>(uin + k * N3 + o));
    const float2 h0 = __ldg(reinterpret_cast<const float2*>(luh + k * N3 + o));
    const float2 hm = __ldg(reinterpret_cast<const float2*>(luh + k * N3 + om));
    const float2 hp = __ldg(reinterpret_cast<const float2*>(luh + k * N3 + op));
    lR[k] = mul2(hnu, sub2(hp, h0));
    lL[k] = mul2(mhnu, sub2(h0, hm));
    lu[k] = add2(__ldg(reinterpret_cast<const float2*>(lout + k * N3 + o)), h0);
  }
  split_flux_vjp2(u, F, gam, lR, lL, lu);
}

// grid (cdiv(n / 2, blockDim.x), cdiv(n, blockDim.y), n B); thread: cells x = 2 t, 2 t + 1
// of row (y, z). TOUT (the x axis run on x <-> y transposed copies): blocks of 16 x 32
// threads cover 32 x 32 cells of a plane, and the result goes out through a shared-memory
// tile in the untransposed layout, cell (z, y, x) of the copies to (z, x, y) of lin.
template <int AXIS, int FC = 1 + AXIS, bool TOUT = false>
__global__ void __launch_bounds__(TOUT ? 512 : 128)
sweep_adj_final2_kernel(const float* __restrict__ uin, const float* __restrict__ lout,
                        const float* __restrict__ luh, float* __restrict__ lin, int n,
                        SArg nua, float gam) {
  pdl_enter();
  constexpr int F = FC;
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int b = blockIdx.z / n;
  const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z - b * n;
  const long long N3 = (long long)n * n * n;
  if (TOUT) {
    __shared__ float tile[5][32][33];  // [field][x - x0][y - y0]
    const int lx = 2 * threadIdx.x, ly = threadIdx.y;
    if (x < n && y < n) {
      float2 lu[5];
      adj_final2_cells<AXIS, F>(uin + (size_t)b * 5 * N3, lout + (size_t)b * 5 * N3,
                                luh + (size_t)b * 5 * N3, n, x, y, z, nua.at(b), gam, lu);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        tile[k][lx][ly] = lu[k].x;
        tile[k][lx + 1][ly] = lu[k].y;
      }
    }
    __syncthreads();
    const int x0 = 2 * blockIdx.x * blockDim.x, y0 = blockIdx.y * blockDim.y;
    float* out = lin + (size_t)b * 5 * N3;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(lin) & 15) == 0) {
      // rows of 32 outputs as eight float4 (y0 + c and n are multiples of 4)
      for (int e = tid; e < 5 * 32 * 8; e += 512) {
        const int k = e >> 8, r = (e >> 3) & 31, c = (e & 7) << 2;
        if (x0 + r < n && y0 + c < n)
          *reinterpret_cast<float4*>(out + k * N3 + ((long long)z * n + x0 + r) * n + y0 + c) =
              make_float4(tile[k][r][c], tile[k][r][c + 1], tile[k][r][c + 2], tile[k][r][c + 3]);
      }
    } else {
      for (int e = tid; e < 5 * 32 * 32; e += 512) {
        const int k = e >> 10, r = (e >> 5) & 31, c = e & 31;
        if (x0 + r < n && y0 + c < n)
          out[k * N3 + ((long long)z * n + x0 + r) * n + y0 + c] = tile[k][r][c];
      }
    }
    return;
  }
  if (x >= n || y >= n) return;
  float2 lu[5];
  adj_final2_cells<AXIS, F>(uin + (size_t)b * 5 * N3, lout + (size_t)b * 5 * N3,
                            luh + (size_t)b * 5 * N3, n, x, y, z, nua.at(b), gam, lu);
  lin += (size_t)b * 5 * N3;
  const long long o = ((long long)z * n + y) * n + x;
#pragma unroll
  for (int k = 0; k < 5; ++k) *reinterpret_cast<float2*>(lin + k * N3 + o) = lu[k];
}

// ------------------------------------------------------------------------- adjoint
// lam_in_k = lam_out_k + lamUh_k + VJP_{F^R,F^L}(U_k; lamF^R_k, lamF^L_k), with
// lamF^R_k = nu/2 (lamUh_{k+1} - lamUh_k), lamF^L_k = -nu/2 (lamUh_k - lamUh_{k-1}), and
// lamUh_j = VJP_{F^R,F^L}(Uh_j; lamFh^R_j, lamFh^L_j) gathered from the limited faces
// t+1/2 (t = j-2 .. j+1) whose adjoint is nu (lam_out_{t+1} - lam_out_t). Output cells need
// U on a 5-cell halo and lam_out on a 3-cell halo; the forward stages are recomputed.
// d(out)/d(nu) = -(F2_+ - F2_-) - nu dF2/dUh . (F_{+} - F_{-})/2 is accumulated into *dnu.
template <int AXIS>
__global__ void __launch_bounds__(SweepCfg<AXIS>::NTA, 2)
sweep_adj_kernel(const float* __restrict__ uin, const float* __restrict__ lout,
                 float* __restrict__ lin, int n, SArg nua, float gam, float eps, DPart dnub) {
  pdl_enter();
  constexpr int S = SweepCfg<AXIS>::SA, W = SweepCfg<AXIS>::WA, NT = SweepCfg<AXIS>::NTA;
  using G = TileGeom<AXIS, S, W, 5>;
  constexpr int NC = G::NC, DS = G::DS, SP = G::SP, CPT = (NC + NT - 1) / NT;
  constexpr int F = 1 + AXIS;
  extern __shared__ float sm[];
  float* sf = sm;            // 10 NC: F^R,F^L of U, then of Uh
  float* sl = sm + 10 * NC;  // 5 NC: lam_out
  float* sh = sm + 15 * NC;  // 5 NC: lamUh
  const long long N3 = (long long)n * n * n;
  const int b = blockIdx.z / n;  // instance
  const int s0 = blockIdx.x * S, w0 = blockIdx.y * W, t = blockIdx.z - b * n;
  uin += (size_t)b * 5 * N3;
  lout += (size_t)b * 5 * N3;
  lin += (size_t)b * 5 * N3;
  const float nu = nua.at(b);
  double* dnu = dnub.at(b);

  float ureg[CPT][5];
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    if (c < NC) {
      const int s = G::s_of(c), w = G::w_of(c), wg = w0 + w;
      const int sgl = wrap_periodic(s0 + s - 5, n);
      float u[5] = {1.f, 0.f, 0.f, 0.f, 1.f};
      float l[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (wg < n) {
        const long long o = goff<AXIS>(sgl, wg, t, n);
#pragma unroll
        for (int k = 0; k < 5; ++k) u[k] = __ldg(uin + k * N3 + o);
        if (s >= 2 && s < SP - 2) {
#pragma unroll
          for (int k = 0; k < 5; ++k) l[k] = __ldg(lout + k * N3 + o);
        }
      }
      float FR[5], FL[5];
      split_flux(u, F, gam, FR, FL);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        ureg[i][k] = u[k];
        sf[k * NC + c] = FR[k];
        sf[(5 + k) * NC + c] = FL[k];
        sl[k * NC + c] = l[k];
      }
    }
  }
  __syncthreads();
  float uh[CPT][5], df1[CPT][5];
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c);
    if (c < NC && s >= 1 && s < SP - 1) {
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const float fp = sf[k * NC + c] - sf[(5 + k) * NC + c + DS];
        const float fm = sf[k * NC + c - DS] - sf[(5 + k) * NC + c];
        df1[i][k] = fp - fm;
        uh[i][k] = ureg[i][k] - 0.5f * nu * df1[i][k];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c);
    if (c < NC && s >= 1 && s < SP - 1) {
      float FR[5], FL[5];
      split_flux(uh[i], F, gam, FR, FL);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        sf[k * NC + c] = FR[k];
        sf[(5 + k) * NC + c] = FL[k];
      }
    }
  }
  __syncthreads();
  float dnu_acc = 0.0f;
  // lamUh_j for j in [4, S+6)
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c), w = G::w_of(c);
    if (c < NC && s >= 4 && s < S + 6) {
      float lR[5], lL[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const float* R = sf + k * NC + c;
        const float* L = sf + (5 + k) * NC + c;
        const float* lo = sl + k * NC + c;
        // face adjoints lam_f(t) = nu (lam_out_{t+1} - lam_out_t), t = j-2 .. j+1
        const float lf_m2 = nu * (lo[-DS] - lo[-2 * DS]);
        const float lf_m1 = nu * (lo[0] - lo[-DS]);
        const float lf_0 = nu * (lo[DS] - lo[0]);
        const float lf_p1 = nu * (lo[2 * DS] - lo[DS]);
        float da, db, acc;
        // right-moving: faces t = j-1, j, j+1
        vanleer_grad(0.5f * (R[0] - R[-DS]), 0.5f * (R[DS] - R[0]), eps, da, db);
        acc = lf_0 * (1.0f + 0.5f * da - 0.5f * db);
        vanleer_grad(0.5f * (R[DS] - R[0]), 0.5f * (R[2 * DS] - R[DS]), eps, da, db);
        acc -= 0.5f * da * lf_p1;
        vanleer_grad(0.5f * (R[-DS] - R[-2 * DS]), 0.5f * (R[0] - R[-DS]), eps, da, db);
        acc += 0.5f * db * lf_m1;
        lR[k] = acc;
        // left-moving: F^L face t = L_{t+1} - phi(0.5(L_{t+1}-L_t), 0.5(L_{t+2}-L_{t+1}))
        vanleer_grad(0.5f * (L[0] - L[-DS]), 0.5f * (L[DS] - L[0]), eps, da, db);  // t=j-1
        acc = -lf_m1 * (1.0f - 0.5f * da + 0.5f * db);
        vanleer_grad(0.5f * (L[DS] - L[0]), 0.5f * (L[2 * DS] - L[DS]), eps, da, db);  // t=j
        acc -= lf_0 * 0.5f * da;
        vanleer_grad(0.5f * (L[-DS] - L[-2 * DS]), 0.5f * (L[0] - L[-DS]), eps, da, db);  // t=j-2
        acc += 0.5f * db * lf_m2;
        lL[k] = acc;
      }
      float luh[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      split_flux_vjp(uh[i], F, gam, lR, lL, luh);
      const int sgl = s0 + s - 5, wg = w0 + w;
      if (s >= 5 && s < S + 5 && sgl < n && wg < n) {
#pragma unroll
        for (int k = 0; k < 5; ++k) dnu_acc -= 0.5f * luh[k] * df1[i][k];
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k * NC + c] = luh[k];
    }
  }
  __syncthreads();
  // outputs s in [5, S+5)
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * NT;
    const int s = G::s_of(c), w = G::w_of(c);
    const int sgl = s0 + s - 5, wg = w0 + w;
    if (c < NC && s >= 5 && s < S + 5 && sgl < n && wg < n) {
      float lR[5], lL[5], lu[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const float* lh = sh + k * NC + c;
        lR[k] = 0.5f * nu * (lh[DS] - lh[0]);
        lL[k] = -0.5f * nu * (lh[0] - lh[-DS]);
        const float lo = sl[k * NC + c];
        lu[k] = lo + lh[0];
        const float fp = face_flux(sf + k * NC + c, sf + (5 + k) * NC + c, DS, eps);
        const float fm = face_flux(sf + k * NC + c - DS, sf + (5 + k) * NC + c - DS, DS, eps);
        dnu_acc -= lo * (fp - fm);
      }
      split_flux_vjp(ureg[i], F, gam, lR, lL, lu);
      const long long o = goff<AXIS>(sgl, wg, t, n);
#pragma unroll
      for (int k = 0; k < 5; ++k) lin[k * N3 + o] = lu[k];
    }
  }
  if (dnu) block_sum_atomic(dnu_acc, dnu);
}

// Kernel variants (SIM_SWEEP_*): the shared-memory tile, or the marching form with line
// segments of 32 or 16 cells (y and z sweeps only: marching along x is not coalesced).
// The default, measured on GB300 for one instance: the tile is fastest up to n ~ 128
// (51 us at 128^3 for every axis); marching with segments of 32 wins for y/z on larger
// grids (335 us vs 386 us at 256^3). The adjoint defaults to the marching pair for every
// axis: y/z directly (2.1x the tile at 256^3), x on x <-> y transposed copies (the x tile
// takes ~320 us at 128^3 against ~170 us for a y/z pair), with segments fitted to whole
// waves (at 128^3 three segments of 43 cells: every block resident at once, 140 us per
// call in the benchmark pass against 156 us with 16-cell segments). sim_autotune times the
// variants per handle.
static int pick_fwd(int axis, int n, int variant) {
  if (axis == 0) return SIM_SWEEP_TILE;
  if (variant != SIM_SWEEP_DEFAULT) return variant;
  return n >= 192 ? SIM_SWEEP_MARCH32 : SIM_SWEEP_TILE;
}

static int pick_adj(int axis, int variant) {
  (void)axis;
  // the paired form is forward only; its adjoint is the fitted marching pair
  return (variant != SIM_SWEEP_DEFAULT && variant != SIM_SWEEP_PAIR) ? variant : SIM_SWEEP_MARCH_FIT;
}

// Block of a line kernel (line_index): the x lanes (n, or n / 2 for two columns per lane)
// in whole warps up to `threads`, and the rest of the block's threads as rows.
static dim3 line_block(int lanes, int threads) {
  const int tx = std::min(threads, 32 * cdiv(lanes, 32));
  return dim3(tx, std::max(1, threads / tx));
}

// Grid of a line kernel over an n^3 grid of B instances with `segs` segments per line.
static dim3 line_grid(int lanes, int n, int B, dim3 blk, int segs) {
  return dim3(cdiv(lanes, blk.x), B * cdiv(n, blk.y), segs);
}

// Segment length of a marching kernel for an n^3 grid of B instances: the number k of
// segments per line that minimises waves(k) x (n / k + halo), a wave being the blocks of
// shape blk that stay resident on all SMs at the kernel's register use (each thread
// streams its segment plus the halo once).
template <class Kern>
static int fit_segment(Kern kernel, int n, int B, int halo, int lanes, dim3 blk) {
  const int block = (int)(blk.x * blk.y);
  // resident blocks on the current device, per kernel, block size and device
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, long long> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 32;
  }
  long long resident = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), dev * 2048 + block);
    auto it = cache.find(key);
    if (it == cache.end()) {
      int sms = 0, per_sm = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess) {
        cudaGetLastError();
        return 32;
      }
      it = cache.emplace(key, per_sm * sms > 0 ? (long long)per_sm * sms : 1).first;
    }
    resident = it->second;
  }
  // blocks of one segment layer
  const long long layer = (long long)cdiv(lanes, blk.x) * cdiv(n, blk.y) * B;
  int best = n, best_cost = 1 << 30;
  for (int k = 1; k <= n; ++k) {
    const int L = cdiv(n, k);
    if (L < 8) break;
    const long long blocks = layer * cdiv(n, L);
    const long long waves = (blocks + resident - 1) / resident;
    const long long cost = waves * (L + halo);
    if (cost < best_cost) {
      best_cost = (int)cost;
      best = L;
    }
  }
  return best;
}

static int segment_length(int variant) {
  return variant == SIM_SWEEP_MARCH16 ? 16 : 32;
}

template <int AXIS>
static sim_status launch_march_t(const float* uin, float* uout, int n, SArg nu, float gam,
                                 float eps, int B, int variant, cudaStream_t st) {
  const dim3 blk = line_block(n, 128);
  const int L = variant == SIM_SWEEP_MARCH_FIT
                    ? fit_segment(sweep_march_kernel<AXIS>, n, B, 6, n, blk)
                    : segment_length(variant);
  DH_CUDA_TRY((launch_pdl(sweep_march_kernel<AXIS>, line_grid(n, n, B, blk, cdiv(n, L)), blk, 0, st, uin, uout, n, nu,
                                                                                 gam, eps, L)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

template <int AXIS, int MINB>
static sim_status launch_march2_mb(const float* uin, float* uout, int n, SArg nu, float gam,
                                   float eps, int B, cudaStream_t st, const float* kick_g,
                                   SArg kick_K) {
  const dim3 blk = line_block(n / 2, 128);
  const int L = fit_segment(sweep_march2_kernel<AXIS, MINB>, n, B, 6, n / 2, blk);
  DH_CUDA_TRY((launch_pdl(sweep_march2_kernel<AXIS, MINB>, line_grid(n / 2, n, B, blk, cdiv(n, L)), blk, 0, st, uin, uout, n, nu, gam, eps, L, kick_g, kick_K)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// Three resident blocks per SM (the registers capped at 168, 12 warps per SM) measured
// fastest: 47 us at 128^3 and 277 us at 256^3 per y or z sweep, against 58 / 347 us at two
// blocks (206 registers) and 66 / 347 us at four (128 registers, spilling).
template <int AXIS>
static sim_status launch_march2_t(const float* uin, float* uout, int n, SArg nu, float gam,
                                  float eps, int B, cudaStream_t st, const float* kick_g,
                                  SArg kick_K) {
  return launch_march2_mb<AXIS, 3>(uin, uout, n, nu, gam, eps, B, st, kick_g, kick_K);
}

// the paired form needs two adjacent x columns per thread: y / z sweeps, n even
static bool takes_pair(int axis, int n, int variant, const void* uin, const void* uout) {
  return axis != 0 && variant == SIM_SWEEP_PAIR && n % 2 == 0 &&
         ((reinterpret_cast<uintptr_t>(uin) | reinterpret_cast<uintptr_t>(uout)) % 8) == 0;
}

template <int AXIS>
static sim_status launch_sweep_t(const float* uin, float* uout, int n, SArg nu, float gam,
                                 float eps, int B, int variant, cudaStream_t st,
                                 const float* kick_g, SArg kick_K) {
  using C = SweepCfg<AXIS>;
  if (takes_pair(AXIS, n, variant, uin, uout))
    return launch_march2_t<AXIS>(uin, uout, n, nu, gam, eps, B, st, kick_g, kick_K);
  if (AXIS != 0 && variant != SIM_SWEEP_TILE && variant != SIM_SWEEP_PAIR) {
    if (kick_g) {
      set_error("internal: the marching forward sweep takes no opening kick");
      return SIM_EINVAL;
    }
    return launch_march_t<AXIS>(uin, uout, n, nu, gam, eps, B, variant, st);
  }
  constexpr int NC = (C::S + 6) * C::W;
  const size_t smem = 15 * NC * sizeof(float);
  dim3 grid(cdiv(n, C::S), cdiv(n, C::W), n * B);
  DH_CUDA_TRY((launch_pdl(sweep_fwd_kernel<AXIS>, grid, C::NT, smem, st, uin, uout, n, nu, gam,
                          eps, kick_g, kick_K)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// out[z][x][y] = in[z][y][x] for the planes of up to two arrays (plane q < np0 of in0 ->
// out0, the rest of in1 -> out1; a plane is n x n floats). 32 x 32 tiles through shared
// memory, TP planes per CTA; VEC: float4 rows (n % 4 == 0, 16-byte aligned arrays). The
// transpose is its own inverse.
struct TPair {
  const float* in0;
  float* out0;
  const float* in1;
  float* out1;
  int np0, np;
};
constexpr int TP = 4;

template <bool VEC>
__global__ void __launch_bounds__(256) transpose_xy_kernel(TPair a, int n) {
  pdl_enter();
  __shared__ float tile[32][33];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int t = threadIdx.x;
  const long long nn = (long long)n * n;
  for (int pi = 0; pi < TP; ++pi) {
    const int q = blockIdx.z * TP + pi;
    if (q >= a.np) break;
    const bool first = q < a.np0;
    const float* in = (first ? a.in0 : a.in1) + (first ? q : q - a.np0) * nn;
    float* out = (first ? a.out0 : a.out1) + (first ? q : q - a.np0) * nn;
    if (pi) __syncthreads();  // the previous plane's tile has been read
    if (VEC) {
      const int r = t >> 3, c = (t & 7) * 4;  // load: tile row r (y), columns c..c+3 (x)
      if (y0 + r < n && x0 + c < n) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(in + (long long)(y0 + r) * n + x0 + c));
        tile[r][c] = v.x;
        tile[r][c + 1] = v.y;
        tile[r][c + 2] = v.z;
        tile[r][c + 3] = v.w;
      }
      __syncthreads();
      if (x0 + r < n && y0 + c < n) {  // store: out row x0 + r, columns y0 + c..c+3
        const float4 v = make_float4(tile[c][r], tile[c + 1][r], tile[c + 2][r], tile[c + 3][r]);
        *reinterpret_cast<float4*>(out + (long long)(x0 + r) * n + y0 + c) = v;
      }
    } else {
      const int tx = t & 31, ty = t >> 5;  // 32 x 8
      for (int j = ty; j < 32; j += 8) {
        const int x = x0 + tx, y = y0 + j;
        if (x < n && y < n) tile[j][tx] = __ldg(in + (long long)y * n + x);
      }
      __syncthreads();
      for (int j = ty; j < 32; j += 8) {
        const int y = y0 + tx, x = x0 + j;  // out row index x, column y
        if (x < n && y < n) out[(long long)x * n + y] = tile[tx][j];
      }
    }
  }
}

// nf planes-of-fields: in0 -> out0 (nf0 fields of n planes), then in1 -> out1 (nf1 fields;
// nf1 = 0 transposes one array)
static sim_status launch_transpose_xy(const float* in0, float* out0, int nf0, const float* in1,
                                      float* out1, int nf1, int n, cudaStream_t st) {
  const TPair a{in0, out0, in1, out1, nf0 * n, (nf0 + nf1) * n};
  const dim3 grid(cdiv(n, 32), cdiv(n, 32), cdiv(a.np, TP));
  const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(in0) | reinterpret_cast<uintptr_t>(out0) |
                                     reinterpret_cast<uintptr_t>(in1) | reinterpret_cast<uintptr_t>(out1)) % 16 == 0);
  if (vec)
    DH_CUDA_TRY((launch_pdl(transpose_xy_kernel<true>, grid, 256, 0, st, a, n)));
  else
    DH_CUDA_TRY((launch_pdl(transpose_xy_kernel<false>, grid, 256, 0, st, a, n)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// Pass 2 of the marching adjoint: the paired packed form when n is even and the arrays are
// 8-byte aligned, else one cell per thread.
template <int AXIS, int FC>
static sim_status launch_adj_final(const float* uin, const float* lout, const float* luh,
                                   float* lin, int n, SArg nu, float gam, int B, cudaStream_t st) {
  const uintptr_t al = reinterpret_cast<uintptr_t>(uin) | reinterpret_cast<uintptr_t>(lout) |
                       reinterpret_cast<uintptr_t>(luh) | reinterpret_cast<uintptr_t>(lin);
  if (AXIS != 0 && n % 2 == 0 && al % 8 == 0) {  // x runs as AXIS 1 on transposed copies
    const dim3 blk = line_block(n / 2, 128);
    const dim3 g(cdiv(n / 2, blk.x), cdiv(n, blk.y), n * B);
    DH_CUDA_TRY((launch_pdl(sweep_adj_final2_kernel<AXIS, FC>, g, blk, 0, st, uin, lout, luh, lin, n, nu, gam)));
  } else {
    const dim3 blk = line_block(n, 256);
    const dim3 g(cdiv(n, blk.x), cdiv(n, blk.y), n * B);
    DH_CUDA_TRY((launch_pdl(sweep_adj_final_kernel<AXIS, FC>, g, blk, 0, st, uin, lout, luh, lin, n, nu, gam)));
  }
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

template <int AXIS>
static sim_status launch_adj_march_t(const float* uin, const float* lout, float* lin, int n,
                                     SArg nu, float gam, float eps, DPart dnu, float* scratch,
                                     int B, int L, cudaStream_t st) {
  if (!scratch) {
    set_error("internal: marching sweep adjoint needs a 5 n^3 scratch buffer per instance");
    return SIM_EINVAL;
  }
  const dim3 blk = line_block(n, 128);
  DH_CUDA_TRY((launch_pdl(sweep_adj_march_kernel<AXIS>, line_grid(n, n, B, blk, cdiv(n, L)), blk, 0, st, uin, lout, scratch, n, nu, gam, eps, dnu, L)));
  DH_LAUNCH_CHECK();
  return launch_adj_final<AXIS, 1 + AXIS>(uin, lout, scratch, lin, n, nu, gam, B, st);
}

// The x adjoint as the y-marching pair on x <-> y transposed copies (momentum component 1
// stays the one along the sweep). scratch: 4 x 5 n^3 floats per instance.
static sim_status launch_adj_x_transposed(const float* uin, const float* lout, float* lin, int n,
                                          SArg nu, float gam, float eps, DPart dnu,
                                          float* scratch, int B, int L, cudaStream_t st) {
  const size_t F5 = (size_t)5 * n * n * n * B;
  float *ut = scratch, *lt = scratch + F5, *it = scratch + 2 * F5, *luh = scratch + 3 * F5;
  DH_TRY(launch_transpose_xy(uin, ut, 5 * B, lout, lt, 5 * B, n, st));
  const dim3 blk = line_block(n, 128);
  DH_CUDA_TRY((launch_pdl(sweep_adj_march_kernel<1, 1>, line_grid(n, n, B, blk, cdiv(n, L)), blk, 0, st, ut, lt, luh, n, nu, gam, eps, dnu, L)));
  DH_LAUNCH_CHECK();
  const uintptr_t al = reinterpret_cast<uintptr_t>(ut) | reinterpret_cast<uintptr_t>(lt) |
                       reinterpret_cast<uintptr_t>(luh);
  if (n % 2 == 0 && al % 8 == 0) {
    // the second pass writes lin in the untransposed layout itself
    const dim3 blk(16, 32);
    const dim3 g(cdiv(n / 2, 16), cdiv(n, 32), n * B);
    DH_CUDA_TRY((launch_pdl(sweep_adj_final2_kernel<1, 1, true>, g, blk, 0, st, ut, lt, luh, lin, n, nu, gam)));
    DH_LAUNCH_CHECK();
    return SIM_OK;
  }
  DH_TRY((launch_adj_final<1, 1>(ut, lt, luh, it, n, nu, gam, B, st)));
  return launch_transpose_xy(it, lin, 5 * B, nullptr, nullptr, 0, n, st);
}

template <int AXIS>
static sim_status launch_sweep_adj_t(const float* uin, const float* lout, float* lin, int n,
                                     SArg nu, float gam, float eps, DPart dnu, float* scratch,
                                     int B, int variant, cudaStream_t st) {
  using C = SweepCfg<AXIS>;
  if (variant != SIM_SWEEP_TILE) {
    const int L = variant == SIM_SWEEP_MARCH_FIT
                      ? fit_segment(sweep_adj_march_kernel<AXIS == 0 ? 1 : AXIS, AXIS == 0 ? 1 : 1 + AXIS>,
                                    n, B, 9, n, line_block(n, 128))
                      : segment_length(variant);
    if (AXIS == 0) {
      if (!scratch) {
        set_error("internal: the transposed x adjoint needs a 20 n^3 scratch buffer per instance");
        return SIM_EINVAL;
      }
      return launch_adj_x_transposed(uin, lout, lin, n, nu, gam, eps, dnu, scratch, B, L, st);
    }
    return launch_adj_march_t<AXIS>(uin, lout, lin, n, nu, gam, eps, dnu, scratch, B, L, st);
  }
  constexpr int NC = (C::SA + 10) * C::WA;
  const size_t smem = 20 * NC * sizeof(float);
  dim3 grid(cdiv(n, C::SA), cdiv(n, C::WA), n * B);
  DH_CUDA_TRY((launch_pdl(sweep_adj_kernel<AXIS>, grid, C::NTA, smem, st, uin, lout, lin, n, nu, gam, eps, dnu)));
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

template <int AXIS>
static sim_status set_sweep_attributes() {
  using C = SweepCfg<AXIS>;
  DH_CUDA_TRY(cudaFuncSetAttribute(sweep_fwd_kernel<AXIS>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(15 * (C::S + 6) * C::W * sizeof(float))));
  DH_CUDA_TRY(cudaFuncSetAttribute(sweep_adj_kernel<AXIS>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(20 * (C::SA + 10) * C::WA * sizeof(float))));
  return SIM_OK;
}

// Shared-memory limits of the sweep kernels, set once per device before its first sweep
// launch (sim_init calls this too, so that no attribute call happens during a capture).
sim_status prepare_sweep_kernels() {
  static std::atomic<unsigned long long> done{0};  // one bit per device index < 64
  int dev = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return SIM_OK;
  DH_TRY(set_sweep_attributes<0>());
  DH_TRY(set_sweep_attributes<1>());
  DH_TRY(set_sweep_attributes<2>());
  done.fetch_or(bit);
  return SIM_OK;
}

sim_status launch_sweep(int axis, const float* uin, float* uout, int n, SArg nu, double gam,
                        double eps, int B, int variant, cudaStream_t st, const float* kick_g,
                        SArg kick_K) {
  DH_TRY(prepare_sweep_kernels());
  if (axis < 0 || axis > 2) {
    set_error("sweep axis must be 0, 1 or 2 (got %d)", axis);
    return SIM_EINVAL;
  }
  const int v = pick_fwd(axis, n, variant);
  const float fg = (float)gam, fe = (float)eps;
  switch (axis) {
    case 0: return launch_sweep_t<0>(uin, uout, n, nu, fg, fe, B, v, st, kick_g, kick_K);
    case 1: return launch_sweep_t<1>(uin, uout, n, nu, fg, fe, B, v, st, kick_g, kick_K);
    default: return launch_sweep_t<2>(uin, uout, n, nu, fg, fe, B, v, st, kick_g, kick_K);
  }
}

bool sweep_takes_kick(int axis, int n, int variant, const float* uin, const float* uout) {
  const int v = pick_fwd(axis, n, variant);
  return v == SIM_SWEEP_TILE || (axis == 0 && v == SIM_SWEEP_PAIR) ||
         takes_pair(axis, n, v, uin, uout);
}

sim_status launch_sweep_adjoint(int axis, const float* uin, const float* lout, float* lin,
                                int n, SArg nu, double gam, double eps, DPart dnu,
                                float* scratch, int B, int variant, cudaStream_t st) {
  DH_TRY(prepare_sweep_kernels());
  if (axis < 0 || axis > 2) {
    set_error("sweep axis must be 0, 1 or 2 (got %d)", axis);
    return SIM_EINVAL;
  }
  const int v = pick_adj(axis, variant);
  const float fg = (float)gam, fe = (float)eps;
  switch (axis) {
    case 0: return launch_sweep_adj_t<0>(uin, lout, lin, n, nu, fg, fe, dnu, scratch, B, v, st);
    case 1: return launch_sweep_adj_t<1>(uin, lout, lin, n, nu, fg, fe, dnu, scratch, B, v, st);
    default: return launch_sweep_adj_t<2>(uin, lout, lin, n, nu, fg, fe, dnu, scratch, B, v, st);
  }
}

}  // namespace dh

extern "C" sim_status sim_sweep(const float* u_in, float* u_out, int32_t n, int32_t axis,
                                double nu, double gamma, double limiter_eps, int32_t variant,
                                void* stream) {
  if (!u_in || !u_out || n < 1 || u_in == u_out || variant < SIM_SWEEP_DEFAULT ||
      variant > SIM_SWEEP_PAIR) {
    dh::set_error("sim_sweep: null/aliased buffers, n < 1 or unknown variant");
    return SIM_EINVAL;
  }
  return dh::launch_sweep(axis, u_in, u_out, n, dh::sarg((float)nu), gamma, limiter_eps, 1,
                          variant, (cudaStream_t)stream, nullptr, dh::sarg(0.0f));
}

extern "C" sim_status sim_sweep_adjoint(const float* u_in, const float* lam_out, float* lam_in,
                                        int32_t n, int32_t axis, double nu, double gamma,
                                        double limiter_eps, double* dnu, int32_t variant,
                                        void* stream) {
  if (!u_in || !lam_out || !lam_in || n < 1 || lam_in == lam_out || lam_in == u_in ||
      variant < SIM_SWEEP_DEFAULT || variant > SIM_SWEEP_PAIR) {
    dh::set_error("sim_sweep_adjoint: null/aliased buffers, n < 1 or unknown variant");
    return SIM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the tile needs no scratch; the marching pairs 20 n^3 floats
  const bool need = variant != SIM_SWEEP_TILE;
  float* scratch = nullptr;
  if (need) DH_CUDA_TRY(cudaMallocAsync((void**)&scratch, 20ull * n * n * n * sizeof(float), st));
  const sim_status r =
      dh::launch_sweep_adjoint(axis, u_in, lam_out, lam_in, n, dh::sarg((float)nu), gamma,
                               limiter_eps, dh::dpart(dnu), scratch, 1, variant, st);
  if (scratch) cudaFreeAsync(scratch, st);
  return r;
}
