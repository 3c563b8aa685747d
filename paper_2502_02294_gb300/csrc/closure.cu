// Learned closure (Sec. 4 of arXiv 2502.02294 lists solver-in-the-loop refinement: a
// network trained against better-resolved runs corrects the coarse solution every step).
//
// Network: four periodic 3x3x3 convolutions 5 -> 16 -> 16 -> 16 -> 5, GELU between them,
// bfloat16 weights and activations, float32 accumulation, applied as a residual update of
// the five gas fields on normalised inputs: u <- u + s * NN((u - mu) / sigma).
//
// Every convolution runs as an implicit GEMM on the tensor cores (tcgen05, M = 128
// positions, K = 16 input channels per tap, accumulators in TMEM). All activations are
// bfloat16 with 16 channels (the 5 gas fields are padded with zeros), so every layer is the
// same 16 -> 16 kernel with zero-padded weights. Activations are stored line-half-major
// ([z][y][2][x][8]): each 8-channel half of a line is a contiguous run of 16-byte positions,
// the row layout of the no-swizzle K-major operand, so an input plane reaches shared memory
// as bulk copies. One padding column on each side of every staged line (pitch P = n + 2)
// makes the operand of an in-plane shift (dy, dx) the same tile moved by (dy P + dx) rows:
// descriptors only, no gather; positions that fall on a padding column give discarded
// results. The three dz taps of one (dy, dx) form one N = 48 operand that updates three
// output planes at once (see the geometry section).
//
// Backward: the gradient with respect to a layer's input is the same convolution with the
// taps mirrored and each tap's matrix transposed (same kernel, other weight packing), its
// epilogue multiplied by GELU' of the previous layer's pre-activation. The weight gradient
// (a reduction over voxels of 27 rank-1 updates of 16 x 16) is a third tensor-core kernel:
// M = (tap, input channel), N = output channel, K = voxels.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "closure.cuh"
#include "pm.cuh"
#include "umma.cuh"

namespace dh {

typedef __nv_bfloat16 bf16;
constexpr int CH = 16;                 // channels of every activation
constexpr int NL = 4;                  // layers
constexpr int WL = 27 * CH * CH;       // padded weights of one layer [tap][ci][co]
constexpr int NPAD = NL * WL + NL * CH;  // padded parameters: weights, then biases [l][co]
constexpr int LAYER_CIN[NL] = {5, 16, 16, 16};
constexpr int LAYER_COUT[NL] = {16, 16, 16, 5};
constexpr int SLK_BEFORE = 8, SLK_AFTER = 136;  // slack positions around the staged region
constexpr int PACK = 27 * 512 / 2;              // bf16 elements of one packed layer

// ------------------------------------------------------------------ geometry
// A CTA owns L output lines (T tiles of 128 positions per plane) of Zc consecutive output
// planes z0 .. z0 + Zc - 1 and marches through the input planes z0 - 1 .. z0 + Zc, which
// stream through a ring of `ring` shared-memory slots ((L + 2) padded lines in two
// 8-channel planes of 16-byte positions, with slack positions around them). Input plane p
// contributes to output planes p - 1, p, p + 1 through the taps dz = +1, 0, -1; for one
// in-plane shift (dy, dx) those three weight blocks sit side by side in one B operand
// (N = 48), so one MMA adds the shifted input to three output-plane accumulators at once:
// 9 MMAs per input plane and tile. The accumulators form a ring of R = 32 / T plane slots
// per tile ([tile][slot][16 columns], output plane o in slot o mod R); an input whose
// output planes wrap around the end of the ring, or lie partly outside the CTA's planes,
// is issued as runs of N = 16 or 32 on the matching rows of the B operand. The epilogue
// drains each output plane once its last input's MMAs are done, zeroes its slot and
// releases it; the MMAs of input i wait for the release of output plane i - R, so they
// may run up to R - 2 input planes ahead of the epilogue. One CTA per SM (all 512 TMEM
// columns); weights, barriers and TMEM are set up once per column of planes.
constexpr int EPI_SETS = 4;                         // epilogue warps per TMEM lane quarter
constexpr int CONV_THREADS = 128 + 128 * EPI_SETS;  // loaders, MMA issuer, epilogue
constexpr int ZC_MAX = 128;           // output planes per CTA
constexpr int NB_MAX = ZC_MAX + 2;    // input planes (and barriers of each kind) per CTA

struct ConvGeom {
  int n, P, L, T, tpl, contig, Zc, R, ring, slot_pos, ncols;
  size_t smem;
};

static int slot_positions(int L, int P) { return SLK_BEFORE + (L + 2) * P + SLK_AFTER; }

static size_t conv_smem(int ring, int L, int P) {
  return (size_t)ring * 2 * slot_positions(L, P) * 16 + 9 * 1536 + 3 * NB_MAX * 8 + 16;
}

static ConvGeom conv_geom(int n, int B) {
  ConvGeom g;
  g.n = n;
  g.P = n + 2;
  const size_t limit = 200 * 1024;
  if (n >= 128) {
    // 128-position tiles inside a line, ceil(n / 128) per line, up to 4 tiles per plane
    g.contig = 0;
    g.tpl = (n + 127) / 128;
    g.L = 4 / g.tpl > 1 ? 4 / g.tpl : 1;
    g.T = g.L * g.tpl;
  } else {
    // tiles run across consecutive padded lines: fewest tiles per plane with T <= 4
    g.contig = 1;
    g.tpl = 0;
    int bestL = 1, bestCost = 1 << 30;
    for (int L = 1; L <= n; ++L) {
      const int T = cdiv((long long)L * g.P, 128);
      if (T > 4 || conv_smem(3, L, g.P) > limit) break;
      const int cost = cdiv(n, L) * T;
      if (cost <= bestCost) {
        bestCost = cost;
        bestL = L;
      }
    }
    g.L = bestL;
    g.T = cdiv((long long)bestL * g.P, 128);
  }
  // a ring of R accumulator planes of 16 columns per tile in 512 columns
  g.R = 32 / g.T;
  g.ncols = 512;
  g.ring = conv_smem(4, g.L, g.P) <= limit ? 4 : 3;
  // output planes per CTA: the split of the planes into chunks that keeps the SMs busiest
  // (whole waves of one CTA per SM), counting the two extra input planes of every chunk
  const int ny = cdiv(n, g.L);
  double best = -1.0;
  g.Zc = n < ZC_MAX ? n : ZC_MAX;
  for (int k = 1; k <= 64; ++k) {
    const int Zc = cdiv(n, k);
    if (Zc > ZC_MAX) continue;
    const long long ctas = (long long)ny * cdiv(n, Zc) * B;
    const double waves = (double)ctas / 152.0;
    const double eff = waves / std::ceil(waves) * (double)Zc / (Zc + 2);
    if (eff > best + 1e-9) {
      best = eff;
      g.Zc = Zc;
    }
    if (Zc <= 2) break;
  }
  g.slot_pos = slot_positions(g.L, g.P);
  // at least 116 KB so that a second CTA never shares the SM (and its 512 TMEM columns)
  g.smem = std::max(conv_smem(g.ring, g.L, g.P), (size_t)116 * 1024);
  return g;
}

// ------------------------------------------------------------------ device helpers
// erfc(|x|) by Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26
// (absolute error below 1.5e-7 for all x >= 0): t = 1 / (1 + p |x|),
// erfc(|x|) ~ (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) e^{-x^2}. Branch-free; e receives
// e^{-x^2}. 1 + erf(x) is then 2 - erfc(|x|) for x >= 0 and erfc(|x|) for x < 0, without
// cancellation on the negative side.
__device__ __forceinline__ float erfc_abs(float ax, float& e) {
  const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
  e = __expf(-ax * ax);
  const float poly =
      fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
           0.254829592f);
  return t * poly * e;
}

// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, on two values with packed float32
// arithmetic (FFMA2 / FMUL2)
__device__ __forceinline__ float2 ff2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 gelu2_f(float2 z) {
  const float2 x = __fmul2_rn(z, ff2(0.70710678118654752f));
  const float2 ax = make_float2(fabsf(x.x), fabsf(x.y));
  const float2 den = __ffma2_rn(ff2(0.3275911f), ax, ff2(1.0f));
  const float2 t = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
  const float2 x2 = __fmul2_rn(ax, ax);
  const float2 e = make_float2(__expf(-x2.x), __expf(-x2.y));
  float2 poly = __ffma2_rn(t, ff2(1.061405429f), ff2(-1.453152027f));
  poly = __ffma2_rn(t, poly, ff2(1.421413741f));
  poly = __ffma2_rn(t, poly, ff2(-0.284496736f));
  poly = __ffma2_rn(t, poly, ff2(0.254829592f));
  const float2 q = __fmul2_rn(__fmul2_rn(t, poly), e);
  // 1 + erf(x) = 2 - q (x >= 0) or q (x < 0)
  const float2 sg = make_float2(x.x >= 0.0f ? -1.0f : 1.0f, x.y >= 0.0f ? -1.0f : 1.0f);
  const float2 base = make_float2(x.x >= 0.0f ? 2.0f : 0.0f, x.y >= 0.0f ? 2.0f : 0.0f);
  const float2 r = __ffma2_rn(sg, q, base);
  return __fmul2_rn(__fmul2_rn(z, ff2(0.5f)), r);
}

// d GELU / dz = Phi(z) + z phi(z), phi(z) = e^{-z^2 / 2} / sqrt(2 pi)
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float x = z * 0.70710678118654752f;
  float e;
  const float q = erfc_abs(fabsf(x), e);
  return 0.5f * (x >= 0.0f ? 2.0f - q : q) + z * 0.3989422804014327f * e;
}

__device__ __forceinline__ int wrapi(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// Activations are bfloat16 [B][z][y][2][x][8]: every line holds its 8-channel halves one
// after the other, each half a contiguous run of 16-byte positions, the row layout of the
// convolution's shared-memory operand (so a line half arrives with one bulk copy).
// Element offset of position x, half h of line `line` = (b n + z) n + y:
__device__ __forceinline__ size_t act_off(long long line, int n, int h, int x) {
  return ((size_t)(line * 2 + h) * n + x) * 8;
}

__device__ __forceinline__ void act_store(bf16* base, long long line, int n, int x,
                                          const float v[16]) {
  uint32_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    w[j] = *reinterpret_cast<const uint32_t*>(&p);
  }
  *reinterpret_cast<uint4*>(base + act_off(line, n, 0, x)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(base + act_off(line, n, 1, x)) = make_uint4(w[4], w[5], w[6], w[7]);
}

struct F5 {
  float v[5];
};

// ------------------------------------------------------------------ convolution
enum { CONV_HIDDEN = 0, CONV_OUT_Y = 1, CONV_OUT_APPLY = 2, CONV_BWD = 3 };

struct ConvArgs {
  const bf16* in;      // activations [B][n][n][2][n][8]
  const bf16* w;       // packed [27][2][16 rows][8]: row = output channel, K = input channel
  const float* bias;   // [16] (forward) or NULL
  int n, P, L, T, tpl, contig, Zc, R, ring, slot_pos, ncols;
  bf16* out;           // HIDDEN / BWD: activations, as in
  float* zout;         // HIDDEN: pre-activation [B][n^3][16] or NULL
  const float* zprev;  // BWD: pre-activation whose GELU' multiplies the result
  float* y;            // OUT_Y: [B][5][n^3]
  float* gas;          // OUT_APPLY: [B][5][n^3], += scale * y
  F5 scale;
  int* err;
  unsigned long long wait_ns;  // limit of each pipeline wait (global-timer nanoseconds)
};

// Limit of the final waits for a CTA's own bulk copies and MMAs in flight: those complete
// without help from other warps, so they are drained even after a pipeline wait gave up.
constexpr unsigned long long kDrainNs = 4000000000ull;

// Bulk copies (async proxy, completion counted in bytes on the plane's mbarrier) of input
// plane gz (periodic) into ring slot `slot_addr`: for each of the L + 2 lines and each
// 8-channel half, the n interior positions (one copy) and the two periodic padding
// positions (16 bytes each). Lane k of the issuing warp copies line half k, k + 32, ...
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ uint32_t plane_tx_bytes(const ConvArgs& a) {
  return (uint32_t)(a.L + 2) * 2u * (uint32_t)(a.n + 2) * 16u;
}

__device__ __forceinline__ void conv_fetch_plane(const ConvArgs& a, const bf16* in, uint32_t slot_addr,
                                                 int gz, int y0, int lane, uint64_t* mbar) {
  const int n = a.n, P = a.P, L = a.L;
  const uint32_t plane_bytes = (uint32_t)a.slot_pos * 16u;
  gz = gz < 0 ? gz + n : (gz >= n ? gz - n : gz);
  for (int k = lane; k < 2 * (L + 2); k += 32) {
    const int ly = k >> 1, h = k & 1;
    const int gy = wrapi(y0 - 1 + ly, n);
    const bf16* src = in + act_off((long long)gz * n + gy, n, h, 0);
    const uint32_t d = slot_addr + (uint32_t)h * plane_bytes + (uint32_t)(SLK_BEFORE + ly * P) * 16u;
    bulk_g2s(d + 16u, src, (uint32_t)n * 16u, mbar);                    // x = 0 .. n - 1
    bulk_g2s(d, src + (size_t)(n - 1) * 8, 16u, mbar);                  // x = -1 -> n - 1
    bulk_g2s(d + (uint32_t)(n + 1) * 16u, src, 16u, mbar);              // x = n -> 0
  }
}

// TMEM zeroing of columns [c0, c1) (multiples of 16) in the 32 lanes of warp w % 4; the
// warps w / 4 = 0 .. nsplit - 1 share the columns
__device__ __forceinline__ void tmem_zero(uint32_t tmem, int c0, int c1, int w, int nsplit) {
  const uint32_t lane_base = (uint32_t)(32 * (w & 3)) << 16;
  uint32_t z[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) z[j] = 0u;
  for (int c = c0 + 16 * (w >> 2); c < c1; c += 16 * nsplit) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(tmem + lane_base + (uint32_t)c),
        "r"(z[0]), "r"(z[1]), "r"(z[2]), "r"(z[3]), "r"(z[4]), "r"(z[5]), "r"(z[6]), "r"(z[7]),
        "r"(z[8]), "r"(z[9]), "r"(z[10]), "r"(z[11]), "r"(z[12]), "r"(z[13]), "r"(z[14]),
        "r"(z[15]));
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 16 zero columns at taddr in this warp's 32 lanes (no wait: tcgen05.wait::st follows)
__device__ __forceinline__ void tmem_zero16_nowait(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

// 16 columns at t0 and 16 at t1 of this thread's TMEM lane, one wait for both loads (one
// asm statement, so no use of the outputs can be placed before the wait)
__device__ __forceinline__ void tmem_ld16x2(uint32_t t0, uint32_t t1, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,"
      "%28,%29,%30,%31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(t0), "r"(t1)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// TMEM column of accumulator slot s of tile t
__device__ __forceinline__ uint32_t acc_col(const ConvArgs& a, int t, int s) {
  return 16u * (uint32_t)(t * a.R + s);
}

// One run of input plane i (ring slot i mod ring) for every tile: block (dy, dx) of the
// weights against the input shifted by (dy, dx), into the len consecutive accumulator slots
// s .. s + len - 1, which hold output planes lo .. lo + len - 1 (relative to z0); output
// plane i - 2 + k takes rows 16 k .. 16 k + 15 of the B operand (dz = 1 - k).
__device__ __forceinline__ void conv_issue_run(const ConvArgs& a, int i, int lo, int len, int s,
                                               uint32_t tmem, uint64_t a_base, uint64_t b_base,
                                               uint32_t slot_units) {
  const int P = a.P, T = a.T;
  const uint64_t a_slot = a_base + (uint64_t)((i % a.ring) * slot_units);
  const uint32_t idesc = len == 3 ? umma_idesc_bf16(128, 48)
                                  : (len == 2 ? umma_idesc_bf16(128, 32) : umma_idesc_bf16(128, 16));
  // rows 16 k0 .. of each 1536-byte block: 8-row groups 128 bytes apart (16-byte units)
  const uint64_t b_run = b_base + (uint64_t)(16 * (lo - (i - 2)));
  // tile-major: the 9 MMAs of one tile chain into the same accumulator (switching the
  // accumulator between consecutive MMAs costs several times a chained MMA)
  for (int t = 0; t < T; ++t) {
    int vb;
    if (a.contig) {
      vb = 128 * t;
    } else {
      const int ly = t / a.tpl;
      vb = ly * P + 1 + 128 * (t - ly * a.tpl);
    }
    const uint32_t d = tmem + acc_col(a, t, s);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int j = (dy + 1) * 3 + (dx + 1);
        const uint64_t db = b_run + (uint64_t)(j * 96);  // 1536-byte blocks
        // descriptors are linear in the start address (16-byte units, low 14 bits)
        const uint64_t da = a_slot + (uint64_t)(SLK_BEFORE + (1 + dy) * P + dx + vb);
        umma_bf16(d, da, db, idesc, 1u);
      }
    }
  }
}

// The MMAs of input plane i: output planes max(0, i - 2) .. min(i, nz - 1), in one run, or
// two where their slots wrap around the end of the ring.
__device__ __forceinline__ void conv_issue_input(const ConvArgs& a, int i, int nz, uint32_t tmem,
                                                 uint64_t a_base, uint64_t b_base,
                                                 uint32_t slot_units) {
  const int lo = max(0, i - 2), hi = min(i, nz - 1);
  const int len = hi - lo + 1, s0 = lo % a.R;
  if (s0 + len <= a.R) {
    conv_issue_run(a, i, lo, len, s0, tmem, a_base, b_base, slot_units);
  } else {
    const int first = a.R - s0;
    conv_issue_run(a, i, lo, first, s0, tmem, a_base, b_base, slot_units);
    conv_issue_run(a, i, lo + first, len - first, 0, tmem, a_base, b_base, slot_units);
  }
}

// Epilogue of row r of tile t of output plane z (all 16 channels).
template <int MODE>
__device__ __forceinline__ void conv_epilogue(const ConvArgs& a, const float acc[16],
                                              const float bias[16], int b, int z, int y0, int t,
                                              int r) {
  const int n = a.n, P = a.P, L = a.L;
  const long long N3 = (long long)n * n * n;
  int ly, x;
  bool valid;
  if (a.contig) {
    const int v = 128 * t + r;
    ly = v / P;
    const int px = v - ly * P;
    x = px - 1;
    valid = px >= 1 && px <= n && ly < L;
  } else {
    ly = t / a.tpl;
    x = 128 * (t - ly * a.tpl) + r;
    valid = x < n;
  }
  const int gy = y0 + ly;
  if (!valid || gy >= n) return;
  const size_t v = ((size_t)z * n + gy) * n + x;
  const long long line = ((long long)b * n + z) * n + gy;
  if (MODE == CONV_HIDDEN) {
    float zc[16], hv[16];
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
      const float2 zz = __fadd2_rn(make_float2(acc[c], acc[c + 1]), make_float2(bias[c], bias[c + 1]));
      const float2 gg = gelu2_f(zz);
      zc[c] = zz.x;
      zc[c + 1] = zz.y;
      hv[c] = gg.x;
      hv[c + 1] = gg.y;
    }
    if (a.zout) {
      float4* zo = reinterpret_cast<float4*>(a.zout + ((size_t)b * N3 + v) * CH);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        zo[q] = make_float4(zc[4 * q], zc[4 * q + 1], zc[4 * q + 2], zc[4 * q + 3]);
    }
    act_store(a.out, line, n, x, hv);
  } else if (MODE == CONV_OUT_Y) {
#pragma unroll
    for (int c = 0; c < 5; ++c) a.y[((size_t)b * 5 + c) * N3 + v] = acc[c] + bias[c];
  } else if (MODE == CONV_OUT_APPLY) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      float* g = a.gas + ((size_t)b * 5 + c) * N3 + v;
      *g += a.scale.v[c] * (acc[c] + bias[c]);
    }
  } else {  // CONV_BWD
    const float4* zp = reinterpret_cast<const float4*>(a.zprev + ((size_t)b * N3 + v) * CH);
    float d[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 zz = __ldg(zp + q);
      d[4 * q] = acc[4 * q] * gelu_grad_f(zz.x);
      d[4 * q + 1] = acc[4 * q + 1] * gelu_grad_f(zz.y);
      d[4 * q + 2] = acc[4 * q + 2] * gelu_grad_f(zz.z);
      d[4 * q + 3] = acc[4 * q + 3] * gelu_grad_f(zz.w);
    }
    act_store(a.out, line, n, x, d);
  }
}

// Warp roles: warp 0 fetches input planes (bulk copies completing on the plane's mbarrier),
// warp 2 lane 0 issues the MMAs of each
// plane once it has landed (and once the slot of its newest output plane is released) and
// commits them to that plane's barrier, warps 4 .. 4 + 4 EPI_SETS - 1 run the epilogue of
// every output plane once its last input's MMAs are done (warp w reads TMEM lanes
// 32 (w % 4) .. + 31 of the tiles t = (w - 4) / 4 mod EPI_SETS), zero its slot and
// release it. Every
// barrier is used once (one per input plane or group), every wait is bounded by a.wait_ns;
// a wait that gives up sets an error flag and its role stops. Before the CTA frees its TMEM
// and exits, the loader waits for every bulk copy it issued and the MMA thread for the
// commit of the last MMAs it issued (kDrainNs each), so nothing asynchronous still writes
// shared or tensor memory. A warp's wait outcome is taken by lane 0 and broadcast, so the
// warp-wide TMEM loads are never reached by part of a warp.

template <int MODE>
__global__ void __launch_bounds__(CONV_THREADS, 1) conv3_kernel(ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int n = a.n;
  const long long N3 = (long long)n * n * n;
  const int b = blockIdx.z, y0 = blockIdx.x * a.L, z0 = blockIdx.y * a.Zc;
  const int nz = min(a.Zc, n - z0);  // output planes of this CTA
  const int nin = nz + 2;            // input planes z0 - 1 .. z0 + nz
  const int R = a.R, ring = a.ring;
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31;
  const uint32_t slot_bytes = 2u * (uint32_t)a.slot_pos * 16u;
  uint8_t* sa = smem;
  uint8_t* sw = smem + ring * slot_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sw + 9 * 1536);  // [NB_MAX]: input landed
  uint64_t* done = full + NB_MAX;                                // [NB_MAX]: its MMAs done
  uint64_t* drained = done + NB_MAX;                             // [NB_MAX]: output released
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drained + NB_MAX);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const bf16* in = a.in + (size_t)b * N3 * CH;
  const uint32_t sa0 = smem_u32(sa);
  const unsigned long long limit = a.wait_ns;

  // setup: slack zeroed, weights staged, barriers, TMEM allocated and zeroed
  const int nslack = SLK_BEFORE + SLK_AFTER;
  for (int i = tid; i < ring * 2 * nslack; i += CONV_THREADS) {
    const int sp = i / nslack, k = i - sp * nslack;
    const int pos = k < SLK_BEFORE ? k : a.slot_pos - SLK_AFTER + (k - SLK_BEFORE);
    *reinterpret_cast<uint4*>(sa + (size_t)sp * a.slot_pos * 16 + (size_t)pos * 16) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  for (int i = tid; i < 9 * 1536 / 16; i += CONV_THREADS)
    reinterpret_cast<uint4*>(sw)[i] = __ldg(reinterpret_cast<const uint4*>(a.w) + i);
  if (tid == 0) {
    for (int i = 0; i < nin; ++i) {
      mbar_init(full + i, 1);
      mbar_init(done + i, 1);
    }
    for (int o = 0; o < nz; ++o) mbar_init(drained + o, 4 * EPI_SETS);
    *sflag = 0;
  }
  if (w == 0) tmem_alloc_warp(tslot, (uint32_t)a.ncols);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  tmem_zero(tmem, 0, a.ncols, w, CONV_THREADS / 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (w < 2) {
    // ---- loader warp: input i into slot i mod ring once input i - ring's MMAs are done;
    //      the plane's barrier completes when all its bytes have landed
    if (w == 0) {
      const uint32_t tx = plane_tx_bytes(a);
      int issued = 0;
      for (int i = 0; i < nin; ++i) {
        uint32_t ok = 1;
        if (i >= ring && lane == 0) ok = mbar_wait_ns(done + (i - ring), 0, limit);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) *sflag = 1;
          break;
        }
        if (lane == 0) {
          uint64_t state;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                       : "=l"(state)
                       : "r"(smem_u32(full + i)), "r"(tx)
                       : "memory");
          (void)state;
        }
        __syncwarp();
        conv_fetch_plane(a, in, sa0 + (uint32_t)(i % ring) * slot_bytes, z0 - 1 + i, y0, lane, full + i);
        issued = i + 1;
      }
      // no copy may still be writing shared memory when the CTA exits
      if (lane == 0)
        for (int i = 0; i < issued; ++i)
          if (!mbar_wait_ns(full + i, 0, kDrainNs)) *sflag = 1;
      __syncwarp();
    }
  } else if (w == 2) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint64_t a_base = umma_desc(sa0, (uint32_t)a.slot_pos * 16u, 128u);
      const uint64_t b_base = umma_desc(smem_u32(sw), 768u, 128u);
      const uint32_t slot_units = slot_bytes >> 4;
      int committed = 0;
      for (int i = 0; i < nin; ++i) {
        // the slot of output plane i last held output plane i - R
        if (i < nz && i >= R && !mbar_wait_ns(drained + (i - R), 0, limit)) {
          *sflag = 1;
          break;
        }
        if (!mbar_wait_ns(full + i, 0, limit)) {
          *sflag = 1;
          break;
        }
        tc_fence_after();
        conv_issue_input(a, i, nz, tmem, a_base, b_base, slot_units);
        umma_commit(done + i);
        committed = i + 1;
      }
      // the commit of the last issued input completes once every MMA issued before it has
      if (committed > 0 && !mbar_wait_ns(done + committed - 1, 0, kDrainNs)) *sflag = 1;
    }
    __syncwarp();
  } else if (w >= 4) {
    // ---- epilogue: output plane z0 + o is final once input o + 2 is in; its accumulator
    //      is slot o mod R. In columns of 12 planes or more, planes are drained two at a
    //      time (one wait for their MMAs, one for both TMEM loads, one for the zeroing of
    //      both slots); short columns take them one by one, so the first starts earlier.
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 of the tiles t = (w - 4) / 4 mod EPI_SETS
    const uint32_t lane_base = (uint32_t)(32 * (w & 3)) << 16;
    const int es = (w - 4) >> 2;
    float bias[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) bias[c] = a.bias ? __ldg(a.bias + c) : 0.0f;
    const int pstep = nz >= 12 ? 2 : 1;
    for (int o = 0; o < nz; o += pstep) {
      const int np = min(pstep, nz - o);  // output planes o .. o + np - 1
      uint32_t ok = 0;
      if (lane == 0) ok = mbar_wait_ns(done + o + np + 1, 0, limit);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *sflag = 1;
        break;
      }
      tc_fence_after();
      const int s0 = o % R, s1 = (o + 1) % R;
      for (int t = es; t < a.T; t += EPI_SETS) {
        if (np == 2) {
          float acc[32];
          tmem_ld16x2(tmem + lane_base + acc_col(a, t, s0), tmem + lane_base + acc_col(a, t, s1), acc);
          conv_epilogue<MODE>(a, acc, bias, b, z0 + o, y0, t, 32 * (w & 3) + lane);
          conv_epilogue<MODE>(a, acc + 16, bias, b, z0 + o + 1, y0, t, 32 * (w & 3) + lane);
        } else {
          float acc[16];
          tmem_ld16(tmem + lane_base + acc_col(a, t, s0), acc);
          conv_epilogue<MODE>(a, acc, bias, b, z0 + o, y0, t, 32 * (w & 3) + lane);
        }
      }
      // clear the slots of planes q + R < nz (reused by output plane q + R) and release them
      // to the MMA thread
      const bool rel0 = o + R < nz, rel1 = np == 2 && o + 1 + R < nz;
      if (rel0) {
        for (int t = es; t < a.T; t += EPI_SETS) {
          tmem_zero16_nowait(tmem + lane_base + acc_col(a, t, s0));
          if (rel1) tmem_zero16_nowait(tmem + lane_base + acc_col(a, t, s1));
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          uint64_t state;
          asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
                       : "=l"(state)
                       : "r"(smem_u32(drained + o))
                       : "memory");
          if (rel1)
            asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
                         : "=l"(state)
                         : "r"(smem_u32(drained + o + 1))
                         : "memory");
          (void)state;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *sflag) atomicExch(a.err, 1);
  if (w == 0) tmem_dealloc_warp(tmem, (uint32_t)a.ncols);
}

static sim_status prepare_conv_kernels() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return SIM_OK;
  const int maxsm = 200 * 1024;
  DH_CUDA_TRY(cudaFuncSetAttribute(conv3_kernel<CONV_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  DH_CUDA_TRY(cudaFuncSetAttribute(conv3_kernel<CONV_OUT_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  DH_CUDA_TRY(cudaFuncSetAttribute(conv3_kernel<CONV_OUT_APPLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  DH_CUDA_TRY(cudaFuncSetAttribute(conv3_kernel<CONV_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  done.fetch_or(bit);
  return SIM_OK;
}

static sim_status launch_conv(int mode, ConvArgs a, int B, cudaStream_t st) {
  const ConvGeom g = conv_geom(a.n, B);
  if (g.smem > 200 * 1024) {
    set_error("closure: grid n = %d needs %zu bytes of shared memory per CTA", a.n, g.smem);
    return SIM_EINVAL;
  }
  // the epilogue drains planes in pairs, waiting for input o + 3 before it releases plane
  // o, and the MMAs of input i wait for the release of plane i - R: R >= 4 keeps that acyclic
  if (g.R < 4 || 16 * g.T * g.R > g.ncols) {
    set_error("closure: grid n = %d needs %d tiles per plane (at most 8)", a.n, g.T);
    return SIM_EINVAL;
  }
  a.P = g.P;
  a.L = g.L;
  a.T = g.T;
  a.tpl = g.tpl;
  a.contig = g.contig;
  a.Zc = g.Zc;
  a.R = g.R;
  a.ring = g.ring;
  a.slot_pos = g.slot_pos;
  a.ncols = g.ncols;
  const dim3 grid(cdiv(a.n, g.L), cdiv(a.n, g.Zc), B);
  switch (mode) {
    case CONV_HIDDEN: conv3_kernel<CONV_HIDDEN><<<grid, CONV_THREADS, g.smem, st>>>(a); break;
    case CONV_OUT_Y: conv3_kernel<CONV_OUT_Y><<<grid, CONV_THREADS, g.smem, st>>>(a); break;
    case CONV_OUT_APPLY: conv3_kernel<CONV_OUT_APPLY><<<grid, CONV_THREADS, g.smem, st>>>(a); break;
    default: conv3_kernel<CONV_BWD><<<grid, CONV_THREADS, g.smem, st>>>(a); break;
  }
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// ------------------------------------------------------------------ weight gradient
// dW[tap][ci][co] = sum_v in[v + off(tap)][ci] dz[v][co] and db[co] = sum_v dz[v][co], as
// tensor-core GEMMs with M = (tap, ci), N = co and K = voxels: 16 consecutive x positions of
// one line per MMA step (a K block). For every K block the producer warps write into a
// shared-memory stage the block's 27 shifted input tiles (16 channels x 16 voxels each: tap t
// at rows 16 (t mod 8) .. + 15 of the M = 128 operand of tap group t / 8) and its dz tile
// (N = 16 rows), every one transposed on the way into the no-swizzle K-major layout (a row is
// 8 voxels of one channel: stmatrix .trans from the fragment of 4-byte channel pairs). One
// thread issues the stage's four M128 N16 K16 MMAs (tap groups 0..3) into four 16-column TMEM
// accumulators that collect all of the CTA's K blocks; the epilogue adds them to dW / db with
// vector atomics. Row 48 of group 3 (tap slot 3, channel 0) is a constant row of ones, so its
// accumulator row is db; the other unused rows of group 3 stay zero. Voxels past the end of a
// line (n not a multiple of 16) have dz = 0.
constexpr int DW_PRODUCERS = 8;                     // producer warps; one more issues the MMAs
constexpr int DW_THREADS = 32 * (DW_PRODUCERS + 1);
constexpr int DW_STAGES = 3;
constexpr int DW_A_BYTES = 4 * 4096;                // four tap groups x 128 rows x 32 bytes
constexpr int DW_STAGE_BYTES = DW_A_BYTES + 512;    // + the dz tile: 16 rows x 32 bytes
constexpr int DW_SMEM = DW_STAGES * DW_STAGE_BYTES + (2 * DW_STAGES + 1) * 8 + 16;
constexpr int DW_CTAS_PER_SM = 4;

struct DwArgs {
  const bf16* in;  // layer input [B][n][n][2][n][8]
  const bf16* dz;  // gradient at the layer's output, same layout
  int n, nxb;      // grid size, K blocks per line
  long long kblocks, per_cta;
  float* dW;  // [27][16][16], accumulated
  float* db;  // [16], accumulated
  int* err;
  unsigned long long wait_ns;
};

// four 8x8 bfloat16 matrices from the mma fragment (lane 4 r + q: row r, columns 2q, 2q + 1
// in register j of matrix j) stored transposed: lane l gives the address of row l mod 8 of
// matrix l / 8
__device__ __forceinline__ void stmatrix_trans4(uint32_t addr, const uint32_t v[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

__global__ void __launch_bounds__(DW_THREADS) conv_dw_kernel(DwArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + DW_STAGES * DW_STAGE_BYTES);
  uint64_t* empty = full + DW_STAGES;
  uint64_t* done = empty + DW_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int n = a.n, nxb = a.nxb;
  const long long kb0 = (long long)blockIdx.x * a.per_cta;
  const long long kb1 = kb0 + a.per_cta < a.kblocks ? kb0 + a.per_cta : a.kblocks;
  const int nkb = (int)(kb1 - kb0);  // >= 1 by the launch
  const uint32_t s0 = smem_u32(smem);
  const unsigned long long limit = a.wait_ns;

  for (int i = tid; i < DW_STAGES * DW_STAGE_BYTES / 16; i += DW_THREADS)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (tid < 2 * DW_STAGES) {
    // group 3, M group 6 (tap slot 3, channels 0-7), K chunk tid & 1, row 0: bfloat16 ones
    const int st = tid >> 1, kc = tid & 1;
    *reinterpret_cast<uint4*>(smem + st * DW_STAGE_BYTES + 3 * 4096 + 6 * 256 + kc * 128) =
        make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  }
  if (tid == 0) {
    for (int st = 0; st < DW_STAGES; ++st) {
      mbar_init(full + st, DW_PRODUCERS);
      mbar_init(empty + st, 1);
    }
    mbar_init(done, 1);
    *sflag = 0;
  }
  if (w == 0) tmem_alloc_warp(tslot, 64u);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (w < DW_PRODUCERS) {
    const long long N3 = (long long)n * n * n;
    const int r = lane >> 2, q = lane & 3;  // fragment row (voxel of an 8-voxel chunk), pair
    const int mj = lane >> 3, row = lane & 7;
    // matrix j = 2 h + kc: channel half h, K chunk kc (voxels 8 kc .. 8 kc + 7)
    const uint32_t row_off = (uint32_t)((mj >> 1) * 256 + (mj & 1) * 128 + row * 16);
    for (int k = 0; k < nkb; ++k) {
      const int st = k % DW_STAGES;
      uint32_t ok = 1;
      if (k >= DW_STAGES && lane == 0) ok = mbar_wait_ns(empty + st, ((k / DW_STAGES) - 1) & 1, limit);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *sflag = 1;
        break;
      }
      long long kb = kb0 + k;
      const int xb = (int)(kb % nxb);
      kb /= nxb;
      const int y = (int)(kb % n);
      kb /= n;
      const int z = (int)(kb % n);
      const int b = (int)(kb / n);
      const int x0 = 16 * xb;
      const uint32_t stage = s0 + (uint32_t)(st * DW_STAGE_BYTES);
      const bf16* inb = a.in + (size_t)b * N3 * CH;
      const bf16* dzb = a.dz + (size_t)b * N3 * CH;
      for (int j = w; j < 28; j += DW_PRODUCERS) {
        uint32_t v[4];
        uint32_t dst;
        if (j < 27) {
          const int ddz = j / 9 - 1, ddy = (j / 3) % 3 - 1, ddx = j % 3 - 1;
          const long long line = (long long)wrapi(z + ddz, n) * n + wrapi(y + ddy, n);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int x = wrapi(x0 + 8 * (m & 1) + r + ddx, n);
            v[m] = __ldg(reinterpret_cast<const unsigned int*>(inb + act_off(line, n, m >> 1, x) + 2 * q));
          }
          dst = stage + (uint32_t)((j >> 3) * 4096 + (j & 7) * 512);
        } else {
          const long long line = (long long)z * n + y;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int x = x0 + 8 * (m & 1) + r;
            v[m] = x < n ? __ldg(reinterpret_cast<const unsigned int*>(dzb + act_off(line, n, m >> 1, x) + 2 * q))
                         : 0u;
          }
          dst = stage + (uint32_t)DW_A_BYTES;
        }
        stmatrix_trans4(dst + row_off, v);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        uint64_t state;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
                     : "=l"(state)
                     : "r"(smem_u32(full + st))
                     : "memory");
        (void)state;
      }
    }
  } else if (lane == 0) {
    // ---- MMA issuer: the stage's four tap groups, then release the stage
    const uint32_t idesc = umma_idesc_bf16(128, 16);
    for (int k = 0; k < nkb; ++k) {
      const int st = k % DW_STAGES;
      if (!mbar_wait_ns(full + st, (k / DW_STAGES) & 1, limit)) {
        *sflag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t stage = s0 + (uint32_t)(st * DW_STAGE_BYTES);
      const uint64_t bdesc = umma_desc(stage + DW_A_BYTES, 128u, 256u);
#pragma unroll
      for (int g = 0; g < 4; ++g)
        umma_bf16(tmem + 16u * g, umma_desc(stage + 4096u * g, 128u, 256u), bdesc, idesc, k > 0 ? 1u : 0u);
      umma_commit(empty + st);
    }
    // completes once every MMA issued above has; waited for before TMEM is read or freed
    umma_commit(done);
    if (!mbar_wait_ns(done, 0, kDrainNs)) *sflag = 1;
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (w < 4 && *sflag == 0) {
    // lane 32 w + l of TMEM = row m: tap slot m / 16 of each group, channel m mod 16
    const int m = 32 * w + lane, slot = m >> 4, ci = m & 15;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(32 * w) << 16) + 16u * g, acc);
      const int t = 8 * g + slot;
      float* dst = t < 27 ? a.dW + (size_t)(t * CH + ci) * CH : (t == 27 && ci == 0 ? a.db : nullptr);
      if (dst)
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4)
          atomicAdd(reinterpret_cast<float4*>(dst) + c4,
                    make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *sflag) atomicExch(a.err, 1);
  if (w == 0) tmem_dealloc_warp(tmem, 64u);
}

static sim_status launch_dw(const bf16* in, const bf16* dz, int n, int B, float* dW, float* db,
                            int* err, unsigned long long wait_ns, cudaStream_t st) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  if (!(done.load() & (1ull << (dev & 63)))) {
    DH_CUDA_TRY(cudaFuncSetAttribute(conv_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM));
    done.fetch_or(1ull << (dev & 63));
  }
  int sms = 0;
  DH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DwArgs a;
  a.in = in;
  a.dz = dz;
  a.n = n;
  a.nxb = cdiv(n, 16);
  a.kblocks = (long long)B * n * n * a.nxb;
  const long long ctas = std::max(1, sms * DW_CTAS_PER_SM);
  a.per_cta = (a.kblocks + ctas - 1) / ctas;
  a.dW = dW;
  a.db = db;
  a.err = err;
  a.wait_ns = wait_ns;
  const int grid = (int)((a.kblocks + a.per_cta - 1) / a.per_cta);
  conv_dw_kernel<<<grid, DW_THREADS, DW_SMEM, st>>>(a);
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// ------------------------------------------------------------------ elementwise kernels
// x[b][v][f] = bf16((gas[b][f][v] - mu_f) / sigma_f), f < 5; channels 5..15 are zero
__global__ void closure_pack_kernel(const float* __restrict__ gas, F5 mu, F5 inv_sigma,
                                    bf16* __restrict__ x, long long N3, int n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= N3) return;
  float v[16];
#pragma unroll
  for (int f = 0; f < 16; ++f) v[f] = 0.0f;
#pragma unroll
  for (int f = 0; f < 5; ++f) v[f] = (gas[((size_t)b * 5 + f) * N3 + i] - mu.v[f]) * inv_sigma.v[f];
  act_store(x, (long long)b * (N3 / n) + i / n, n, (int)(i % n), v);
}

// loss += norm sum (y - (tgt - in) / s)^2 over 5 fields; dz4 = bf16(2 norm (y - t))
__global__ void closure_loss_kernel(const float* __restrict__ y, const float* __restrict__ gin,
                                    const float* __restrict__ gtg, F5 inv_s, float norm,
                                    bf16* __restrict__ dz4, double* __restrict__ loss,
                                    long long N3, int n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  float acc = 0.0f;
  if (i < N3) {
    float g[16];
#pragma unroll
    for (int f = 0; f < 16; ++f) g[f] = 0.0f;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const size_t o = ((size_t)b * 5 + f) * N3 + i;
      const float t = (gtg[o] - gin[o]) * inv_s.v[f];
      const float d = y[o] - t;
      acc += d * d;
      g[f] = 2.0f * norm * d;
    }
    act_store(dz4, (long long)b * (N3 / n) + i / n, n, (int)(i % n), g);
  }
  block_sum_atomic(acc * norm, loss);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int count, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Packed weights, per layer 9 blocks (dy, dx) of [kc][48 rows][8]: row 16 d + c holds output
// channel c of tap dz = 1 - d (the input plane's contribution to output planes p - 1, p,
// p + 1 in that order), K = input channel 8 kc + e. Forward: W[tap][k][c]; backward (the
// transposed, mirrored convolution): W[26 - tap][c][k].
__global__ void repack_kernel(const float* __restrict__ W, bf16* __restrict__ wf,
                              bf16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over NL * PACK
  if (i >= NL * PACK) return;
  const int l = i / PACK;
  const int r = i - l * PACK;
  const int j = r / 768, e = r % 768;
  const int kc = e / 384, row = (e / 8) % 48, el = e % 8;
  const int dz = 1 - row / 16, c = row % 16, k = 8 * kc + el;
  const int tap = (dz + 1) * 9 + j;
  const float* Wl = W + (size_t)l * WL;
  wf[i] = __float2bfloat16_rn(Wl[(tap * CH + k) * CH + c]);
  wb[i] = __float2bfloat16_rn(Wl[((26 - tap) * CH + c) * CH + k]);
}

}  // namespace dh

// ===================================================================== closure object
using namespace dh;

struct sim_closure_s {
  cudaStream_t st = 0;
  float mu[5] = {0, 0, 0, 0, 0}, inv_sigma[5] = {1, 1, 1, 1, 1}, scale[5] = {1, 1, 1, 1, 1};
  float* prm = nullptr;   // NPAD: padded weights then biases (float32 master copy)
  float* grad = nullptr;  // NPAD
  float *m = nullptr, *v = nullptr;
  int adam_t = 0;
  bf16 *wf = nullptr, *wb = nullptr;  // NL x PACK each
  int* err = nullptr;
  unsigned long long wait_ns = 1000000000ull;  // 1 s per tensor-core pipeline wait
  double* loss = nullptr;
  // workspace
  int wn = 0, wB = 0;
  bool wtrain = false;
  uint64_t gen = 0;  // bumped whenever the workspace moves (captured graphs must be redone)
  bf16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *d1 = nullptr, *d2 = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *y = nullptr;
  std::vector<void*> ws;
};

namespace dh {

static void ws_free(sim_closure_s* c) {
  for (void* p : c->ws) cudaFree(p);
  c->ws.clear();
  c->x = c->a1 = c->a2 = c->a3 = c->d1 = c->d2 = nullptr;
  c->z1 = c->z2 = c->z3 = c->y = nullptr;
  c->wn = c->wB = 0;
}

template <class T>
static sim_status ws_alloc(sim_closure_s* c, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error("closure: cudaMalloc(%zu bytes) failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return SIM_ENOMEM;
  }
  c->ws.push_back(*p);
  return SIM_OK;
}

sim_status closure_prepare(sim_closure_s* c, int n, int B, bool training) {
  DH_TRY(prepare_conv_kernels());
  if (c->wn == n && c->wB >= B && (c->wtrain || !training)) return SIM_OK;
  // the old buffers may be in use on any stream (a simulation's, this closure's)
  DH_CUDA_TRY(cudaDeviceSynchronize());
  ws_free(c);
  c->gen += 1;
  const size_t V = (size_t)n * n * n * B;
  DH_TRY(ws_alloc(c, &c->x, V * CH));
  DH_TRY(ws_alloc(c, &c->a1, V * CH));
  DH_TRY(ws_alloc(c, &c->a2, V * CH));
  if (training) {
    DH_TRY(ws_alloc(c, &c->a3, V * CH));
    DH_TRY(ws_alloc(c, &c->d1, V * CH));
    DH_TRY(ws_alloc(c, &c->d2, V * CH));
    DH_TRY(ws_alloc(c, &c->z1, V * CH));
    DH_TRY(ws_alloc(c, &c->z2, V * CH));
    DH_TRY(ws_alloc(c, &c->z3, V * CH));
    DH_TRY(ws_alloc(c, &c->y, V * 5));
  }
  c->wn = n;
  c->wB = B;
  c->wtrain = training;
  return SIM_OK;
}

static ConvArgs conv_args(sim_closure_s* c, int l, bool backward, const bf16* in, int n) {
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.in = in;
  a.w = (backward ? c->wb : c->wf) + (size_t)l * PACK;
  a.bias = backward ? nullptr : c->prm + NL * WL + l * CH;
  a.n = n;
  a.err = c->err;
  a.wait_ns = c->wait_ns;
  for (int f = 0; f < 5; ++f) a.scale.v[f] = c->scale[f];
  return a;
}

static F5 f5(const float* v) {
  F5 r;
  for (int f = 0; f < 5; ++f) r.v[f] = v[f];
  return r;
}

// Forward through the four layers. mode CONV_OUT_APPLY adds s y to `gas`; CONV_OUT_Y
// writes y (and, for training, every pre-activation).
static sim_status closure_forward(sim_closure_s* c, const float* gas, int n, int B, int mode,
                                  float* gas_apply, bool keep, cudaStream_t st) {
  const long long N3 = (long long)n * n * n;
  closure_pack_kernel<<<dim3(cdiv(N3, 256), B), 256, 0, st>>>(gas, f5(c->mu), f5(c->inv_sigma),
                                                              c->x, N3, n);
  DH_LAUNCH_CHECK();
  bf16* acts[4] = {c->x, c->a1, c->a2, keep ? c->a3 : c->a1};
  float* zs[3] = {keep ? c->z1 : nullptr, keep ? c->z2 : nullptr, keep ? c->z3 : nullptr};
  for (int l = 0; l < 3; ++l) {
    ConvArgs a = conv_args(c, l, false, acts[l], n);
    a.out = acts[l + 1];
    a.zout = zs[l];
    DH_TRY(launch_conv(CONV_HIDDEN, a, B, st));
  }
  ConvArgs a = conv_args(c, 3, false, acts[3], n);
  if (mode == CONV_OUT_APPLY) {
    a.gas = gas_apply;
    return launch_conv(CONV_OUT_APPLY, a, B, st);
  }
  a.y = c->y;
  return launch_conv(CONV_OUT_Y, a, B, st);
}

uint64_t closure_generation(const sim_closure_s* c) { return c->gen; }

sim_status closure_apply(sim_closure_s* c, float* gas, int n, int B, cudaStream_t st) {
  if (c->wn != n || c->wB < B) {
    set_error("closure: workspace not prepared for n = %d, B = %d", n, B);
    return SIM_EINVAL;
  }
  return closure_forward(c, gas, n, B, CONV_OUT_APPLY, gas, false, st);
}

// loss and the gradient of every parameter (c->grad, overwritten) for one batch
static sim_status closure_backprop(sim_closure_s* c, const float* gas, const float* target,
                                   int n, int B, cudaStream_t st) {
  const long long N3 = (long long)n * n * n;
  DH_TRY(closure_forward(c, gas, n, B, CONV_OUT_Y, nullptr, true, st));
  DH_CUDA_TRY(cudaMemsetAsync(c->loss, 0, sizeof(double), st));
  DH_CUDA_TRY(cudaMemsetAsync(c->grad, 0, NPAD * sizeof(float), st));
  F5 inv_s;
  for (int f = 0; f < 5; ++f) inv_s.v[f] = 1.0f / c->scale[f];
  const float norm = (float)(1.0 / (5.0 * (double)N3 * B));
  closure_loss_kernel<<<dim3(cdiv(N3, 256), B), 256, 0, st>>>(c->y, gas, target, inv_s, norm,
                                                              c->d1, c->loss, N3, n);
  DH_LAUNCH_CHECK();
  // layer l: input activation acts[l], pre-activation of layer l - 1: zs[l - 1]
  const bf16* acts[4] = {c->x, c->a1, c->a2, c->a3};
  const float* zs[3] = {c->z1, c->z2, c->z3};
  bf16* dcur = c->d1;
  bf16* dnext = c->d2;
  for (int l = 3; l >= 0; --l) {
    DH_TRY(launch_dw(acts[l], dcur, n, B, c->grad + (size_t)l * WL, c->grad + NL * WL + l * CH,
                     c->err, c->wait_ns, st));
    if (l == 0) break;
    ConvArgs a = conv_args(c, l, true, dcur, n);
    a.out = dnext;
    a.zprev = zs[l - 1];
    DH_TRY(launch_conv(CONV_BWD, a, B, st));
    bf16* t = dcur;
    dcur = dnext;
    dnext = t;
  }
  return SIM_OK;
}

static sim_status repack(sim_closure_s* c, cudaStream_t st) {
  repack_kernel<<<cdiv(NL * PACK, 256), 256, 0, st>>>(c->prm, c->wf, c->wb);
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

// flat weight vector (real layer shapes) <-> padded parameters
static void flat_to_pad(const float* flat, std::vector<float>& pad) {
  pad.assign(NPAD, 0.0f);
  size_t o = 0;
  for (int l = 0; l < NL; ++l) {
    const int ci = LAYER_CIN[l], co = LAYER_COUT[l];
    for (int t = 0; t < 27; ++t)
      for (int i = 0; i < ci; ++i)
        for (int j = 0; j < co; ++j) pad[(size_t)l * WL + (t * CH + i) * CH + j] = flat[o++];
    for (int j = 0; j < co; ++j) pad[NL * WL + l * CH + j] = flat[o++];
  }
}

static void pad_to_flat(const std::vector<float>& pad, float* flat) {
  size_t o = 0;
  for (int l = 0; l < NL; ++l) {
    const int ci = LAYER_CIN[l], co = LAYER_COUT[l];
    for (int t = 0; t < 27; ++t)
      for (int i = 0; i < ci; ++i)
        for (int j = 0; j < co; ++j) flat[o++] = pad[(size_t)l * WL + (t * CH + i) * CH + j];
    for (int j = 0; j < co; ++j) flat[o++] = pad[NL * WL + l * CH + j];
  }
}

// Reads and clears the timeout flag (the closure's stream must be idle).
static int check_err(sim_closure_s* c) {
  int e = 0;
  cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) cudaMemset(c->err, 0, sizeof(int));
  return e;
}

// ------------------------------------------------------------------ coarse / fine pairing
// fine half-complex mode <- coarse mode (band-limited interpolation, Nyquist split)
__global__ void refine_map_kernel(const cufftComplex* __restrict__ Wc, int nc,
                                  cufftComplex* __restrict__ Xf, int nf, float s) {
  const int nhf = nf / 2 + 1, nhc = nc / 2 + 1;
  const long long NCf = (long long)nf * nf * nhf;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NCf) return;
  const int kx = (int)(i % nhf);
  const long long r = i / nhf;
  int ky = (int)(r % nf), kz = (int)(r / nf);
  if (ky > nf / 2) ky -= nf;
  if (kz > nf / 2) kz -= nf;
  const bool even = (nc % 2 == 0);
  const int lim = nc / 2;  // |k| <= nc/2 (even: the Nyquist index; odd: (nc-1)/2)
  float f = s;
  bool in = kx <= lim && abs(ky) <= lim && abs(kz) <= lim;
  if (in && even) {
    if (kx == lim) f *= 0.5f;
    if (abs(ky) == lim) f *= 0.5f;
    if (abs(kz) == lim) f *= 0.5f;
  }
  cufftComplex out = make_cuFloatComplex(0.0f, 0.0f);
  if (in) {
    const int cy = ky < 0 ? ky + nc : ky, cz = kz < 0 ? kz + nc : kz;
    const cufftComplex w = Wc[((long long)cz * nc + cy) * nhc + kx];
    out = make_cuFloatComplex(f * w.x, f * w.y);
  }
  Xf[i] = out;
}

// coarse cell j = tent-weighted mean of the 27 fine cells around fine cell 2j
__global__ void restrict_gas_kernel(const float* __restrict__ gf, int nf,
                                    float* __restrict__ gc) {
  const int nc = nf / 2;
  const long long NCc = (long long)nc * nc * nc, NFf = (long long)nf * nf * nf;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int bf = blockIdx.y;  // instance x field
  if (i >= NCc) return;
  const int x = (int)(i % nc), y = (int)((i / nc) % nc), z = (int)(i / ((long long)nc * nc));
  const float w[3] = {0.25f, 0.5f, 0.25f};
  const float* src = gf + (size_t)bf * NFf;
  float acc = 0.0f;
  for (int c = 0; c < 3; ++c) {
    const int fz = wrapi(2 * z + c - 1, nf);
    for (int bb = 0; bb < 3; ++bb) {
      const int fy = wrapi(2 * y + bb - 1, nf);
      const float* row = src + ((size_t)fz * nf + fy) * nf;
      const float wzy = w[c] * w[bb];
      for (int a = 0; a < 3; ++a) acc += wzy * w[a] * row[wrapi(2 * x + a - 1, nf)];
    }
  }
  gc[(size_t)bf * NCc + i] = acc;
}

__global__ void restrict_part_kernel(const float* __restrict__ pf, int nf, float* __restrict__ pc) {
  const int nc = nf / 2;
  const long long NCc = (long long)nc * nc * nc, NFf = (long long)nf * nf * nf;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int bc = blockIdx.y;  // instance x component
  if (i >= NCc) return;
  const int x = (int)(i % nc), y = (int)((i / nc) % nc), z = (int)(i / ((long long)nc * nc));
  pc[(size_t)bc * NCc + i] = pf[(size_t)bc * NFf + ((size_t)(2 * z) * nf + 2 * y) * nf + 2 * x];
}

}  // namespace dh

// ===================================================================== C ABI
extern "C" {

sim_status sim_closure_create(const float* weights, void* stream, sim_closure_t** out) {
  if (!out) {
    set_error("sim_closure_create: out is NULL");
    return SIM_EINVAL;
  }
  *out = nullptr;
  sim_closure_s* c = new sim_closure_s();
  c->st = (cudaStream_t)stream;
  auto bad = [&](sim_status s) {
    sim_closure_destroy(c);
    return s;
  };
  if (cudaMalloc((void**)&c->prm, NPAD * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&c->grad, NPAD * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&c->m, NPAD * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&c->v, NPAD * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&c->wf, (size_t)NL * PACK * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc((void**)&c->wb, (size_t)NL * PACK * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc((void**)&c->err, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->loss, sizeof(double)) != cudaSuccess) {
    set_error("sim_closure_create: cudaMalloc failed");
    return bad(SIM_ENOMEM);
  }
  std::vector<float> pad(NPAD, 0.0f);
  if (weights) flat_to_pad(weights, pad);
  if (cudaMemcpy(c->prm, pad.data(), NPAD * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->m, 0, NPAD * sizeof(float)) != cudaSuccess ||
      cudaMemset(c->v, 0, NPAD * sizeof(float)) != cudaSuccess ||
      cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess) {
    set_error("sim_closure_create: upload failed");
    return bad(SIM_ECUDA);
  }
  sim_status r = prepare_conv_kernels();
  if (r == SIM_OK) r = repack(c, c->st);
  if (r != SIM_OK) return bad(r);
  *out = c;
  return SIM_OK;
}

void sim_closure_destroy(sim_closure_t* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  ws_free(c);
  for (void* p : {(void*)c->prm, (void*)c->grad, (void*)c->m, (void*)c->v, (void*)c->wf,
                  (void*)c->wb, (void*)c->err, (void*)c->loss})
    if (p) cudaFree(p);
  delete c;
}

sim_status sim_closure_set_norm(sim_closure_t* c, const float* mu, const float* sigma,
                                const float* scale) {
  if (!c || !mu || !sigma || !scale) return SIM_EINVAL;
  for (int f = 0; f < 5; ++f)
    if (!(sigma[f] > 0) || !(scale[f] > 0)) {
      set_error("sim_closure_set_norm: sigma and scale must be > 0");
      return SIM_EINVAL;
    }
  for (int f = 0; f < 5; ++f) {
    c->mu[f] = mu[f];
    c->inv_sigma[f] = 1.0f / sigma[f];
    c->scale[f] = scale[f];
  }
  return SIM_OK;
}

sim_status sim_closure_get_weights(sim_closure_t* c, float* host_out) {
  if (!c || !host_out) return SIM_EINVAL;
  std::vector<float> pad(NPAD);
  DH_CUDA_TRY(cudaStreamSynchronize(c->st));
  DH_CUDA_TRY(cudaMemcpy(pad.data(), c->prm, NPAD * sizeof(float), cudaMemcpyDeviceToHost));
  pad_to_flat(pad, host_out);
  return SIM_OK;
}

sim_status sim_closure_set_weights(sim_closure_t* c, const float* host_in) {
  if (!c || !host_in) return SIM_EINVAL;
  std::vector<float> pad;
  flat_to_pad(host_in, pad);
  DH_CUDA_TRY(cudaStreamSynchronize(c->st));
  DH_CUDA_TRY(cudaMemcpy(c->prm, pad.data(), NPAD * sizeof(float), cudaMemcpyHostToDevice));
  DH_CUDA_TRY(cudaMemset(c->m, 0, NPAD * sizeof(float)));
  DH_CUDA_TRY(cudaMemset(c->v, 0, NPAD * sizeof(float)));
  c->adam_t = 0;
  return repack(c, c->st);
}

sim_status sim_closure_forward(sim_closure_t* c, const float* gas, int32_t n, int32_t B,
                               float* y) {
  if (!c || !gas || !y || n < 2 || B < 1) {
    set_error("sim_closure_forward: invalid arguments");
    return SIM_EINVAL;
  }
  DH_TRY(closure_prepare(c, n, B, true));
  DH_TRY(closure_forward(c, gas, n, B, CONV_OUT_Y, nullptr, false, c->st));
  DH_CUDA_TRY(cudaMemcpyAsync(y, c->y, (size_t)B * 5 * n * n * n * sizeof(float),
                              cudaMemcpyDeviceToDevice, c->st));
  return SIM_OK;
}

sim_status sim_closure_apply(sim_closure_t* c, float* gas, int32_t n, int32_t B) {
  if (!c || !gas || n < 2 || B < 1) {
    set_error("sim_closure_apply: invalid arguments");
    return SIM_EINVAL;
  }
  DH_TRY(closure_prepare(c, n, B, false));
  return closure_apply(c, gas, n, B, c->st);
}

sim_status sim_closure_gradient(sim_closure_t* c, const float* gas, const float* target,
                                int32_t n, int32_t B, double* loss_host, float* grad_host) {
  if (!c || !gas || !target || n < 2 || B < 1) {
    set_error("sim_closure_gradient: invalid arguments");
    return SIM_EINVAL;
  }
  DH_TRY(closure_prepare(c, n, B, true));
  DH_TRY(closure_backprop(c, gas, target, n, B, c->st));
  DH_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (check_err(c)) {
    set_error("closure: a tensor-core wait timed out");
    return SIM_ETIMEOUT;
  }
  if (loss_host) DH_CUDA_TRY(cudaMemcpy(loss_host, c->loss, sizeof(double), cudaMemcpyDeviceToHost));
  if (grad_host) {
    std::vector<float> pad(NPAD);
    DH_CUDA_TRY(cudaMemcpy(pad.data(), c->grad, NPAD * sizeof(float), cudaMemcpyDeviceToHost));
    pad_to_flat(pad, grad_host);
  }
  return SIM_OK;
}

sim_status sim_closure_train_step(sim_closure_t* c, const float* gas, const float* target,
                                  int32_t n, int32_t B, double lr, double* loss_out) {
  if (!c || !gas || !target || n < 2 || B < 1 || !(lr > 0)) {
    set_error("sim_closure_train_step: invalid arguments");
    return SIM_EINVAL;
  }
  DH_TRY(closure_prepare(c, n, B, true));
  DH_TRY(closure_backprop(c, gas, target, n, B, c->st));
  c->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  adam_kernel<<<cdiv(NPAD, 256), 256, 0, c->st>>>(
      c->prm, c->grad, c->m, c->v, NPAD, (float)lr, (float)b1, (float)b2, 1e-8f,
      (float)(1.0 - std::pow(b1, c->adam_t)), (float)(1.0 - std::pow(b2, c->adam_t)));
  DH_LAUNCH_CHECK();
  DH_TRY(repack(c, c->st));
  if (loss_out)
    DH_CUDA_TRY(cudaMemcpyAsync(loss_out, c->loss, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  return SIM_OK;
}

sim_status sim_closure_set_wait_limit(sim_closure_t* c, int64_t ns) {
  if (!c || ns < 0) {
    set_error("sim_closure_set_wait_limit: invalid arguments");
    return SIM_EINVAL;
  }
  c->wait_ns = (unsigned long long)ns;
  return SIM_OK;
}

sim_status sim_closure_status(sim_closure_t* c) {
  if (!c) return SIM_EINVAL;
  DH_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (check_err(c)) {
    set_error("closure: a tensor-core wait timed out");
    return SIM_ETIMEOUT;
  }
  return SIM_OK;
}

sim_status sim_refine_noise(const float* w_c, int32_t n_c, float* w_f, int32_t n_f,
                            double scale, void* stream) {
  if (!w_c || !w_f || n_c < 2 || n_f <= n_c) {
    set_error("sim_refine_noise: invalid arguments (need n_f > n_c >= 2)");
    return SIM_EINVAL;
  }
  FFTPlans* pc = shared_plans(n_c);
  FFTPlans* pf = shared_plans(n_f);
  if (!pc || !pf) return SIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const long long NCc = (long long)n_c * n_c * (n_c / 2 + 1);
  const long long NCf = (long long)n_f * n_f * (n_f / 2 + 1);
  cufftComplex* buf = nullptr;
  DH_CUDA_TRY(cudaMallocAsync((void**)&buf, (NCc + NCf) * sizeof(cufftComplex), st));
  sim_status r = pc->set_stream(st);
  if (r == SIM_OK) r = pf->set_stream(st);
  if (r == SIM_OK && cufftExecR2C(pc->r2c1, const_cast<float*>(w_c), buf) != CUFFT_SUCCESS) {
    set_error("sim_refine_noise: cufftExecR2C failed");
    r = SIM_ECUDA;
  }
  if (r == SIM_OK) {
    const float s = (float)(scale / ((double)n_c * n_c * n_c));
    refine_map_kernel<<<cdiv(NCf, 256), 256, 0, st>>>(buf, n_c, buf + NCc, n_f, s);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("sim_refine_noise: launch failed");
      r = SIM_ECUDA;
    }
  }
  if (r == SIM_OK && cufftExecC2R(pf->c2r1, buf + NCc, w_f) != CUFFT_SUCCESS) {
    set_error("sim_refine_noise: cufftExecC2R failed");
    r = SIM_ECUDA;
  }
  cudaFreeAsync(buf, st);
  return r;
}

sim_status sim_restrict_gas(const float* gas_f, int32_t n_f, float* gas_c, int32_t B,
                            void* stream) {
  if (!gas_f || !gas_c || n_f < 2 || n_f % 2 || B < 1) {
    set_error("sim_restrict_gas: invalid arguments (n_f even)");
    return SIM_EINVAL;
  }
  const long long NCc = (long long)(n_f / 2) * (n_f / 2) * (n_f / 2);
  restrict_gas_kernel<<<dim3(cdiv(NCc, 256), 5 * B), 256, 0, (cudaStream_t)stream>>>(gas_f, n_f, gas_c);
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

sim_status sim_restrict_particles(const float* part_f, int32_t n_f, float* part_c, int32_t B,
                                  void* stream) {
  if (!part_f || !part_c || n_f < 2 || n_f % 2 || B < 1) {
    set_error("sim_restrict_particles: invalid arguments (n_f even)");
    return SIM_EINVAL;
  }
  const long long NCc = (long long)(n_f / 2) * (n_f / 2) * (n_f / 2);
  restrict_part_kernel<<<dim3(cdiv(NCc, 256), 6 * B), 256, 0, (cudaStream_t)stream>>>(part_f, n_f, part_c);
  DH_LAUNCH_CHECK();
  return SIM_OK;
}

}  // extern "C"
