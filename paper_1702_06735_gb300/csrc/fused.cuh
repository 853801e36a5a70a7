// One persistent kernel per likelihood evaluation.
//
// A block (one per SM) has eight warps, one event per thread.  Its event
// tiles move global -> shared with one bulk copy per tile (tiles are
// contiguous in memory) into a ring of stages; each stage completes on its
// own mbarrier, and the last warp to release a stage (a shared-memory count)
// issues the copy of the tile that refills it, so no block barrier is taken
// per tile.  The block
//   1. derives the per-evaluation constants from the parameter vector
//      (lineshape constants, coefficients of each component in A_f and
//      Abar_f, time-integral weights of the normalisation) while its first
//      tiles are in flight,
//   2. processes its data tiles (tiles b, b + grid, ...): lineshapes and
//      components (or the stored component cache), Eq. (mix) in its
//      factorised form in double precision, ln B and its adjoint,
//   3. processes its MC tiles: components, the normalisation matrix
//      I_jk = <a_j^* a_k> and the adjoint of the time-integrated rate.
// Each block then writes its partial sums; the last block to finish sums the
// partials of all blocks in a fixed order (double-float arithmetic) and forms
// N, the NLL and the gradient.  Every wait is bounded and reports
// TDMIX_ERR_TIMEOUT.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "device_tables.hpp"
#include "eval.cuh"
#include "gram_tc.cuh"
#include "kinematics.cuh"

namespace tdmix {

// How a block accumulates the MC normalisation matrix over its tiles:
//   kGramRegs    per-thread register accumulators of every entry (up to 8
//                shared components), block sums at the end;
//   kGramTensor  tcgen05 MMAs per tile on exact fixed-point pieces,
//                folded into double-float accumulators (fp32 path, any
//                supported U; see gram_tc.cuh);
//   kGramShared  per tile the components are written to shared memory and
//                thread q sums the q-th entry over the tile's events (fp64
//                path beyond 8 components).
enum GramMode { kGramRegs = 0, kGramTensor = 1, kGramShared = 2 };

constexpr int kTile = kTileEvents;
constexpr int kWarps = kTile / 32;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s
constexpr int kStageBudget = 192 * 1024;     // shared memory for the tile ring
// The cached pass (component cache in, no MC tiles) runs kCachedBlocksPerSM
// blocks per SM: its ring gets under half the budget, so that both blocks'
// shared memory fits.
constexpr int kStageBudgetCached = 88 * 1024;

// Per-evaluation constants in double precision (shared memory of a block).
struct CtaConst {
  double m0[kMaxRes], g0[kMaxRes], m2[kMaxRes], kappa[kMaxRes];
  double dlk_dm[kMaxRes], dlk_dg[kMaxRes];  // d ln kappa / d m0, d ln kappa / d Gamma0
  double cA[kMaxComp][2], cB[kMaxComp][2];
  double x, y, gamma, tau, alpha, beta, gc, dc, ia, ic;
  int chain_comp[kMaxChains], chain_amp[kMaxChains], floating[kMaxParams];
  int nonfinite, domain;
  double p[kMaxParams];  // the parameter vector
};

static_assert(sizeof(CtaConst) % 8 == 0, "copied in 8-byte words");

// d ln kappa / d m0 and d ln kappa / d Gamma0 of resonance r (gradient only):
// ln kappa = 2 ln m0 + ln Gamma0 - (2L+1)/2 ln q0^2 - 2 ln F_L(z0), z0 = q0^2 r^2,
// d q0^2 / d m0 = 2 m0 (u^2 - (ma^2 - mb^2)^2) / (4 u^2), u = m0^2, and
// q0^2 = lambda / (4u), so 1 / (2 q0^2) = 2u / lambda.
__device__ inline void kappa_log_derivatives(const ModelConst& km, int r, double m0, double g0, CtaConst& cc) {
  const int shape = km.res_shape[r];
  if (shape == SHAPE_CONST) {
    cc.dlk_dm[r] = rcp<double>(m0);
    cc.dlk_dg[r] = rcp<double>(g0);
  } else if (shape == SHAPE_MDW) {
    const int L = km.res_L[r];
    const double r2 = km.r_res * km.r_res;
    const double a = km.res_ma[r] * km.res_ma[r], b = km.res_mb[r] * km.res_mb[r];
    const double u = m0 * m0;
    const double iu = rcp<double>(u), im0 = m0 * iu;  // 1/u, 1/m0
    const double lam = u * u + a * a + b * b - 2.0 * (u * a + u * b + a * b);
    const double q02 = 0.25 * lam * iu;
    const double z0 = q02 * r2;
    const double dq2 = 0.5 * m0 * (u * u - (a - b) * (a - b)) * iu * iu;
    const double dlnF = L == 0 ? 0.0 : (L == 1 ? -0.5 * rcp<double>(1.0 + z0)
                                               : -0.5 * (3.0 + 2.0 * z0) * rcp<double>(9.0 + 3.0 * z0 + z0 * z0));
    cc.dlk_dm[r] = 2.0 * im0 - (2 * L + 1) * dq2 * (2.0 * rcp<double>(lam)) * u - 2.0 * dlnF * r2 * dq2;
    cc.dlk_dg[r] = rcp<double>(g0);
  } else {
    cc.dlk_dm[r] = cc.dlk_dg[r] = 0.0;
  }
}

// Block-wide copy of `bytes` (a multiple of 8) in 8-byte words.
__device__ __forceinline__ void copy_words(void* dst, const void* src, int bytes) {
  uint2* d = static_cast<uint2*>(dst);
  const uint2* q = static_cast<const uint2*>(src);
  for (int i = threadIdx.x; i < bytes / 8; i += blockDim.x) d[i] = q[i];
}

// Per-evaluation constants, derived by the kTile threads of a block in
// parallel.  derive_load brings the parameter vector (device memory, or the
// kernel parameters when `dparams` is null) and the model tables into shared
// memory; after a barrier, derive_compute has thread c place chain c's
// coefficient, thread 64 + r derive resonance r's constants, thread 96 the
// mixing weights and, with RES_GRAD, thread 128 + r the log-derivatives of
// kappa_r.
// m0 Gamma(s) = kappa X(s) with, for a mass-dependent width,
// kappa = m0^2 Gamma0 / (q0^(2L+1) F_L(q0 r)^2); with
// lambda = Kallen(m0^2, ma^2, mb^2) = 4 m0^2 q0^2 this is
// kappa = 2 m0^3 Gamma0 G_L(z0) (4 m0^2)^L lambda^-(2L+1)/2, G_L = 1/F_L^2
// (1, 1 + z, 9 + 3z + z^2), z0 = q0^2 r^2; a constant width has
// kappa = m0 Gamma0.  Only reciprocal square roots and Newton reciprocals
// sit on the dependent chains (double precision is slow to issue on this
// GPU).  derive_compute ends without a barrier: the caller synchronises.
template <class T, int U>
__device__ inline void derive_load(const double* __restrict__ dparams, const double* hp, const ModelConst& km,
                                   CtaConst& cc, BlockConst<T>& bc) {
  const int tid = threadIdx.x;
  const int nc = km.n_chains, np = km.n_params;
  for (int k = tid; k < np; k += kTile) {
    cc.p[k] = dparams ? dparams[k] : hp[k];
    cc.floating[k] = km.floating[k];
  }
  for (int j = tid; j < U; j += kTile) {  // components without a chain in A (or Abar) keep 0
    cc.cA[j][0] = cc.cA[j][1] = cc.cB[j][0] = cc.cB[j][1] = 0.0;
    bc.cab[j] = Quad<T>{T(0), T(0), T(0), T(0)};
    bc.cab_lo[j] = Quad<T>{T(0), T(0), T(0), T(0)};
  }
  for (int c = tid; c < nc; c += kTile) {
    cc.chain_comp[c] = km.chain_comp[c];
    cc.chain_amp[c] = km.chain_amp[c];
  }
  if (tid == 0) {
    cc.nonfinite = cc.domain = 0;
    cc.gamma = km.gamma;
    cc.tau = km.tau;
  }
}

template <class T, int U, int NR, bool RES_GRAD = false>
__device__ inline void derive_compute(const ModelConst& km, CtaConst& cc, BlockConst<T>& bc) {
  const int tid = threadIdx.x;
  const int nc = km.n_chains, np = km.n_params;
  const double* sp = cc.p;
  for (int k = tid; k < np; k += kTile)
    if (!isfinite(sp[k])) atomicOr(&cc.nonfinite, 1);
  if (tid < nc) {  // each (amplitude, component) has at most one chain
    const int j = cc.chain_comp[tid];
    const bool in_a = cc.chain_amp[tid] == 0;
    double(*dst)[2] = in_a ? cc.cA : cc.cB;
    T* hi = in_a ? &bc.cab[j].x : &bc.cab[j].z;  // (re, im) adjacent
    T* lo = in_a ? &bc.cab_lo[j].x : &bc.cab_lo[j].z;
    for (int q = 0; q < 2; ++q) {
      const double v = sp[2 * tid + q];
      dst[j][q] = v;
      hi[q] = T(v);
      lo[q] = T(v - double(T(v)));
    }
  }
  if (tid >= 64 && tid < 64 + NR) {
    const int r = tid - 64;
    const int shape = km.res_shape[r], L = km.res_L[r];
    const double ma = km.res_ma[r], mb = km.res_mb[r], rr = km.r_res;
    const double m0 = sp[2 * nc + 2 * r], g0 = sp[2 * nc + 2 * r + 1];
    const double u = m0 * m0;
    double kap = 0;
    if (shape != SHAPE_NONE && !(m0 > 0 && g0 > 0)) atomicOr(&cc.domain, 1);
    if (shape == SHAPE_CONST) {
      kap = m0 * g0;
    } else if (shape == SHAPE_MDW) {
      const double a2 = ma * ma, b2 = mb * mb;
      const double lam = u * u + a2 * a2 + b2 * b2 - 2.0 * (u * a2 + u * b2 + a2 * b2);
      if (!(lam > 0)) atomicOr(&cc.domain, 1);
      const double rs = rsqrt(lam);                                  // lambda^-1/2
      const double z0 = lam * (0.25 * rr * rr) * rcp<double>(u);     // (q0 r)^2, off the rsqrt chain
      double g = 1.0, w = rs;                                        // G_L(z0) and lambda^-(2L+1)/2 (4u)^L
      if (L == 1) {
        g = 1.0 + z0;
        w = rs * rs * rs * (4.0 * u);
      } else if (L == 2) {
        g = 9.0 + z0 * (3.0 + z0);
        const double r2s = rs * rs;
        w = rs * r2s * r2s * (16.0 * u * u);
      }
      kap = 2.0 * m0 * u * g0 * g * w;
    }
    cc.m0[r] = m0;
    cc.g0[r] = g0;
    cc.m2[r] = u;
    cc.kappa[r] = kap;
    Quad<T> R;
    if constexpr (sizeof(T) == 4) {
      const float hi = float(u);
      R.x = hi;
      R.y = float(u - double(hi));
    } else {
      R.x = T(u);
      R.y = T(0);
    }
    R.z = T(kap);
    R.w = T(kap - double(T(kap)));
    bc.res[r] = R;
  }
  if (RES_GRAD && tid >= 128 && tid < 128 + NR) {
    const int r = tid - 128;
    kappa_log_derivatives(km, r, sp[2 * nc + 2 * r], sp[2 * nc + 2 * r + 1], cc);
  }
  // mixing weights on one thread (two independent reciprocals)
  if (tid == 96) {
    const double x = sp[2 * nc + 2 * NR], y = sp[2 * nc + 2 * NR + 1];
    if (!(fabs(y) < 1.0)) atomicOr(&cc.domain, 1);
    const double ia = rcp<double>(1.0 - y * y), ic = rcp<double>(1.0 + x * x);
    cc.x = x;
    cc.y = y;
    cc.ia = ia;
    cc.ic = ic;
    cc.alpha = ia + ic;
    cc.beta = (x * x + y * y) * ia * ic;
    cc.gc = y * ia;
    cc.dc = x * ic;
    bc.x = x;
    bc.y = y;
    bc.gamma = cc.gamma;
    bc.hx = 0.5 * x * cc.gamma;
    bc.hy = 0.5 * y * cc.gamma;
    bc.xf = float(x);
    bc.yf = float(y);
    bc.gammaf = float(cc.gamma);
    const DF hx2 = df_from_double(bc.hx), hy2 = df_from_double(bc.hy);
    bc.hxh = hx2.hi;
    bc.hxl = hx2.lo;
    bc.hyh = hy2.hi;
    bc.hyl = hy2.lo;
    // decay-time limits of the mixing-series tiers: |x|, |y| Gamma t / 2 <= 0.02, 0.1
    const double mg = fmax(fabs(x), fabs(y)) * cc.gamma;
    const double ig = mg > 0 ? rcp<double>(mg) : INFINITY;
    bc.tlim[0] = static_cast<unsigned long long>(__double_as_longlong(0.04 * ig));
    bc.tlim[1] = static_cast<unsigned long long>(__double_as_longlong(0.2 * ig));
    bc.mix = Quad<T>{T(cc.alpha), T(cc.beta), T(cc.gc), T(cc.dc)};
  }
}

// The per-evaluation constants of one parameter vector, derived once for a
// whole batch of evaluations (k_derive) instead of in every block of every
// evaluation: a block of a batched evaluation copies its record into shared
// memory, which takes one global-load latency, where deriving the constants
// takes chains of dependent double-precision operations (about 2 us on this
// GPU, where each such operation has a latency of ~70 cycles).
template <class T>
struct alignas(16) DerivedConst {
  CtaConst cc;
  BlockConst<T> bc;
};

// Block k derives the constants of parameter vector params[k * np ..) into
// out[k] (the same steps as a k_eval block, with the log-derivatives of
// kappa).
template <class P, class S>
__global__ void __launch_bounds__(kTileEvents) k_derive(const double* __restrict__ params, int np,
                                                       const __grid_constant__ ModelConst km,
                                                       DerivedConst<typename P::T>* out) {
  using T = typename P::T;
  __shared__ CtaConst cc;
  __shared__ BlockConst<T> bc;
  derive_load<T, S::U>(params + size_t(blockIdx.x) * np, nullptr, km, cc, bc);
  __syncthreads();
  derive_compute<T, S::U, S::NR, true>(km, cc, bc);
  __syncthreads();
  copy_words(&out[blockIdx.x].cc, &cc, sizeof(CtaConst));
  copy_words(&out[blockIdx.x].bc, &bc, sizeof(BlockConst<T>));
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

__device__ __forceinline__ float2 to_df(double v) {
  const float hi = float(v);
  return make_float2(hi, float(v - double(hi)));
}

// Shuffle-tree sum over the 32 lanes of a warp (result in lane 0).
template <class V>
__device__ __forceinline__ V warp_sum(V a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
  return a;
}

// Warp sums of NQ per-lane floats by a butterfly reduce-scatter over groups
// of 32 values: in the step with offset `off` (16, 8, 4, 2, 1) a lane keeps
// half of its remaining partial sums (the upper half if bit `off` of its lane
// index is set), adds the copy lane ^ off holds of them and sends it the
// other half.  After the five steps lane l holds the warp sum of value l of
// the group, which it writes to row[l].  31 shuffles per group of 32 values,
// against 5 per value for one shuffle tree each; the order of the additions
// is fixed, so the sums are bitwise repeatable.
template <int NQ>
__device__ __forceinline__ void warp_sums_butterfly(const float (&vt)[NQ], float* row, int lane) {
  constexpr int NG = (NQ + 31) / 32;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = g * 32 + i < NQ ? vt[g * 32 + i] : 0.f;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < off; ++i) {
        const float send = up ? v[i] : v[i + off];
        const float keep = up ? v[i + off] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    if (g * 32 + lane < NQ) row[g * 32 + lane] = v[0];
  }
}

// Block sum of per-thread values vt[0 .. NQ) into double-float pairs
// out[q] = (hi, lo), in a fixed order: inside each warp a butterfly (fp32) or
// shuffle trees (fp64), then the warp sums in warp order.  fp32: everything on the FP32 pipe (TwoSum
// across warps); converting each warp sum to double would cost a whole warp
// instruction on the slow fp64 pipe per value, even for one active lane.
// fp64: double shuffle trees and sums, rounded to a pair at the end.
// `red` is shared scratch of kWarps x NQ values; ends with a barrier.
template <class T, int NQ>
__device__ inline void block_sum_df(const T (&vt)[NQ], T* red, float2* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if constexpr (sizeof(T) == 4) {
    warp_sums_butterfly<NQ>(vt, red + warp * NQ, lane);
  } else {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const T s = warp_sum(vt[q]);
      if (lane == 0) red[warp * NQ + q] = s;
    }
  }
  __syncthreads();
  for (int q = tid; q < NQ; q += blockDim.x) {
    if constexpr (sizeof(T) == 4) {
      float s = 0.f, e = 0.f;
      for (int w = 0; w < kTile / 32; ++w) {
        float t, err;
        two_sum(s, red[w * NQ + q], t, err);
        s = t;
        e += err;
      }
      float t, err;  // renormalise (hi, lo)
      two_sum(s, e, t, err);
      out[q] = make_float2(t, err);
    } else {
      double s = 0;
      for (int w = 0; w < kTile / 32; ++w) s += red[w * NQ + q];
      out[q] = to_df(s);
    }
  }
  __syncthreads();
}

template <class P, class S, int GRAM = kGramRegs>
struct Layout {
  using T = typename P::T;
  static constexpr int U = S::U, NR = S::NR;
  static constexpr int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  static constexpr int WMC = 1 + NRE + NIM + 2 * NR;  // sum w, Re I (j<=k), Im I (j<k), s1, s2
  static constexpr int WD = 5 + 4 * U + 2 * NR;       // sum ln B, n_bad, d/dx, d/dy, gA, gB, s1, s2, n recomputed
  static constexpr int W = WMC + WD;
  static constexpr int NPL_FULL = Planes<P, S>::W0;    // invariants, width factors, spin factors
  static constexpr int NPL_CACHE = 2 * U;             // component cache (re, im)
  // bytes of one stage: planes, then one 8-byte-per-event plane (t; the MC
  // weights need at most as much)
  static constexpr int stage_bytes(bool full) {
    return (full ? NPL_FULL : NPL_CACHE) * kTile * int(sizeof(T)) + kTile * 8;
  }
  // shared memory after the ring used by the tensor-core normalisation matrix
  static constexpr int extra_bytes(bool full) {
    return (full && GRAM == kGramTensor) ? TcGram<U>::extra_bytes : 0;
  }
  // ring depth: as many stages as fit the budget, 2 to 6 (the lookahead must
  // cover the memory latency under full load, a few microseconds)
  // blocks per SM of the cached pass: kCachedBlocksPerSM on the fp32 path up to
  // 8 components (within 128 registers), else one
  static constexpr int cached_blocks = (P::kF32 && U <= 8) ? kCachedBlocksPerSM : 1;
  static constexpr int stages(bool full) {
    const int budget = full || cached_blocks == 1 ? kStageBudget : kStageBudgetCached;
    const int n = (budget - extra_bytes(full)) / stage_bytes(full);
    return n < 2 ? 2 : (n > 6 ? 6 : n);
  }
  // bytes of one tile in global memory (SampleDev::tile_bytes / cache_tile_bytes)
  static constexpr int64_t data_tile_bytes() { return int64_t(NPL_FULL) * kTile * sizeof(T) + kTile * 8; }
  static constexpr int64_t mc_tile_bytes(bool weighted) {
    return int64_t(NPL_FULL) * kTile * sizeof(T) + (weighted ? kTile * sizeof(T) : 0);
  }
  static constexpr int64_t cache_tile_bytes() { return int64_t(NPL_CACHE) * kTile * sizeof(T) + kTile * 8; }
  // the last block copies the partial rows of `g` blocks into shared memory
  // (whole 16-byte units) when they fit; otherwise it reads them from global
  // memory (L2)
  static constexpr int partial_bytes(int g) { return W * g * 8 + 16; }
  static constexpr bool partials_in_smem(int g) { return partial_bytes(g) <= kStageBudget; }
  // dynamic shared memory: the stage ring and the normalisation-matrix
  // buffers, reused by the last block for the partial rows of up to `ld`
  // blocks
  static constexpr int smem_bytes(bool full, int ld) {
    const int st = stages(full) * stage_bytes(full) + extra_bytes(full);
    const int pa = partials_in_smem(ld) ? partial_bytes(ld) : 0;
    return st > pa ? st : pa;
  }
};

// The cached fp32 data pass with the gradient (and the serving kernel's)
// forms A and Abar with the coefficients rounded to fp32, c_hi = fl32(c),
// and leaves out the residues dc = c - c_hi (below 2^-24 |c|).  Since it
// also sums the holomorphic sensitivities gA_j = sum_e (d ln B_e / dA)
// a_j(e) and gB_j (the coefficient gradient), the residues enter the sum
// of ln B to first order in the finish instead of once per event:
//   sum ln B(c) = sum ln B(c_hi) + 2 Re sum_j (gA_j dcA_j + gB_j dcB_j) + O(|dc|^2),
// the neglected term about 2^-48 relative.  ds holds [sum ln B, n_bad,
// d/dx, d/dy, Re gA, Im gA, Re gB, Im gB, ...].  Component j's share (0 for
// j >= U); the finish sums the shares over the lanes of a warp, since
// double-precision conversions and arithmetic in one dependent chain would
// take microseconds on this GPU.
template <int U>
__device__ inline double coef_residue_term(const CtaConst& cc, const double* ds, int j) {
  if (j >= U) return 0.0;
  const double ar = cc.cA[j][0] - double(float(cc.cA[j][0])), ai = cc.cA[j][1] - double(float(cc.cA[j][1]));
  const double br = cc.cB[j][0] - double(float(cc.cB[j][0])), bi = cc.cB[j][1] - double(float(cc.cB[j][1]));
  return 2.0 * ((ds[4 + j] * ar - ds[4 + U + j] * ai) + (ds[4 + 2 * U + j] * br - ds[4 + 3 * U + j] * bi));
}

// Likelihood from the MC column totals `mcs` and the data column totals
// `ds` of one sample: writes [nll, N, n_bad or status, sum ln B,
// n recomputed, grad...]
// to `res` (and the NLL and gradient to `onll`, `og` when not null).
//   N = <alpha |A|^2 + beta |Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*)> / Gamma
// is Eq. (mix) integrated over t in [0, inf) and averaged over the MC sample
// (alpha = 1/(1-y^2) + 1/(1+x^2), beta = 1/(1-y^2) - 1/(1+x^2),
// gc = y/(1-y^2), dc = x/(1+x^2)); with S_jk = sum_e w_e a_j^* a_k and
// I = S / sum w: <|A|^2> = cA^H I cA, <|Abar|^2> = cB^H I cB,
// <A Abar*> = cB^H I cA.   NLL = -sum ln B + Gamma sum t + N_d ln N.
// The vectors S cA, S cB come first (one product per thread, shuffle sums
// over k), then the four quadratic forms from them (c^H (S c)): fp64 issue
// throughput, not latency, bounds this block-wide work on this GPU, and this
// order needs about a third of the fp64 instructions of forming each
// quadratic form from S directly.  Warp 0 then takes the logarithm while
// warps 1-7 form the gradient.  Used by the
// last block of an evaluation and, in serving, by the last chunk of each
// request (256 threads).
// COEF_RESIDUE: the data sums were formed with the coefficients rounded to
// fp32 (see coef_residue_term).
template <class S, bool COEF_RESIDUE = false>
__device__ inline void finish_likelihood(double* res, double* onll, double* og, int nc, int np, const CtaConst& cc,
                                         const double* mcs, const double* ds, double Nd, double sum_t, double inv_sw,
                                         bool want_grad, bool have_res_grad, int timed_out, const double2* logtab,
                                         unsigned long long* trace) {
  constexpr int U = S::U, NR = S::NR;
  constexpr int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  static_assert(U <= 16, "lane groups of at most 16 over the components");
  __shared__ double vv[2][U][2];  // S cA, S cB (unnormalised)
  __shared__ double sh[4];        // AA, BB, Xr, Xi (unnormalised)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int status = timed_out ? -7 : (cc.nonfinite ? -5 : (cc.domain ? -6 : 0));
  if (status != 0) {
    for (int k = tid; k < kResHeader + np; k += blockDim.x) {
      const double v = k == 2 ? double(status) : nan("");
      res[k] = v;
      if (k == 0 && onll) *onll = v;
      if (k >= kResHeader && og) og[k - kResHeader] = v;
    }
    return;
  }
  // S_jk (Hermitian) from the packed totals: Re over j <= k, Im over j < k
  auto s_at = [&](int j, int k, double& sr, double& si) {
    const int lo = j < k ? j : k, hi = j < k ? k : j;
    sr = mcs[1 + lo * U - lo * (lo - 1) / 2 + (hi - lo)];
    si = j == k ? 0.0 : mcs[1 + NRE + lo * (U - 1) - lo * (lo - 1) / 2 + (hi - lo - 1)];
    if (j > k) si = -si;
  };
  // (1) v = S c for c = cA (which 0) and cB (which 1): thread = (which, j, k)
  //     in groups of KG lanes over k, shuffle sums within the group
  constexpr int KG = U <= 1 ? 1 : (U <= 2 ? 2 : (U <= 4 ? 4 : (U <= 8 ? 8 : 16)));
  constexpr int PAIRS_PER_PASS = kTile / KG;
  for (int p0 = 0; p0 < 2 * U; p0 += PAIRS_PER_PASS) {
    const int pr = p0 + tid / KG, k = tid % KG;
    const int which = pr / U, j = pr % U;
    double re = 0, im = 0;
    if (pr < 2 * U && k < U) {
      const double(*c)[2] = which ? cc.cB : cc.cA;
      double sr, si;
      s_at(j, k, sr, si);
      re = sr * c[k][0] - si * c[k][1];
      im = sr * c[k][1] + si * c[k][0];
    }
#pragma unroll
    for (int off = 1; off < KG; off <<= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (pr < 2 * U && k == 0) {
      vv[which][j][0] = re;
      vv[which][j][1] = im;
    }
  }
  __syncthreads();
  // (2) the four forms from v: f = 0: cA^H vA, 1: cB^H vB, 2 / 3: Re / Im cB^H vA
  if (tid < (4 * KG + 31) / 32 * 32) {  // whole warps, for the shuffles
    const int f = tid / KG, j = tid % KG;
    double acc = 0;
    if (f < 4 && j < U) {
      const double(*cl)[2] = f == 0 ? cc.cA : cc.cB;
      const double* v = vv[f == 1 ? 1 : 0][j];
      acc = f == 3 ? cl[j][0] * v[1] - cl[j][1] * v[0] : cl[j][0] * v[0] + cl[j][1] * v[1];
    }
#pragma unroll
    for (int off = 1; off < KG; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (f < 4 && j == 0) sh[f] = acc;
  }
  __syncthreads();
  const double al = cc.alpha, be = cc.beta, gc = cc.gc, dc = cc.dc, x = cc.x, y = cc.y, gamma = cc.gamma;
  const double AA = sh[0], BB = sh[1], Xr = sh[2], Xi = sh[3];
  const double nbar = (al * AA + be * BB - 2.0 * gc * Xr - 2.0 * dc * Xi) * inv_sw;
  if (warp == 0) {  // the logarithm; warp 0 takes no part in the gradient
    double cres = 0.0;  // lane 0: the coefficient residue term, one component per lane
    if constexpr (COEF_RESIDUE) cres = warp_sum(coef_residue_term<U>(cc, ds, lane));
    if (tid == 0) {
      const double N = nbar * cc.tau;
      const double sum_lnb = ds[0] + cres, nbad = ds[1];
      double nll = -sum_lnb + gamma * sum_t + Nd * log_table(N, logtab);
      if (nbad > 0 || !(N > 0)) nll = nan("");
      res[0] = nll;
      res[1] = N;
      res[2] = nbad;
      res[3] = sum_lnb;
      res[4] = ds[4 + 4 * U + 2 * NR];
      if (onll) *onll = nll;
      if (trace) trace[6] = global_ns();
    }
    return;
  }
  if (!want_grad) return;
  auto put = [&](int k, double v) {
    res[kResHeader + k] = v;
    if (og) og[k] = v;
  };
  // d(N_d ln N) = N_d dnbar / nbar, applied to unnormalised sensitivities
  // data columns: [sum ln B, n_bad, d/dx, d/dy, Re gA, Im gA, Re gB, Im gB, s1, s2]
  // chains on threads 32.., resonances on threads 160.., x and y on thread 224
  const double sc = Nd * rcp<double>(nbar) * inv_sw;
  if (tid - 32 < nc) {  // nc <= 64: threads 32 .. 95
    const int ch = tid - 32;
    const int j = cc.chain_comp[ch];
    const double(*vA)[2] = vv[0];
    const double(*vB)[2] = vv[1];
    double dnr, dni, gr, gi;
    if (cc.chain_amp[ch] == 0) {
      dnr = 2 * al * vA[j][0] - 2 * gc * vB[j][0] + 2 * dc * vB[j][1];
      dni = 2 * al * vA[j][1] - 2 * gc * vB[j][1] - 2 * dc * vB[j][0];
      gr = ds[4 + j];
      gi = ds[4 + U + j];
    } else {
      dnr = 2 * be * vB[j][0] - 2 * gc * vA[j][0] - 2 * dc * vA[j][1];
      dni = 2 * be * vB[j][1] - 2 * gc * vA[j][1] + 2 * dc * vA[j][0];
      gr = ds[4 + 2 * U + j];
      gi = ds[4 + 3 * U + j];
    }
    // d sum ln B / d Re c = 2 Re(g), d / d Im c = -2 Im(g)
    put(2 * ch, cc.floating[2 * ch] ? -(2 * gr) + sc * dnr : 0.0);
    put(2 * ch + 1, cc.floating[2 * ch + 1] ? 2 * gi + sc * dni : 0.0);
  }
  if (tid >= 160 && tid < 160 + NR) {
    const int r = tid - 160;
    const double m0 = cc.m0[r];
    double dm_n = 0, dg_n = 0, dm_d = 0, dg_d = 0;
    if (have_res_grad) {
      // d n / d m0 = -4 m0 s1 - 2 dkappa/dm0 s2, d n / d Gamma0 = -2 dkappa/dGamma0 s2
      const double dk_dm = cc.kappa[r] * cc.dlk_dm[r], dk_dg = cc.kappa[r] * cc.dlk_dg[r];
      const double s1m = mcs[1 + NRE + NIM + r], s2m = mcs[1 + NRE + NIM + NR + r];
      dm_n = -4 * m0 * s1m - 2 * dk_dm * s2m;
      dg_n = -2 * dk_dg * s2m;
      const double s1d = ds[4 + 4 * U + r], s2d = ds[4 + 4 * U + NR + r];
      dm_d = -4 * m0 * s1d - 2 * dk_dm * s2d;
      dg_d = -2 * dk_dg * s2d;
    }
    const int k = 2 * nc + 2 * r;
    put(k, cc.floating[k] ? -dm_d + sc * dm_n : 0.0);
    put(k + 1, cc.floating[k + 1] ? -dg_d + sc * dg_n : 0.0);
  }
  if (tid == 224) {
    const double ia = cc.ia, ic = cc.ic;
    const double dal_dx = -2 * x * ic * ic, dal_dy = 2 * y * ia * ia;
    const double dbe_dx = 2 * x * ic * ic, dbe_dy = 2 * y * ia * ia;
    const double dgc_dy = (1 + y * y) * ia * ia, ddc_dx = (1 - x * x) * ic * ic;
    const double dn_dx = dal_dx * AA + dbe_dx * BB - 2 * ddc_dx * Xi;
    const double dn_dy = dal_dy * AA + dbe_dy * BB - 2 * dgc_dy * Xr;
    const int k = 2 * nc + 2 * NR;
    put(k, cc.floating[k] ? -ds[2] + sc * dn_dx : 0.0);
    put(k + 1, cc.floating[k + 1] ? -ds[3] + sc * dn_dy : 0.0);
  }
}

// RATES: the variant that writes per-event rates (a.rates); on the fp32
// path it also recomputes the ill-conditioned data events in double-float,
// so that every reported rate is within 1e-5 of its double-precision value.
// Likelihood evaluations without rates keep the fp32 ln B of those few
// events (their effect on the NLL is orders of magnitude below its 1e-3
// tolerance) and do not carry the recomputation's code.
// GRAM: how the MC normalisation matrix is accumulated (GramMode).
template <class P, class S, bool FULL, bool GRAD, bool WEIGHTED, bool RATES = false, int GRAM = kGramRegs>
__global__ void __launch_bounds__(kTile, FULL ? 1 : Layout<P, S, GRAM>::cached_blocks)
    k_eval(const __grid_constant__ EvalArgs a) {
  using T = typename P::T;
  using LY = Layout<P, S, GRAM>;
  static_assert(GRAM != kGramTensor || P::kF32, "tensor-core normalisation matrix on the fp32 path");
  static_assert(GRAM != kGramRegs || S::U <= 8, "register accumulation of the normalisation matrix up to 8 components");
  constexpr bool TCG = FULL && GRAM == kGramTensor;
  constexpr bool SMG = FULL && GRAM == kGramShared;
  constexpr int U = S::U, NR = S::NR, NRE = LY::NRE, NIM = LY::NIM, WMC = LY::WMC, WD = LY::WD;
  constexpr int NPL = FULL ? LY::NPL_FULL : LY::NPL_CACHE;
  constexpr int NST = LY::stages(FULL);
  constexpr int STB = LY::stage_bytes(FULL);
  constexpr int TE = kTile;
  constexpr int ES = int(sizeof(T));
  static_assert(NR <= 32 && kMaxChains <= 64, "thread roles of derive_compute");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NST], part_bar;
  __shared__ unsigned released[NST];  // warps done with the stage's current tile
  __shared__ unsigned s_issued;       // items whose copy has been issued
  __shared__ CtaConst cc;
  __shared__ BlockConst<T> bc;
  constexpr int RED_MC = GRAM == kGramRegs ? WMC : 1 + 2 * NR;  // per-thread MC columns summed over the block
  __shared__ T red[kWarps * (RED_MC > WD ? RED_MC : WD)];
  __shared__ double red_lnb[kWarps];
  __shared__ float2 rowp[LY::W];   // this block's partial row (double-float)
  __shared__ double colsum[LY::W];
  __shared__ unsigned s_last, s_timeout;
  __shared__ double2 logtab[kLogTable];
  __shared__ float4 logtab_f[P::kF32 ? kLogTable : 1];  // the same entries as double-float pairs
  // tensor-core normalisation matrix: MMA completion, TMEM base, column
  // exponents of the last three tiles (written, read, being reset)
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t s_tmem;
  __shared__ unsigned s_E[3][TCG ? TcGram<U>::CP : 1];
  __shared__ float2 mc_small[1 + 2 * kMaxRes];  // block sums of the MC weight and lineshape sensitivities

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  // the cached fp32 pass with the gradient forms A, Abar with the fp32
  // coefficients and adds their rounding residues in the finish
  // (coef_residue_term); the full pass, where the data tiles are a small
  // share of the work, applies them per event
  constexpr bool CRES = P::kF32 && GRAD && !FULL;
  // The next evaluation of a batch may start its blocks as this one's blocks exit.
  // The cached path reads the component cache and the stored MC totals that
  // the evaluation before it wrote, so it waits for that one first.
  grid_dependents_launch();
  if constexpr (!FULL) grid_dependency_wait();
  unsigned long long* trace = a.trace ? a.trace + size_t(blockIdx.x) * kTracePhases : nullptr;
  if (trace && tid == 0) trace[0] = global_ns();
  const SampleDev& dd = a.data;
  const SampleDev& dmc = a.mc;
  // Block b takes the contiguous range of MC tiles mc_ranges[b] ..
  // mc_ranges[b + 1] and then the data tiles b, b + G, ..., chosen on the
  // host so that every block carries about the same cost.  The assignment depends only on
  // the sizes and the grid, so every run sums in the same order.
  const int64_t b = blockIdx.x;
  const int64_t n_dt = dd.n_tiles;
  const int64_t my_data = n_dt > b ? (n_dt - 1 - b) / G + 1 : 0;
  const int64_t mc_begin = FULL ? a.mc_ranges[b] : 0, mc_end = FULL ? a.mc_ranges[b + 1] : 0;
  const int64_t my_mc = mc_end - mc_begin;  // items 0 .. my_mc - 1: MC tiles, then the data tiles
  const int64_t my_items = my_mc + my_data;

  // ---- one bulk copy of work item k (a whole tile) into stage k % NST
  auto issue = [&](int64_t k) {
    const int st = int(k % NST);
    const void* src;
    uint32_t bytes;
    if (k >= my_mc) {
      const int64_t tile = b + (k - my_mc) * G;
      if constexpr (FULL) {
        src = static_cast<const unsigned char*>(dd.planes) + tile * dd.tile_bytes;
        bytes = uint32_t(dd.tile_bytes);
      } else {
        src = static_cast<const unsigned char*>(dd.cache) + tile * dd.cache_tile_bytes;
        bytes = uint32_t(dd.cache_tile_bytes);
      }
    } else {
      const int64_t tile = mc_begin + k;
      src = static_cast<const unsigned char*>(dmc.planes) + tile * dmc.tile_bytes;
      bytes = uint32_t(dmc.tile_bytes);
    }
    mbar_arrive_expect_tx(&full_bar[st], bytes);
    bulk_g2s(smem_raw + st * STB, src, bytes, &full_bar[st]);
  };

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full_bar[s], 1);
      released[s] = 0;
    }
    mbar_init(&part_bar, 1);
    if constexpr (TCG) mbar_init(&mma_bar, 1);
    mbar_fence_init();
    // the first tile does not depend on the parameters (the test hook
    // withholds block 0's, so that its bounded wait runs out)
    if (my_items > 0 && !(a.withhold_first_copy && b == 0)) issue(0);
  }
  // tensor-core normalisation matrix: TMEM for the accumulator (warp 0),
  // zeroed operand buffer and accumulators, per-tile column exponents
  const TcGramSmem<U> tg = TcGramSmem<U>::at(smem_raw + NST * STB);
  if constexpr (TCG) {
    if (warp == 0) tmem_alloc(&s_tmem, TcGram<U>::TMEM_COLS);
    tg.init();
    for (int v = tid; v < 3 * TcGram<U>::CP; v += kTile) (&s_E[0][0])[v] = 0u;
  }
  if (!FULL)  // stored MC totals of the fixed lineshapes
    for (int v = tid; v < WMC; v += kTile) colsum[v] = a.gram_store[v];
  for (int j = tid; j < kLogTable; j += kTile) {
    const double2 v = static_cast<const double2*>(a.logtab)[j];
    logtab[j] = v;
    if constexpr (P::kF32) {
      const DF r = df_from_double(v.x), l = df_from_double(v.y);
      logtab_f[j] = make_float4(r.hi, r.lo, l.hi, l.lo);
    }
  }
  // the parameter loads go out before the other tile copies flood the memory system
  if (a.derived) {  // constants derived once for a batch
    const auto* rec = static_cast<const DerivedConst<T>*>(a.derived);
    copy_words(&cc, &rec->cc, sizeof(CtaConst));
    copy_words(&bc, &rec->bc, sizeof(BlockConst<T>));
  } else {
    derive_load<T, U>(a.params, a.hp, a.km, cc, bc);
  }
  if constexpr (TCG) tc_fence_before_sync();
  __syncthreads();
  uint32_t tmem = 0;
  if constexpr (TCG) {
    tc_fence_after_sync();
    tmem = s_tmem;
  }
  if (tid == 0) {
    const int64_t first = my_items < NST ? my_items : NST;
    for (int64_t k = 1; k < first; ++k) issue(k);
    s_issued = unsigned(first);
  }
  if (!a.derived) derive_compute<T, U, NR, GRAD && FULL>(a.km, cc, bc);
  __syncthreads();
  if (trace && tid == 0) trace[1] = global_ns();

  bool timed_out = false;
  uint32_t st = 0, ph = 0;
  int64_t k = 0;
  // This warp is done with item k (stage st).  The last of the eight warps
  // to get here issues the copy of item k + NST into the same stage; the
  // count is reset before that copy is issued, and a warp adds to it again
  // only after the copy has completed on the stage's barrier.
  auto release = [&]() {
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&released[st], 1u) == kWarps - 1) {
        __threadfence_block();
        released[st] = 0;
        if (k + NST < my_items) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(k + NST);
          atomicMax(&s_issued, unsigned(k + NST + 1));
        }
      }
    }
    if (++st == NST) {
      st = 0;
      ph ^= 1u;
    }
  };

  {
    // ---- MC tiles
    if constexpr (FULL && GRAM == kGramRegs) {
      T sw = 0, gre[NRE], gim[NIM > 0 ? NIM : 1], s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
      for (int q = 0; q < NRE; ++q) gre[q] = 0;
#pragma unroll
      for (int q = 0; q < (NIM > 0 ? NIM : 1); ++q) gim[q] = 0;
#pragma unroll
      for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;
      for (; k < my_mc && !timed_out; ++k) {
        const int64_t tile = mc_begin + k;
        const bool ok = mbar_wait_bounded(&full_bar[st], ph, kWaitNs);
        if (__any_sync(0xffffffffu, !ok)) {
          timed_out = true;
          break;
        }
        const int64_t i = tile * TE + tid;
        if (i < dmc.n) {
          const unsigned char* stage = smem_raw + st * STB;
          const T* sbase = reinterpret_cast<const T*>(stage);
          const SmemSrc<P, S, TE> src{sbase, tid, false};
          EventCore<P, S> ev;
          // fp32 with the gradient, up to 8 components: keep the term products for backprop_q
          constexpr bool KEEPQ = GRAD && P::kF32 && U <= 8;
          T qr[KEEPQ ? U * S::NO : 1], qi[KEEPQ ? U * S::NO : 1];
          ev.lineshapes(src, bc);
          if constexpr (KEEPQ) ev.components_q(src, qr, qi);
          else ev.components(src);
          const T w = WEIGHTED ? reinterpret_cast<const T*>(stage + NPL * TE * ES)[tid] : T(1);
          sw += w;
          int kr = 0, ki = 0;
#pragma unroll
          for (int j = 0; j < U; ++j) {
            const T wr = WEIGHTED ? w * ev.ar[j] : ev.ar[j], wi = WEIGHTED ? w * ev.ai[j] : ev.ai[j];
#pragma unroll
            for (int kk = j; kk < U; ++kk) {
              gre[kr] = fma(wr, ev.ar[kk], gre[kr]);
              gre[kr] = fma(wi, ev.ai[kk], gre[kr]);
              ++kr;
              if (kk > j) {
                gim[ki] = fma(wr, ev.ai[kk], gim[ki]);
                gim[ki] = fma(-wi, ev.ar[kk], gim[ki]);
                ++ki;
              }
            }
          }
          if constexpr (GRAD) {
            T Ar, Ai, Br, Bi;
            ev.amplitudes(bc, Ar, Ai, Br, Bi);
            // n = alpha|A|^2 + beta|Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*);
            // dn = 2 Re(uA dA + uB dAbar), uA = alpha A* - (gc - i dc) Abar*,
            // uB = beta Abar* - (gc + i dc) A*.
            const Quad<T> M = bc.mix;  // {alpha, beta, gc, dc}
            const T uAr = M.x * Ar - M.z * Br + M.w * Bi;
            const T uAi = -M.x * Ai + M.z * Bi + M.w * Br;
            const T uBr = M.y * Br - M.z * Ar - M.w * Ai;
            const T uBi = -M.y * Bi + M.z * Ai - M.w * Ar;
            if constexpr (KEEPQ) ev.template backprop_q<WEIGHTED>(bc, qr, qi, uAr, uAi, uBr, uBi, w, s1, s2);
            else ev.template backprop_lineshapes<WEIGHTED>(src, bc, uAr, uAi, uBr, uBi, w, s1, s2);
          }
        }
        release();
      }
      T vt[WMC];
      vt[0] = sw;
#pragma unroll
      for (int q = 0; q < NRE; ++q) vt[1 + q] = gre[q];
#pragma unroll
      for (int q = 0; q < NIM; ++q) vt[1 + NRE + q] = gim[q];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        vt[1 + NRE + NIM + r] = s1[r];
        vt[1 + NRE + NIM + NR + r] = s2[r];
      }
      block_sum_df<T, WMC>(vt, red, rowp);
    }
    if constexpr (TCG || SMG) {
      // Block-synchronous tiles: every thread takes part in every barrier,
      // and a bounded wait that gives up stops all of them.
      using TG = TcGram<U>;
      constexpr int CPX = TCG ? TG::CP : 1;
      if constexpr (SMG) static_assert(2 * U * TE * 8 <= STB, "the components of a tile fit its stage");
      timed_out = __syncthreads_or(timed_out) != 0;
      T sw = 0, s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
      for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;
      // kGramShared: this thread's entry of the normalisation sums, Re over
      // j <= k for q < NRE, Im over j < k after that (row-major)
      double gacc = 0.0;
      int gj = 0, gk = 0;
      const bool g_re = tid < NRE;
      if constexpr (SMG) {
        int r = g_re ? tid : tid - NRE;
        for (;;) {
          const int len = g_re ? U - gj : U - 1 - gj;
          if (r < len || gj >= U) break;
          r -= len;
          ++gj;
        }
        gk = g_re ? gj + r : gj + 1 + r;
      }
      int t3 = 0;
      uint32_t mma_phase = 0;
      bool mma_in_flight = false;
      for (; k < my_mc && !timed_out; ++k) {
        const int64_t tile = mc_begin + k;
        const bool ok = mbar_wait_bounded(&full_bar[st], ph, kWaitNs);
        const int64_t i = tile * TE + tid;
        const bool valid = ok && i < dmc.n;
        unsigned char* stage = smem_raw + st * STB;
        const T* sbase = reinterpret_cast<const T*>(stage);
        const SmemSrc<P, S, TE> src{sbase, tid, false};
        EventCore<P, S> ev;
        T w = T(0);
        if (valid) {
          ev.lineshapes(src, bc);
          ev.components(src);
          w = WEIGHTED ? reinterpret_cast<const T*>(stage + NPL * TE * ES)[tid] : T(1);
          sw += w;
        } else {
#pragma unroll
          for (int j = 0; j < U; ++j) ev.ar[j] = ev.ai[j] = T(0);
        }
        const T sq = WEIGHTED ? sqrt(w) : T(1);  // G = X^T X with sqrt(w) in each row
        // the adjoint of the time-integrated rate (needs this tile's planes)
        auto adjoint = [&]() {
          if constexpr (GRAD) {
            if (valid) {
              T Ar, Ai, Br, Bi;
              ev.amplitudes(bc, Ar, Ai, Br, Bi);
              const Quad<T> M = bc.mix;  // {alpha, beta, gc, dc}, see the register variant
              const T uAr = M.x * Ar - M.z * Br + M.w * Bi;
              const T uAi = -M.x * Ai + M.z * Bi + M.w * Br;
              const T uBr = M.y * Br - M.z * Ar - M.w * Ai;
              const T uBi = -M.y * Bi + M.z * Ai - M.w * Ar;
              ev.template backprop_lineshapes<WEIGHTED>(src, bc, uAr, uAi, uBr, uBi, w, s1, s2);
            }
          }
        };
        if constexpr (TCG) {
          float x[CPX];
#pragma unroll
          for (int c = 0; c < CPX; ++c) x[c] = 0.f;
#pragma unroll
          for (int j = 0; j < U; ++j) {
            x[j] = float(ev.ar[j] * sq);
            x[U + j] = float(ev.ai[j] * sq);
          }
          // largest exponent of each column over the tile
          unsigned mine = 0;
#pragma unroll
          for (int c = 0; c < CPX; ++c) {
            const unsigned e = __reduce_max_sync(0xffffffffu, exp_bits(x[c]));
            if (lane == c) mine = e;
          }
          if (lane < CPX) atomicMax(&s_E[t3][lane], mine < 7u ? 7u : mine);
          if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
          }
          if (tid < CPX) s_E[t3 == 0 ? 2 : t3 - 1][tid] = 0u;  // buffer of tile k + 2
          tg.store_pieces(x, s_E[t3], tid);
          __syncthreads();
          if (tid == 0) tg.issue(tmem, &mma_bar);
          mma_in_flight = true;
          adjoint();
          const bool ok2 = mbar_wait_bounded(&mma_bar, mma_phase, kWaitNs);
          mma_phase ^= 1u;
          tc_fence_after_sync();
          if (ok2) mma_in_flight = false;
          tg.stage(tmem);
          tc_fence_before_sync();
          if (__syncthreads_or(!ok2)) {
            timed_out = true;
            break;
          }
          tg.fold(s_E[t3]);
          t3 = t3 == 2 ? 0 : t3 + 1;
        } else {
          adjoint();
          if (__syncthreads_or(!ok)) {  // every thread is done with the planes
            timed_out = true;
            break;
          }
          T* X = reinterpret_cast<T*>(stage);  // [2U][256] components, re then im
#pragma unroll
          for (int j = 0; j < U; ++j) {
            X[j * TE + tid] = ev.ar[j] * sq;
            X[(U + j) * TE + tid] = ev.ai[j] * sq;
          }
          __syncthreads();
          if (tid < NRE + NIM) {
            const T* xj = X + gj * TE;
            const T* xk = X + gk * TE;
            const T* yj = X + (U + gj) * TE;
            const T* yk = X + (U + gk) * TE;
            // lanes start at different events (no shared-memory bank conflicts)
            for (int e0 = 0; e0 < TE; ++e0) {
              const int e = (e0 + lane) & (TE - 1);
              gacc = g_re ? fma(xj[e], xk[e], fma(yj[e], yk[e], gacc)) : fma(xj[e], yk[e], fma(-yj[e], xk[e], gacc));
            }
          }
          __syncthreads();  // before the stage is refilled
        }
        release();
      }
      if constexpr (TCG) {
        if (mma_in_flight && tid == 0)  // a wait gave up: let the MMA finish before TMEM is freed
          mbar_wait_bounded(&mma_bar, mma_phase ^ 1u, kWaitNs);
      }
      T vt[1 + 2 * NR];
      vt[0] = sw;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        vt[1 + r] = s1[r];
        vt[1 + NR + r] = s2[r];
      }
      block_sum_df<T, 1 + 2 * NR>(vt, red, mc_small);  // ends with a barrier
      for (int v = tid; v < 1 + 2 * NR; v += blockDim.x) rowp[v == 0 ? 0 : NRE + NIM + v] = mc_small[v];
      if constexpr (TCG) tg.finish(rowp + 1, rowp + 1 + NRE);
      if constexpr (SMG)
        if (tid < NRE + NIM) rowp[1 + tid] = to_df(gacc);
    }
    if (trace && tid == 0) trace[2] = global_ns();

    // ---- data tiles (after the MC tiles).  Everything up to here only
    // read memory that no evaluation writes (event planes, parameters,
    // constants), so it may overlap the end of the previous evaluation of a
    // batch; the component cache, the rates, the partial rows and the
    // completion counter are written only after that evaluation completed.
    grid_dependency_wait();
    {
      double lnb = 0.0;     // sum ln B = lnb + lexp ln 2 (fp64 path)
      DF lnbf{0.0f, 0.0f};  // the same as a double-float pair (fp32 path)
      int bad = 0, lexp = 0, n_rec = 0;
      T gx = 0, gy = 0, gAr[U], gAi[U], gBr[U], gBi[U], s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
      for (int j = 0; j < U; ++j) gAr[j] = gAi[j] = gBr[j] = gBi[j] = 0;
#pragma unroll
      for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;
      for (; k < my_items && !timed_out; ++k) {
        const int64_t tile = b + (k - my_mc) * G;
        const bool ok = mbar_wait_bounded(&full_bar[st], ph, kWaitNs);
        if (__any_sync(0xffffffffu, !ok)) {
          timed_out = true;
          break;
        }
        const int64_t i = tile * TE + tid;
        if (i < dd.n) {
          const unsigned char* stage = smem_raw + st * STB;
          const T* sbase = reinterpret_cast<const T*>(stage);
          // decay time: a double (fp64 path) or a double-float pair (fp32 path)
          const double t_e = P::kF32 ? 0.0 : reinterpret_cast<const double*>(stage + NPL * TE * ES)[tid];
          const float2 t_f = P::kF32 ? reinterpret_cast<const float2*>(stage + NPL * TE * ES)[tid] : float2{0.f, 0.f};
          const SmemSrc<P, S, TE> src{sbase, tid, false};
          EventCore<P, S> ev;
          constexpr bool RECOMPUTE = RATES && FULL && P::kF32;
          // fp32 full evaluation with the gradient, up to 8 components: keep the
          // term products for backprop_q
          constexpr bool KEEPQ = FULL && GRAD && P::kF32 && !RECOMPUTE && U <= 8;
          T sc[RECOMPUTE ? U : 1];
          T qr[KEEPQ ? U * S::NO : 1], qi[KEEPQ ? U * S::NO : 1];
          if constexpr (FULL) {
            ev.lineshapes(src, bc);
            if constexpr (KEEPQ) ev.components_q(src, qr, qi);
            else ev.template components<RECOMPUTE>(src, sc);
            T* cache = reinterpret_cast<T*>(static_cast<unsigned char*>(dd.cache) + tile * dd.cache_tile_bytes);
#pragma unroll
            for (int j = 0; j < U; ++j) {
              cache[j * TE + tid] = ev.ar[j];
              cache[(U + j) * TE + tid] = ev.ai[j];
            }
          } else {
#pragma unroll
            for (int j = 0; j < U; ++j) {
              ev.ar[j] = sbase[j * TE + tid];
              ev.ai[j] = sbase[(U + j) * TE + tid];
            }
          }
          T Ar_, Ai_, Br_, Bi_;
          ev.template amplitudes<!CRES>(bc, Ar_, Ai_, Br_, Bi_);
          T tAr, tAi, tBr, tBi;
          bool ok_ev;
          if constexpr (P::kF32) {
            DF Ad[4] = {DF{Ar_, 0.0f}, DF{Ai_, 0.0f}, DF{Br_, 0.0f}, DF{Bi_, 0.0f}};
            if constexpr (RECOMPUTE) {
              if (ill_conditioned<U>(bc, sc, Ar_, Ai_, Br_, Bi_, t_f.x)) {
                df_amplitudes<S>(sbase, dd.lo + tile * int64_t(S::NX + U * S::NO) * TE, tid, bc, Ad);
                n_rec += 1;
              }
            }
            ok_ev = mix_event_df<GRAD>(bc, logtab, logtab_f, Ad[0], Ad[1], Ad[2], Ad[3], t_f.x, t_f.y, lnbf, lexp,
                                       a.rates ? a.rates + i : nullptr, tAr, tAi, tBr, tBi, gx, gy);
          } else {
            ok_ev = mix_event<P, GRAD>(bc, logtab, Ar_, Ai_, Br_, Bi_, Ar_, Ai_, Br_, Bi_, t_e, lnb, lexp,
                                       a.rates ? a.rates + i : nullptr, tAr, tAi, tBr, tBi, gx, gy);
          }
          if (ok_ev) {
            if constexpr (GRAD) {
#pragma unroll
              for (int j = 0; j < U; ++j) {
                cmac(gAr[j], gAi[j], tAr, tAi, ev.ar[j], ev.ai[j]);
                cmac(gBr[j], gBi[j], tBr, tBi, ev.ar[j], ev.ai[j]);
              }
              if constexpr (KEEPQ) ev.template backprop_q<false>(bc, qr, qi, tAr, tAi, tBr, tBi, T(1), s1, s2);
              else if constexpr (FULL) ev.template backprop_lineshapes<false>(src, bc, tAr, tAi, tBr, tBi, T(1), s1, s2);
            }
          } else {
            bad += 1;
          }
        }
        release();
      }
      // block sums of the data accumulators -> rowp[WMC ..]
      {
        __shared__ int red_bad[kWarps], red_rec[kWarps];
        const double v0 = warp_sum(fma(double(lexp), kLn2, P::kF32 ? df_to_double(lnbf) : lnb));
        const int v1 = warp_sum(bad);
        const int v2 = warp_sum(n_rec);
        if (lane == 0) {
          red_lnb[warp] = v0;
          red_bad[warp] = v1;
          red_rec[warp] = v2;
        }
        T vt[WD - 3];
        vt[0] = gx;
        vt[1] = gy;
#pragma unroll
        for (int j = 0; j < U; ++j) {
          vt[2 + j] = gAr[j];
          vt[2 + U + j] = gAi[j];
          vt[2 + 2 * U + j] = gBr[j];
          vt[2 + 3 * U + j] = gBi[j];
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          vt[2 + 4 * U + r] = s1[r];
          vt[2 + 4 * U + NR + r] = s2[r];
        }
        block_sum_df<T, WD - 3>(vt, red, rowp + WMC + 2);  // ends with a barrier
        if (tid == 0) {
          double sl = 0;
          int sb = 0, sr = 0;
          for (int w = 0; w < kWarps; ++w) {
            sl += red_lnb[w];
            sb += red_bad[w];
            sr += red_rec[w];
          }
          rowp[WMC] = to_df(sl);
          rowp[WMC + 1] = make_float2(float(sb), 0.f);
          rowp[WMC + WD - 1] = make_float2(float(sr), 0.f);
        }
      }
    }
    if (trace && tid == 0) trace[3] = global_ns();
  }
  if constexpr (TCG) tc_fence_before_sync();
  const int block_timed_out = __syncthreads_or(timed_out);
  if constexpr (TCG) {
    if (warp == 0) {
      tc_fence_after_sync();
      tmem_dealloc(tmem, TcGram<U>::TMEM_COLS);
    }
  }
  if (block_timed_out && tid == 0) {
    // copies no warp waited for (the last one of each stage) land before
    // shared memory is reused or released
    const int64_t n_is = s_issued;
    for (int64_t q = n_is > NST ? n_is - NST : 0; q < n_is; ++q)
      mbar_wait_bounded(&full_bar[q % NST], uint32_t((q / NST) & 1), kWaitNs);
  }

  // ---- block partials (row b of [G][W]), then the last block reduces
  float2* part = static_cast<float2*>(a.part);
  for (int v = FULL ? tid : WMC + tid; v < LY::W; v += blockDim.x) part[size_t(b) * LY::W + v] = rowp[v];
  __syncthreads();
  if (trace && tid == 0) trace[4] = global_ns();
  if (tid == 0) {
    // the barrier orders every thread's partial stores before this release;
    // the last block's acquire then sees all blocks' partials
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    const unsigned old = atomicAdd(a.counter, block_timed_out ? 0x10001u : 1u);
    s_last = (old & 0xffffu) == unsigned(G - 1);
    s_timeout = (old >> 16) + (block_timed_out ? 1u : 0u);
    if (s_last) asm volatile("fence.acq_rel.gpu;" ::: "memory");
  }
  __syncthreads();
  if (!s_last) {
    if (trace && tid == 0) trace[5] = trace[6] = trace[7] = trace[4];
    return;
  }
  {
    // The partial rows of all blocks ([G][W] double-float pairs) come into
    // shared memory (the idle stage ring) by one bulk copy when they fit,
    // else they are read from global memory (L2).  Thread (column c, half h)
    // sums the rows of its half in order with TwoSum, lanes on consecutive
    // columns (no bank conflicts); the halves are combined through shared
    // memory.
    constexpr int HC = kTile / 2;
    __shared__ float2 half_sum[HC];
    const bool parts_smem = LY::partials_in_smem(G);
    const float2* sp = parts_smem ? reinterpret_cast<const float2*>(smem_raw) : part;
    if (parts_smem) {
      if (tid == 0) {
        asm volatile("fence.proxy.async;" ::: "memory");
        const uint32_t bytes = (uint32_t(G) * uint32_t(LY::W) * 8u + 15u) & ~15u;
        mbar_arrive_expect_tx(&part_bar, bytes);
        bulk_g2s(smem_raw, part, bytes, &part_bar);
      }
      const bool ok = mbar_wait_bounded(&part_bar, 0, kWaitNs);
      if (__syncthreads_or(!ok) && tid == 0) s_timeout += 1u;
    }
    const int c0 = FULL ? 0 : WMC;
    const int ncol = LY::W - c0;
    const int half_rows = (G + 1) / 2;
    const int h = tid / HC;
    for (int cb = 0; cb < ncol; cb += HC) {
      const int c = cb + tid % HC;
      float s = 0.f, er = 0.f;
      if (c < ncol) {
        // rows in four interleaved chains (independent loads and adds), then
        // the chains combined in order
        const float2* col = sp + c0 + c;
        const int r0 = h * half_rows, r1 = h ? G : half_rows;
        float s4[4] = {0.f, 0.f, 0.f, 0.f}, e4[4] = {0.f, 0.f, 0.f, 0.f};
        int rb = r0;
        for (; rb + 4 <= r1; rb += 4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 v = col[size_t(rb + q) * LY::W];
            float t, err;
            two_sum(s4[q], v.x, t, err);
            s4[q] = t;
            e4[q] += err + v.y;
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (rb + q < r1) {
            const float2 v = col[size_t(rb + q) * LY::W];
            float t, err;
            two_sum(s4[q], v.x, t, err);
            s4[q] = t;
            e4[q] += err + v.y;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float t, err;
          two_sum(s, s4[q], t, err);
          s = t;
          er += err + e4[q];
        }
        if (h == 1) half_sum[c - cb] = make_float2(s, er);
      }
      __syncthreads();
      if (h == 0 && c < ncol) {
        const float2 o = half_sum[c - cb];
        float t, err;
        two_sum(s, o.x, t, err);
        colsum[c0 + c] = double(t) + (double(er) + double(o.y) + double(err));
      }
      __syncthreads();
    }
    if (FULL)
      for (int v = tid; v < WMC; v += blockDim.x) a.gram_store[v] = colsum[v];
  }
  if (trace && tid == 0) trace[5] = global_ns();
  if (tid == 0) *a.counter = 0u;
  finish_likelihood<S, CRES>(a.result, a.out_nll, a.out_grad, a.km.n_chains, a.km.n_params, cc, colsum, colsum + WMC,
                       double(dd.n), a.sum_t, a.inv_sum_w, GRAD, FULL && GRAD, s_timeout != 0, logtab, trace);
  __syncthreads();
  if (trace && tid == 0) trace[7] = global_ns();
}

}  // namespace tdmix
