// One persistent kernel per likelihood evaluation.
//
// Every block (one per SM):
//   1. starts bulk asynchronous copies of its first two event tiles,
//   2. derives the per-evaluation constants from the parameter vector
//      (lineshape constants, coefficients of each component in A_f and
//      Abar_f, time-integral weights of the normalisation),
//   3. processes its data tiles (tiles b, b + grid, ...): lineshapes and
//      components (or the stored component cache), Eq. (mix) in its
//      factorised form in double precision, ln B and its adjoint,
//   4. processes its MC tiles: components, the normalisation matrix
//      I_jk = <a_j^* a_k> and the adjoint of the time-integrated rate,
//   5. writes its partial sums; the last block to finish sums the partials
//      of all blocks in a fixed order (double-float arithmetic) and forms
//      N, the NLL and the gradient.
// Tiles move global -> shared by cp.async.bulk completing on mbarriers, two
// stages deep; every wait is bounded and reports TDMIX_ERR_TIMEOUT.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "device_tables.hpp"
#include "eval.cuh"
#include "kinematics.cuh"

namespace tdmix {

constexpr int kTile = 256;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

// Per-evaluation constants in double precision (shared memory of a block).
struct CtaConst {
  double m0[kMaxRes], g0[kMaxRes], m2[kMaxRes], kappa[kMaxRes], dk_dm[kMaxRes], dk_dg[kMaxRes];
  double cA[kMaxComp][2], cB[kMaxComp][2];
  double x, y, gamma, alpha, beta, gc, dc, ia, ic;
  int chain_comp[kMaxChains], chain_amp[kMaxChains], floating[kMaxChains * 2 + 2 * kMaxRes + 2];
  int nonfinite, domain;
};

__device__ inline double dlnF_dz_dev(int L, double z) {
  if (L == 0) return 0.0;
  if (L == 1) return -0.5 / (1.0 + z);
  return -0.5 * (3.0 + 2.0 * z) / (9.0 + 3.0 * z + z * z);
}

// Threads of the block in parallel: first every parameter and model table
// entry is loaded into shared memory, then thread r derives resonance r's
// constants, thread c places chain c's coefficient and two threads the
// mixing weights.  m0 Gamma(s) = kappa X(s) with, for a mass-dependent
// width, kappa = m0^2 Gamma0 / (q0^(2L+1) F_L(q0 r)^2); with
// lambda = Kallen(m0^2, ma^2, mb^2) = 4 m0^2 q0^2 this is
// kappa = 2 m0^3 Gamma0 G_L(z0) (4 m0^2)^L lambda^-(2L+1)/2, G_L = 1/F_L^2
// (1, 1 + z, 9 + 3z + z^2), z0 = q0^2 r^2; a constant width has
// kappa = m0 Gamma0.  Only one reciprocal square root and one division sit
// on the dependent chain (double precision is slow to issue on this GPU).
template <class T>
__device__ inline void derive_constants(const double* __restrict__ params, const DevModel* __restrict__ dm,
                                        const int* __restrict__ floating, CtaConst& cc, BlockConst<T>& bc) {
  __shared__ double sp[kMaxChains * 2 + 2 * kMaxRes + 2];
  __shared__ int s_nc, s_nr, s_u, s_np;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_nc = dm->n_chains;
    s_nr = dm->NR;
    s_u = dm->U;
    s_np = dm->n_params;
    cc.nonfinite = cc.domain = 0;
    cc.gamma = dm->gamma;
  }
  __syncthreads();
  const int nc = s_nc, NR = s_nr, U = s_u, np = s_np;
  for (int k = tid; k < np; k += blockDim.x) {
    const double v = params[k];
    sp[k] = v;
    cc.floating[k] = floating[k];
    if (!isfinite(v)) atomicOr(&cc.nonfinite, 1);
  }
  for (int j = tid; j < U; j += blockDim.x) cc.cA[j][0] = cc.cA[j][1] = cc.cB[j][0] = cc.cB[j][1] = 0.0;
  for (int c = tid; c < nc; c += blockDim.x) {
    cc.chain_comp[c] = dm->chain_comp[c];
    cc.chain_amp[c] = dm->chain_amp[c];
  }
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    double(*dst)[2] = cc.chain_amp[c] == 0 ? cc.cA : cc.cB;
    dst[cc.chain_comp[c]][0] = sp[2 * c];
    dst[cc.chain_comp[c]][1] = sp[2 * c + 1];
  }
  for (int r = tid; r < NR; r += blockDim.x) {
    const int shape = dm->res_shape[r], L = dm->res_L[r];
    const double ma = dm->res_ma[r], mb = dm->res_mb[r], rr = dm->r_res;
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
      const double rs = rsqrt(lam);                  // lambda^-1/2
      const double z0 = lam * rr * rr / (4.0 * u);   // (q0 r)^2, off the rsqrt chain
      double g = 1.0, w = rs;                        // G_L(z0) and lambda^-(2L+1)/2 (4u)^L
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
    if constexpr (sizeof(T) == 4) {
      const float hi = float(u);
      bc.m2[r] = hi;
      bc.m2_lo[r] = float(u - double(hi));
    } else {
      bc.m2[r] = T(u);
      bc.m2_lo[r] = T(0);
    }
    bc.kappa[r] = T(kap);
    bc.kappa_lo[r] = T(kap - double(T(kap)));
  }
  // mixing weights: thread 32 and 33 each take one reciprocal
  if (tid == 32 || tid == 33) {
    const double x = sp[2 * nc + 2 * NR], y = sp[2 * nc + 2 * NR + 1];
    if (tid == 32) {
      if (!(fabs(y) < 1.0)) atomicOr(&cc.domain, 1);
      cc.ia = 1.0 / (1.0 - y * y);
      cc.y = y;
    } else {
      cc.ic = 1.0 / (1.0 + x * x);
      cc.x = x;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const double x = cc.x, y = cc.y, ia = cc.ia, ic = cc.ic;
    cc.alpha = ia + ic;
    cc.beta = (x * x + y * y) * ia * ic;
    cc.gc = y * ia;
    cc.dc = x * ic;
    bc.x = x;
    bc.y = y;
    bc.gamma = cc.gamma;
    bc.alpha = T(cc.alpha);
    bc.beta = T(cc.beta);
    bc.gc = T(cc.gc);
    bc.dc = T(cc.dc);
  }
  for (int j = tid; j < U; j += blockDim.x) {
    for (int q = 0; q < 2; ++q) {
      bc.cA[j][q] = T(cc.cA[j][q]);
      bc.cB[j][q] = T(cc.cB[j][q]);
      bc.cA_lo[j][q] = T(cc.cA[j][q] - double(bc.cA[j][q]));
      bc.cB_lo[j][q] = T(cc.cB[j][q] - double(bc.cB[j][q]));
    }
  }
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

template <class P, class S>
struct Layout {
  using T = typename P::T;
  static constexpr int U = S::U, NR = S::NR;
  static constexpr int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  static constexpr int WMC = 1 + NRE + NIM + 2 * NR;  // sum w, Re I (j<=k), Im I (j<k), s1, s2
  static constexpr int WD = 4 + 4 * U + 2 * NR;       // sum ln B, n_bad, d/dx, d/dy, gA, gB, s1, s2
  static constexpr int W = WMC + WD;
  static constexpr int NPL_FULL = Planes<P, S>::W0;    // invariants, width factors, spin factors
  static constexpr int NPL_CACHE = 2 * U;             // component cache (re, im)
  // bytes of one stage: planes, then one 8-byte-per-event plane (t or w)
  static constexpr int stage_bytes(bool full) {
    return (full ? NPL_FULL : NPL_CACHE) * kTile * int(sizeof(T)) + kTile * 8;
  }
  // dynamic shared memory: two stages, reused by the last block for the
  // partial array of `ld` blocks
  static constexpr int smem_bytes(bool full, int ld) {
    const int st = 2 * stage_bytes(full), pa = W * ld * 8;
    return st > pa ? st : pa;
  }
};

// dkappa/dm0 and dkappa/dGamma0 of resonance r (used for the gradient only):
// ln kappa = 2 ln m0 + ln Gamma0 - (2L+1)/2 ln q0^2 - 2 ln F_L(z0), z0 = q0^2 r^2,
// d q0^2 / d m0 = 2 m0 (u^2 - (ma^2 - mb^2)^2) / (4 u^2), u = m0^2.
__device__ inline void kappa_derivatives(const DevModel* dm, int r, double m0, double g0, double kap, CtaConst& cc) {
  const int shape = dm->res_shape[r];
  if (shape == SHAPE_CONST) {
    cc.dk_dm[r] = g0;
    cc.dk_dg[r] = m0;
  } else if (shape == SHAPE_MDW) {
    const int L = dm->res_L[r];
    const double r2 = dm->r_res * dm->r_res;
    const double a = dm->res_ma[r] * dm->res_ma[r], b = dm->res_mb[r] * dm->res_mb[r];
    const double u = m0 * m0;
    const double q02 = breakup2(u, a, b);
    const double z0 = q02 * r2;
    const double dq2 = 2.0 * m0 * (u * u - (a - b) * (a - b)) / (4.0 * u * u);
    const double dlnk = 2.0 / m0 - (2 * L + 1) * dq2 / (2.0 * q02) - 2.0 * dlnF_dz_dev(L, z0) * r2 * dq2;
    cc.dk_dm[r] = kap * dlnk;
    cc.dk_dg[r] = kap / g0;
  } else {
    cc.dk_dm[r] = cc.dk_dg[r] = 0.0;
  }
}

// Last block: normalisation, NLL and gradient from the column totals.
//   N = <alpha |A|^2 + beta |Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*)> / Gamma
// is Eq. (mix) integrated over t in [0, inf) and averaged over the MC sample
// (alpha = 1/(1-y^2) + 1/(1+x^2), beta = 1/(1-y^2) - 1/(1+x^2),
// gc = y/(1-y^2), dc = x/(1+x^2)); with S_jk = sum_e w_e a_j^* a_k and
// I = S / sum w: <|A|^2> = cA^H I cA, <|Abar|^2> = cB^H I cB,
// <A Abar*> = cB^H I cA.   NLL = -sum ln B + Gamma sum t + N_d ln N.
// Work is spread over threads so that only short chains of double-precision
// operations are dependent; the logarithm runs on one thread while the
// others form the gradient.
// Likelihood from the MC column totals `mcs` and the data column totals
// `ds` of one sample: writes [nll, N, n_bad or status, sum ln B, grad...]
// to `res`.  Used by the last block of an evaluation and, in serving, by the
// last chunk of each request.  `err` is a bounded-wait failure flag (read
// and cleared).
template <class S>
__device__ inline void finish_likelihood(double* res, int nc, int np, const CtaConst& cc, const double* mcs,
                                         const double* ds, double Nd, double sum_t, double inv_sw, bool want_grad,
                                         bool have_res_grad, int* err, unsigned long long* trace) {
  constexpr int U = S::U, NR = S::NR;
  constexpr int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  __shared__ double prod[2][U][U][2];
  __shared__ double vv[2][U][2];  // S cA, S cB (unnormalised)
  __shared__ double sh[8];        // AA, BB, Xr, Xi (unnormalised), nbar, sc
  const int tid = threadIdx.x;
  const int timed_out = *err;
  const int status = timed_out ? -7 : (cc.nonfinite ? -5 : (cc.domain ? -6 : 0));
  if (status != 0) {
    __syncthreads();
    if (tid == 0 && timed_out) *err = 0;
    for (int k = tid; k < kResHeader + np; k += blockDim.x) res[k] = k == 2 ? double(status) : nan("");
    return;
  }
  // products S_jk c_k, thread (which, j, k)
  for (int e = tid; e < 2 * U * U; e += blockDim.x) {
    const int which = e / (U * U), j = (e / U) % U, k = e % U;
    const int lo = j < k ? j : k, hi = j < k ? k : j;
    const int ire = lo * U - lo * (lo - 1) / 2 + (hi - lo);
    const int iim = lo * (U - 1) - lo * (lo - 1) / 2 + (hi - lo - 1);
    const double sr = mcs[1 + ire];
    const double si = j == k ? 0.0 : (j < k ? mcs[1 + NRE + iim] : -mcs[1 + NRE + iim]);
    const double cr = which ? cc.cB[k][0] : cc.cA[k][0], ci = which ? cc.cB[k][1] : cc.cA[k][1];
    prod[which][j][k][0] = sr * cr - si * ci;
    prod[which][j][k][1] = sr * ci + si * cr;
  }
  __syncthreads();
  for (int e = tid; e < 2 * U; e += blockDim.x) {
    const int which = e / U, j = e % U;
    double re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      re += prod[which][j][k][0];
      im += prod[which][j][k][1];
    }
    vv[which][j][0] = re;
    vv[which][j][1] = im;
  }
  __syncthreads();
  if (tid < 4) {
    // tid 0: cA^H S cA, 1: cB^H S cB, 2/3: Re/Im cB^H S cA
    const double(*c)[2] = tid == 0 ? cc.cA : cc.cB;
    const int w = tid == 1 ? 1 : 0;
    double acc = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      if (tid == 3) acc += c[j][0] * vv[w][j][1] - c[j][1] * vv[w][j][0];
      else acc += c[j][0] * vv[w][j][0] + c[j][1] * vv[w][j][1];
    }
    sh[tid] = acc;
  }
  __syncthreads();
  const double al = cc.alpha, be = cc.beta, gc = cc.gc, dc = cc.dc, x = cc.x, y = cc.y, gamma = cc.gamma;
  const double AA = sh[0], BB = sh[1], Xr = sh[2], Xi = sh[3];
  const double nbar = (al * AA + be * BB - 2.0 * gc * Xr - 2.0 * dc * Xi) * inv_sw;
  if (want_grad && tid == 32) sh[5] = Nd / nbar;  // d(N_d ln N) = N_d dnbar / nbar
  __syncthreads();
  if (tid == 0) {
    const double N = nbar / gamma;
    const double sum_lnb = ds[0], nbad = ds[1];
    double nll = -sum_lnb + gamma * sum_t + Nd * log(N);
    if (nbad > 0 || !(N > 0)) nll = nan("");
    res[0] = nll;
    res[1] = N;
    res[2] = nbad;
    res[3] = sum_lnb;
    if (timed_out) *err = 0;
    if (trace) trace[6] = global_ns();
  }
  if (!want_grad) return;
  const double sc = sh[5] * inv_sw;  // applied to unnormalised sensitivities
  // data columns: [sum ln B, n_bad, d/dx, d/dy, Re gA, Im gA, Re gB, Im gB, s1, s2]
  // chains on threads 32.., resonances on threads 160.., x and y on thread 224
  // (thread 0 is busy with the logarithm)
  for (int ch = tid - 32; ch >= 0 && ch < nc; ch += blockDim.x) {
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
    res[kResHeader + 2 * ch] = cc.floating[2 * ch] ? -(2 * gr) + sc * dnr : 0.0;
    res[kResHeader + 2 * ch + 1] = cc.floating[2 * ch + 1] ? 2 * gi + sc * dni : 0.0;
  }
  for (int r = tid - 160; r >= 0 && r < NR; r += blockDim.x) {
    const double m0 = cc.m0[r];
    double dm_n = 0, dg_n = 0, dm_d = 0, dg_d = 0;
    if (have_res_grad) {
      // d n / d m0 = -4 m0 s1 - 2 dkappa/dm0 s2, d n / d Gamma0 = -2 dkappa/dGamma0 s2
      const double s1m = mcs[1 + NRE + NIM + r], s2m = mcs[1 + NRE + NIM + NR + r];
      dm_n = -4 * m0 * s1m - 2 * cc.dk_dm[r] * s2m;
      dg_n = -2 * cc.dk_dg[r] * s2m;
      const double s1d = ds[4 + 4 * U + r], s2d = ds[4 + 4 * U + NR + r];
      dm_d = -4 * m0 * s1d - 2 * cc.dk_dm[r] * s2d;
      dg_d = -2 * cc.dk_dg[r] * s2d;
    }
    const int k = 2 * nc + 2 * r;
    res[kResHeader + k] = cc.floating[k] ? -dm_d + sc * dm_n : 0.0;
    res[kResHeader + k + 1] = cc.floating[k + 1] ? -dg_d + sc * dg_n : 0.0;
  }
  if (tid == 224) {
    const double ia = cc.ia, ic = cc.ic;
    const double dal_dx = -2 * x * ic * ic, dal_dy = 2 * y * ia * ia;
    const double dbe_dx = 2 * x * ic * ic, dbe_dy = 2 * y * ia * ia;
    const double dgc_dy = (1 + y * y) * ia * ia, ddc_dx = (1 - x * x) * ic * ic;
    const double dn_dx = dal_dx * AA + dbe_dx * BB - 2 * ddc_dx * Xi;
    const double dn_dy = dal_dy * AA + dbe_dy * BB - 2 * dgc_dy * Xr;
    const int k = 2 * nc + 2 * NR;
    res[kResHeader + k] = cc.floating[k] ? -ds[2] + sc * dn_dx : 0.0;
    res[kResHeader + k + 1] = cc.floating[k + 1] ? -ds[3] + sc * dn_dy : 0.0;
  }
}

template <class S>
__device__ inline void final_epilogue(const EvalArgs& a, CtaConst& cc, const double* colsum, bool want_grad,
                                      bool have_res_grad, unsigned long long* trace) {
  constexpr int WMC = Layout<PrecF64, S>::WMC;
  finish_likelihood<S>(a.result, a.dm->n_chains, a.dm->n_params, cc, colsum, colsum + WMC, double(a.data.n),
                       a.sum_t, a.inv_sum_w, want_grad, have_res_grad, a.err, trace);
}

template <class P, class S, bool FULL, bool GRAD, bool WEIGHTED>
__global__ void __launch_bounds__(kTile, 1) k_eval(EvalArgs a, const int* __restrict__ floating) {
  using T = typename P::T;
  using LY = Layout<P, S>;
  using PL = Planes<P, S>;
  constexpr int U = S::U, NR = S::NR, NRE = LY::NRE, NIM = LY::NIM, WMC = LY::WMC, WD = LY::WD;
  constexpr int NPL = FULL ? LY::NPL_FULL : LY::NPL_CACHE;
  constexpr int TE = kTile;
  constexpr int ES = int(sizeof(T));
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ CtaConst cc;
  __shared__ BlockConst<T> bc;
  __shared__ double red[kTile / 32][WMC > WD ? WMC : WD];
  __shared__ double colsum[LY::W];
  __shared__ unsigned is_last;

  const int tid = threadIdx.x;
  const int G = gridDim.x;
  unsigned long long* trace = a.trace ? a.trace + size_t(blockIdx.x) * kTracePhases : nullptr;
  if (trace && tid == 0) trace[0] = global_ns();
  const SampleDev& dd = a.data;
  const SampleDev& dmc = a.mc;
  const int64_t n_dt = (dd.n + TE - 1) / TE;
  const int64_t n_mt = FULL ? (dmc.n + TE - 1) / TE : 0;
  // Block b takes data tiles b, b + G, ... and then the contiguous range of
  // MC tiles mc_ranges[b] .. mc_ranges[b + 1], chosen on the host so that
  // every block carries about the same cost.  The assignment depends only on
  // the sizes and the grid, so every run sums in the same order.
  const int64_t b = blockIdx.x;
  const int64_t my_data = n_dt > b ? (n_dt - 1 - b) / G + 1 : 0;
  const int64_t mc_begin = FULL ? a.mc_ranges[b] : 0, mc_end = FULL ? a.mc_ranges[b + 1] : 0;
  const int64_t my_items = my_data + (mc_end - mc_begin);
  const int stage_bytes = LY::stage_bytes(FULL);
  unsigned char* stage[2] = {smem_raw, smem_raw + stage_bytes};

  // ---- bulk copies of one work item into a stage
  auto issue = [&](int64_t k) {
    const int st = int(k & 1);
    const bool is_data = k < my_data;
    const SampleDev& s = is_data ? dd : dmc;
    const int64_t off = (is_data ? b + k * G : mc_begin + (k - my_data)) * TE;
    uint32_t bytes = uint32_t(NPL) * TE * ES;
    const bool extra = is_data || WEIGHTED;
    if (extra) bytes += is_data ? TE * 8 : TE * ES;
    mbar_arrive_expect_tx(&bars[st], bytes);
    T* dst = reinterpret_cast<T*>(stage[st]);
    for (int p = 0; p < NPL; ++p) {
      const T* src;
      if constexpr (FULL) {
        if (p < PL::X0) src = static_cast<const T*>(s.s) + p * s.pitch;
        else if (p < PL::K0) src = static_cast<const T*>(s.x) + (p - PL::X0) * s.pitch;
        else src = static_cast<const T*>(s.k) + (p - PL::K0) * s.pitch;
      } else {
        src = static_cast<const T*>(s.cache) + p * s.pitch;
      }
      bulk_g2s(dst + p * TE, src + off, TE * ES, &bars[st]);
    }
    unsigned char* ex = stage[st] + NPL * TE * ES;
    if (is_data) bulk_g2s(ex, dd.t + off, TE * 8, &bars[st]);
    else if (WEIGHTED) bulk_g2s(ex, static_cast<const T*>(dmc.w) + off, TE * ES, &bars[st]);
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    if (my_items > 0) issue(0);
    if (my_items > 1) issue(1);
  }
  derive_constants<T>(a.params, a.dm, floating, cc, bc);
  __syncthreads();
  if (trace && tid == 0) trace[1] = global_ns();

  int64_t k = 0;
  bool timed_out = false;

  // ---- data tiles
  {
    double lnb = 0.0;
    int bad = 0;
    T gx = 0, gy = 0, gAr[U], gAi[U], gBr[U], gBi[U], s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
    for (int j = 0; j < U; ++j) gAr[j] = gAi[j] = gBr[j] = gBi[j] = 0;
#pragma unroll
    for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;
    T* cache = static_cast<T*>(dd.cache);
    for (; k < my_data; ++k) {
      const int64_t item = b + k * G;
      const int st = int(k & 1);
      const bool ok = mbar_wait_bounded(&bars[st], uint32_t((k >> 1) & 1), kWaitNs);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      const int64_t i = item * TE + tid;
      if (i < dd.n) {
        const T* sbase = reinterpret_cast<const T*>(stage[st]);
        const double t_e = reinterpret_cast<const double*>(stage[st] + NPL * TE * ES)[tid];
        const SmemSrc<P, S, TE> src{sbase, tid, false};
        EventCore<P, S> ev;
        if constexpr (FULL) {
          ev.lineshapes(src, bc);
          ev.components(src);
#pragma unroll
          for (int j = 0; j < U; ++j) {
            cache[j * dd.pitch + i] = ev.ar[j];
            cache[(U + j) * dd.pitch + i] = ev.ai[j];
          }
        } else {
#pragma unroll
          for (int j = 0; j < U; ++j) {
            ev.ar[j] = sbase[j * TE + tid];
            ev.ai[j] = sbase[(U + j) * TE + tid];
          }
        }
        T Ar_, Ai_, Br_, Bi_;
        ev.template amplitudes<true>(bc, Ar_, Ai_, Br_, Bi_);
        // Eq. (mix) as 2 |cosh(w) A - sinh(w) Abar|^2, w = (y + i x) Gamma t / 2, in double.
        const double Ar = Ar_, Ai = Ai_, Br = Br_, Bi = Bi_;
        const double gt = bc.gamma * t_e;
        double cha, sha, cb, sb;
        mixing_trig(0.5 * bc.y * gt, 0.5 * bc.x * gt, cha, sha, cb, sb);
        const double chr = cha * cb, chi = sha * sb;  // cosh(w)
        const double shr = sha * cb, shi = cha * sb;  // sinh(w)
        const double Zr = chr * Ar - chi * Ai - (shr * Br - shi * Bi);
        const double Zi = chr * Ai + chi * Ar - (shr * Bi + shi * Br);
        const double z2 = Zr * Zr + Zi * Zi;
        const double B = 2.0 * z2;
        if (a.rates) a.rates[i] = exp(-gt) * B;
        if (B > 0.0 && B < INFINITY) {
          lnb += log(B);
          if constexpr (GRAD) {
            // d ln B = 2 Re(V dZ), V = Z* / |Z|^2; dZ = cosh(w) dA - sinh(w) dAbar
            // + (sinh(w) A - cosh(w) Abar) dw; dw/dy = Gamma t / 2, dw/dx = i Gamma t / 2.
            // The sensitivities are formed in the working precision; in fp32
            // cosh(w), sinh(w) and Z are re-derived in fp32 rather than
            // converted from their fp64 values.
            T cr, ci, sr, si, Zrt, Zit;
            if constexpr (P::kF32) {
              const float gtf = float(bc.gamma) * float(t_e);
              float chf, shf, cbf, sbf;
              mixing_trig_f32(0.5f * float(bc.y) * gtf, 0.5f * float(bc.x) * gtf, chf, shf, cbf, sbf);
              cr = chf * cbf; ci = shf * sbf; sr = shf * cbf; si = chf * sbf;
              Zrt = 0; Zit = 0;
              cmac(Zrt, Zit, cr, ci, Ar_, Ai_);
              cmac(Zrt, Zit, -sr, -si, Br_, Bi_);
            } else {
              cr = chr; ci = chi; sr = shr; si = shi;
              Zrt = Zr; Zit = Zi;
            }
            const T iz = rcp<T>(fma(Zrt, Zrt, Zit * Zit));
            const T Vr = Zrt * iz, Vi = -Zit * iz;
            const T tAr = fma(Vr, cr, -Vi * ci), tAi = fma(Vr, ci, Vi * cr);
            const T tBr = -fma(Vr, sr, -Vi * si), tBi = -fma(Vr, si, Vi * sr);
            T Dr = 0, Di = 0;
            cmac(Dr, Di, sr, si, Ar_, Ai_);
            cmac(Dr, Di, -cr, -ci, Br_, Bi_);
            const T tg = P::kF32 ? T(float(bc.gamma) * float(t_e)) : T(gt);
            gy = fma(tg, fma(Vr, Dr, -Vi * Di), gy);
            gx = fma(-tg, fma(Vr, Di, Vi * Dr), gx);
#pragma unroll
            for (int j = 0; j < U; ++j) {
              cmac(gAr[j], gAi[j], tAr, tAi, ev.ar[j], ev.ai[j]);
              cmac(gBr[j], gBi[j], tBr, tBi, ev.ar[j], ev.ai[j]);
            }
            if constexpr (FULL) ev.template backprop_lineshapes<false>(src, bc, tAr, tAi, tBr, tBi, T(1), s1, s2);
          }
        } else {
          bad += 1;
        }
      }
      __syncthreads();  // stage consumed
      if (tid == 0 && k + 2 < my_items) issue(k + 2);
    }
    // block sum of the data accumulators -> colsum[WMC ..]
    const int lane = tid & 31, warp = tid >> 5;
    {
      const double v0 = warp_sum(lnb), v1 = warp_sum(double(bad));
      if (lane == 0) {
        red[warp][0] = v0;
        red[warp][1] = v1;
      }
    }
    T vt[WD - 2];
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
#pragma unroll
    for (int q = 0; q < WD - 2; ++q) {
      const T s = warp_sum(vt[q]);
      if (lane == 0) red[warp][2 + q] = double(s);
    }
    __syncthreads();
    for (int v = tid; v < WD; v += blockDim.x) {
      double s = 0;
      for (int w = 0; w < kTile / 32; ++w) s += red[w][v];
      colsum[WMC + v] = s;
    }
    __syncthreads();
  }

  if (trace && tid == 0) trace[2] = global_ns();

  // ---- MC tiles
  if constexpr (FULL) {
    T sw = 0, gre[NRE], gim[NIM > 0 ? NIM : 1], s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
    for (int q = 0; q < NRE; ++q) gre[q] = 0;
#pragma unroll
    for (int q = 0; q < (NIM > 0 ? NIM : 1); ++q) gim[q] = 0;
#pragma unroll
    for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;
    for (; k < my_items && !timed_out; ++k) {
      const int64_t item = mc_begin + (k - my_data);
      const int st = int(k & 1);
      const bool ok = mbar_wait_bounded(&bars[st], uint32_t((k >> 1) & 1), kWaitNs);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      const int64_t i = item * TE + tid;
      if (i < dmc.n) {
        const T* sbase = reinterpret_cast<const T*>(stage[st]);
        const SmemSrc<P, S, TE> src{sbase, tid, false};
        EventCore<P, S> ev;
        ev.lineshapes(src, bc);
        ev.components(src);
        const T w = WEIGHTED ? reinterpret_cast<const T*>(stage[st] + NPL * TE * ES)[tid] : T(1);
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
          const T uAr = bc.alpha * Ar - bc.gc * Br + bc.dc * Bi;
          const T uAi = -bc.alpha * Ai + bc.gc * Bi + bc.dc * Br;
          const T uBr = bc.beta * Br - bc.gc * Ar - bc.dc * Ai;
          const T uBi = -bc.beta * Bi + bc.gc * Ai - bc.dc * Ar;
          ev.template backprop_lineshapes<WEIGHTED>(src, bc, uAr, uAi, uBr, uBi, w, s1, s2);
        }
      }
      __syncthreads();
      if (tid == 0 && k + 2 < my_items) issue(k + 2);
    }
    const int lane = tid & 31, warp = tid >> 5;
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
#pragma unroll
    for (int q = 0; q < WMC; ++q) {
      const T s = warp_sum(vt[q]);
      if (lane == 0) red[warp][q] = double(s);
    }
    __syncthreads();
    for (int v = tid; v < WMC; v += blockDim.x) {
      double s = 0;
      for (int w = 0; w < kTile / 32; ++w) s += red[w][v];
      colsum[v] = s;
    }
    __syncthreads();
  }
  if (trace && tid == 0) trace[3] = global_ns();
  if (timed_out) {
    // let copies still in flight land before the block exits
    if (tid == 0) {
      atomicOr(a.err, 1);
      for (int64_t q = k; q < my_items && q < k + 2; ++q)
        mbar_wait_bounded(&bars[q & 1], uint32_t((q >> 1) & 1), kWaitNs);
    }
    __syncthreads();
  }

  // ---- block partials (column-major, [W][ld]), then the last block reduces
  float2* part = static_cast<float2*>(a.part);
  for (int v = tid; v < LY::W; v += blockDim.x)
    part[size_t(v) * a.ld + blockIdx.x] = (FULL || v >= WMC) ? to_df(colsum[v]) : make_float2(0.f, 0.f);
  __threadfence();
  __syncthreads();
  if (trace && tid == 0) trace[4] = global_ns();
  if (tid == 0) is_last = atomicAdd(a.counter, 1u) == unsigned(G - 1);
  __syncthreads();
  if (!is_last) {
    if (trace && tid == 0) trace[5] = trace[6] = trace[7] = trace[4];
    return;
  }
  __threadfence();
  {
    // The partial array (column-major, [W][ld] double-float pairs) is brought
    // into shared memory (the now idle tile stages) by one bulk copy, then
    // warps 0-6 sum it, two threads per column, double-float (TwoSum)
    // accumulation, halves combined by one shuffle.  Warp 7 meanwhile derives
    // the parameter-only gradient constants.
    const int c0 = FULL ? 0 : WMC;
    const int ncol = LY::W - c0;
    float2* sp = reinterpret_cast<float2*>(smem_raw);
    if (tid == 0) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_init(&bars[2], 1);
      mbar_fence_init();
      const uint32_t bytes = uint32_t(ncol) * uint32_t(a.ld) * 8u;
      mbar_arrive_expect_tx(&bars[2], bytes);
      bulk_g2s(sp, part + size_t(c0) * a.ld, bytes, &bars[2]);
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bars[2], 0, kWaitNs);
    if (__syncthreads_or(!ok) && tid == 0) atomicOr(a.err, 1);
    if (tid < 224) {
      // every lane of warps 0-6 runs the same number of iterations, so the
      // full-warp shuffle below is reached by all of them
      const int half_rows = (G + 1) / 2;
      for (int e0 = 0; e0 < 2 * ncol; e0 += 224) {
        const int e = e0 + tid;
        const bool act = e < 2 * ncol;
        const int c = e / 2, h = e & 1;
        float s = 0.f, er = 0.f;
        if (act) {
          const float2* col = sp + size_t(c) * a.ld;
          const int r0 = h * half_rows, r1 = h ? G : half_rows;
          for (int rb = r0; rb < r1; ++rb) {
            const float2 v = col[rb];
            float t, err;
            two_sum(s, v.x, t, err);
            s = t;
            er += err + v.y;
          }
        }
        const float so = __shfl_xor_sync(0xffffffffu, s, 1), eo = __shfl_xor_sync(0xffffffffu, er, 1);
        if (act && h == 0) {
          float t, err;
          two_sum(s, so, t, err);
          colsum[c0 + c] = double(t) + (double(er) + double(eo) + double(err));
        }
      }
    } else if (GRAD && FULL) {
      for (int r = tid - 224; r < NR; r += 32)
        kappa_derivatives(a.dm, r, cc.m0[r], cc.g0[r], cc.kappa[r], cc);
    }
    __syncthreads();
    for (int v = tid; v < WMC; v += blockDim.x) {
      if (FULL) a.gram_store[v] = colsum[v];
      else colsum[v] = a.gram_store[v];
    }
  }
  __syncthreads();
  if (trace && tid == 0) trace[5] = global_ns();
  __syncthreads();
  if (tid == 0) *a.counter = 0u;
  final_epilogue<S>(a, cc, colsum, GRAD, FULL && GRAD, trace);
  __syncthreads();
  if (trace && tid == 0) trace[7] = global_ns();
}

}  // namespace tdmix
