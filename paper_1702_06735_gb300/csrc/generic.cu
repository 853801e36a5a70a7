// Likelihood evaluation of amplitude models whose structure is not compiled
// into the library.
//
// The specialised kernel (fused.cuh) has the model structure - which
// lineshapes multiply into which term of which component - fixed at compile
// time, so every per-event array lives in registers.  A model with any
// other structure is evaluated here from the runtime tables of DevModel:
// the same quantities (Sec. 3: lineshapes, components with their spin and
// barrier factors and Bose orderings, the coherent sums A_f and Abar_f;
// Eq. (mix) with ln B; the Monte Carlo normalisation of Sec. 3.1 with the
// closed-form time integrals; the adjoint of all of it), in double
// precision whatever precision the context was created with.  Per-event
// arrays indexed through the tables live in thread-local memory, so this
// path is several times slower than a specialised one; it lets a user
// compose a model (Sec. 3) without rebuilding the library.  It also
// evaluates models with a decay-time resolution (resolution.cuh), an
// extension the paper leaves out.
//
// Two launches per evaluation, on the planes the kinematic precompute wrote
// (fp64 tile-major layout of SampleDev):
//   k_generic_tiles   one block per SM, 256 threads, one event per thread:
//                     block b takes the MC tiles mc_ranges[b] ..
//                     mc_ranges[b + 1] and the data tiles b, b + G, ...,
//                     and writes row b of the [G][W] double partial sums;
//   k_generic_finish  one block: sums the rows in block order (so results
//                     are bitwise repeatable) and forms N, the NLL and the
//                     gradient.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "fused.cuh"
#include "kernels.hpp"
#include "resolution.cuh"

namespace tdmix {
namespace {

constexpr int kGT = kTileEvents;  // threads per block = events per tile
constexpr int kGW = kGT / 32;
constexpr int kMaxNRE = kMaxComp * (kMaxComp + 1) / 2, kMaxNIM = kMaxComp * (kMaxComp - 1) / 2;
constexpr int kMaxWMC = 1 + kMaxNRE + kMaxNIM + 2 * kMaxRes;
constexpr int kMaxWD = 5 + 4 * kMaxComp + 2 * kMaxRes;
constexpr int kMaxW = kMaxWMC + kMaxWD;

// Column counts of a partial row: MC [sum w, Re S_jk (j <= k), Im S_jk
// (j < k), s1_r, s2_r], then data [sum ln B, n_bad, d/dx, d/dy, Re gA_j,
// Im gA_j, Re gB_j, Im gB_j, s1_r, s2_r, n recomputed (always 0 here)].
struct GWidths {
  int U, NR, NRE, NIM, WMC, WD, W;
  __host__ __device__ GWidths(int u, int nr)
      : U(u), NR(nr), NRE(u * (u + 1) / 2), NIM(u * (u - 1) / 2), WMC(1 + NRE + NIM + 2 * nr),
        WD(5 + 4 * u + 2 * nr), W(WMC + WD) {}
};

// Per-evaluation constants of one block (double precision).
struct GConst {
  int U, NO, NB, NR, NS, NX, NT, nc, np;
  int term_bw[kMaxTerms][2];
  int bw_res[kMaxBW], bw_splane[kMaxBW], bw_xplane[kMaxBW];
  double m2[kMaxRes], kappa[kMaxRes];
  double cA[kMaxComp][2], cB[kMaxComp][2];
  double alpha, beta, gc, dc;  // weights of the time-integrated rate (see finish_likelihood)
  BlockConst<double> bc;       // mixing constants read by mix_event
};

// kappa of resonance r, with m0 Gamma(s) = kappa X(s) and X(s) = q^(2L+1)
// F_L(q r)^2 / sqrt(s) the width plane of the precompute: kappa = m0^2
// Gamma0 / (q0^(2L+1) F_L(q0 r)^2) for a mass-dependent width (Sec. 3
// lineshapes), m0 Gamma0 for a constant one, 0 without a lineshape.
__device__ double generic_kappa(const ModelConst& km, int r, double m0, double g0) {
  const int shape = km.res_shape[r];
  if (shape == SHAPE_CONST) return m0 * g0;
  if (shape != SHAPE_MDW) return 0.0;
  const int L = km.res_L[r];
  const double u = m0 * m0;
  const double q02 = breakup2(u, km.res_ma[r] * km.res_ma[r], km.res_mb[r] * km.res_mb[r]);
  double qp = sqrt(q02);
  for (int l = 0; l < L; ++l) qp *= q02;
  const double F = barrier(L, q02 * km.r_res * km.r_res);
  return u * g0 / (qp * F * F);
}

// Derives the block's constants from the parameter vector (kernel
// parameters or device memory) and the structure tables.
__device__ void generic_derive(const EvalArgs& a, GConst& g) {
  const int tid = threadIdx.x;
  const DevModel& dm = *a.dm;
  const ModelConst& km = a.km;
  if (tid == 0) {
    g.U = dm.U;
    g.NO = dm.NO;
    g.NB = dm.NB;
    g.NR = dm.NR;
    g.NS = dm.NS;
    g.NX = dm.NX;
    g.NT = dm.U * dm.NO;
    g.nc = km.n_chains;
    g.np = km.n_params;
  }
  for (int t = tid; t < dm.U * dm.NO; t += kGT) {
    g.term_bw[t][0] = dm.term_bw[t][0];
    g.term_bw[t][1] = dm.term_bw[t][1];
  }
  for (int b = tid; b < dm.NB; b += kGT) {
    g.bw_res[b] = dm.bw_res[b];
    g.bw_splane[b] = dm.bw_splane[b];
    g.bw_xplane[b] = dm.bw_xplane[b];
  }
  for (int j = tid; j < kMaxComp; j += kGT) g.cA[j][0] = g.cA[j][1] = g.cB[j][0] = g.cB[j][1] = 0.0;
  __syncthreads();
  auto par = [&](int k) { return a.params ? a.params[k] : a.hp[k]; };
  const int nc = km.n_chains;
  if (tid < nc) {  // each (amplitude, component) has at most one chain
    const int j = km.chain_comp[tid];
    double(*dst)[2] = km.chain_amp[tid] == 0 ? g.cA : g.cB;
    dst[j][0] = par(2 * tid);
    dst[j][1] = par(2 * tid + 1);
  }
  if (tid >= 64 && tid < 64 + dm.NR) {
    const int r = tid - 64;
    const double m0 = par(2 * nc + 2 * r), g0 = par(2 * nc + 2 * r + 1);
    g.m2[r] = m0 * m0;
    g.kappa[r] = generic_kappa(km, r, m0, g0);
  }
  if (tid == 96) {
    const double x = par(2 * nc + 2 * dm.NR), y = par(2 * nc + 2 * dm.NR + 1);
    const double ia = 1.0 / (1.0 - y * y), ic = 1.0 / (1.0 + x * x);
    g.alpha = ia + ic;
    g.beta = (x * x + y * y) * ia * ic;
    g.gc = y * ia;
    g.dc = x * ic;
    const double gamma = km.gamma;
    g.bc.x = x;
    g.bc.y = y;
    g.bc.gamma = gamma;
    g.bc.hx = 0.5 * x * gamma;
    g.bc.hy = 0.5 * y * gamma;
    // decay-time limits of the mixing-series tiers (see mix_event)
    const double mg = fmax(fabs(x), fabs(y)) * gamma;
    const double ig = mg > 0 ? 1.0 / mg : INFINITY;
    g.bc.tlim[0] = static_cast<unsigned long long>(__double_as_longlong(0.04 * ig));
    g.bc.tlim[1] = static_cast<unsigned long long>(__double_as_longlong(0.2 * ig));
  }
  __syncthreads();
}

// One event's lineshapes BW_b = 1 / (m0^2 - s - i kappa X_b(s)) and
// components a_j = sum_o K_{j,o} prod_{b of (j,o)} BW_b from the planes of
// its tile (plane p of this event at pl[p * 256]).
struct GEvent {
  double bwr[kMaxBW], bwi[kMaxBW], xs[kMaxBW];
  double ar[kMaxComp], ai[kMaxComp];

  __device__ void eval(const GConst& g, const double* pl) {
    const int X0 = g.NS, K0 = g.NS + g.NX;
    for (int b = 0; b < g.NB; ++b) {
      const int r = g.bw_res[b], xp = g.bw_xplane[b];
      const double delta = g.m2[r] - pl[g.bw_splane[b] * kGT];
      const double X = xp >= 0 ? pl[(X0 + xp) * kGT] : 1.0;
      const double im = g.kappa[r] * X;
      const double inv = 1.0 / (delta * delta + im * im);
      bwr[b] = delta * inv;
      bwi[b] = im * inv;
      xs[b] = X;
    }
    for (int j = 0; j < g.U; ++j) {
      double sr = 0, si = 0;
      for (int o = 0; o < g.NO; ++o) {
        const int t = j * g.NO + o;
        const int b0 = g.term_bw[t][0], b1 = g.term_bw[t][1];
        const double K = pl[(K0 + t) * kGT];
        double pr = 1.0, pi = 0.0;
        if (b0 >= 0 && b1 >= 0) {
          pr = bwr[b0] * bwr[b1] - bwi[b0] * bwi[b1];
          pi = bwr[b0] * bwi[b1] + bwi[b0] * bwr[b1];
        } else if (b0 >= 0 || b1 >= 0) {
          const int bb = b0 >= 0 ? b0 : b1;
          pr = bwr[bb];
          pi = bwi[bb];
        }
        sr += K * pr;
        si += K * pi;
      }
      ar[j] = sr;
      ai[j] = si;
    }
  }

  __device__ void amplitudes(const GConst& g, double& Ar, double& Ai, double& Br, double& Bi) const {
    Ar = Ai = Br = Bi = 0;
    for (int j = 0; j < g.U; ++j) {
      cmac(Ar, Ai, g.cA[j][0], g.cA[j][1], ar[j], ai[j]);
      cmac(Br, Bi, g.cB[j][0], g.cB[j][1], ar[j], ai[j]);
    }
  }

  // Given gA = df/dA and gB = df/dAbar of a real f (df = 2 Re(gA dA + gB
  // dAbar)), adds wt sum_{b of r} Re(H_b) to s1[r] and wt sum_{b of r} X_b
  // Im(H_b) to s2[r], H_b = (df/dBW_b) BW_b^2 (then df/dm0 = -4 m0 s1 -
  // 2 dkappa/dm0 s2 and df/dGamma0 = -2 dkappa/dGamma0 s2).
  __device__ void backprop(const GConst& g, const double* pl, double gAr, double gAi, double gBr, double gBi,
                           double wt, double* s1, double* s2) const {
    double Gr[kMaxBW], Gi[kMaxBW];
    for (int b = 0; b < g.NB; ++b) Gr[b] = Gi[b] = 0;
    const int K0 = g.NS + g.NX;
    for (int j = 0; j < g.U; ++j) {
      double Wr = 0, Wi = 0;
      cmac(Wr, Wi, gAr, gAi, g.cA[j][0], g.cA[j][1]);
      cmac(Wr, Wi, gBr, gBi, g.cB[j][0], g.cB[j][1]);
      for (int o = 0; o < g.NO; ++o) {
        const int t = j * g.NO + o;
        const int b0 = g.term_bw[t][0], b1 = g.term_bw[t][1];
        if (b0 < 0 && b1 < 0) continue;
        const double K = pl[(K0 + t) * kGT];
        const double wr = K * Wr, wi = K * Wi;
        if (b0 >= 0 && b1 >= 0) {
          cmac(Gr[b0], Gi[b0], wr, wi, bwr[b1], bwi[b1]);
          cmac(Gr[b1], Gi[b1], wr, wi, bwr[b0], bwi[b0]);
        } else {
          const int bb = b0 >= 0 ? b0 : b1;
          Gr[bb] += wr;
          Gi[bb] += wi;
        }
      }
    }
    for (int b = 0; b < g.NB; ++b) {
      const int r = g.bw_res[b];
      const double qr = bwr[b] * bwr[b] - bwi[b] * bwi[b], qi = 2 * bwr[b] * bwi[b];
      const double Hr = Gr[b] * qr - Gi[b] * qi, Hi = Gr[b] * qi + Gi[b] * qr;
      s1[r] += wt * Hr;
      s2[r] += wt * xs[b] * Hi;
    }
  }
};

// Sums per-thread values v(c) of nq columns over the block into out[c]
// (shuffle trees in each warp, then the warp sums in warp order).  `red`
// is shared scratch of kGW * nq doubles.
template <class F>
__device__ void block_columns(int nq, F v, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < nq; ++c) {
    const double s = warp_sum(v(c));
    if (lane == 0) red[warp * nq + c] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nq; c += kGT) {
    double s = 0;
    for (int w = 0; w < kGW; ++w) s += red[w * nq + c];
    out[c] = s;
  }
  __syncthreads();
}

// PASS 0: MC and data tiles; with a background the data pass needs N first:
// PASS 1 runs the MC tiles only, k_generic_norm forms N, and PASS 2 the data
// tiles (each event's density (1 - f) R / N + f B_bkg).
template <bool GRAD, int PASS>
__global__ void __launch_bounds__(kGT, 1) k_generic_tiles(const __grid_constant__ EvalArgs a) {
  __shared__ GConst g;
  __shared__ double red[kGW * kMaxWD];
  __shared__ double row[kMaxW];
  extern __shared__ double xcomp[];  // [2U + 1][256]: re planes, im planes, weights of one MC tile
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x, G = gridDim.x;
  generic_derive(a, g);
  const GWidths wd(g.U, g.NR);
  const int U = g.U, NR = g.NR;
  const SampleDev& dmc = a.mc;
  const SampleDev& dd = a.data;

  // ---- MC tiles: normalisation sums and the adjoint of the time-integrated rate
  if (PASS != 2) {
    double sw = 0, s1[kMaxRes], s2[kMaxRes];
    for (int r = 0; r < NR; ++r) s1[r] = s2[r] = 0;
    // thread q < NRE + NIM owns sum entry q: Re S_jk over j <= k, then Im S_jk over j < k (row-major)
    const bool g_re = tid < wd.NRE;
    int gj = 0, gk = 0;
    {
      int rr = g_re ? tid : tid - wd.NRE;
      for (;;) {
        const int len = g_re ? U - gj : U - 1 - gj;
        if (rr < len || gj >= U) break;
        rr -= len;
        ++gj;
      }
      gk = g_re ? gj + rr : gj + 1 + rr;
    }
    double gacc = 0;
    const int npl = g.NS + g.NX + g.NT;
    for (int64_t tile = a.mc_ranges[b]; tile < a.mc_ranges[b + 1]; ++tile) {
      const double* pl = reinterpret_cast<const double*>(static_cast<const unsigned char*>(dmc.planes) +
                                                         tile * dmc.tile_bytes) + tid;
      const bool valid = tile * kGT + tid < dmc.n;
      GEvent ev;
      double w = 0;
      if (valid) {
        ev.eval(g, pl);
        w = dmc.weighted ? pl[npl * kGT] : 1.0;
        sw += w;
        if (GRAD) {
          double Ar, Ai, Br, Bi;
          ev.amplitudes(g, Ar, Ai, Br, Bi);
          // n = alpha |A|^2 + beta |Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*),
          // dn = 2 Re(uA dA + uB dAbar)
          const double uAr = g.alpha * Ar - g.gc * Br + g.dc * Bi;
          const double uAi = -g.alpha * Ai + g.gc * Bi + g.dc * Br;
          const double uBr = g.beta * Br - g.gc * Ar - g.dc * Ai;
          const double uBi = -g.beta * Bi + g.gc * Ai - g.dc * Ar;
          ev.backprop(g, pl, uAr, uAi, uBr, uBi, w, s1, s2);
        }
      } else {
        for (int j = 0; j < U; ++j) ev.ar[j] = ev.ai[j] = 0;
      }
      for (int j = 0; j < U; ++j) {
        xcomp[j * kGT + tid] = ev.ar[j];
        xcomp[(U + j) * kGT + tid] = ev.ai[j];
      }
      xcomp[2 * U * kGT + tid] = w;
      __syncthreads();
      if (tid < wd.NRE + wd.NIM) {
        const double* xj = xcomp + gj * kGT;
        const double* yj = xcomp + (U + gj) * kGT;
        const double* xk = xcomp + gk * kGT;
        const double* yk = xcomp + (U + gk) * kGT;
        const double* wt = xcomp + 2 * U * kGT;
        for (int e = 0; e < kGT; ++e)
          gacc += wt[e] * (g_re ? xj[e] * xk[e] + yj[e] * yk[e] : xj[e] * yk[e] - yj[e] * xk[e]);
      }
      __syncthreads();
    }
    const int nq = 1 + 2 * NR;
    block_columns(
        nq, [&](int c) { return c == 0 ? sw : (c <= NR ? s1[c - 1] : s2[c - 1 - NR]); }, red, red + kGW * nq);
    for (int c = tid; c < nq; c += kGT) row[c == 0 ? 0 : wd.NRE + wd.NIM + c] = red[kGW * nq + c];
    if (tid < wd.NRE + wd.NIM) row[1 + tid] = gacc;
    __syncthreads();
  }

  // ---- data tiles: ln B of Eq. (mix) and its adjoint (with a background:
  // ln of the mixture density and the adjoint weighted by the signal share)
  if (PASS != 1) {
    double lnb = 0, gx = 0, gy = 0, nbad = 0, sum_ws = 0;
    const double* part_in = static_cast<const double*>(a.part);
    const double Nsig = PASS == 2 ? part_in[size_t(G) * wd.W] : 0.0;  // N from k_generic_norm
    const double fb = a.km.bkg_fraction, taub = a.km.bkg_tau;
    int lexp = 0;
    double gAr[kMaxComp], gAi[kMaxComp], gBr[kMaxComp], gBi[kMaxComp], s1[kMaxRes], s2[kMaxRes];
    const double2* logtab = static_cast<const double2*>(a.logtab);
    for (int j = 0; j < U; ++j) gAr[j] = gAi[j] = gBr[j] = gBi[j] = 0;
    for (int r = 0; r < NR; ++r) s1[r] = s2[r] = 0;
    const int npl = g.NS + g.NX + g.NT;
    for (int64_t tile = b; tile < dd.n_tiles; tile += G) {
      const int64_t i = tile * kGT + tid;
      if (i >= dd.n) continue;
      const double* pl = reinterpret_cast<const double*>(static_cast<const unsigned char*>(dd.planes) +
                                                         tile * dd.tile_bytes) + tid;
      GEvent ev;
      ev.eval(g, pl);
      double Ar, Ai, Br, Bi, tAr, tAi, tBr, tBi;
      ev.amplitudes(g, Ar, Ai, Br, Bi);
      const double t_e = pl[npl * kGT];
      bool ok;
      double R = 0, gxe = 0, gye = 0;  // the event's rate and its d ln R / dx, d ln R / dy
      if (a.km.sigma_t > 0) {  // Eq. (mix) folded with the decay-time resolution: ln R, R with e^{-Gamma t}
        ok = resolved_rate<GRAD>(Ar, Ai, Br, Bi, t_e, g.bc.x, g.bc.y, g.bc.gamma, a.km.sigma_t, R, tAr, tAi, tBr,
                                 tBi, gxe, gye);
        if (ok && PASS == 0) lnb += log(R);
      } else {
        double lnb_e = 0;
        int lexp_e = 0;
        ok = mix_event<PrecF64, GRAD>(g.bc, logtab, Ar, Ai, Br, Bi, Ar, Ai, Br, Bi, t_e, lnb_e, lexp_e, &R, tAr, tAi,
                                      tBr, tBi, gxe, gye);
        if (ok && PASS == 0) {
          lnb += lnb_e;
          lexp += lexp_e;
        }
      }
      if (a.rates) a.rates[i] = R;
      double ws = 1.0;  // weight of the signal sensitivities: 1, or the signal share of the mixture
      if (PASS == 2 && ok) {
        // background density: e^{-t/tau_b} / tau_b in the true time, folded with the resolution if any
        double Bb;
        if (a.km.sigma_t > 0) {
          Cplx K, dK;
          fold_exp(t_e, Cplx{1.0 / taub, 0.0}, a.km.sigma_t, K, dK);
          Bb = K.re / taub;
        } else {
          Bb = t_e >= 0 ? exp(-t_e / taub) / taub : 0.0;
        }
        const double Ls = (1.0 - fb) * R / Nsig, L = Ls + fb * Bb;
        ok = L > 0 && L < INFINITY;
        if (ok) {
          lnb += log(L);
          ws = Ls / L;
          sum_ws += ws;
        }
      }
      if (!ok) {
        nbad += 1;
        continue;
      }
      if (GRAD) {
        gx += ws * gxe;
        gy += ws * gye;
        tAr *= ws;
        tAi *= ws;
        tBr *= ws;
        tBi *= ws;
        for (int j = 0; j < U; ++j) {
          cmac(gAr[j], gAi[j], tAr, tAi, ev.ar[j], ev.ai[j]);
          cmac(gBr[j], gBi[j], tBr, tBi, ev.ar[j], ev.ai[j]);
        }
        ev.backprop(g, pl, tAr, tAi, tBr, tBi, 1.0, s1, s2);
      }
    }
    const double lnb_t = fma(double(lexp), kLn2, lnb);
    const int nq = wd.WD - 1;  // all data columns but the recomputed count
    block_columns(
        nq,
        [&](int c) {
          if (c < 4) return c == 0 ? lnb_t : (c == 1 ? nbad : (c == 2 ? gx : gy));
          c -= 4;
          if (c < 4 * U) {
            const int q = c / U, j = c % U;
            return q == 0 ? gAr[j] : (q == 1 ? gAi[j] : (q == 2 ? gBr[j] : gBi[j]));
          }
          c -= 4 * U;
          return c < NR ? s1[c] : s2[c - NR];
        },
        red, row + wd.WMC);
    // the last data column: 0, or with a background the sum of the signal shares
    {
      const double v = warp_sum(sum_ws);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double sws = 0;
        for (int w = 0; w < kGW; ++w) sws += red[w];
        row[wd.W - 1] = PASS == 2 ? sws : 0.0;
      }
      __syncthreads();
    }
  }
  double* part = static_cast<double*>(a.part);
  for (int c = PASS == 2 ? wd.WMC + tid : tid; c < (PASS == 1 ? wd.WMC : wd.W); c += kGT) part[b * wd.W + c] = row[c];
}

// Sums the partial rows of G blocks in block order and writes the result
// vector [nll, N, n_bad or status, sum ln B, 0, grad...] (and the NLL and
// gradient to out_nll, out_grad when given), the MC column totals to
// gram_store.  The formulas are those of finish_likelihood:
//   N = tau <alpha |A|^2 + beta |Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*)>
//   NLL = -sum ln B + Gamma sum t + N_data ln N.
// mode 0: the result; mode 1 (background, between the MC and the data
// pass): only N, into part[G * W]; mode 2 (background, last): the result of
// the mixture, NLL = -sum ln((1 - f) R/N + f B), its normalisation term
// weighted by the sum of the events' signal shares instead of N_data.
__global__ void __launch_bounds__(kGT) k_generic_finish(const __grid_constant__ EvalArgs a, int G, int want_grad,
                                                        int mode) {
  __shared__ double col[kMaxW];
  __shared__ CtaConst cc;  // d ln kappa / d m0, d ln kappa / d Gamma0 (kappa_log_derivatives)
  const int tid = threadIdx.x;
  const DevModel& dm = *a.dm;
  const ModelConst& km = a.km;
  const GWidths wd(dm.U, dm.NR);
  const int U = dm.U, NR = dm.NR, nc = km.n_chains, np = km.n_params;
  const double* part = static_cast<const double*>(a.part);
  for (int c = tid; c < wd.W; c += kGT) {
    double s = 0;
    for (int q = 0; q < G; ++q) s += part[size_t(q) * wd.W + c];
    col[c] = s;
  }
  auto par = [&](int k) { return a.params ? a.params[k] : a.hp[k]; };
  if (tid < NR) {
    const double m0 = par(2 * nc + 2 * tid), g0 = par(2 * nc + 2 * tid + 1);
    if (m0 > 0 && g0 > 0) kappa_log_derivatives(km, tid, m0, g0, cc);
  }
  __syncthreads();
  if (mode != 1)
    for (int c = tid; c < wd.WMC; c += kGT) a.gram_store[c] = col[c];
  if (tid != 0) return;
  auto put = [&](int k, double v) {
    a.result[k] = v;
    if (k == 0 && a.out_nll) *a.out_nll = v;
    if (k >= kResHeader && a.out_grad) a.out_grad[k - kResHeader] = v;
  };
  // parameter screening (device parameter vectors are not screened on the host)
  int status = 0;
  for (int k = 0; k < np; ++k)
    if (!isfinite(par(k))) status = -5;
  if (status == 0) {
    for (int r = 0; r < NR; ++r) {
      if (km.res_shape[r] == SHAPE_NONE) continue;
      const double m0 = par(2 * nc + 2 * r), g0 = par(2 * nc + 2 * r + 1);
      if (!(m0 > 0 && g0 > 0)) status = -6;
      if (km.res_shape[r] == SHAPE_MDW) {
        const double u = m0 * m0, a2 = km.res_ma[r] * km.res_ma[r], b2 = km.res_mb[r] * km.res_mb[r];
        if (!(u * u + a2 * a2 + b2 * b2 - 2.0 * (u * a2 + u * b2 + a2 * b2) > 0)) status = -6;
      }
    }
    if (!(fabs(par(np - 1)) < 1.0)) status = -6;
    if (km.sigma_t > 0 && !(fabs(par(np - 2)) * km.gamma * km.sigma_t * 0.70710678118654752 <= kMaxResolutionMix))
      status = -6;
  }
  double* n_out = const_cast<double*>(part) + size_t(G) * wd.W;  // N for the data pass of a background
  if (status != 0) {
    if (mode == 1) *n_out = nan("");
    else
      for (int k = 0; k < kResHeader + np; ++k) put(k, k == 2 ? double(status) : nan(""));
    return;
  }
  double cA[kMaxComp][2] = {}, cB[kMaxComp][2] = {};
  for (int c = 0; c < nc; ++c) {
    double(*dst)[2] = km.chain_amp[c] == 0 ? cA : cB;
    dst[km.chain_comp[c]][0] = par(2 * c);
    dst[km.chain_comp[c]][1] = par(2 * c + 1);
  }
  const double x = par(2 * nc + 2 * NR), y = par(2 * nc + 2 * NR + 1), gamma = km.gamma;
  const double ia = 1.0 / (1.0 - y * y), ic = 1.0 / (1.0 + x * x);
  const double al = ia + ic, be = (x * x + y * y) * ia * ic, gc = y * ia, dc = x * ic;
  // S_jk = sum_e w_e a_j^* a_k (Hermitian) from the packed totals; v = S c
  auto s_at = [&](int j, int k, double& sr, double& si) {
    const int lo = j < k ? j : k, hi = j < k ? k : j;
    sr = col[1 + lo * U - lo * (lo - 1) / 2 + (hi - lo)];
    si = j == k ? 0.0 : col[1 + wd.NRE + lo * (U - 1) - lo * (lo - 1) / 2 + (hi - lo - 1)];
    if (j > k) si = -si;
  };
  double vA[kMaxComp][2], vB[kMaxComp][2];
  double AA = 0, BB = 0, Xr = 0, Xi = 0;
  for (int j = 0; j < U; ++j) {
    double ar = 0, ai = 0, br = 0, bi = 0;
    for (int k = 0; k < U; ++k) {
      double sr, si;
      s_at(j, k, sr, si);
      cmac(ar, ai, sr, si, cA[k][0], cA[k][1]);
      cmac(br, bi, sr, si, cB[k][0], cB[k][1]);
    }
    vA[j][0] = ar;
    vA[j][1] = ai;
    vB[j][0] = br;
    vB[j][1] = bi;
    AA += cA[j][0] * ar + cA[j][1] * ai;  // Re(cA^* vA)
    BB += cB[j][0] * br + cB[j][1] * bi;
    Xr += cB[j][0] * ar + cB[j][1] * ai;  // Re(cB^* vA)
    Xi += cB[j][0] * ai - cB[j][1] * ar;  // Im(cB^* vA)
  }
  const double inv_sw = a.inv_sum_w;
  const double nbar = (al * AA + be * BB - 2.0 * gc * Xr - 2.0 * dc * Xi) * inv_sw;
  const double N = nbar * km.tau;
  if (mode == 1) {
    *n_out = N;
    return;
  }
  const double* ds = col + wd.WMC;
  // the weight of d ln N: the number of data events, or with a background the sum of their signal shares
  const double Nd = mode == 2 ? ds[wd.WD - 1] : double(a.data.n);
  // sum ln B leaves out e^{-Gamma t}; the folded rates of a decay-time resolution include it; with a
  // background the data pass summed ln of the whole normalised density
  double nll = mode == 2 ? -ds[0] : -ds[0] + (km.sigma_t > 0 ? 0.0 : gamma * a.sum_t) + Nd * log(N);
  if (ds[1] > 0 || !(N > 0)) nll = nan("");
  put(0, nll);
  put(1, N);
  put(2, ds[1]);
  put(3, ds[0]);
  put(4, 0.0);
  if (!want_grad) return;
  const double sc = Nd / nbar * inv_sw;
  for (int ch = 0; ch < nc; ++ch) {
    const int j = km.chain_comp[ch];
    double dnr, dni, gr, gi;
    if (km.chain_amp[ch] == 0) {
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
    put(kResHeader + 2 * ch, km.floating[2 * ch] ? -(2 * gr) + sc * dnr : 0.0);
    put(kResHeader + 2 * ch + 1, km.floating[2 * ch + 1] ? 2 * gi + sc * dni : 0.0);
  }
  for (int r = 0; r < NR; ++r) {
    const double m0 = par(2 * nc + 2 * r), g0 = par(2 * nc + 2 * r + 1);
    const double kap = generic_kappa(km, r, m0, g0);
    const double dk_dm = kap * cc.dlk_dm[r], dk_dg = kap * cc.dlk_dg[r];
    const double* mcs = col;
    const double s1m = mcs[1 + wd.NRE + wd.NIM + r], s2m = mcs[1 + wd.NRE + wd.NIM + NR + r];
    const double s1d = ds[4 + 4 * U + r], s2d = ds[4 + 4 * U + NR + r];
    const double dm_n = -4 * m0 * s1m - 2 * dk_dm * s2m, dg_n = -2 * dk_dg * s2m;
    const double dm_d = -4 * m0 * s1d - 2 * dk_dm * s2d, dg_d = -2 * dk_dg * s2d;
    const int k = 2 * nc + 2 * r;
    put(kResHeader + k, km.floating[k] ? -dm_d + sc * dm_n : 0.0);
    put(kResHeader + k + 1, km.floating[k + 1] ? -dg_d + sc * dg_n : 0.0);
  }
  const double dal_dx = -2 * x * ic * ic, dal_dy = 2 * y * ia * ia;
  const double dbe_dx = 2 * x * ic * ic, dbe_dy = 2 * y * ia * ia;
  const double dgc_dy = (1 + y * y) * ia * ia, ddc_dx = (1 - x * x) * ic * ic;
  const double dn_dx = dal_dx * AA + dbe_dx * BB - 2 * ddc_dx * Xi;
  const double dn_dy = dal_dy * AA + dbe_dy * BB - 2 * dgc_dy * Xr;
  const int k = 2 * nc + 2 * NR;
  put(kResHeader + k, km.floating[k] ? -ds[2] + sc * dn_dx : 0.0);
  put(kResHeader + k + 1, km.floating[k + 1] ? -ds[3] + sc * dn_dy : 0.0);
}

int g_generic_smem_set[64] = {};
std::mutex g_generic_mu;

template <bool GRAD, int PASS>
cudaError_t launch_tiles(int grid, int smem, cudaStream_t st, const EvalArgs& a) {
  k_generic_tiles<GRAD, PASS><<<grid, kGT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PASS>
cudaError_t allow_tiles_smem(int smem) {
  cudaError_t e = cudaFuncSetAttribute(k_generic_tiles<true, PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_generic_tiles<false, PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

}  // namespace

// Launcher behind ShapeOps::eval for the generic path (every evaluation is
// a full one; `full` and `pdl` do not apply).
cudaError_t generic_eval(bool /*full*/, bool grad, int grid, bool /*pdl*/, cudaStream_t st, const EvalArgs& a) {
  // [2U + 1][256] doubles of one MC tile's components and weights, for the largest U
  const int smem = (2 * kMaxComp + 1) * kGT * int(sizeof(double));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    // the attribute acts per device: set once per device (every time beyond the table's devices)
    std::lock_guard<std::mutex> lk(g_generic_mu);
    const bool known = dev >= 0 && dev < 64;
    if (!known || !g_generic_smem_set[dev]) {
      if ((e = allow_tiles_smem<0>(smem)) || (e = allow_tiles_smem<1>(smem)) || (e = allow_tiles_smem<2>(smem)))
        return e;
      if (known) g_generic_smem_set[dev] = 1;
    }
  }
  if (a.km.bkg_fraction > 0) {  // MC pass, N, data pass with the mixture, result
    e = grad ? launch_tiles<true, 1>(grid, smem, st, a) : launch_tiles<false, 1>(grid, smem, st, a);
    if (e != cudaSuccess) return e;
    k_generic_finish<<<1, kGT, 0, st>>>(a, grid, 0, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = grad ? launch_tiles<true, 2>(grid, smem, st, a) : launch_tiles<false, 2>(grid, smem, st, a);
    if (e != cudaSuccess) return e;
    k_generic_finish<<<1, kGT, 0, st>>>(a, grid, grad ? 1 : 0, 2);
    return cudaGetLastError();
  }
  e = grad ? launch_tiles<true, 0>(grid, smem, st, a) : launch_tiles<false, 0>(grid, smem, st, a);
  if (e != cudaSuccess) return e;
  k_generic_finish<<<1, kGT, 0, st>>>(a, grid, grad ? 1 : 0, 0);
  return cudaGetLastError();
}

}  // namespace tdmix
