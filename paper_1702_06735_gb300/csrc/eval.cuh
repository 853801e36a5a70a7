// Per-event kernels of the likelihood, specialised at compile time on the
// structure of an amplitude model (its lineshape/term tables) and on the
// precision of the per-event arithmetic.
//
// One thread evaluates one event at a time (grid-stride loop):
//   lineshapes  BW_b = 1 / (m0^2 - s - i kappa_r X_b(s))      (Sec. 3, lineshapes)
//   components  a_j = sum_o K_{j,o} prod_{b in (j,o)} BW_b     (Sec. 3, chains with
//               form and spin factors K, Bose orderings o, recurring blocks shared)
//   amplitudes  A = sum_j cA_j a_j,  Abar = sum_j cB_j a_j     (Sec. 3, coherent sum)
//   data:       B = 2 |cosh(w) A - sinh(w) Abar|^2, w = (y + i x) Gamma t / 2,
//               which equals the right-hand side of Eq. (mix); ln B is summed
//   MC:         I_jk = <a_j^* a_k>, from which the normalisation of Sec. 3.1
//               with closed-form time integrals follows in the final kernel
//   adjoint:    d/d(c, x, y, m0, Gamma0) of ln B (data) and of the
//               time-integrated rate (MC), accumulated alongside.
// Block partials are written to one row per block and summed in a fixed
// order by the final kernel, so results are bitwise repeatable.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_tables.hpp"

namespace tdmix {

struct PrecF64 {
  using T = double;
  static constexpr bool kF32 = false;
};
struct PrecF32 {
  using T = float;
  static constexpr bool kF32 = true;
};

template <class T>
__device__ __forceinline__ T rcp(T v);
template <>
__device__ __forceinline__ double rcp<double>(double v) { return __drcp_rn(v); }
template <>
__device__ __forceinline__ float rcp<float>(float v) { return __frcp_rn(v); }

// Per-block copy of the per-evaluation constants in the working precision.
template <class T>
struct BlockConst {
  T m2[kMaxRes], m2_lo[kMaxRes], kappa[kMaxRes];
  T cA[kMaxComp][2], cB[kMaxComp][2];
  T alpha, beta, gc, dc;
  double x, y, gamma;
};

template <class P>
__device__ inline void load_block_const(const EvalConst* __restrict__ ec, int NR, int U,
                                        BlockConst<typename P::T>& bc) {
  int t = threadIdx.x;
  if (t < NR) {
    if constexpr (P::kF32) {
      bc.m2[t] = ec->m2_hi[t];
      bc.m2_lo[t] = ec->m2_lo[t];
      bc.kappa[t] = ec->kappa_f[t];
    } else {
      bc.m2[t] = ec->m2[t];
      bc.m2_lo[t] = 0;
      bc.kappa[t] = ec->kappa[t];
    }
  }
  if (t < U) {
    if constexpr (P::kF32) {
      bc.cA[t][0] = ec->cAf[t][0]; bc.cA[t][1] = ec->cAf[t][1];
      bc.cB[t][0] = ec->cBf[t][0]; bc.cB[t][1] = ec->cBf[t][1];
    } else {
      bc.cA[t][0] = ec->cA[t][0]; bc.cA[t][1] = ec->cA[t][1];
      bc.cB[t][0] = ec->cB[t][0]; bc.cB[t][1] = ec->cB[t][1];
    }
  }
  if (t == 0) {
    if constexpr (P::kF32) {
      bc.alpha = ec->alpha_f; bc.beta = ec->beta_f; bc.gc = ec->gc_f; bc.dc = ec->dc_f;
    } else {
      bc.alpha = ec->alpha; bc.beta = ec->beta; bc.gc = ec->gc; bc.dc = ec->dc;
    }
    bc.x = ec->x;
    bc.y = ec->y;
    bc.gamma = ec->gamma;
  }
}

// Warp + block tree reduction of NV doubles per thread into one row (fixed order).
template <int NV>
__device__ inline void block_reduce_row(double (&v)[NV], double* __restrict__ row, double* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) smem[warp * NV + k] = a;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += smem[w * NV + k];
    row[k] = a;
  }
}

template <class P, class S>
struct EventCore {
  using T = typename P::T;
  static constexpr int U = S::U, NO = S::NO, NB = S::NB, NR = S::NR;
  T bwr[NB > 0 ? NB : 1], bwi[NB > 0 ? NB : 1], xs[NB > 0 ? NB : 1];
  T ar[U], ai[U];

  __device__ __forceinline__ void lineshapes(const SampleDev& d, int64_t i, const BlockConst<T>& bc) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int r = S::bres(b), sp = S::bs(b), xp = S::bx(b);
      T delta;
      if constexpr (P::kF32) {
        const float* s = static_cast<const float*>(d.s);
        float hi = __ldg(s + sp * d.pitch + i);
        float lo = __ldg(s + (S::NS + sp) * d.pitch + i);
        delta = (bc.m2[r] - hi) + (bc.m2_lo[r] - lo);
      } else {
        const double* s = static_cast<const double*>(d.s);
        delta = bc.m2[r] - __ldg(s + sp * d.pitch + i);
      }
      T X = T(1);
      if (xp >= 0) X = __ldg(static_cast<const T*>(d.x) + xp * d.pitch + i);
      T im = bc.kappa[r] * X;
      T inv = rcp<T>(delta * delta + im * im);
      bwr[b] = delta * inv;
      bwi[b] = im * inv;
      xs[b] = X;
    }
  }

  __device__ __forceinline__ T kfac(const SampleDev& d, int t, int64_t i) const {
    return __ldg(static_cast<const T*>(d.k) + t * d.pitch + i);
  }

  __device__ __forceinline__ void components(const SampleDev& d, int64_t i) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      T sr = 0, si = 0;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const int t = j * NO + o;
        const int b0 = S::tb0(t), b1 = S::tb1(t);
        T K = kfac(d, t, i);
        T pr, pi;
        if (b0 >= 0 && b1 >= 0) {
          pr = bwr[b0] * bwr[b1] - bwi[b0] * bwi[b1];
          pi = bwr[b0] * bwi[b1] + bwi[b0] * bwr[b1];
        } else if (b0 >= 0) {
          pr = bwr[b0]; pi = bwi[b0];
        } else if (b1 >= 0) {
          pr = bwr[b1]; pi = bwi[b1];
        } else {
          pr = 1; pi = 0;
        }
        sr += K * pr;
        si += K * pi;
      }
      ar[j] = sr;
      ai[j] = si;
    }
  }

  __device__ __forceinline__ void amplitudes(const BlockConst<T>& bc, T& Ar, T& Ai, T& Br, T& Bi) const {
    Ar = Ai = Br = Bi = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      Ar += bc.cA[j][0] * ar[j] - bc.cA[j][1] * ai[j];
      Ai += bc.cA[j][0] * ai[j] + bc.cA[j][1] * ar[j];
      Br += bc.cB[j][0] * ar[j] - bc.cB[j][1] * ai[j];
      Bi += bc.cB[j][0] * ai[j] + bc.cB[j][1] * ar[j];
    }
  }

  // Given the holomorphic sensitivities gA = df/dA, gB = df/dAbar of a real
  // f (df = 2 Re(gA dA + gB dAbar)), accumulate per resonance
  //   s1_r += wt * sum_{b of r} Re(H_b),  s2_r += wt * sum_{b of r} X_b Im(H_b),
  // with H_b = (df/dBW_b) BW_b^2; then df/dm0 = -4 m0 s1 - 2 dkappa/dm0 s2 and
  // df/dGamma0 = -2 dkappa/dGamma0 s2 (the factor 2 Re already included).
  __device__ __forceinline__ void backprop_lineshapes(const SampleDev& d, int64_t i, const BlockConst<T>& bc,
                                                      T gAr, T gAi, T gBr, T gBi, T wt, T (&s1)[NR > 0 ? NR : 1],
                                                      T (&s2)[NR > 0 ? NR : 1]) const {
    if constexpr (NB > 0) {
      T Gr[NB], Gi[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) Gr[b] = Gi[b] = 0;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        // W_j = gA cA_j + gB cB_j
        T Wr = gAr * bc.cA[j][0] - gAi * bc.cA[j][1] + gBr * bc.cB[j][0] - gBi * bc.cB[j][1];
        T Wi = gAr * bc.cA[j][1] + gAi * bc.cA[j][0] + gBr * bc.cB[j][1] + gBi * bc.cB[j][0];
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          const int t = j * NO + o;
          const int b0 = S::tb0(t), b1 = S::tb1(t);
          if (b0 < 0 && b1 < 0) continue;
          T K = kfac(d, t, i);
          T wr = K * Wr, wi = K * Wi;
          if (b0 >= 0 && b1 >= 0) {
            Gr[b0] += wr * bwr[b1] - wi * bwi[b1];
            Gi[b0] += wr * bwi[b1] + wi * bwr[b1];
            Gr[b1] += wr * bwr[b0] - wi * bwi[b0];
            Gi[b1] += wr * bwi[b0] + wi * bwr[b0];
          } else {
            const int bb = b0 >= 0 ? b0 : b1;
            Gr[bb] += wr;
            Gi[bb] += wi;
          }
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int r = S::bres(b);
        T qr = bwr[b] * bwr[b] - bwi[b] * bwi[b];
        T qi = 2 * bwr[b] * bwi[b];
        T Hr = Gr[b] * qr - Gi[b] * qi;
        T Hi = Gr[b] * qi + Gi[b] * qr;
        s1[r] += wt * Hr;
        s2[r] += wt * xs[b] * Hi;
      }
    }
  }
};

// MC kernel: Gram matrix I_jk (upper triangle), sum of weights and, when
// GRAD, the resonance-parameter sensitivities of the time-integrated rate.
// Row: [sum w, Re I (j<=k), Im I (j<k), s1 (NR), s2 (NR)].
template <class P, class S, bool GRAD>
__global__ void __launch_bounds__(256) k_mc(SampleDev d, const EvalConst* __restrict__ ec,
                                            double* __restrict__ rows) {
  using T = typename P::T;
  constexpr int U = S::U, NR = S::NR;
  constexpr int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  constexpr int NV = 1 + NRE + NIM + 2 * NR;
  __shared__ BlockConst<T> bc;
  __shared__ double red[8 * NV];
  load_block_const<P>(ec, NR, U, bc);
  __syncthreads();

  T sw = 0, gre[NRE], gim[NIM > 0 ? NIM : 1];
  T s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
  for (int k = 0; k < NRE; ++k) gre[k] = 0;
#pragma unroll
  for (int k = 0; k < (NIM > 0 ? NIM : 1); ++k) gim[k] = 0;
#pragma unroll
  for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;

  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < d.n; i += stride) {
    EventCore<P, S> ev;
    ev.lineshapes(d, i, bc);
    ev.components(d, i);
    T w = d.w ? __ldg(static_cast<const T*>(d.w) + i) : T(1);
    sw += w;
    int kr = 0, ki = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      T wr = w * ev.ar[j], wi = w * ev.ai[j];
#pragma unroll
      for (int k = j; k < U; ++k) {
        gre[kr++] += wr * ev.ar[k] + wi * ev.ai[k];
        if (k > j) gim[ki++] += wr * ev.ai[k] - wi * ev.ar[k];
      }
    }
    if constexpr (GRAD) {
      T Ar, Ai, Br, Bi;
      ev.amplitudes(bc, Ar, Ai, Br, Bi);
      // n = alpha|A|^2 + beta|Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*);
      // dn = 2 Re(uA dA + uB dAbar), uA = alpha A* - (gc - i dc) Abar*,
      // uB = beta Abar* - (gc + i dc) A*.
      T uAr = bc.alpha * Ar - bc.gc * Br + bc.dc * Bi;
      T uAi = -bc.alpha * Ai + bc.gc * Bi + bc.dc * Br;
      T uBr = bc.beta * Br - bc.gc * Ar - bc.dc * Ai;
      T uBi = -bc.beta * Bi + bc.gc * Ai - bc.dc * Ar;
      ev.backprop_lineshapes(d, i, bc, uAr, uAi, uBr, uBi, w, s1, s2);
    }
  }

  double v[NV];
  v[0] = double(sw);
#pragma unroll
  for (int k = 0; k < NRE; ++k) v[1 + k] = double(gre[k]);
#pragma unroll
  for (int k = 0; k < NIM; ++k) v[1 + NRE + k] = double(gim[k]);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    v[1 + NRE + NIM + r] = double(s1[r]);
    v[1 + NRE + NIM + NR + r] = double(s2[r]);
  }
  block_reduce_row<NV>(v, rows + size_t(blockIdx.x) * NV, red);
}

// Data kernel.  FROM_CACHE reads the components a_j stored by an earlier
// pass instead of recomputing them (parameters other than masses and widths
// moved).  GRAD accumulates d ln B / d(theta).  Optional per-event output:
// rate e^{-Gamma t} B.
// Row: [sum ln B, n_bad, d/dx, d/dy, Re gA (U), Im gA (U), Re gB (U), Im gB (U),
//       s1 (NR), s2 (NR)] where gA_j = sum_e (d ln B/dA) a_j.
template <class P, class S, bool FROM_CACHE, bool GRAD>
__global__ void __launch_bounds__(256) k_data(SampleDev d, const EvalConst* __restrict__ ec,
                                              double* __restrict__ rows, double* __restrict__ rates) {
  using T = typename P::T;
  constexpr int U = S::U, NR = S::NR;
  constexpr int NRG = (GRAD && !FROM_CACHE) ? NR : 0;
  constexpr int NV = 4 + 4 * U + 2 * NR;
  __shared__ BlockConst<T> bc;
  __shared__ double red[8 * NV];
  load_block_const<P>(ec, NR, U, bc);
  __syncthreads();

  double lnb = 0, bad = 0, gx = 0, gy = 0;
  T gAr[U], gAi[U], gBr[U], gBi[U];
  T s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
  for (int j = 0; j < U; ++j) gAr[j] = gAi[j] = gBr[j] = gBi[j] = 0;
#pragma unroll
  for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;

  T* cache = static_cast<T*>(d.cache);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < d.n; i += stride) {
    EventCore<P, S> ev;
    if constexpr (FROM_CACHE) {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        ev.ar[j] = __ldg(cache + j * d.pitch + i);
        ev.ai[j] = __ldg(cache + (U + j) * d.pitch + i);
      }
    } else {
      ev.lineshapes(d, i, bc);
      ev.components(d, i);
#pragma unroll
      for (int j = 0; j < U; ++j) {
        cache[j * d.pitch + i] = ev.ar[j];
        cache[(U + j) * d.pitch + i] = ev.ai[j];
      }
    }
    T Ar_, Ai_, Br_, Bi_;
    ev.amplitudes(bc, Ar_, Ai_, Br_, Bi_);
    // Eq. (mix) in its factorised form, in double precision.
    const double Ar = Ar_, Ai = Ai_, Br = Br_, Bi = Bi_;
    const double gt = bc.gamma * __ldg(d.t + i);
    const double ha = 0.5 * bc.y * gt, hb = 0.5 * bc.x * gt;
    double sb, cb;
    sincos(hb, &sb, &cb);
    const double cha = cosh(ha), sha = sinh(ha);
    const double chr = cha * cb, chi = sha * sb;   // cosh(w)
    const double shr = sha * cb, shi = cha * sb;   // sinh(w)
    const double Zr = chr * Ar - chi * Ai - (shr * Br - shi * Bi);
    const double Zi = chr * Ai + chi * Ar - (shr * Bi + shi * Br);
    const double z2 = Zr * Zr + Zi * Zi;
    const double B = 2.0 * z2;
    const bool ok = B > 0.0 && B < INFINITY;
    if (rates) rates[i] = exp(-gt) * B;
    if (!ok) {
      bad += 1.0;
      continue;
    }
    lnb += log(B);
    if constexpr (GRAD) {
      // d ln B = 2 Re(V dZ), V = Z* / |Z|^2; dZ = cosh(w) dA - sinh(w) dAbar
      // + (sinh(w) A - cosh(w) Abar) dw, dw/dy = Gamma t / 2, dw/dx = i Gamma t / 2.
      const double iz = 1.0 / z2;
      const double Vr = Zr * iz, Vi = -Zi * iz;
      const double pAr = Vr * chr - Vi * chi, pAi = Vr * chi + Vi * chr;
      const double pBr = -(Vr * shr - Vi * shi), pBi = -(Vr * shi + Vi * shr);
      const double Dr = shr * Ar - shi * Ai - (chr * Br - chi * Bi);
      const double Di = shr * Ai + shi * Ar - (chr * Bi + chi * Br);
      const double VDr = Vr * Dr - Vi * Di, VDi = Vr * Di + Vi * Dr;
      gy += gt * VDr;
      gx -= gt * VDi;
      const T tAr = T(pAr), tAi = T(pAi), tBr = T(pBr), tBi = T(pBi);
#pragma unroll
      for (int j = 0; j < U; ++j) {
        gAr[j] += tAr * ev.ar[j] - tAi * ev.ai[j];
        gAi[j] += tAr * ev.ai[j] + tAi * ev.ar[j];
        gBr[j] += tBr * ev.ar[j] - tBi * ev.ai[j];
        gBi[j] += tBr * ev.ai[j] + tBi * ev.ar[j];
      }
      if constexpr (NRG > 0) ev.backprop_lineshapes(d, i, bc, tAr, tAi, tBr, tBi, T(1), s1, s2);
    }
  }

  double v[NV];
  v[0] = lnb;
  v[1] = bad;
  v[2] = gx;
  v[3] = gy;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    v[4 + j] = double(gAr[j]);
    v[4 + U + j] = double(gAi[j]);
    v[4 + 2 * U + j] = double(gBr[j]);
    v[4 + 3 * U + j] = double(gBi[j]);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    v[4 + 4 * U + r] = double(s1[r]);
    v[4 + 4 * U + NR + r] = double(s2[r]);
  }
  block_reduce_row<NV>(v, rows + size_t(blockIdx.x) * NV, red);
}

}  // namespace tdmix
