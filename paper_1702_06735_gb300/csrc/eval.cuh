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

#include "async_copy.cuh"
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
// MUFU reciprocal refined by one Newton-Raphson step r + r (1 - v r):
// relative error ~ (2^-22)^2 before the final rounding, i.e. within an ulp
// of the correctly rounded reciprocal, for positive normal v.
template <>
__device__ __forceinline__ float rcp<float>(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  const float e = fmaf(-v, r, 1.0f);
  return fmaf(r, e, r);
}

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

// cosh, sinh of a and cos, sin of b.  For |a|, |b| <= 0.1 (the mixing
// arguments y Gamma t / 2, x Gamma t / 2 of every event with t below ~40
// lifetimes at percent-level x, y) the Maclaurin series truncated after the
// z^5 term (z = a^2 or b^2) is used: the first omitted term is below 3e-21
// relative.  Otherwise the CUDA math library is called.
__device__ __forceinline__ void mixing_trig(double a, double b, double& cha, double& sha, double& cb, double& sb) {
  if (fabs(a) <= 0.1 && fabs(b) <= 0.1) {
    const double za = a * a, zb = b * b;
    cha = 1.0 + za * (1.0 / 2 + za * (1.0 / 24 + za * (1.0 / 720 + za * (1.0 / 40320 + za * (1.0 / 3628800)))));
    sha = a * (1.0 + za * (1.0 / 6 + za * (1.0 / 120 + za * (1.0 / 5040 + za * (1.0 / 362880 + za * (1.0 / 39916800))))));
    cb = 1.0 - zb * (1.0 / 2 - zb * (1.0 / 24 - zb * (1.0 / 720 - zb * (1.0 / 40320 - zb * (1.0 / 3628800)))));
    sb = b * (1.0 - zb * (1.0 / 6 - zb * (1.0 / 120 - zb * (1.0 / 5040 - zb * (1.0 / 362880 - zb * (1.0 / 39916800))))));
  } else {
    cha = cosh(a);
    sha = sinh(a);
    sincos(b, &sb, &cb);
  }
}

// Reduces, per block, ND double and NT working-precision values per thread
// (warp shuffle tree, then the warps' partials summed in double in warp
// order) and stores them column-major: value v of block b goes to
// part[v * ld + b].  Fixed order, so results are bitwise repeatable.
template <class T, int ND, int NT>
__device__ inline void block_reduce_store(const double (&vd)[ND > 0 ? ND : 1], const T (&vt)[NT > 0 ? NT : 1],
                                          double* __restrict__ part, int64_t ld, double* smem) {
  constexpr int NV = ND + NT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    double a = vd[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) smem[warp * NV + k] = a;
  }
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    T a = vt[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) smem[warp * NV + ND + k] = double(a);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += smem[w * NV + k];
    part[k * ld + blockIdx.x] = a;
  }
}

// acc += a * b for complex numbers held as (re, im) pairs.
template <class T>
__device__ __forceinline__ void cmac(T& accr, T& acci, T ar, T ai, T br, T bi) {
  accr = fma(ar, br, accr);
  accr = fma(-ai, bi, accr);
  acci = fma(ar, bi, acci);
  acci = fma(ai, br, acci);
}

// Where one event's precomputed planes are read from.  Plane numbering:
// invariants (fp32: hi planes then lo planes), width factors X, spin x
// barrier factors K, then the optional MC weight.
template <class P, class S>
struct Planes {
  static constexpr int NSP = P::kF32 ? 2 * S::NS : S::NS;
  static constexpr int X0 = NSP, K0 = NSP + S::NX, W0 = NSP + S::NX + S::U * S::NO;
};

template <class P, class S>
struct GlobalSrc {
  using T = typename P::T;
  const SampleDev& d;
  int64_t i;
  __device__ __forceinline__ T s_hi(int sp) const {
    return __ldg(static_cast<const T*>(d.s) + sp * d.pitch + i);
  }
  __device__ __forceinline__ T s_lo(int sp) const {
    return __ldg(static_cast<const T*>(d.s) + (S::NS + sp) * d.pitch + i);
  }
  __device__ __forceinline__ T x(int xp) const { return __ldg(static_cast<const T*>(d.x) + xp * d.pitch + i); }
  __device__ __forceinline__ T k(int t) const { return __ldg(static_cast<const T*>(d.k) + t * d.pitch + i); }
  __device__ __forceinline__ T w() const { return d.w ? __ldg(static_cast<const T*>(d.w) + i) : T(1); }
};

template <class P, class S, int TE>
struct SmemSrc {
  using T = typename P::T;
  using L = Planes<P, S>;
  const T* base;  // this stage; plane p at base[p * TE]
  int tid;
  bool weighted;
  __device__ __forceinline__ T s_hi(int sp) const { return base[sp * TE + tid]; }
  __device__ __forceinline__ T s_lo(int sp) const { return base[(S::NS + sp) * TE + tid]; }
  __device__ __forceinline__ T x(int xp) const { return base[(L::X0 + xp) * TE + tid]; }
  __device__ __forceinline__ T k(int t) const { return base[(L::K0 + t) * TE + tid]; }
  __device__ __forceinline__ T w() const { return weighted ? base[L::W0 * TE + tid] : T(1); }
};

template <class P, class S>
struct EventCore {
  using T = typename P::T;
  static constexpr int U = S::U, NO = S::NO, NB = S::NB, NR = S::NR;
  T bwr[NB > 0 ? NB : 1], bwi[NB > 0 ? NB : 1], xs[NB > 0 ? NB : 1];
  T ar[U], ai[U];

  template <class Src>
  __device__ __forceinline__ void lineshapes(const Src& src, const BlockConst<T>& bc) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int r = S::bres(b), sp = S::bs(b), xp = S::bx(b);
      T delta;
      if constexpr (P::kF32) {
        delta = (bc.m2[r] - src.s_hi(sp)) + (bc.m2_lo[r] - src.s_lo(sp));
      } else {
        delta = bc.m2[r] - src.s_hi(sp);
      }
      T X = T(1);
      if (xp >= 0) X = src.x(xp);
      T im = bc.kappa[r] * X;
      T inv = rcp<T>(fma(delta, delta, im * im));
      bwr[b] = delta * inv;
      bwi[b] = im * inv;
      xs[b] = X;
    }
  }

  template <class Src>
  __device__ __forceinline__ void components(const Src& src) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      T sr = 0, si = 0;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const int t = j * NO + o;
        const int b0 = S::tb0(t), b1 = S::tb1(t);
        T K = src.k(t);
        T pr, pi;
        if (b0 >= 0 && b1 >= 0) {
          pr = fma(bwr[b0], bwr[b1], -bwi[b0] * bwi[b1]);
          pi = fma(bwr[b0], bwi[b1], bwi[b0] * bwr[b1]);
        } else if (b0 >= 0) {
          pr = bwr[b0]; pi = bwi[b0];
        } else if (b1 >= 0) {
          pr = bwr[b1]; pi = bwi[b1];
        } else {
          pr = 1; pi = 0;
        }
        sr = fma(K, pr, sr);
        si = fma(K, pi, si);
      }
      ar[j] = sr;
      ai[j] = si;
    }
  }

  __device__ __forceinline__ void amplitudes(const BlockConst<T>& bc, T& Ar, T& Ai, T& Br, T& Bi) const {
    Ar = Ai = Br = Bi = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      cmac(Ar, Ai, bc.cA[j][0], bc.cA[j][1], ar[j], ai[j]);
      cmac(Br, Bi, bc.cB[j][0], bc.cB[j][1], ar[j], ai[j]);
    }
  }

  // Given the holomorphic sensitivities gA = df/dA, gB = df/dAbar of a real
  // f (df = 2 Re(gA dA + gB dAbar)), accumulate per resonance
  //   s1_r += wt * sum_{b of r} Re(H_b),  s2_r += wt * sum_{b of r} X_b Im(H_b),
  // with H_b = (df/dBW_b) BW_b^2; then df/dm0 = -4 m0 s1 - 2 dkappa/dm0 s2 and
  // df/dGamma0 = -2 dkappa/dGamma0 s2 (the factor 2 Re already included).
  template <bool WEIGHTED, class Src>
  __device__ __forceinline__ void backprop_lineshapes(const Src& src, const BlockConst<T>& bc,
                                                      T gAr, T gAi, T gBr, T gBi, T wt, T (&s1)[NR > 0 ? NR : 1],
                                                      T (&s2)[NR > 0 ? NR : 1]) const {
    if constexpr (NB > 0) {
      T Gr[NB], Gi[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) Gr[b] = Gi[b] = 0;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        // W_j = gA cA_j + gB cB_j
        T Wr = 0, Wi = 0;
        cmac(Wr, Wi, gAr, gAi, bc.cA[j][0], bc.cA[j][1]);
        cmac(Wr, Wi, gBr, gBi, bc.cB[j][0], bc.cB[j][1]);
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          const int t = j * NO + o;
          const int b0 = S::tb0(t), b1 = S::tb1(t);
          if (b0 < 0 && b1 < 0) continue;
          T K = src.k(t);
          T wr = K * Wr, wi = K * Wi;
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
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int r = S::bres(b);
        const T qr = fma(bwr[b], bwr[b], -bwi[b] * bwi[b]);
        const T qi = 2 * bwr[b] * bwi[b];
        const T Hr = fma(Gr[b], qr, -Gi[b] * qi);
        const T Hi = fma(Gr[b], qi, Gi[b] * qr);
        if (WEIGHTED) {
          s1[r] = fma(wt, Hr, s1[r]);
          s2[r] = fma(wt * xs[b], Hi, s2[r]);
        } else {
          s1[r] += Hr;
          s2[r] = fma(xs[b], Hi, s2[r]);
        }
      }
    }
  }
};

// MC kernel: Gram matrix I_jk (upper triangle), sum of weights and, when
// GRAD, the resonance-parameter sensitivities of the time-integrated rate.
// Row: [sum w, Re I (j<=k), Im I (j<k), s1 (NR), s2 (NR)].
// Persistent: block b takes tiles b, b + grid, ... of kMcTile events; each
// tile's planes are brought into shared memory by bulk asynchronous copies
// (one per plane) completing on an mbarrier, two stages deep, so the copy of
// tile k+2 overlaps the arithmetic of tile k.
constexpr int kMcTile = 256;

template <class P, class S>
__host__ __device__ constexpr int mc_planes(bool weighted) {
  return Planes<P, S>::W0 + (weighted ? 1 : 0);
}

template <class P, class S, bool GRAD, bool WEIGHTED>
__global__ void __launch_bounds__(kMcTile, 1) k_mc(SampleDev d, const EvalConst* __restrict__ ec,
                                                   double* __restrict__ part, int64_t ld, int* __restrict__ err) {
  using T = typename P::T;
  using L = Planes<P, S>;
  constexpr int TE = kMcTile;
  constexpr int U = S::U, NR = S::NR;
  constexpr int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  constexpr int NV = 1 + NRE + NIM + 2 * NR;
  extern __shared__ __align__(1024) unsigned char tile_smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ BlockConst<T> bc;
  __shared__ double red[8 * NV];
  const int tid = threadIdx.x;
  constexpr bool weighted = WEIGHTED;
  const int npl = L::W0 + (weighted ? 1 : 0);
  const uint32_t stage_elems = uint32_t(npl) * TE;
  T* stage[2] = {reinterpret_cast<T*>(tile_smem), reinterpret_cast<T*>(tile_smem) + stage_elems};
  const int64_t n_tiles = (d.n + TE - 1) / TE;
  const int64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  load_block_const<P>(ec, NR, U, bc);
  __syncthreads();

  auto plane_src = [&](int p, int64_t tile) -> const T* {
    const int64_t off = tile * TE;
    if (p < L::X0) return static_cast<const T*>(d.s) + p * d.pitch + off;
    if (p < L::K0) return static_cast<const T*>(d.x) + (p - L::X0) * d.pitch + off;
    if (p < L::W0) return static_cast<const T*>(d.k) + (p - L::K0) * d.pitch + off;
    return static_cast<const T*>(d.w) + off;
  };
  auto issue = [&](int64_t k) {
    const int st = int(k & 1);
    const int64_t tile = blockIdx.x + k * gridDim.x;
    mbar_arrive_expect_tx(&bars[st], stage_elems * uint32_t(sizeof(T)));
    for (int p = 0; p < npl; ++p)
      bulk_g2s(stage[st] + p * TE, plane_src(p, tile), TE * uint32_t(sizeof(T)), &bars[st]);
  };
  if (tid == 0) {
    if (my_tiles > 0) issue(0);
    if (my_tiles > 1) issue(1);
  }

  T sw = 0, gre[NRE], gim[NIM > 0 ? NIM : 1];
  T s1[NR > 0 ? NR : 1], s2[NR > 0 ? NR : 1];
#pragma unroll
  for (int k = 0; k < NRE; ++k) gre[k] = 0;
#pragma unroll
  for (int k = 0; k < (NIM > 0 ? NIM : 1); ++k) gim[k] = 0;
#pragma unroll
  for (int r = 0; r < (NR > 0 ? NR : 1); ++r) s1[r] = s2[r] = 0;

  int64_t k = 0;
  for (; k < my_tiles; ++k) {
    const int st = int(k & 1);
    const bool ok = mbar_wait_bounded(&bars[st], uint32_t((k >> 1) & 1), 1000000000ull);
    if (__syncthreads_or(!ok)) break;
    const int64_t i = (blockIdx.x + k * gridDim.x) * TE + tid;
    if (i < d.n) {
      const SmemSrc<P, S, TE> src{stage[st], tid, weighted};
      EventCore<P, S> ev;
      ev.lineshapes(src, bc);
      ev.components(src);
      const T w = src.w();
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
        T uAr = bc.alpha * Ar - bc.gc * Br + bc.dc * Bi;
        T uAi = -bc.alpha * Ai + bc.gc * Bi + bc.dc * Br;
        T uBr = bc.beta * Br - bc.gc * Ar - bc.dc * Ai;
        T uBi = -bc.beta * Bi + bc.gc * Ai - bc.dc * Ar;
        ev.template backprop_lineshapes<WEIGHTED>(src, bc, uAr, uAi, uBr, uBi, w, s1, s2);
      }
    }
    __syncthreads();  // stage st fully consumed
    if (tid == 0 && k + 2 < my_tiles) issue(k + 2);
  }
  if (k < my_tiles) {
    // a copy did not arrive in time: report, let copies in flight land, stop
    if (tid == 0) {
      atomicOr(err, 1);
      for (int64_t q = k; q < my_tiles && q < k + 2; ++q)
        mbar_wait_bounded(&bars[q & 1], uint32_t((q >> 1) & 1), 1000000000ull);
    }
    __syncthreads();
  }

  double vd[1] = {0.0};
  T vt[NV];
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
  block_reduce_store<T, 0, NV>(vd, vt, part, ld, red);
}

// Data kernel.  FROM_CACHE reads the components a_j stored by an earlier
// pass instead of recomputing them (parameters other than masses and widths
// moved).  GRAD accumulates d ln B / d(theta).  Optional per-event output:
// rate e^{-Gamma t} B.
// Row: [sum ln B, n_bad, d/dx, d/dy, Re gA (U), Im gA (U), Re gB (U), Im gB (U),
//       s1 (NR), s2 (NR)] where gA_j = sum_e (d ln B/dA) a_j.
constexpr int kDataThreads = 128;

template <class P, class S, bool FROM_CACHE, bool GRAD>
__global__ void __launch_bounds__(kDataThreads) k_data(SampleDev d, const EvalConst* __restrict__ ec,
                                                       double* __restrict__ part, int64_t ld,
                                                       double* __restrict__ rates) {
  using T = typename P::T;
  constexpr int U = S::U, NR = S::NR;
  constexpr int NRG = (GRAD && !FROM_CACHE) ? NR : 0;
  constexpr int NV = 4 + 4 * U + 2 * NR;
  __shared__ BlockConst<T> bc;
  __shared__ double red[8 * NV];
  load_block_const<P>(ec, NR, U, bc);
  __syncthreads();

  double lnb = 0, bad = 0;
  T gx = 0, gy = 0;
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
      const GlobalSrc<P, S> src{d, i};
      ev.lineshapes(src, bc);
      ev.components(src);
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
    double cha, sha, cb, sb;
    mixing_trig(ha, hb, cha, sha, cb, sb);
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
      // Sensitivities in the working precision.
      const T iz = rcp<T>(T(z2));
      const T Vr = T(Zr) * iz, Vi = -T(Zi) * iz;
      const T cr = T(chr), ci = T(chi), sr = T(shr), si = T(shi);
      const T tAr = fma(Vr, cr, -Vi * ci), tAi = fma(Vr, ci, Vi * cr);
      const T tBr = -fma(Vr, sr, -Vi * si), tBi = -fma(Vr, si, Vi * sr);
      T Dr = 0, Di = 0;
      cmac(Dr, Di, sr, si, Ar_, Ai_);
      cmac(Dr, Di, -cr, -ci, Br_, Bi_);
      const T tg = T(gt);
      gy = fma(tg, fma(Vr, Dr, -Vi * Di), gy);
      gx = fma(-tg, fma(Vr, Di, Vi * Dr), gx);
#pragma unroll
      for (int j = 0; j < U; ++j) {
        cmac(gAr[j], gAi[j], tAr, tAi, ev.ar[j], ev.ai[j]);
        cmac(gBr[j], gBi[j], tBr, tBi, ev.ar[j], ev.ai[j]);
      }
      if constexpr (NRG > 0)
        ev.template backprop_lineshapes<false>(GlobalSrc<P, S>{d, i}, bc, tAr, tAi, tBr, tBi, T(1), s1, s2);
    }
  }

  const double vd[2] = {lnb, bad};
  T vt[NV - 2];
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
  block_reduce_store<T, 2, NV - 2>(vd, vt, part, ld, red);
}

}  // namespace tdmix
