// Per-event building blocks of the likelihood kernels, specialised at
// compile time on the structure of an amplitude model (its lineshape/term
// tables) and on the precision of the per-event arithmetic.
//
// One thread evaluates one event at a time:
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
// Every sum is formed in a fixed order, so results are bitwise repeatable.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "device_tables.hpp"
#include "df.cuh"

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
// Hardware reciprocal approximation refined by two Newton-Raphson steps
// r <- r + r (1 - v r): each step squares the relative error, so from the
// approximation's ~2^-23 the result is within an ulp or two of 1/v (not
// correctly rounded), for positive normal v.
template <>
__device__ __forceinline__ double rcp<double>(double v) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
  double e = fma(-v, r, 1.0);
  r = fma(r, e, r);
  e = fma(-v, r, 1.0);
  return fma(r, e, r);
}
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

// The reciprocal of a lineshape's denominator: in fp32 the hardware
// approximation alone (rcp.approx.ftz.f32, within one ulp of the correctly
// rounded reciprocal for positive normal v, measured by tdmix_test_math), in
// fp64 rcp<double> (the approximation is ~2^-23 there).
template <class T>
__device__ __forceinline__ T rcp_lineshape(T v) {
  if constexpr (sizeof(T) == 4) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  } else {
    return rcp<double>(v);
  }
}

// Four values read together (one 128-bit shared load in fp32, two in fp64).
template <class T>
struct alignas(4 * sizeof(T)) Quad {
  T x, y, z, w;
};

// Per-block copy of the per-evaluation constants in the working precision,
// grouped by use so that each group is one vector load per event.
template <class T>
struct BlockConst {
  // working-precision values; in fp32 the lo parts carry the rounding
  // residual of the double-precision constant (value = hi + lo), so that no
  // systematic fp32 rounding enters every event in the same direction
  Quad<T> res[kMaxRes];     // resonance r: {m0^2, its lo part, kappa, its lo part}
  Quad<T> cab[kMaxComp];    // component j: {Re cA, Im cA, Re cB, Im cB}
  Quad<T> cab_lo[kMaxComp]; // their lo parts
  Quad<T> mix;              // {alpha, beta, gc, dc}
  double x, y, gamma;
  double hx, hy;                       // x Gamma / 2, y Gamma / 2
  float xf, yf, gammaf;                // fp32 copies for the fp32 adjoint
  float hxh, hxl, hyh, hyl;            // x Gamma / 2 and y Gamma / 2 as double-float pairs (fp32 path)
  unsigned long long tlim[2];          // bit patterns of the decay times below which
                                       // |x|, |y| Gamma t / 2 <= 0.02 (resp. 0.1)
};

// cosh, sinh of a and cos, sin of b.  The mixing arguments y Gamma t / 2,
// x Gamma t / 2 are small: at percent-level x, y, |a|, |b| <= 0.02 holds for
// decay times below ~6.5 lifetimes (nearly every event); there (tier 0) the
// Maclaurin series through the z^3 term (z = a^2 or b^2) is used (first
// omitted term below 7e-19 relative); for |a|, |b| <= 0.1 (tier 1, t below
// ~40 lifetimes) the series run through z^5 (first omitted term below
// 3e-21); otherwise (tier 2) the CUDA math library is called.  The caller
// picks the tier from the decay time (BlockConst::tlim).
__device__ __forceinline__ void mixing_trig(double a, double b, int tier, double& cha, double& sha, double& cb,
                                            double& sb) {
  if (tier == 0) {
    const double za = a * a, zb = b * b;
    cha = 1.0 + za * (1.0 / 2 + za * (1.0 / 24 + za * (1.0 / 720)));
    sha = a * (1.0 + za * (1.0 / 6 + za * (1.0 / 120 + za * (1.0 / 5040))));
    cb = 1.0 - zb * (1.0 / 2 - zb * (1.0 / 24 - zb * (1.0 / 720)));
    sb = b * (1.0 - zb * (1.0 / 6 - zb * (1.0 / 120 - zb * (1.0 / 5040))));
  } else if (tier == 1) {
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

// Natural logarithm by Tang's table-driven method (P. T. P. Tang, ACM Trans.
// Math. Softw. 16 (1990) 378): v = 2^e m with m in [1, 2); F = 1 + j/128 is
// the grid point nearest m, so m - F is exact and r = (m - F) / F has
// |r| <= 2^-8; then ln v = e ln 2 + ln F + ln(1 + r), the last from its
// Taylor series through r^6 (first omitted term below 2^-58).  tab[j] holds
// {1/F, ln F} for j = 0 .. 128, made on the host in extended precision.  About
// ten double-precision operations against several tens for the library
// logarithm.  The error is below 2^-52 absolute for |ln v| < 1 and relative
// above (near v = 1 the terms e ln 2 and ln F cancel, so it is not small
// relative to ln v there; the likelihood sums logarithms and needs the
// absolute accuracy).  Positive normal v only (the library function takes
// the rest).
constexpr int kLogTable = 129;
constexpr double kLn2 = 0.69314718055994530942;
// ln v = e ln 2 + the returned value (the caller sums the exponents as
// integers and multiplies by ln 2 once).
__device__ __forceinline__ double log_table_split(double v, const double2* tab, int& e) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  if (bits - 0x0010000000000000ull >= 0x7FE0000000000000ull) {  // not positive normal
    e = 0;
    return log(v);
  }
  const unsigned long long frac = bits & 0x000FFFFFFFFFFFFFull;
  e = int(bits >> 52) - 1023;
  const double m = __longlong_as_double(static_cast<long long>(frac | 0x3FF0000000000000ull));
  const unsigned long long j = (frac + (1ull << 44)) >> 45;  // nearest multiple of 1/128, 0 .. 128
  const double F = __longlong_as_double(static_cast<long long>(0x3FF0000000000000ull + (j << 45)));  // 1 + j/128
  const double2 t = tab[int(j)];
  const double r = (m - F) * t.x;
  const double p = fma(r, fma(r, fma(r, fma(r, -1.0 / 6, 1.0 / 5), -1.0 / 4), 1.0 / 3), -0.5);
  const double l1p = fma(r * r, p, r);
  return t.y + l1p;
}

__device__ __forceinline__ double log_table(double v, const double2* tab) {
  int e;
  const double m = log_table_split(v, tab, e);
  return fma(double(e), kLn2, m);
}

// Single-precision version for |a|, |b| <= 0.1 (Maclaurin series through the
// z^3 term, first omitted term below 3e-13 relative), CUDA's functions otherwise.
__device__ __forceinline__ void mixing_trig_f32(float a, float b, float& cha, float& sha, float& cb, float& sb) {
  if (fabsf(a) <= 0.1f && fabsf(b) <= 0.1f) {
    const float za = a * a, zb = b * b;
    cha = 1.0f + za * (1.0f / 2 + za * (1.0f / 24 + za * (1.0f / 720)));
    sha = a * (1.0f + za * (1.0f / 6 + za * (1.0f / 120 + za * (1.0f / 5040))));
    cb = 1.0f - zb * (1.0f / 2 - zb * (1.0f / 24 - zb * (1.0f / 720)));
    sb = b * (1.0f - zb * (1.0f / 6 - zb * (1.0f / 120 - zb * (1.0f / 5040))));
  } else {
    cha = coshf(a);
    sha = sinhf(a);
    sincosf(b, &sb, &cb);
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
      const Quad<T> R = bc.res[r];
      T delta;
      if constexpr (P::kF32) {
        delta = (R.x - src.s_hi(sp)) + (R.y - src.s_lo(sp));
      } else {
        delta = R.x - src.s_hi(sp);
      }
      T X = T(1);
      if (xp >= 0) X = src.x(xp);
      T im;
      if constexpr (P::kF32) im = fma(R.z, X, R.w * X);
      else im = R.z * X;
      T inv = rcp_lineshape<T>(fma(delta, delta, im * im));
      bwr[b] = delta * inv;
      bwi[b] = im * inv;
      xs[b] = X;
    }
  }

  // With SCALE, sc[j] receives sum_o |K_{j,o}| (|Re P| + |Im P|) for the
  // lineshape products P of component j: an upper bound (within a factor
  // sqrt 2) of sum_o |K_{j,o} P|, the magnitude the rounding errors of a_j
  // scale with.
  template <bool SCALE = false, class Src>
  __device__ __forceinline__ void components(const Src& src, T* sc = nullptr) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      T sr = 0, si = 0, sm = 0;
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
        if constexpr (SCALE) sm = fma(fabs(K), fabs(pr) + fabs(pi), sm);
      }
      ar[j] = sr;
      ai[j] = si;
      if constexpr (SCALE) sc[j] = sm;
    }
  }

  // components() that also keeps every term's product Q_t = K_t prod BW
  // (the term's contribution to its component) for backprop_q.
  template <class Src>
  __device__ __forceinline__ void components_q(const Src& src, T (&qr)[U * NO], T (&qi)[U * NO]) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      T sr = 0, si = 0;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const int t = j * NO + o;
        const int b0 = S::tb0(t), b1 = S::tb1(t);
        const T K = src.k(t);
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
        qr[t] = K * pr;
        qi[t] = K * pi;
        sr += qr[t];
        si += qi[t];
      }
      ar[j] = sr;
      ai[j] = si;
    }
  }

  // backprop_lineshapes from the kept term products: with W_j = gA cA_j +
  // gB cB_j, df/dBW_b = Z_b / BW_b, Z_b = sum over the terms t of b of
  // W_j(t) Q_t (a term holding b twice counts twice), so H_b = (df/dBW_b)
  // BW_b^2 = Z_b BW_b.  The same sums as backprop_lineshapes with fewer
  // operations: no K reloads, no BW_b^2.
  template <bool WEIGHTED>
  __device__ __forceinline__ void backprop_q(const BlockConst<T>& bc, const T (&qr)[U * NO], const T (&qi)[U * NO],
                                             T gAr, T gAi, T gBr, T gBi, T wt, T (&s1)[NR > 0 ? NR : 1],
                                             T (&s2)[NR > 0 ? NR : 1]) const {
    if constexpr (NB > 0) {
      T Zr[NB], Zi[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) Zr[b] = Zi[b] = 0;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        T Wr = 0, Wi = 0;
        const Quad<T> C = bc.cab[j];
        cmac(Wr, Wi, gAr, gAi, C.x, C.y);
        cmac(Wr, Wi, gBr, gBi, C.z, C.w);
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          const int t = j * NO + o;
          const int b0 = S::tb0(t), b1 = S::tb1(t);
          if (b0 < 0 && b1 < 0) continue;
          const T zr = fma(Wr, qr[t], -Wi * qi[t]), zi = fma(Wr, qi[t], Wi * qr[t]);
          if (b0 >= 0) {
            Zr[b0] += zr;
            Zi[b0] += zi;
          }
          if (b1 >= 0) {
            Zr[b1] += zr;
            Zi[b1] += zi;
          }
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int r = S::bres(b);
        const T Hr = fma(Zr[b], bwr[b], -Zi[b] * bwi[b]);
        const T Hi = fma(Zr[b], bwi[b], Zi[b] * bwr[b]);
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

  // LO: also add the low parts of the coefficients (fp32 data events, whose
  // ln B enters the likelihood one by one).
  template <bool LO = false>
  __device__ __forceinline__ void amplitudes(const BlockConst<T>& bc, T& Ar, T& Ai, T& Br, T& Bi) const {
    Ar = Ai = Br = Bi = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      if constexpr (LO && P::kF32) {
        const Quad<T> L = bc.cab_lo[j];
        cmac(Ar, Ai, L.x, L.y, ar[j], ai[j]);
        cmac(Br, Bi, L.z, L.w, ar[j], ai[j]);
      }
      const Quad<T> C = bc.cab[j];
      cmac(Ar, Ai, C.x, C.y, ar[j], ai[j]);
      cmac(Br, Bi, C.z, C.w, ar[j], ai[j]);
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
        const Quad<T> C = bc.cab[j];
        cmac(Wr, Wi, gAr, gAi, C.x, C.y);
        cmac(Wr, Wi, gBr, gBi, C.z, C.w);
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

// Sensitivities of ln B = ln 2|Z|^2, Z = cosh(w) A - sinh(w) Abar, with
// cosh w = cr + i ci and sinh w = sr + i si: d ln B = 2 Re(V dZ), V = 1/Z,
// dZ = cosh(w) dA - sinh(w) dAbar + (sinh(w) A - cosh(w) Abar) dw, dw/dy =
// Gamma t / 2, dw/dx = i Gamma t / 2 (tg = Gamma t).  Writes tA = V cosh(w),
// tB = -V sinh(w) and adds d ln B / dy, d ln B / dx to gy, gx.
template <class T>
__device__ __forceinline__ void mix_adjoint(T cr, T ci, T sr, T si, T Zr, T Zi, T Ar, T Ai, T Br, T Bi, T tg, T& tAr,
                                            T& tAi, T& tBr, T& tBi, T& gx, T& gy) {
  const T iz = rcp<T>(fma(Zr, Zr, Zi * Zi));
  const T Vr = Zr * iz, Vi = -Zi * iz;
  tAr = fma(Vr, cr, -Vi * ci);
  tAi = fma(Vr, ci, Vi * cr);
  tBr = -fma(Vr, sr, -Vi * si);
  tBi = -fma(Vr, si, Vi * sr);
  T Dr = 0, Di = 0;
  cmac(Dr, Di, sr, si, Ar, Ai);
  cmac(Dr, Di, -cr, -ci, Br, Bi);
  gy = fma(tg, fma(Vr, Dr, -Vi * Di), gy);
  gx = fma(-tg, fma(Vr, Di, Vi * Dr), gx);
}

// One data event's rate from its amplitudes A, Abar and decay time: Eq. (mix) as B = 2 |cosh(w) A - sinh(w) Abar|^2 with
// w = (y + i x) Gamma t / 2, in double precision.  For a B that is positive
// and finite, adds ln B to the pair (lnb, lexp) as lnb + lexp ln 2 and
// returns true; with GRAD it also forms the
// sensitivities of ln B: d ln B = 2 Re(tA dA + tB dAbar) and adds
// d ln B / dx, d ln B / dy to gx, gy.  d ln B = 2 Re(V dZ), V = Z* / |Z|^2,
// dZ = cosh(w) dA - sinh(w) dAbar + (sinh(w) A - cosh(w) Abar) dw,
// dw/dy = Gamma t / 2, dw/dx = i Gamma t / 2.  The sensitivities are formed
// in the working precision; in fp32, cosh(w), sinh(w) and Z are re-derived
// in fp32 rather than converted from their fp64 values.  `rate` (optional)
// receives e^{-Gamma t} B.
// Ar .. Bi are the amplitudes the rate is formed from (double precision);
// Ar_ .. Bi_ the working-precision ones the sensitivities are formed from
// (the same values unless the data event was recomputed in double-float).
template <class P, bool GRAD>
__device__ __forceinline__ bool mix_event(const BlockConst<typename P::T>& bc, const double2* logtab, double Ar,
                                          double Ai, double Br, double Bi, typename P::T Ar_, typename P::T Ai_,
                                          typename P::T Br_, typename P::T Bi_, double t_e, double& lnb, int& lexp,
                                          double* rate, typename P::T& tAr, typename P::T& tAi, typename P::T& tBr,
                                          typename P::T& tBi, typename P::T& gx, typename P::T& gy) {
  using T = typename P::T;
  const double gt = bc.gamma * t_e;
  const unsigned long long tb = static_cast<unsigned long long>(__double_as_longlong(t_e));
  const int tier = tb <= bc.tlim[0] ? 0 : (tb <= bc.tlim[1] ? 1 : 2);  // t < 0 or NaN: tier 2
  double cha, sha, cb, sb;
  mixing_trig(bc.hy * t_e, bc.hx * t_e, tier, cha, sha, cb, sb);
  const double chr = cha * cb, chi = sha * sb;  // cosh(w)
  const double shr = sha * cb, shi = cha * sb;  // sinh(w)
  const double Zr = chr * Ar - chi * Ai - (shr * Br - shi * Bi);
  const double Zi = chr * Ai + chi * Ar - (shr * Bi + shi * Br);
  const double z2 = Zr * Zr + Zi * Zi;  // B = 2 z2: ln B = ln z2 + ln 2
  if (rate) *rate = exp(-gt) * (2.0 * z2);
  const unsigned long long bb = static_cast<unsigned long long>(__double_as_longlong(z2));
  if (bb - 1ull >= 0x7FEFFFFFFFFFFFFFull) return false;  // B <= 0, infinite or NaN
  int e;
  lnb += log_table_split(z2, logtab, e);
  lexp += e + 1;
  if constexpr (GRAD) {
    if constexpr (P::kF32) {
      const float tg = bc.gammaf * float(t_e);
      float chf, shf, cbf, sbf;
      mixing_trig_f32(0.5f * bc.yf * tg, 0.5f * bc.xf * tg, chf, shf, cbf, sbf);
      const float cr = chf * cbf, ci = shf * sbf, sr = shf * cbf, si = chf * sbf;
      float Zrt = 0, Zit = 0;
      cmac(Zrt, Zit, cr, ci, Ar_, Ai_);
      cmac(Zrt, Zit, -sr, -si, Br_, Bi_);
      mix_adjoint<T>(cr, ci, sr, si, Zrt, Zit, Ar_, Ai_, Br_, Bi_, tg, tAr, tAi, tBr, tBi, gx, gy);
    } else {
      mix_adjoint<T>(chr, chi, shr, shi, Zr, Zi, Ar_, Ai_, Br_, Bi_, gt, tAr, tAi, tBr, tBi, gx, gy);
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Eq. (mix) of the fp32 path in double-float arithmetic.
//
// GB300 runs double-precision arithmetic at about 1/64 of the FP32 rate, so
// the ~45 fp64 operations per event of mix_event bound the data pass by the
// FP64 pipe, far below the memory rate at which its inputs arrive.  Here the
// same quantities are formed from float pairs (value = hi + lo, about 48
// significant bits) on the FP32 pipe: the mixing arguments a = y Gamma t / 2,
// b = x Gamma t / 2 from the decay time and the constants as pairs; for
// |a|, |b| <= 0.1 the Maclaurin series of cosh, sinh, cos, sin with their
// leading terms in pairs and the tails (below 4e-4 relative) in floats;
//   P = cosh a cos b - 1,  Q = sinh a sin b,  R = sinh a cos b,  S = cosh a sin b,
// so that cosh w = 1 + P + i Q and sinh w = R + i S;
//   Z = A + (P + i Q) A - (R + i S) Abar,  B = 2 |Z|^2,
// with every product and sum in pairs (errors about 2^-48 of the operands'
// magnitudes, as fp64's 2^-53); ln |Z|^2 by Tang's table method with the
// table entries, the reduced argument and the leading series terms in pairs.
// The mixing factors are within ~1e-15 of their values for |a|, |b| <= 0.02
// (decay times below ~6.5 lifetimes at percent-level x, y) and ~1e-12 up to
// 0.1; ln B within ~1e-15 absolute of ln of the computed B.  Larger
// arguments (and B that is not a normal float) take mix_event.
// ---------------------------------------------------------------------------

// 1/6 as a double-float pair.
constexpr float kSixthHi = 1.0f / 6.0f;
constexpr float kSixthLo = float(1.0 / 6.0 - double(1.0f / 6.0f));

// The four mixing factors P, Q, R, S for |a.hi|, |b.hi| <= 0.1.
__device__ __forceinline__ void mixing_factors_df(DF a, DF b, DF& Pm, DF& Q, DF& R, DF& S) {
  const DF a2 = df_mul(a, a), b2 = df_mul(b, b);
  const float za = a2.hi, zb = b2.hi;
  // cosh a - 1 = a^2 (1/2 + ta), 1 - cos b = b^2 (1/2 - tb); series through
  // z^5 (first omitted term below 2e-21 relative at |a|, |b| = 0.1)
  const float ta = za * (1.0f / 24 + za * (1.0f / 720 + za * (1.0f / 40320 + za * (1.0f / 3628800))));
  const float tb = zb * (1.0f / 24 - zb * (1.0f / 720 - zb * (1.0f / 40320 - zb * (1.0f / 3628800))));
  const DF Ca = df_mul(a2, df_fast_two_sum(0.5f, ta));
  const DF Cb = df_mul(b2, df_fast_two_sum(0.5f, -tb));
  // sinh a - a = a a^2 (1/6 + sa), b - sin b = b b^2 (1/6 - sb)
  const float sa = za * (1.0f / 120 + za * (1.0f / 5040 + za * (1.0f / 362880 + za * (1.0f / 39916800))));
  const float sb = zb * (1.0f / 120 - zb * (1.0f / 5040 - zb * (1.0f / 362880 - zb * (1.0f / 39916800))));
  const DF Sa = df_mul(df_mul(a, a2), df_add_s(DF{kSixthHi, kSixthLo}, DF{sa, 0.0f}));
  const DF Sb = df_mul(df_mul(b, b2), df_add_s(DF{kSixthHi, kSixthLo}, DF{-sb, 0.0f}));
  const DF sha = df_add_s(a, Sa), snb = df_sub_s(b, Sb);  // sinh a, sin b
  Pm = df_sub_s(df_sub_s(Ca, Cb), df_mul(Ca, Cb));
  Q = df_mul(sha, snb);
  R = df_sub_s(sha, df_mul(sha, Cb));
  S = df_add_s(snb, df_mul(snb, Ca));
}

// ln v = e ln 2 + l for a double-float v whose hi part is a positive float
// with exponent in [-100, 125] (returns false otherwise: below 2^-100 the lo
// part of a pair can be subnormal and carry fewer bits).  v = 2^e m,
// m in [1, 2); F = 1 + j/128 the grid point nearest m (m - F exact),
// r = (m - F) / F with |r| <= 2^-8 (the pair 1/F from the table), then
// ln v = e ln 2 + ln F + ln(1 + r), ln(1 + r) = r - r^2/2 (pairs) +
// r^3 (1/3 - r/4 + r^2/5 - r^3/6 + r^4/7) (float; first omitted term below
// 2^-67).  tab[j] = {1/F hi, lo, ln F hi, lo}.
__device__ __forceinline__ bool log_df(DF v, const float4* tab, int& e, DF& l) {
  const unsigned bits = __float_as_uint(v.hi);
  const unsigned be = bits >> 23;                      // sign and biased exponent
  if (be < 27u || be > 252u) return false;             // not positive, or exponent outside [-100, 125]
  e = int(be) - 127;
  const unsigned frac = bits & 0x007FFFFFu;
  const float mh = __uint_as_float(frac | 0x3F800000u);
  const float ml = v.lo * __uint_as_float(unsigned(127 - e) << 23);  // lo scaled by 2^-e (exact)
  const unsigned j = (frac + (1u << 15)) >> 16;        // nearest multiple of 1/128, 0 .. 128
  const float F = __uint_as_float(0x3F800000u + (j << 16));
  const float4 t = tab[j];
  const DF r = df_mul(df_two_sum(mh - F, ml), DF{t.x, t.y});
  const DF r2 = df_mul(r, r);
  const float rh = r.hi;
  const float c = rh * rh * rh * (1.0f / 3 + rh * (-0.25f + rh * (0.2f + rh * (-1.0f / 6 + rh * (1.0f / 7)))));
  const DF l1 = df_add_s(df_add_s(r, DF{-0.5f * r2.hi, -0.5f * r2.lo}), DF{c, 0.0f});
  l = df_add_s(DF{t.z, t.w}, l1);
  return true;
}

// The fp32 path's counterpart of mix_event<PrecF32, GRAD>: A, Abar as
// double-float pairs (lo parts zero unless the event was recomputed), the
// decay time as a pair (th, tl); ln B is added to the pair (lnb, lexp) as
// lnb + lexp ln 2 with lnb a double-float accumulator.  The sensitivities
// are formed in fp32 from the leading parts of the mixing factors and Z.
template <bool GRAD>
__device__ __forceinline__ bool mix_event_df(const BlockConst<float>& bc, const double2* logtab, const float4* logtab_f,
                                             DF Ar, DF Ai, DF Br, DF Bi, float th, float tl, DF& lnb, int& lexp,
                                             double* rate, float& tAr, float& tAi, float& tBr, float& tBi, float& gx,
                                             float& gy) {
  const DF t{th, tl};
  const DF a = df_mul(DF{bc.hyh, bc.hyl}, t), b = df_mul(DF{bc.hxh, bc.hxl}, t);
  if (!(fabsf(a.hi) <= 0.1f && fabsf(b.hi) <= 0.1f)) {  // long decay times, or t not finite
    double l = 0.0;
    const bool ok = mix_event<PrecF32, GRAD>(bc, logtab, df_to_double(Ar), df_to_double(Ai), df_to_double(Br),
                                             df_to_double(Bi), Ar.hi, Ai.hi, Br.hi, Bi.hi, df_to_double(t), l, lexp,
                                             rate, tAr, tAi, tBr, tBi, gx, gy);
    lnb = df_add_s(lnb, df_from_double(l));
    return ok;
  }
  DF Pm, Q, R, S;
  mixing_factors_df(a, b, Pm, Q, R, S);
  const DF Zr = df_add_s(Ar, df_sub_s(df_sub_s(df_mul(Pm, Ar), df_mul(Q, Ai)), df_sub_s(df_mul(R, Br), df_mul(S, Bi))));
  const DF Zi = df_add_s(Ai, df_sub_s(df_add_s(df_mul(Pm, Ai), df_mul(Q, Ar)), df_add_s(df_mul(R, Bi), df_mul(S, Br))));
  const DF z2 = df_add_s(df_mul(Zr, Zr), df_mul(Zi, Zi));  // B = 2 z2
  if (rate) *rate = exp(-bc.gamma * df_to_double(t)) * (2.0 * df_to_double(z2));
  int e;
  DF l;
  if (log_df(z2, logtab_f, e, l)) {
    lnb = df_add_s(lnb, l);
    lexp += e + 1;
  } else {
    // B <= 0, not finite, or outside the float exponent range: double precision
    const double v = df_to_double(z2);
    const unsigned long long bb = static_cast<unsigned long long>(__double_as_longlong(v));
    if (bb - 1ull >= 0x7FEFFFFFFFFFFFFFull) return false;
    lnb = df_add_s(lnb, df_from_double(log_table_split(v, logtab, e)));
    lexp += e + 1;
  }
  if constexpr (GRAD)
    mix_adjoint<float>(1.0f + Pm.hi, Q.hi, R.hi, S.hi, Zr.hi, Zi.hi, Ar.hi, Ai.hi, Br.hi, Bi.hi, bc.gammaf * th, tAr,
                       tAi, tBr, tBi, gx, gy);
  return true;
}

// ---------------------------------------------------------------------------
// Ill-conditioned data events of the fp32 path.
//
// The fp32 amplitudes carry rounding errors of a few ulps of the magnitudes
// of their terms, S = sum over chains and Bose orderings of |c T|, so the
// relative error of an event's rate grows like S / |Z| (Z = cosh(w) A -
// sinh(w) Abar, B = 2 |Z|^2): about 5e-7 S / |Z| at worst.  Events whose
// estimate of S / |Z| exceeds kRecomputeCond are recomputed: lineshapes,
// components and A, Abar again in double-float from the double-float
// inputs (invariants s = hi + lo in the tile; width and spin x barrier
// factors from their hi planes in the tile and their lo planes in
// SampleDev::lo; constants and coefficients as hi + lo pairs), which
// leaves the rate within ~1e-12 of its value for any condition met in
// practice.  Events below the threshold stay within 5e-7 x 16 = 8e-6.
constexpr float kRecomputeCond = 16.0f;

// Condition estimate of one fp32 data event: true if
// S_Z > kRecomputeCond |Z|, with S_Z = cosh|w| S_A + sinh|w| S_B an upper
// bound of the magnitude the errors of Z scale with (|cosh w| <= cosh|w|,
// |sinh w| <= sinh|w|, |w| <= |a| + |b|) and Z formed in fp32.
template <int U>
__device__ __forceinline__ bool ill_conditioned(const BlockConst<float>& bc, const float (&sc)[U], float Ar, float Ai,
                                                float Br, float Bi, float t_e) {
  float SA = 0.f, SB = 0.f;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const Quad<float> C = bc.cab[j];
    SA = fmaf(fabsf(C.x) + fabsf(C.y), sc[j], SA);
    SB = fmaf(fabsf(C.z) + fabsf(C.w), sc[j], SB);
  }
  const float tg = bc.gammaf * t_e;
  const float a = 0.5f * bc.yf * tg, b = 0.5f * bc.xf * tg;
  float cha, sha, cb, sb, chw, shw, c0, s0;
  mixing_trig_f32(a, b, cha, sha, cb, sb);
  mixing_trig_f32(fabsf(a) + fabsf(b), 0.f, chw, shw, c0, s0);
  const float cr = cha * cb, ci = sha * sb, sr = sha * cb, si = cha * sb;
  const float Zr = cr * Ar - ci * Ai - (sr * Br - si * Bi);
  const float Zi = cr * Ai + ci * Ar - (sr * Bi + si * Br);
  const float SZ = chw * SA + shw * SB;
  return SZ * SZ > (kRecomputeCond * kRecomputeCond) * (Zr * Zr + Zi * Zi);
}

// A and Abar of one fp32 data event recomputed in double-float.  `stage`
// is the event tile in shared memory (planes of SmemSrc), `lo` this tile's
// lo planes ([NX + U NO][256] floats: width factors, then spin x barrier
// factors), e the event's slot.  Out of line: it runs for few events, and
// its registers must not add to the main loop's.
template <class S>
__device__ __noinline__ void df_amplitudes(const float* __restrict__ stage, const float* __restrict__ lo, int e,
                                           const BlockConst<float>& bc, DF* out) {
  constexpr int TE = kTileEvents;
  constexpr int NB = S::NB, NO = S::NO, U = S::U, NS = S::NS, NX = S::NX;
  constexpr int X0 = 2 * NS, K0 = 2 * NS + NX;
  DF bwr[NB > 0 ? NB : 1], bwi[NB > 0 ? NB : 1];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int r = S::bres(b), sp = S::bs(b), xp = S::bx(b);
    const Quad<float> R = bc.res[r];
    const DF delta = df_sub(DF{R.x, R.y}, DF{stage[sp * TE + e], stage[(NS + sp) * TE + e]});
    const DF X = xp >= 0 ? DF{stage[(X0 + xp) * TE + e], lo[xp * TE + e]} : DF{1.0f, 0.0f};
    const DF im = df_mul(DF{R.z, R.w}, X);
    const DF inv = df_rcp(df_add(df_mul(delta, delta), df_mul(im, im)));
    bwr[b] = df_mul(delta, inv);
    bwi[b] = df_mul(im, inv);
  }
  DF Ar{0.f, 0.f}, Ai{0.f, 0.f}, Br{0.f, 0.f}, Bi{0.f, 0.f};
#pragma unroll
  for (int j = 0; j < U; ++j) {
    DF sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int t = j * NO + o;
      const int b0 = S::tb0(t), b1 = S::tb1(t);
      const DF K{stage[(K0 + t) * TE + e], lo[(NX + t) * TE + e]};
      DF pr, pi;
      if (b0 >= 0 && b1 >= 0) {
        pr = df_sub(df_mul(bwr[b0], bwr[b1]), df_mul(bwi[b0], bwi[b1]));
        pi = df_add(df_mul(bwr[b0], bwi[b1]), df_mul(bwi[b0], bwr[b1]));
      } else if (b0 >= 0) {
        pr = bwr[b0];
        pi = bwi[b0];
      } else if (b1 >= 0) {
        pr = bwr[b1];
        pi = bwi[b1];
      } else {
        pr = DF{1.0f, 0.0f};
        pi = DF{0.0f, 0.0f};
      }
      sr = df_add(sr, df_mul(K, pr));
      si = df_add(si, df_mul(K, pi));
    }
    const Quad<float> C = bc.cab[j], L = bc.cab_lo[j];
    const DF car{C.x, L.x}, cai{C.y, L.y}, cbr{C.z, L.z}, cbi{C.w, L.w};
    Ar = df_add(Ar, df_sub(df_mul(car, sr), df_mul(cai, si)));
    Ai = df_add(Ai, df_add(df_mul(car, si), df_mul(cai, sr)));
    Br = df_add(Br, df_sub(df_mul(cbr, sr), df_mul(cbi, si)));
    Bi = df_add(Bi, df_add(df_mul(cbr, si), df_mul(cbi, sr)));
  }
  out[0] = Ar;
  out[1] = Ai;
  out[2] = Br;
  out[3] = Bi;
}

}  // namespace tdmix
