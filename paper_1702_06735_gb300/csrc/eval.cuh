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
      T inv = rcp<T>(fma(delta, delta, im * im));
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
    T cr, ci, sr, si, Zrt, Zit, tg;
    if constexpr (P::kF32) {
      const float tf = float(t_e);
      tg = bc.gammaf * tf;
      float chf, shf, cbf, sbf;
      mixing_trig_f32(0.5f * bc.yf * tg, 0.5f * bc.xf * tg, chf, shf, cbf, sbf);
      cr = chf * cbf; ci = shf * sbf; sr = shf * cbf; si = chf * sbf;
      Zrt = 0; Zit = 0;
      cmac(Zrt, Zit, cr, ci, Ar_, Ai_);
      cmac(Zrt, Zit, -sr, -si, Br_, Bi_);
    } else {
      cr = chr; ci = chi; sr = shr; si = shi;
      Zrt = Zr; Zit = Zi;
      tg = gt;
    }
    const T iz = rcp<T>(fma(Zrt, Zrt, Zit * Zit));
    const T Vr = Zrt * iz, Vi = -Zit * iz;
    tAr = fma(Vr, cr, -Vi * ci);
    tAi = fma(Vr, ci, Vi * cr);
    tBr = -fma(Vr, sr, -Vi * si);
    tBi = -fma(Vr, si, Vi * sr);
    T Dr = 0, Di = 0;
    cmac(Dr, Di, sr, si, Ar_, Ai_);
    cmac(Dr, Di, -cr, -ci, Br_, Bi_);
    gy = fma(tg, fma(Vr, Dr, -Vi * Di), gy);
    gx = fma(-tg, fma(Vr, Di, Vi * Dr), gx);
  }
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
                                                float Br, float Bi, double t_e) {
  float SA = 0.f, SB = 0.f;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const Quad<float> C = bc.cab[j];
    SA = fmaf(fabsf(C.x) + fabsf(C.y), sc[j], SA);
    SB = fmaf(fabsf(C.z) + fabsf(C.w), sc[j], SB);
  }
  const float tg = bc.gammaf * float(t_e);
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
                                           const BlockConst<float>& bc, double* out) {
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
  out[0] = df_to_double(Ar);
  out[1] = df_to_double(Ai);
  out[2] = df_to_double(Br);
  out[3] = df_to_double(Bi);
}

}  // namespace tdmix
