// Decay-time resolution: the rate of Eq. (mix) folded with a Gaussian of
// width sigma in the measured time (an extension; the paper's sensitivity
// study has no resolution, Sec. 4).  Double precision.
//
// Each exponential term folds in closed form: for Re a > 0,
//   K(t; a) = int_0^inf e^{-a t'} G(t - t'; sigma) dt'
//           = 1/2 e^{-t^2 / (2 sigma^2)} w(xi),  xi = i (a sigma^2 - t) / (sigma sqrt 2),
// w the Faddeeva function w(z) = e^{-z^2} erfc(-i z); in the lower half
// plane w(xi) = 2 e^{-xi^2} - w(-xi), where 1/2 e^{-t^2/(2 sigma^2)} 2 e^{-xi^2}
// = e^{-a t + a^2 sigma^2 / 2}, the unfolded exponential with its shift.
// With a = Gamma (1 -+ y) (cosh, sinh: real a) and a = Gamma (1 - i x)
// (cos + i sin), the four time functions of Eq. (mix) follow.  The
// derivative in a (for the gradient in x and y) is
//   dK/da = (a sigma^2 - t) K - sigma^2 G(t; sigma).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace tdmix {

struct Cplx {
  double re, im;
};
__device__ __forceinline__ Cplx cadd(Cplx a, Cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cplx csub(Cplx a, Cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cplx cscale(Cplx a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ Cplx cdiv(Cplx a, Cplx b) {
  const double d = 1.0 / (b.re * b.re + b.im * b.im);
  return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
__device__ __forceinline__ Cplx cexp(Cplx a) {
  double s, c;
  sincos(a.im, &s, &c);
  const double e = exp(a.re);
  return {e * c, e * s};
}

constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1 / sqrt(pi)

// Faddeeva function w(z) for Im z >= 0 and |Re z| <= 0.3 (the arguments
// of the folds: Re xi = x Gamma sigma / sqrt 2 is small).  Two methods, both
// from the mathematics of w:
//   |z| >= 8: Laplace's continued fraction
//       w(z) = (i / sqrt pi) / (z - (1/2) / (z - 1 / (z - (3/2) / (z - ...)))),
//     thirty levels evaluated from the bottom;
//   |z| < 8: the Taylor series around the imaginary-axis point i v (v = Im z)
//     in the real offset d = Re z, from w(i v) = erfcx(v) (the CUDA math
//     library) and the derivatives w' = -2 z w + 2 i / sqrt pi,
//     w^(n+1) = -2 z w^(n) - 2 n w^(n-1), thirty terms.
// Against scipy's wofz over |Re z| <= 0.3, 0 <= Im z <= 500 both agree with
// the reference to 6e-15 relative (checked in double precision on the host).
__device__ inline Cplx faddeeva_upper(Cplx z) {
  if (z.re * z.re + z.im * z.im >= 64.0) {
    Cplx r = {0.0, 0.0};
    for (int n = 30; n >= 1; --n) r = cdiv(Cplx{0.5 * n, 0.0}, csub(z, r));
    return cdiv(Cplx{0.0, kInvSqrtPi}, csub(z, r));
  }
  const double d = z.re;
  const Cplx z0 = {0.0, z.im};
  Cplx wm = {erfcx(z.im), 0.0};                                     // w(i v)
  Cplx wn = cadd(cscale(cmul(z0, wm), -2.0), Cplx{0.0, 2.0 * kInvSqrtPi});  // w'(i v)
  Cplx sum = cadd(wm, cscale(wn, d));
  double fac = d;  // d^n / n!
  for (int n = 1; n < 30; ++n) {
    const Cplx wp = csub(cscale(cmul(z0, wn), -2.0), cscale(wm, 2.0 * n));
    fac *= d / (n + 1);
    sum = cadd(sum, cscale(wp, fac));
    wm = wn;
    wn = wp;
  }
  return sum;
}

// K(t; a) and dK/da for Re a > 0 (see the top of the file).
__device__ inline void fold_exp(double t, Cplx a, double sigma, Cplx& K, Cplx& dK) {
  const double s2 = sigma * sigma, r = 1.0 / (sigma * 1.41421356237309504880);
  const Cplx xi = {-a.im * s2 * r, (a.re * s2 - t) * r};  // i (a sigma^2 - t) / (sigma sqrt 2)
  const double g = exp(-0.5 * t * t / s2);
  if (xi.im >= 0.0) {
    K = cscale(faddeeva_upper(xi), 0.5 * g);
  } else {
    const Cplx w = faddeeva_upper(Cplx{-xi.re, -xi.im});
    const Cplx e = cexp(cadd(cscale(a, -t), cscale(cmul(a, a), 0.5 * s2)));  // e^{-a t + a^2 sigma^2 / 2}
    K = csub(e, cscale(w, 0.5 * g));
  }
  // dK/da = (a sigma^2 - t) K - sigma^2 G(t), G(t) = g / (sigma sqrt(2 pi))
  dK = csub(cmul(Cplx{a.re * s2 - t, a.im * s2}, K), Cplx{s2 * g * r * kInvSqrtPi, 0.0});
}

// The folded rate R of one event from its amplitudes A, Abar and measured
// time t, with the holomorphic sensitivities of ln R (d ln R = 2 Re(tA dA +
// tB dAbar)) and d ln R / dx, d ln R / dy (added to gx, gy).  Returns false
// for R <= 0 or not finite.
//   R = (|A|^2 + |Abar|^2) Cch + (|A|^2 - |Abar|^2) Ccos - 2 Re(A Abar*) Csh - 2 Im(A Abar*) Csin,
//   Cch, Csh = Re(K(Gamma(1-y)) +- K(Gamma(1+y))) / 2,  Ccos + i Csin = K(Gamma(1 - i x)).
template <bool GRAD>
__device__ inline bool resolved_rate(double Ar, double Ai, double Br, double Bi, double t, double x, double y,
                                     double gamma, double sigma, double& R, double& tAr, double& tAi, double& tBr,
                                     double& tBi, double& gx, double& gy) {
  Cplx km, dkm, kp, dkp, kc, dkc;
  fold_exp(t, Cplx{gamma * (1.0 - y), 0.0}, sigma, km, dkm);
  fold_exp(t, Cplx{gamma * (1.0 + y), 0.0}, sigma, kp, dkp);
  fold_exp(t, Cplx{gamma, -gamma * x}, sigma, kc, dkc);
  const double cch = 0.5 * (km.re + kp.re), csh = 0.5 * (km.re - kp.re);
  const double cco = kc.re, csn = kc.im;
  const double A2 = Ar * Ar + Ai * Ai, B2 = Br * Br + Bi * Bi;
  const double Xr = Ar * Br + Ai * Bi, Xi = Ai * Br - Ar * Bi;  // A Abar*
  R = (A2 + B2) * cch + (A2 - B2) * cco - 2.0 * Xr * csh - 2.0 * Xi * csn;
  if (!(R > 0.0) || !(R < INFINITY)) return false;
  if (GRAD) {
    const double iR = 1.0 / R;
    // dR/dA = A* (Cch + Ccos) - Abar* (Csh - i Csin), dR/dAbar = Abar* (Cch - Ccos) - A* (Csh + i Csin)
    const double pa = cch + cco, pb = cch - cco;
    tAr = (Ar * pa - (Br * csh - Bi * csn)) * iR;
    tAi = (-Ai * pa - (-Bi * csh - Br * csn)) * iR;
    tBr = (Br * pb - (Ar * csh + Ai * csn)) * iR;
    tBi = (-Bi * pb - (-Ai * csh + Ar * csn)) * iR;
    // da/dy = -Gamma (a-), +Gamma (a+); da/dx = -i Gamma (a of cos + i sin)
    const double dch_dy = 0.5 * gamma * (dkp.re - dkm.re), dsh_dy = -0.5 * gamma * (dkm.re + dkp.re);
    const Cplx dc_dx = cmul(dkc, Cplx{0.0, -gamma});
    gy += ((A2 + B2) * dch_dy - 2.0 * Xr * dsh_dy) * iR;
    gx += ((A2 - B2) * dc_dx.re - 2.0 * Xi * dc_dx.im) * iR;
  }
  return true;
}

}  // namespace tdmix
