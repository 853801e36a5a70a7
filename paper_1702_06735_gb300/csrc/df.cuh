// Double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  The building blocks are
// the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2),
// Fast-TwoSum (Dekker 1971, |a| >= |b|) and TwoProd by one fused
// multiply-add; addition follows the accurate ("IEEE") double-double sum of
// Hida, Li and Bailey (QD library, 2001), which keeps its relative accuracy
// when the operands cancel, and multiplication the product with the
// FMA-based TwoProd of the leading parts.
// Used where a single-precision result would lose too much and the
// double-precision pipe of this GPU (about 1/64 of the FP32 rate) would cost
// more: Eq. (mix) and ln B of the fp32 path's data events, and the
// recomputation of ill-conditioned ones.
#pragma once
#include <cuda_runtime.h>

namespace tdmix {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return DF{s, b - (s - a)};
}

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return DF{s, (a - (s - bp)) + (b - bp)};
}

__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = a * b;
  return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  const DF t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

// Sum whose error is bounded by about 2^-48 (|a| + |b|) rather than by the
// size of the result (the "sloppy" double-double sum): enough where the
// accuracy is wanted relative to the operands, as in the mixing formula.
__device__ __forceinline__ DF df_add_s(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF df_sub_s(DF a, DF b) { return df_add_s(a, DF{-b.hi, -b.lo}); }

// A double as a double-float (48 of its 53 bits).
__device__ __forceinline__ DF df_from_double(double v) {
  const float hi = float(v);
  return DF{hi, float(v - double(hi))};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF p = df_two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return df_fast_two_sum(p.hi, p.lo);
}

// 1 / a for a > 0: r0 = 1 / a.hi in single precision, then one Newton step
// r = r0 + r0 (1 - a r0) with the residual 1 - a r0 formed in double-float
// (it is of order 2^-23, so r0 times its leading float suffices).
__device__ __forceinline__ DF df_rcp(DF a) {
  const float r0 = 1.0f / a.hi;
  const DF e = df_sub(DF{1.0f, 0.0f}, df_mul(a, DF{r0, 0.0f}));
  return df_fast_two_sum(r0, r0 * e.hi);
}

// Exact value of a double-float as a double (48 bits fit in 53).
__device__ __forceinline__ double df_to_double(DF a) { return double(a.hi) + double(a.lo); }

}  // namespace tdmix
