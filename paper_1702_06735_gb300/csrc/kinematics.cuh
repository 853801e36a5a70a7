// Device-side Lorentz algebra, barrier factors and spin factors (Sec. 3
// building blocks), used once per event load by the precompute kernel
// (double precision) and by the event generator (double, and single
// precision for its pre-screen).
// Metric (+,-,-,-); four-vectors hold contravariant (E, px, py, pz).
#pragma once
#include <cuda_runtime.h>

#include "model.hpp"

namespace tdmix {

// Four-vector in the working precision T (double for the event loader,
// float for the generator's pre-screen).
template <class T>
struct V4T {
  T e, x, y, z;
};
using V4 = V4T<double>;

template <class T>
__device__ __forceinline__ V4T<T> operator+(V4T<T> a, V4T<T> b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T>
__device__ __forceinline__ V4T<T> operator-(V4T<T> a, V4T<T> b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T>
__device__ __forceinline__ V4T<T> operator*(T s, V4T<T> a) { return {s * a.e, s * a.x, s * a.y, s * a.z}; }
template <class T>
__device__ __forceinline__ T dot(V4T<T> a, V4T<T> b) { return a.e * b.e - a.x * b.x - a.y * b.y - a.z * b.z; }

// Relative momentum r = a - b of P -> (a, b) with its component along P removed.
template <class T>
__device__ __forceinline__ V4T<T> tvec(V4T<T> P, V4T<T> a, V4T<T> b) {
  V4T<T> r = a - b;
  return r - (dot(r, P) / dot(P, P)) * P;
}

// epsilon_{mu nu rho sigma} a^mu b^nu c^rho d^sigma, epsilon_{0123} = +1:
// the determinant of the 4x4 matrix with rows a, b, c, d.
template <class T>
__device__ __forceinline__ T levi(V4T<T> a, V4T<T> b, V4T<T> c, V4T<T> d) {
  T m01 = c.e * d.x - c.x * d.e, m02 = c.e * d.y - c.y * d.e, m03 = c.e * d.z - c.z * d.e;
  T m12 = c.x * d.y - c.y * d.x, m13 = c.x * d.z - c.z * d.x, m23 = c.y * d.z - c.z * d.y;
  T M0 = b.x * m23 - b.y * m13 + b.z * m12;
  T M1 = b.e * m23 - b.y * m03 + b.z * m02;
  T M2 = b.e * m13 - b.x * m03 + b.z * m01;
  T M3 = b.e * m12 - b.x * m02 + b.y * m01;
  return a.e * M0 - a.x * M1 + a.y * M2 - a.z * M3;
}

// Squared two-body breakup momentum of mass^2 s into masses^2 a2, b2, >= 0.
template <class T>
__device__ __forceinline__ T breakup2(T s, T a2, T b2) {
  T l = s * s + a2 * a2 + b2 * b2 - T(2) * (s * a2 + s * b2 + a2 * b2);
  return fmax(l / (T(4) * s), T(0));
}

// Blatt-Weisskopf factor without its q^L part, z = (q r)^2.
template <class T>
__device__ __forceinline__ T barrier(int L, T z) {
  if (L == 0) return T(1);
  if (L == 1) return T(1) / sqrt(T(1) + z);
  return T(1) / sqrt(T(9) + T(3) * z + z * z);
}

// Spin factor times barrier factors of one ordering of one chain; a, b, c, d
// in the chain's particle order.  VV_*: D -> R1(a b) R2(c d);
// AP_S: D -> R1 d, R1 -> R2 c (S-wave), R2 -> (a b).
template <class T>
__device__ inline T spin_barrier(int spin, V4T<T> a, V4T<T> b, V4T<T> c, V4T<T> d, T r, T rD) {
  if (spin == SPIN_NR) return T(1);
  V4T<T> PD = a + b + c + d;
  T mD2 = dot(PD, PD);
  if (spin == SPIN_AP_S) {
    V4T<T> P2 = a + b;
    V4T<T> P1 = P2 + c;
    T s1 = dot(P1, P1), s2 = dot(P2, P2);
    V4T<T> L = tvec(PD, P1, d);
    V4T<T> t2 = tvec(P2, a, b);
    T S = dot(L, t2) - dot(L, P1) * dot(t2, P1) / s1;
    T qD2 = breakup2(mD2, s1, dot(d, d));
    T q22 = breakup2(s2, dot(a, a), dot(b, b));
    return S * barrier(1, qD2 * rD * rD) * barrier(1, q22 * r * r);
  }
  V4T<T> P1 = a + b, P2 = c + d;
  T s1 = dot(P1, P1), s2 = dot(P2, P2);
  V4T<T> t1 = tvec(P1, a, b), t2 = tvec(P2, c, d);
  T S;
  int LD;
  if (spin == SPIN_VV_S) {
    S = dot(t1, t2);
    LD = 0;
  } else if (spin == SPIN_VV_P) {
    S = levi(PD, P1 - P2, t1, t2);
    LD = 1;
  } else {
    V4T<T> L = tvec(PD, P1, P2);
    S = dot(t1, L) * dot(t2, L) - (T(1) / T(3)) * dot(L, L) * (dot(t1, t2) - dot(t1, PD) * dot(t2, PD) / mD2);
    LD = 2;
  }
  T qD2 = breakup2(mD2, s1, s2);
  T q12 = breakup2(s1, dot(a, a), dot(b, b));
  T q22 = breakup2(s2, dot(c, c), dot(d, d));
  return S * barrier(LD, qD2 * rD * rD) * barrier(1, q12 * r * r) * barrier(1, q22 * r * r);
}

}  // namespace tdmix
