// Device-side Lorentz algebra, barrier factors and spin factors (Sec. 3
// building blocks), used once per event load by the precompute kernel.
// Metric (+,-,-,-); four-vectors hold contravariant (E, px, py, pz).
#pragma once
#include <cuda_runtime.h>

#include "model.hpp"

namespace tdmix {

struct V4 {
  double e, x, y, z;
};

__device__ __forceinline__ V4 operator+(V4 a, V4 b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V4 operator-(V4 a, V4 b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V4 operator*(double s, V4 a) { return {s * a.e, s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V4 a, V4 b) { return a.e * b.e - a.x * b.x - a.y * b.y - a.z * b.z; }

// Relative momentum r = a - b of P -> (a, b) with its component along P removed.
__device__ __forceinline__ V4 tvec(V4 P, V4 a, V4 b) {
  V4 r = a - b;
  return r - (dot(r, P) / dot(P, P)) * P;
}

// epsilon_{mu nu rho sigma} a^mu b^nu c^rho d^sigma, epsilon_{0123} = +1:
// the determinant of the 4x4 matrix with rows a, b, c, d.
__device__ __forceinline__ double levi(V4 a, V4 b, V4 c, V4 d) {
  double m01 = c.e * d.x - c.x * d.e, m02 = c.e * d.y - c.y * d.e, m03 = c.e * d.z - c.z * d.e;
  double m12 = c.x * d.y - c.y * d.x, m13 = c.x * d.z - c.z * d.x, m23 = c.y * d.z - c.z * d.y;
  double M0 = b.x * m23 - b.y * m13 + b.z * m12;
  double M1 = b.e * m23 - b.y * m03 + b.z * m02;
  double M2 = b.e * m13 - b.x * m03 + b.z * m01;
  double M3 = b.e * m12 - b.x * m02 + b.y * m01;
  return a.e * M0 - a.x * M1 + a.y * M2 - a.z * M3;
}

// Squared two-body breakup momentum of mass^2 s into masses^2 a2, b2, >= 0.
__device__ __forceinline__ double breakup2(double s, double a2, double b2) {
  double l = s * s + a2 * a2 + b2 * b2 - 2.0 * (s * a2 + s * b2 + a2 * b2);
  return fmax(l / (4.0 * s), 0.0);
}

// Blatt-Weisskopf factor without its q^L part, z = (q r)^2.
__device__ __forceinline__ double barrier(int L, double z) {
  if (L == 0) return 1.0;
  if (L == 1) return 1.0 / sqrt(1.0 + z);
  return 1.0 / sqrt(9.0 + 3.0 * z + z * z);
}

// Spin factor times barrier factors of one ordering of one chain; a, b, c, d
// in the chain's particle order.  VV_*: D -> R1(a b) R2(c d);
// AP_S: D -> R1 d, R1 -> R2 c (S-wave), R2 -> (a b).
__device__ inline double spin_barrier(int spin, V4 a, V4 b, V4 c, V4 d, double r, double rD) {
  if (spin == SPIN_NR) return 1.0;
  V4 PD = a + b + c + d;
  double mD2 = dot(PD, PD);
  if (spin == SPIN_AP_S) {
    V4 P2 = a + b;
    V4 P1 = P2 + c;
    double s1 = dot(P1, P1), s2 = dot(P2, P2);
    V4 L = tvec(PD, P1, d);
    V4 t2 = tvec(P2, a, b);
    double S = dot(L, t2) - dot(L, P1) * dot(t2, P1) / s1;
    double qD2 = breakup2(mD2, s1, dot(d, d));
    double q22 = breakup2(s2, dot(a, a), dot(b, b));
    return S * barrier(1, qD2 * rD * rD) * barrier(1, q22 * r * r);
  }
  V4 P1 = a + b, P2 = c + d;
  double s1 = dot(P1, P1), s2 = dot(P2, P2);
  V4 t1 = tvec(P1, a, b), t2 = tvec(P2, c, d);
  double S;
  int LD;
  if (spin == SPIN_VV_S) {
    S = dot(t1, t2);
    LD = 0;
  } else if (spin == SPIN_VV_P) {
    S = levi(PD, P1 - P2, t1, t2);
    LD = 1;
  } else {
    V4 L = tvec(PD, P1, P2);
    S = dot(t1, L) * dot(t2, L) -
        (1.0 / 3.0) * dot(L, L) * (dot(t1, t2) - dot(t1, PD) * dot(t2, PD) / mD2);
    LD = 2;
  }
  double qD2 = breakup2(mD2, s1, s2);
  double q12 = breakup2(s1, dot(a, a), dot(b, b));
  double q22 = breakup2(s2, dot(c, c), dot(d, d));
  return S * barrier(LD, qD2 * rD * rD) * barrier(1, q12 * r * r) * barrier(1, q22 * r * r);
}

}  // namespace tdmix
