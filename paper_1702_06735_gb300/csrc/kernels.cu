// Model-independent kernels run once per event load: kinematic precompute
// and the fixed-order sum of the decay times or MC weights.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "device_tables.hpp"
#include "kernels.hpp"
#include "kinematics.cuh"

namespace tdmix {

// ---------------------------------------------------------------------------
// Kinematic precompute (one thread per event, fp64): invariants s, width
// factors X(s) = q^(2L+1) F_L(q r)^2 / sqrt(s) and the spin x barrier factor
// K_{j,o} of every component ordering.  None depends on fit parameters.
// Written tile-major (the layout of SampleDev): event i is slot i % 256 of
// tile i / 256; after the planes of a tile come its decay times (data: a
// double each in fp64 tiles, a double-float pair in fp32 tiles) or weights
// (weighted MC); the decay times also go to the component-cache tile.
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(256) k_precompute(Momenta mom, int64_t n, const DevModel* __restrict__ dm,
                                                    unsigned char* planes, int64_t tile_bytes, int npl,
                                                    const double* __restrict__ t, const double* __restrict__ w,
                                                    unsigned char* cache, int64_t cache_tile_bytes,
                                                    float* __restrict__ lo) {
  using T = typename std::conditional<F32, float, double>::type;
  constexpr int TE = kTileEvents;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t tile = i / TE;
  const int e = int(i % TE);
  T* out = reinterpret_cast<T*>(planes + tile * tile_bytes);
  V4 p[4];
  for (int a = 0; a < 4; ++a)
    p[a] = {__ldg(mom.p[a][0] + i), __ldg(mom.p[a][1] + i), __ldg(mom.p[a][2] + i), __ldg(mom.p[a][3] + i)};
  const int NS = dm->NS, NX = dm->NX, NT = dm->U * dm->NO;
  const int NSP = F32 ? 2 * NS : NS;
  double sv[kMaxSPlanes];
  for (int sp = 0; sp < NS; ++sp) {
    V4 P = {0, 0, 0, 0};
    const int mask = dm->splane_mask[sp];
    for (int a = 0; a < 4; ++a)
      if (mask & (1 << a)) P = P + p[a];
    const double s = dot(P, P);
    sv[sp] = s;
    if (F32) {
      const float hi = float(s);
      out[sp * TE + e] = hi;
      out[(NS + sp) * TE + e] = float(s - double(hi));
    } else {
      out[sp * TE + e] = T(s);
    }
  }
  for (int xp = 0; xp < NX; ++xp) {
    const double s = sv[dm->xplane_s[xp]];
    const int L = dm->xplane_L[xp];
    const double ma = dm->xplane_ma[xp], mb = dm->xplane_mb[xp];
    const double q2 = breakup2(s, ma * ma, mb * mb);
    const double q = sqrt(q2);
    double qp = q;
    for (int l = 0; l < L; ++l) qp *= q2;
    const double F = barrier(L, q2 * dm->r_res * dm->r_res);
    const double X = qp * F * F / sqrt(s);
    out[(NSP + xp) * TE + e] = T(X);
    if (F32 && lo) lo[(tile * (NX + NT) + xp) * TE + e] = float(X - double(float(X)));
  }
  for (int k = 0; k < NT; ++k) {
    const int* pt = dm->term_parts[k];
    const double K = spin_barrier(dm->term_spin[k], p[pt[0]], p[pt[1]], p[pt[2]], p[pt[3]], dm->r_res,
                                  dm->r_parent);
    out[(NSP + NX + k) * TE + e] = T(K);
    if (F32 && lo) lo[(tile * (NX + NT) + NX + k) * TE + e] = float(K - double(float(K)));
  }
  unsigned char* extra = planes + tile * tile_bytes + int64_t(npl) * TE * sizeof(T);
  if (t) {
    // the decay time: a double (fp64 tiles) or a double-float pair (fp32 tiles)
    unsigned char* tc = cache ? cache + tile * cache_tile_bytes + int64_t(2 * dm->U) * TE * sizeof(T) : nullptr;
    if constexpr (F32) {
      const float hi = float(t[i]);
      const float2 v = make_float2(hi, float(t[i] - double(hi)));
      reinterpret_cast<float2*>(extra)[e] = v;
      if (tc) reinterpret_cast<float2*>(tc)[e] = v;
    } else {
      reinterpret_cast<double*>(extra)[e] = t[i];
      if (tc) reinterpret_cast<double*>(tc)[e] = t[i];
    }
  } else if (w) {
    reinterpret_cast<T*>(extra)[e] = T(w[i]);
  }
}

void launch_precompute(bool f32, const Momenta& mom, int64_t n, const DevModel* dm, void* planes, int64_t tile_bytes,
                       int npl, const double* t, const double* w, void* cache, int64_t cache_tile_bytes, float* lo,
                       cudaStream_t st) {
  if (n <= 0) return;
  const int threads = 256;
  const unsigned blocks = unsigned((n + threads - 1) / threads);
  auto* pl = static_cast<unsigned char*>(planes);
  auto* ca = static_cast<unsigned char*>(cache);
  if (f32) k_precompute<true><<<blocks, threads, 0, st>>>(mom, n, dm, pl, tile_bytes, npl, t, w, ca, cache_tile_bytes,
                                                         lo);
  else k_precompute<false><<<blocks, threads, 0, st>>>(mom, n, dm, pl, tile_bytes, npl, t, w, ca, cache_tile_bytes,
                                                          nullptr);
}

// Fixed-order sum of a vector (one block).
__global__ void __launch_bounds__(1024) k_sum(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double part[1024];
  double a = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += v[i];
  part[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

void launch_sum(const double* v, int64_t n, double* out, cudaStream_t st) {
  k_sum<<<1, 1024, 0, st>>>(v, n, out);
}

}  // namespace tdmix
