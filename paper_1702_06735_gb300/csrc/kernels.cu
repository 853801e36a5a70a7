// Model-independent kernels run once per event load: kinematic precompute,
// sum of decay times, weight conversion.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "device_tables.hpp"
#include "kernels.hpp"
#include "kinematics.cuh"

namespace tdmix {

// ---------------------------------------------------------------------------
// Kinematic precompute (one thread per event, fp64): invariants s, width
// factors X(s) = q^(2L+1) F_L(q r)^2 / sqrt(s) and the spin x barrier factor
// K_{j,o} of every component ordering.  None depends on fit parameters.
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(256) k_precompute(Momenta mom, int64_t n, int64_t pitch,
                                                    const DevModel* __restrict__ dm, void* s_out,
                                                    void* x_out, void* k_out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V4 p[4];
  for (int a = 0; a < 4; ++a)
    p[a] = {__ldg(mom.p[a][0] + i), __ldg(mom.p[a][1] + i), __ldg(mom.p[a][2] + i), __ldg(mom.p[a][3] + i)};
  const int NS = dm->NS, NX = dm->NX, NT = dm->U * dm->NO;
  double sv[kMaxSPlanes];
  for (int sp = 0; sp < NS; ++sp) {
    V4 P = {0, 0, 0, 0};
    const int mask = dm->splane_mask[sp];
    for (int a = 0; a < 4; ++a)
      if (mask & (1 << a)) P = P + p[a];
    const double s = dot(P, P);
    sv[sp] = s;
    if (F32) {
      float hi = float(s);
      float lo = float(s - double(hi));
      static_cast<float*>(s_out)[sp * pitch + i] = hi;
      static_cast<float*>(s_out)[(NS + sp) * pitch + i] = lo;
    } else {
      static_cast<double*>(s_out)[sp * pitch + i] = s;
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
    if (F32) static_cast<float*>(x_out)[xp * pitch + i] = float(X);
    else static_cast<double*>(x_out)[xp * pitch + i] = X;
  }
  for (int t = 0; t < NT; ++t) {
    const int* pt = dm->term_parts[t];
    const double K = spin_barrier(dm->term_spin[t], p[pt[0]], p[pt[1]], p[pt[2]], p[pt[3]], dm->r_res,
                                  dm->r_parent);
    if (F32) static_cast<float*>(k_out)[t * pitch + i] = float(K);
    else static_cast<double*>(k_out)[t * pitch + i] = K;
  }
}

void launch_precompute(bool f32, const Momenta& mom, int64_t n, int64_t pitch, const DevModel* dm, void* s_out,
                       void* x_out, void* k_out, cudaStream_t st) {
  if (n <= 0) return;
  const int threads = 256;
  const unsigned blocks = unsigned((n + threads - 1) / threads);
  if (f32) k_precompute<true><<<blocks, threads, 0, st>>>(mom, n, pitch, dm, s_out, x_out, k_out);
  else k_precompute<false><<<blocks, threads, 0, st>>>(mom, n, pitch, dm, s_out, x_out, k_out);
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

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = float(in[i]);
}

void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_to_f32<<<unsigned((n + 255) / 256), 256, 0, st>>>(in, out, n);
}

}  // namespace tdmix
