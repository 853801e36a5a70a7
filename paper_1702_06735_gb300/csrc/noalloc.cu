// Allocation-free log-likelihood sum over a caller-provided component cache.
//
// Some callers cannot allocate device memory at the time they evaluate: code
// recorded into a CUDA graph, code that runs under an external memory
// manager that owns every device allocation, or a real-time loop that must
// not block on the allocator.  This entry point serves them: it reads the
// caller's inputs, writes the caller's output and keeps its block partial
// sums in a fixed-size file-scope device array instead of allocating.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/tdmix.h"
#include "model.hpp"

namespace {

constexpr int kThreads = 256;

// Block-partial scratch shared by every call on a device (2 doubles per
// block).  Every GPU that loads this library holds it until the process exits.
__device__ __align__(256) double g_noalloc_scratch[TDMIX_NOALLOC_MAX_BLOCKS * 2];

// Device address of g_noalloc_scratch, looked up once per device.
double* g_scratch_addr[TDMIX_NOALLOC_MAX_DEVICES];
std::once_flag g_scratch_once[TDMIX_NOALLOC_MAX_DEVICES];
cudaError_t g_scratch_err[TDMIX_NOALLOC_MAX_DEVICES];

__global__ void __launch_bounds__(kThreads) k_loglik_partials(int U, int64_t n, int64_t ld,
                                                              const double* __restrict__ a_re,
                                                              const double* __restrict__ a_im,
                                                              const double* __restrict__ t,
                                                              const double* __restrict__ cA,
                                                              const double* __restrict__ cB, double x, double y,
                                                              double gamma, double* __restrict__ scratch) {
  __shared__ double c[4 * tdmix::kMaxComp];
  __shared__ double red[2][kThreads / 32];
  for (int k = threadIdx.x; k < 2 * U; k += blockDim.x) {
    c[k] = cA[k];
    c[2 * tdmix::kMaxComp + k] = cB[k];
  }
  __syncthreads();
  double lnb = 0.0, bad = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double Ar = 0, Ai = 0, Br = 0, Bi = 0;
    for (int j = 0; j < U; ++j) {
      const double ar = a_re[j * ld + i], ai = a_im[j * ld + i];
      const double car = c[2 * j], cai = c[2 * j + 1];
      const double cbr = c[2 * tdmix::kMaxComp + 2 * j], cbi = c[2 * tdmix::kMaxComp + 2 * j + 1];
      Ar += car * ar - cai * ai;
      Ai += car * ai + cai * ar;
      Br += cbr * ar - cbi * ai;
      Bi += cbr * ai + cbi * ar;
    }
    // B = 2 |cosh(w) A - sinh(w) Abar|^2, w = (y + i x) gamma t / 2
    const double gt = gamma * t[i];
    const double a = 0.5 * y * gt, b = 0.5 * x * gt;
    double sb, cb;
    sincos(b, &sb, &cb);
    const double cha = cosh(a), sha = sinh(a);
    const double chr = cha * cb, chi = sha * sb, shr = sha * cb, shi = cha * sb;
    const double Zr = chr * Ar - chi * Ai - (shr * Br - shi * Bi);
    const double Zi = chr * Ai + chi * Ar - (shr * Bi + shi * Br);
    const double B = 2.0 * (Zr * Zr + Zi * Zi);
    if (B > 0.0 && B < INFINITY) lnb += log(B);
    else bad += 1.0;
  }
  for (int off = 16; off > 0; off >>= 1) {
    lnb += __shfl_down_sync(0xffffffffu, lnb, off);
    bad += __shfl_down_sync(0xffffffffu, bad, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = lnb;
    red[1][warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0, q = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      s += red[0][w];
      q += red[1][w];
    }
    scratch[2 * blockIdx.x] = s;
    scratch[2 * blockIdx.x + 1] = q;
  }
}

__global__ void k_loglik_finish(int nblocks, const double* __restrict__ scratch, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0, q = 0;
  for (int b = 0; b < nblocks; ++b) {
    s += scratch[2 * b];
    q += scratch[2 * b + 1];
  }
  out[0] = s;
  out[1] = q;
}

}  // namespace

extern "C" int tdmix_loglik_components_noalloc(int U, int64_t n, const double* a_re, const double* a_im, int64_t ld,
                                               const double* t, const double* cA, const double* cB, double x,
                                               double y, double gamma, double* out, void* stream) {
  if (U < 1 || U > tdmix::kMaxComp || n < 1 || ld < n || !a_re || !a_im || !t || !cA || !cB || !out)
    return TDMIX_ERR_ARG;
  if (!(fabs(y) < 1.0) || !(gamma > 0)) return TDMIX_ERR_DOMAIN;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TDMIX_ERR_CUDA;
  if (dev < 0 || dev >= TDMIX_NOALLOC_MAX_DEVICES) return TDMIX_ERR_ARG;
  std::call_once(g_scratch_once[dev], [dev] {
    void* p = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    g_scratch_addr[dev] = static_cast<double*>(p);
  });
  if (g_scratch_err[dev] != cudaSuccess || !g_scratch_addr[dev]) return TDMIX_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // a failure left by earlier, unrelated work must not be reported here
  const int64_t want = (n + kThreads - 1) / kThreads;
  const int blocks = int(want < TDMIX_NOALLOC_MAX_BLOCKS ? want : TDMIX_NOALLOC_MAX_BLOCKS);
  k_loglik_partials<<<blocks, kThreads, 0, st>>>(U, n, ld, a_re, a_im, t, cA, cB, x, y, gamma, g_scratch_addr[dev]);
  k_loglik_finish<<<1, 32, 0, st>>>(blocks, g_scratch_addr[dev], out);
  return cudaGetLastError() == cudaSuccess ? TDMIX_OK : TDMIX_ERR_CUDA;
}
