// Self-test entry of the hand-written device arithmetic (a library
// extension for testing): evaluates one of the kernels' math routines, or
// the CUDA function it stands in for, over a caller's argument vector, so
// that tests can compare the two directly.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/tdmix.h"
#include "eval.cuh"
#include "kernels.hpp"
#include "philox.cuh"

namespace {

using namespace tdmix;

// which: see tdmix_test_math in the header.  Outputs per argument: one
// double, or four for the mixing-series codes.
__global__ void k_test_math(int which, int64_t n, const double* __restrict__ in, double* __restrict__ out,
                            const double2* __restrict__ tab) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = in[i];
  switch (which) {
    case TDMIX_MATH_LOG_TABLE: out[i] = log_table(v, tab); break;
    case TDMIX_MATH_LOG_CUDA: out[i] = log(v); break;
    case TDMIX_MATH_RCP_F64: out[i] = rcp<double>(v); break;
    case TDMIX_MATH_DIV_F64: out[i] = 1.0 / v; break;
    case TDMIX_MATH_RCP_F32: out[i] = double(rcp<float>(float(v))); break;
    case TDMIX_MATH_DIV_F32: out[i] = double(1.0f / float(v)); break;
    case TDMIX_MATH_DF_RCP: {
      const float hi = float(v);
      out[i] = df_to_double(df_rcp(DF{hi, float(v - double(hi))}));
      break;
    }
    case TDMIX_MATH_MIX_TIER0:
    case TDMIX_MATH_MIX_TIER1:
    case TDMIX_MATH_MIX_TIER2: {
      double ch, sh, c, s;
      mixing_trig(v, v, which - TDMIX_MATH_MIX_TIER0, ch, sh, c, s);
      out[4 * i] = ch;
      out[4 * i + 1] = sh;
      out[4 * i + 2] = c;
      out[4 * i + 3] = s;
      break;
    }
    default: break;
  }
}

__global__ void k_test_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                              uint32_t* out) {
  const Philox4 r = philox4x32_10(Philox4{{c0, c1, c2, c3}}, k0, k1);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

}  // namespace

extern "C" int tdmix_test_philox(const uint32_t* counter, const uint32_t* key, uint32_t* out) {
  if (!counter || !key || !out) return TDMIX_ERR_ARG;
  cudaGetLastError();
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, 4 * sizeof(uint32_t)) != cudaSuccess) return TDMIX_ERR_NOMEM;
  k_test_philox<<<1, 1>>>(counter[0], counter[1], counter[2], counter[3], key[0], key[1], d);
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpy(out, d, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d);
  return ok ? TDMIX_OK : TDMIX_ERR_CUDA;
}

extern "C" int tdmix_test_math(int which, int64_t n, const double* in, double* out) {
  if (n < 1 || !in || !out || which < 0 || which >= TDMIX_MATH_CODES) return TDMIX_ERR_ARG;
  const int per = which >= TDMIX_MATH_MIX_TIER0 ? 4 : 1;
  cudaGetLastError();
  const std::vector<double> tab = make_log_table();
  double *d_in = nullptr, *d_out = nullptr, *d_tab = nullptr;
  int rc = TDMIX_OK;
  if (cudaMalloc(&d_in, n * sizeof(double)) != cudaSuccess || cudaMalloc(&d_out, per * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_tab, tab.size() * sizeof(double)) != cudaSuccess) {
    rc = TDMIX_ERR_NOMEM;
  } else if (cudaMemcpy(d_in, in, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = TDMIX_ERR_CUDA;
  } else {
    k_test_math<<<unsigned((n + 255) / 256), 256>>>(which, n, d_in, d_out, reinterpret_cast<const double2*>(d_tab));
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d_out, per * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = TDMIX_ERR_CUDA;
  }
  cudaFree(d_in);
  cudaFree(d_out);
  cudaFree(d_tab);
  return rc;
}
