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

// One record {Ar, Ai, Br, Bi, t, x, y, Gamma} of the Eq. (mix) codes: the
// amplitudes are rounded to float and the decay time to a double-float pair
// for both paths, so that they start from the same values.
struct MixCase {
  float Ar, Ai, Br, Bi;
  DF t;
  BlockConst<float> bf;
  BlockConst<double> bd;
};

__device__ MixCase mix_case(const double* r) {
  MixCase c;
  c.Ar = float(r[0]);
  c.Ai = float(r[1]);
  c.Br = float(r[2]);
  c.Bi = float(r[3]);
  c.t = df_from_double(r[4]);
  const double x = r[5], y = r[6], g = r[7];
  const double hx = 0.5 * x * g, hy = 0.5 * y * g;
  const double mg = fmax(fabs(x), fabs(y)) * g;
  const double ig = mg > 0 ? 1.0 / mg : INFINITY;
  const unsigned long long t0 = static_cast<unsigned long long>(__double_as_longlong(0.04 * ig));
  const unsigned long long t1 = static_cast<unsigned long long>(__double_as_longlong(0.2 * ig));
  c.bf.x = c.bd.x = x;
  c.bf.y = c.bd.y = y;
  c.bf.gamma = c.bd.gamma = g;
  c.bf.hx = c.bd.hx = hx;
  c.bf.hy = c.bd.hy = hy;
  c.bf.xf = c.bd.xf = float(x);
  c.bf.yf = c.bd.yf = float(y);
  c.bf.gammaf = c.bd.gammaf = float(g);
  const DF hx2 = df_from_double(hx), hy2 = df_from_double(hy);
  c.bf.hxh = hx2.hi;
  c.bf.hxl = hx2.lo;
  c.bf.hyh = hy2.hi;
  c.bf.hyl = hy2.lo;
  c.bf.tlim[0] = c.bd.tlim[0] = t0;
  c.bf.tlim[1] = c.bd.tlim[1] = t1;
  return c;
}

// which: see tdmix_test_math in the header.  Outputs per argument: one
// double, or four for the mixing-series and Eq. (mix) codes.
__global__ void k_test_math(int which, int64_t n, const double* __restrict__ in, double* __restrict__ out,
                            const double2* __restrict__ tab, const float4* __restrict__ tab_f) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (which == TDMIX_MATH_MIX_DF || which == TDMIX_MATH_MIX_F64) {
    const MixCase c = mix_case(in + 8 * i);
    double rate = 0.0, lnb = 0.0;
    int lexp = 0;
    bool ok;
    float f0, f1, f2, f3, gx = 0.f, gy = 0.f;
    if (which == TDMIX_MATH_MIX_DF) {
      DF l{0.0f, 0.0f};
      ok = mix_event_df<false>(c.bf, tab, tab_f, DF{c.Ar, 0.0f}, DF{c.Ai, 0.0f}, DF{c.Br, 0.0f}, DF{c.Bi, 0.0f},
                               c.t.hi, c.t.lo, l, lexp, &rate, f0, f1, f2, f3, gx, gy);
      lnb = df_to_double(l);
    } else {
      double d0, d1, d2, d3, dx = 0.0, dy = 0.0;
      ok = mix_event<PrecF64, false>(c.bd, tab, c.Ar, c.Ai, c.Br, c.Bi, c.Ar, c.Ai, c.Br, c.Bi, df_to_double(c.t),
                                     lnb, lexp, &rate, d0, d1, d2, d3, dx, dy);
    }
    out[4 * i] = ok ? fma(double(lexp), kLn2, lnb) : NAN;
    out[4 * i + 1] = rate;
    out[4 * i + 2] = ok ? 1.0 : 0.0;
    out[4 * i + 3] = 0.0;
    return;
  }
  const double v = in[i];
  switch (which) {
    case TDMIX_MATH_LOG_DF: {
      int e;
      DF l;
      out[i] = log_df(df_from_double(v), tab_f, e, l) ? fma(double(e), kLn2, df_to_double(l)) : NAN;
      break;
    }
    case TDMIX_MATH_LOG_TABLE: out[i] = log_table(v, tab); break;
    case TDMIX_MATH_LOG_CUDA: out[i] = log(v); break;
    case TDMIX_MATH_RCP_F64: out[i] = rcp<double>(v); break;
    case TDMIX_MATH_DIV_F64: out[i] = 1.0 / v; break;
    case TDMIX_MATH_RCP_F32: out[i] = double(rcp<float>(float(v))); break;
    case TDMIX_MATH_DIV_F32: out[i] = double(1.0f / float(v)); break;
    case TDMIX_MATH_RCP_APPROX_F32: out[i] = double(rcp_lineshape<float>(float(v))); break;
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
  const bool mix = which == TDMIX_MATH_MIX_DF || which == TDMIX_MATH_MIX_F64;
  const int per = (which >= TDMIX_MATH_MIX_TIER0 && which <= TDMIX_MATH_MIX_TIER2) || mix ? 4 : 1;
  const int per_in = mix ? 8 : 1;
  cudaGetLastError();
  const std::vector<double> tab = make_log_table();
  // the table as double-float pairs {1/F hi, lo, ln F hi, lo}, split as the kernels split it
  std::vector<float> tab_f(tab.size() * 2);
  for (size_t k = 0; k < tab.size(); ++k) {
    const float hi = float(tab[k]);
    tab_f[2 * k] = hi;
    tab_f[2 * k + 1] = float(tab[k] - double(hi));
  }
  double *d_in = nullptr, *d_out = nullptr, *d_tab = nullptr;
  float* d_tab_f = nullptr;
  int rc = TDMIX_OK;
  if (cudaMalloc(&d_in, per_in * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_out, per * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_tab, tab.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_tab_f, tab_f.size() * sizeof(float)) != cudaSuccess) {
    rc = TDMIX_ERR_NOMEM;
  } else if (cudaMemcpy(d_in, in, per_in * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d_tab_f, tab_f.data(), tab_f.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = TDMIX_ERR_CUDA;
  } else {
    k_test_math<<<unsigned((n + 255) / 256), 256>>>(which, n, d_in, d_out, reinterpret_cast<const double2*>(d_tab),
                                                    reinterpret_cast<const float4*>(d_tab_f));
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d_out, per * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = TDMIX_ERR_CUDA;
  }
  cudaFree(d_in);
  cudaFree(d_out);
  cudaFree(d_tab);
  cudaFree(d_tab_f);
  return rc;
}
