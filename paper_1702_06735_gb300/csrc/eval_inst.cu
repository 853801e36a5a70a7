// Instantiates the per-event kernels for every compiled model structure in
// one precision (TDMIX_PREC_F32 = 0: fp64 path, 1: fp32 precision path).
#include <string>

#include "eval.cuh"
#include "kernels.hpp"
#include "shapes_gen.h"

#ifndef TDMIX_PREC_F32
#error "define TDMIX_PREC_F32"
#endif

namespace tdmix {

#if TDMIX_PREC_F32
using Prec = PrecF32;
#define TDMIX_FIND find_shape_ops_f32
#else
using Prec = PrecF64;
#define TDMIX_FIND find_shape_ops_f64
#endif

namespace {  // internal linkage: this file is compiled once per precision

// Per-thread register accumulation of the Gram matrix is used up to this
// many components.
constexpr int kMaxRegisterGramU = 8;

template <class S>
struct Ops {
  static constexpr bool kOk = S::U <= kMaxRegisterGramU;
  static cudaError_t mc(bool grad, int grid, cudaStream_t st, const SampleDev& d, const EvalConst* ec,
                        double* part, int64_t ld, int* err) {
    if constexpr (kOk) {
      using T = typename Prec::T;
      const bool weighted = d.w != nullptr;
      const int smem = 2 * mc_planes<Prec, S>(weighted) * kMcTile * int(sizeof(T));
      auto kern = grad ? (weighted ? k_mc<Prec, S, true, true> : k_mc<Prec, S, true, false>)
                       : (weighted ? k_mc<Prec, S, false, true> : k_mc<Prec, S, false, false>);
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      kern<<<grid, kMcTile, smem, st>>>(d, ec, part, ld, err);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t data(bool from_cache, bool grad, int grid, cudaStream_t st, const SampleDev& d,
                          const EvalConst* ec, double* part, int64_t ld, double* rates) {
    if constexpr (kOk) {
      auto kern = from_cache ? (grad ? k_data<Prec, S, true, true> : k_data<Prec, S, true, false>)
                             : (grad ? k_data<Prec, S, false, true> : k_data<Prec, S, false, false>);
      kern<<<grid, kDataThreads, 0, st>>>(d, ec, part, ld, rates);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static int mc_bps(bool) { return 1; }  // persistent: one block per SM
  static int data_bps(bool from_cache, bool grad) {
    int n = 0;
    if constexpr (kOk) {
      if (from_cache) {
        if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, true, true>, kDataThreads, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, true, false>, kDataThreads, 0);
      } else {
        if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, false, true>, kDataThreads, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, false, false>, kDataThreads, 0);
      }
    }
    return n;
  }
};

}  // namespace

const ShapeOps* TDMIX_FIND(const std::string& sig) {
#define TDMIX_SHAPE_ENTRY(S)                                                                          \
  if (Ops<shapes::S>::kOk && sig == shapes::S::sig()) {                                               \
    static const ShapeOps o = {shapes::S::sig(),                                                      \
                               shapes::S::U,                                                          \
                               shapes::S::NR,                                                         \
                               1 + shapes::S::U * shapes::S::U + 2 * shapes::S::NR,                   \
                               4 + 4 * shapes::S::U + 2 * shapes::S::NR,                              \
                               kDataThreads,                                                          \
                               &Ops<shapes::S>::mc,                                                   \
                               &Ops<shapes::S>::data,                                                 \
                               &Ops<shapes::S>::mc_bps,                                               \
                               &Ops<shapes::S>::data_bps};                                            \
    return &o;                                                                                        \
  }
  TDMIX_FOR_EACH_SHAPE(TDMIX_SHAPE_ENTRY)
#undef TDMIX_SHAPE_ENTRY
  return nullptr;
}

}  // namespace tdmix
