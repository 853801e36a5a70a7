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
                        double* rows) {
    if constexpr (kOk) {
      if (grad) k_mc<Prec, S, true><<<grid, 256, 0, st>>>(d, ec, rows);
      else k_mc<Prec, S, false><<<grid, 256, 0, st>>>(d, ec, rows);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t data(bool from_cache, bool grad, int grid, cudaStream_t st, const SampleDev& d,
                          const EvalConst* ec, double* rows, double* rates) {
    if constexpr (kOk) {
      if (from_cache) {
        if (grad) k_data<Prec, S, true, true><<<grid, 256, 0, st>>>(d, ec, rows, rates);
        else k_data<Prec, S, true, false><<<grid, 256, 0, st>>>(d, ec, rows, rates);
      } else {
        if (grad) k_data<Prec, S, false, true><<<grid, 256, 0, st>>>(d, ec, rows, rates);
        else k_data<Prec, S, false, false><<<grid, 256, 0, st>>>(d, ec, rows, rates);
      }
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static int mc_bps(bool grad) {
    int n = 0;
    if constexpr (kOk) {
      if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mc<Prec, S, true>, 256, 0);
      else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mc<Prec, S, false>, 256, 0);
    }
    return n;
  }
  static int data_bps(bool from_cache, bool grad) {
    int n = 0;
    if constexpr (kOk) {
      if (from_cache) {
        if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, true, true>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, true, false>, 256, 0);
      } else {
        if (grad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, false, true>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_data<Prec, S, false, false>, 256, 0);
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
