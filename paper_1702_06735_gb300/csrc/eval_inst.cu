// Instantiates the per-event kernels for every compiled model structure in
// one precision (TDMIX_PREC_F32 = 0: fp64 path, 1: fp32 precision path).
#include <atomic>
#include <string>

#include "fused.cuh"
#include "serve.cuh"
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

constexpr int kMaxDevices = 64;

// Raises the dynamic shared-memory limit of kernel `f` to `smem` bytes on the
// current device once (cudaFuncSetAttribute acts per device); `seen` holds
// the largest size allowed so far per device.  Safe to call from several
// host threads.
template <class F>
cudaError_t allow_smem(F* f, int smem, std::atomic<int> (&seen)[kMaxDevices]) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (smem <= seen[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int cur = seen[dev].load(std::memory_order_relaxed);
  while (cur < smem && !seen[dev].compare_exchange_weak(cur, smem, std::memory_order_release)) {
  }
  return cudaSuccess;
}

template <class S>
struct Ops {
  static constexpr bool kOk = S::U <= kMaxRegisterGramU;
  template <bool FULL, bool GRAD, bool W>
  static cudaError_t launch(int grid, cudaStream_t st, const EvalArgs& a) {
    const int smem = Layout<Prec, S>::smem_bytes(FULL, int(a.ld));
    static std::atomic<int> seen[kMaxDevices];  // per instantiation and device
    const cudaError_t e = allow_smem(k_eval<Prec, S, FULL, GRAD, W>, smem, seen);
    if (e != cudaSuccess) return e;
    k_eval<Prec, S, FULL, GRAD, W><<<grid, kTile, smem, st>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t eval(bool full, bool grad, int grid, cudaStream_t st, const EvalArgs& a) {
    if constexpr (kOk) {
      const bool w = a.mc.weighted != 0;
      if (full) {
        if (grad) return w ? launch<true, true, true>(grid, st, a) : launch<true, true, false>(grid, st, a);
        return w ? launch<true, false, true>(grid, st, a) : launch<true, false, false>(grid, st, a);
      }
      return grad ? launch<false, true, false>(grid, st, a) : launch<false, false, false>(grid, st, a);
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t serve(bool grad, int grid, cudaStream_t st, const ServeArgs& a) {
    if constexpr (kOk) {
      const int smem = ServeLayout<Prec, S>::smem_bytes();
      static std::atomic<int> seen_g[kMaxDevices], seen_n[kMaxDevices];
      auto kern = grad ? k_serve<Prec, S, true> : k_serve<Prec, S, false>;
      const cudaError_t e = allow_smem(kern, smem, grad ? seen_g : seen_n);
      if (e != cudaSuccess) return e;
      kern<<<grid, kTile, smem, st>>>(a);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
};

}  // namespace

const ShapeOps* TDMIX_FIND(const std::string& sig) {
#define TDMIX_SHAPE_ENTRY(S)                                                                  \
  if (Ops<shapes::S>::kOk && sig == shapes::S::sig()) {                                       \
    using LY_ = Layout<Prec, shapes::S>;                                                      \
    static const ShapeOps o = {shapes::S::sig(), shapes::S::U, shapes::S::NR, LY_::WMC, LY_::WD, \
                               LY_::NPL_FULL, LY_::data_tile_bytes(), LY_::mc_tile_bytes(false), \
                               LY_::mc_tile_bytes(true), LY_::cache_tile_bytes(),               \
                               &Ops<shapes::S>::eval, &Ops<shapes::S>::serve};                \
    return &o;                                                                                \
  }
  TDMIX_FOR_EACH_SHAPE(TDMIX_SHAPE_ENTRY)
#undef TDMIX_SHAPE_ENTRY
  return nullptr;
}

}  // namespace tdmix
