// Instantiates the per-event kernels for every compiled model structure in
// one precision (TDMIX_PREC_F32 = 0: fp64 path, 1: fp32 precision path).
#include <mutex>
#include <string>

#include "fused.cuh"
#include "generate.cuh"
#include "serve.cuh"
#include "kernels.hpp"
#include "shapes_gen.h"
#include "../../include/tdmix.h"

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

// Raises the dynamic shared-memory limit of kernel `f` to at least `smem`
// bytes on the current device (cudaFuncSetAttribute acts per device); `seen`
// holds the limit set so far per device.  Safe to call from several host
// threads: the check, the attribute call and the update run under one
// mutex per device, and the limit only ever grows (it is set to the larger
// of the request and what was set before).
struct SmemLimit {
  std::mutex mu[kMaxDevices];
  int seen[kMaxDevices] = {};
};

template <class F>
cudaError_t allow_smem(F* f, int smem, SmemLimit& lim) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  std::lock_guard<std::mutex> g(lim.mu[dev]);
  if (smem <= lim.seen[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  lim.seen[dev] = smem;
  return cudaSuccess;
}

template <class S>
struct Ops {
  // normalisation-matrix accumulation available for this structure
  static constexpr bool kRegs = S::U <= kMaxRegisterGramU;
  static constexpr bool kTensor = Prec::kF32 && S::U <= 16;
  static constexpr bool kShared = !Prec::kF32 && !kRegs && S::U <= 16;
  static constexpr bool kOk = kRegs || kTensor || kShared;
  // the mode of the cached path (no MC tiles: the mode only names the kernel)
  static constexpr int kCacheGram = kRegs ? kGramRegs : (Prec::kF32 ? kGramTensor : kGramShared);

  template <bool FULL, bool GRAD, bool W, bool RATES, int GRAM>
  static cudaError_t launch(int grid, bool pdl, cudaStream_t st, const EvalArgs& a) {
    const int smem = Layout<Prec, S, GRAM>::smem_bytes(FULL, int(a.ld));
    static SmemLimit seen;  // per instantiation
    const cudaError_t e = allow_smem(k_eval<Prec, S, FULL, GRAD, W, RATES, GRAM>, smem, seen);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(kTile);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_eval<Prec, S, FULL, GRAD, W, RATES, GRAM>, a);
  }
  template <int GRAM>
  static cudaError_t eval_full(bool grad, int grid, bool pdl, cudaStream_t st, const EvalArgs& a) {
    const bool w = a.mc.weighted != 0;
    if (a.rates && !grad)  // per-event rates (always a full evaluation without gradient)
      return w ? launch<true, false, true, true, GRAM>(grid, pdl, st, a)
               : launch<true, false, false, true, GRAM>(grid, pdl, st, a);
    if (grad)
      return w ? launch<true, true, true, false, GRAM>(grid, pdl, st, a)
               : launch<true, true, false, false, GRAM>(grid, pdl, st, a);
    return w ? launch<true, false, true, false, GRAM>(grid, pdl, st, a)
             : launch<true, false, false, false, GRAM>(grid, pdl, st, a);
  }
  static cudaError_t eval(bool full, bool grad, int grid, bool pdl, cudaStream_t st, const EvalArgs& a) {
    if constexpr (kOk) {
      if (!full)
        return grad ? launch<false, true, false, false, kCacheGram>(grid, pdl, st, a)
                    : launch<false, false, false, false, kCacheGram>(grid, pdl, st, a);
      if constexpr (Prec::kF32) {
        if constexpr (kRegs)
          if (a.gram_pref != TDMIX_GRAM_TENSOR) return eval_full<kGramRegs>(grad, grid, pdl, st, a);
        return eval_full<kGramTensor>(grad, grid, pdl, st, a);
      } else {
        if (a.gram_pref == TDMIX_GRAM_TENSOR) return cudaErrorNotSupported;
        if constexpr (kRegs) return eval_full<kGramRegs>(grad, grid, pdl, st, a);
        else return eval_full<kGramShared>(grad, grid, pdl, st, a);
      }
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t derive(int K, const double* params, int np, const ModelConst& km, void* out, cudaStream_t st) {
    k_derive<Prec, S><<<K, kTile, 0, st>>>(params, np, km, static_cast<DerivedConst<typename Prec::T>*>(out));
    return cudaGetLastError();
  }
  static cudaError_t serve(int grid, cudaStream_t st, const ServeLoopArgs& a) {
    if constexpr (kOk) {
      const int smem = ServeLayout<Prec, S>::smem_bytes();
      static SmemLimit seen;
      const cudaError_t e = allow_smem(k_serve_loop<Prec, S, true>, smem, seen);
      if (e != cudaSuccess) return e;
      k_serve_loop<Prec, S, true><<<grid, kTile, smem, st>>>(a);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
};

}  // namespace

#if !TDMIX_PREC_F32
namespace {
template <class S>
struct Gen {
  static cudaError_t pass1(int grid, cudaStream_t st, const GenArgs& a) {
    k_gen_pass1<S><<<grid, kGenThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t pass2(int grid, cudaStream_t st, const GenArgs& a) {
    k_gen_pass2<S><<<grid, kGenThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
};
}  // namespace

// The generator evaluates the rate in double precision whatever the
// precision of the context, so it is compiled once (here).
const GenOps* find_gen_ops(const std::string& sig) {
#define TDMIX_GEN_ENTRY(S)                                                    \
  if (sig == shapes::S::sig()) {                                              \
    static const GenOps o = {&Gen<shapes::S>::pass1, &Gen<shapes::S>::pass2}; \
    return &o;                                                                \
  }
  TDMIX_FOR_EACH_SHAPE(TDMIX_GEN_ENTRY)
#undef TDMIX_GEN_ENTRY
  return nullptr;
}
#endif

const ShapeOps* TDMIX_FIND(const std::string& sig) {
#define TDMIX_SHAPE_ENTRY(S)                                                                  \
  if (Ops<shapes::S>::kOk && sig == shapes::S::sig()) {                                       \
    using LY_ = Layout<Prec, shapes::S>;                                                      \
    static const ShapeOps o = {shapes::S::sig(), shapes::S::U, shapes::S::NR, LY_::WMC, LY_::WD, \
                               LY_::NPL_FULL, LY_::data_tile_bytes(), LY_::mc_tile_bytes(false), \
                               LY_::mc_tile_bytes(true), LY_::cache_tile_bytes(),               \
                               &Ops<shapes::S>::eval, &Ops<shapes::S>::serve,                 \
                               ServeLayout<Prec, shapes::S>::WR, &Ops<shapes::S>::derive,     \
                               int64_t(sizeof(DerivedConst<typename Prec::T>)), LY_::cached_blocks}; \
    return &o;                                                                                \
  }
  TDMIX_FOR_EACH_SHAPE(TDMIX_SHAPE_ENTRY)
#undef TDMIX_SHAPE_ENTRY
  return nullptr;
}

}  // namespace tdmix
