// Host-side launchers of the kernels (declarations shared by the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "device_tables.hpp"

namespace tdmix {

struct Momenta {
  const double* p[4][4];  // [particle][E, px, py, pz], device planes
};

// Kinematic precompute into the tile-major planes of a sample (see
// SampleDev); t (data) and w (weighted MC) are device f64 arrays or null;
// cache (data) receives the decay times of its tiles, or null; lo (fp32
// data) receives the rounding residuals of the width and spin x barrier
// factors (SampleDev::lo), or null.
void launch_precompute(bool f32, const Momenta& mom, int64_t n, const DevModel* dm, void* planes, int64_t tile_bytes,
                       int npl, const double* t, const double* w, void* cache, int64_t cache_tile_bytes, float* lo,
                       cudaStream_t st);
void launch_sum(const double* v, int64_t n, double* out, cudaStream_t st);

// Launcher of the model-specialised evaluation kernel.
struct ShapeOps {
  const char* signature;
  int U, NR;
  int mc_width;    // MC columns of a block-partial row
  int data_width;  // data columns
  // full: recompute components and run the MC tiles; otherwise read the
  // component cache and reuse the stored MC totals.
  int n_planes;    // event planes per tile (NPL)
  int64_t data_tile_bytes, mc_tile_bytes, mc_tile_bytes_weighted, cache_tile_bytes;
  // pdl: launched with programmatic stream serialization, so that it may
  // start while the evaluation before it in the stream finishes (the kernel
  // waits for that one before it writes anything a later one reads)
  cudaError_t (*eval)(bool full, bool grad, int grid, bool pdl, cudaStream_t st, const EvalArgs& a);
  // the persistent serving loop (see serve.cuh)
  cudaError_t (*serve)(int grid, cudaStream_t st, const ServeLoopArgs& a);
  int serve_row_stride;  // float2 entries per chunk-partial row
  // per-evaluation constants of K parameter vectors (device, K x np) into
  // `out` (K records of derived_bytes), for the evaluations of a batch
  // (EvalArgs::derived); null where the path derives them itself
  cudaError_t (*derive)(int K, const double* params, int np, const ModelConst& km, void* out, cudaStream_t st);
  int64_t derived_bytes;
  int cached_blocks;  // blocks per SM of the cached pass (component cache in, no MC tiles)
};

// Launcher of the runtime-table evaluation (generic.cu) for model
// structures without a compiled specialisation; fits ShapeOps::eval.
cudaError_t generic_eval(bool full, bool grad, int grid, bool pdl, cudaStream_t st, const EvalArgs& a);

// Table of the kernels' logarithm ({1/F, ln F} pairs, F = 1 + j/128).
std::vector<double> make_log_table();

struct GenArgs;
// Launchers of the event generator of one model structure (generate.cuh):
// pass 1 (accept bits, block counts, largest weight) and pass 2 (write the
// accepted events), grid blocks of kGenPerBlock candidates each.
struct GenOps {
  cudaError_t (*pass1)(int grid, cudaStream_t st, const GenArgs& a);
  cudaError_t (*pass2)(int grid, cudaStream_t st, const GenArgs& a);
};
const GenOps* find_gen_ops(const std::string& signature);

// Specialisation compiled for a model signature, or null.
const ShapeOps* find_shape_ops(const std::string& signature, bool f32);

}  // namespace tdmix
