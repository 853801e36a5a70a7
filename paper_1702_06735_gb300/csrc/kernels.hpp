// Host-side launchers of the kernels (declarations shared by the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "device_tables.hpp"

namespace tdmix {

struct Momenta {
  const double* p[4][4];  // [particle][E, px, py, pz], device planes
};

void launch_precompute(bool f32, const Momenta& mom, int64_t n, int64_t pitch, const DevModel* dm, void* s_out,
                       void* x_out, void* k_out, cudaStream_t st);
void launch_sum(const double* v, int64_t n, double* out, cudaStream_t st);
void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t st);

// Launcher of the model-specialised evaluation kernel.
struct ShapeOps {
  const char* signature;
  int U, NR;
  int mc_width;    // MC columns of a block-partial row
  int data_width;  // data columns
  // full: recompute components and run the MC tiles; otherwise read the
  // component cache and reuse the stored MC totals.
  cudaError_t (*eval)(bool full, bool grad, int grid, cudaStream_t st, const EvalArgs& a, const int* floating);
  // batched evaluation of serving requests (see serve.cuh)
  cudaError_t (*serve)(bool grad, int grid, cudaStream_t st, const ServeArgs& a);
};

// Specialisation compiled for a model signature, or null.
const ShapeOps* find_shape_ops(const std::string& signature, bool f32);

}  // namespace tdmix
