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

struct FinalArgs {
  const DevModel* dm;
  const EvalConst* ec;
  const double* mc_part;    // null: use gram_store from an earlier pass
  int n_mc_rows;
  int64_t mc_ld;
  const double* data_part;
  int n_data_rows;
  int64_t data_ld;
  double* colsum;           // scratch: one double per reduced column
  unsigned* counter;        // scratch: blocks done (returned to 0 by the last block)
  double* gram_store;
  int64_t n_data;
  double sum_t;
  const int* floating;
  int want_grad;
  int have_res_grad;
  int* err;          // set by kernels whose bounded waits gave up; read and cleared here
  double* result;
};

void launch_precompute(bool f32, const Momenta& mom, int64_t n, int64_t pitch, const DevModel* dm, void* s_out,
                       void* x_out, void* k_out, cudaStream_t st);
void launch_sum(const double* v, int64_t n, double* out, cudaStream_t st);
void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t st);
void launch_prepare(const double* params, const DevModel* dm, EvalConst* ec, cudaStream_t st);
void launch_final(const FinalArgs& fa, int mc_width, int data_width, cudaStream_t st);

// Launchers of the model-specialised per-event kernels.
struct ShapeOps {
  const char* signature;
  int U, NR;
  int mc_row_width;
  int data_row_width;
  int data_threads;
  // Block partials are stored column-major: value v of block b at part[v * ld + b].
  cudaError_t (*mc)(bool grad, int grid, cudaStream_t st, const SampleDev& d, const EvalConst* ec, double* part,
                    int64_t ld, int* err);
  cudaError_t (*data)(bool from_cache, bool grad, int grid, cudaStream_t st, const SampleDev& d,
                      const EvalConst* ec, double* part, int64_t ld, double* rates);
  int (*mc_blocks_per_sm)(bool grad);
  int (*data_blocks_per_sm)(bool from_cache, bool grad);
};

// Specialisation compiled for a model signature, or null.
const ShapeOps* find_shape_ops(const std::string& signature, bool f32);

}  // namespace tdmix
