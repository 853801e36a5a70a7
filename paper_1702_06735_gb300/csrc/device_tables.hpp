// Plain-old-data tables shared between the host library and the kernels.
#pragma once
#include <cstdint>

#include "model.hpp"

namespace tdmix {

// Model structure as the kernels read it (device global memory, written once).
struct DevModel {
  int U, NO, NB, NR, NS, NX, n_chains, n_params;
  int chain_comp[kMaxChains];
  int chain_amp[kMaxChains];
  int res_shape[kMaxRes];
  int res_L[kMaxRes];
  double res_ma[kMaxRes], res_mb[kMaxRes];
  double r_res, r_parent, gamma;
  int term_spin[kMaxTerms];
  int term_parts[kMaxTerms][4];
  int splane_mask[kMaxSPlanes];
  int xplane_s[kMaxXPlanes];
  int xplane_L[kMaxXPlanes];
  double xplane_ma[kMaxXPlanes], xplane_mb[kMaxXPlanes];
};

// Device view of one event sample (data or phase-space MC).
struct SampleDev {
  int64_t n, pitch;
  void* s;            // invariants: fp64 [NS][pitch]; fp32 [2][NS][pitch] (hi, lo)
  void* x;            // width factors X(s) [NX][pitch]
  void* k;            // spin x barrier factors [U*NO][pitch]
  const double* t;    // decay times (data)
  const void* w;      // event weights (MC) or null
  void* cache;        // per-event components [2][U][pitch] (data)
};

// Arguments of the fused evaluation kernel.
struct EvalArgs {
  SampleDev data, mc;
  const double* params;
  const DevModel* dm;
  void* part;            // float2 [width][ld] double-float block partials (MC columns, then data columns)
  int64_t ld;            // leading dimension of part (>= grid)
  double* gram_store;    // MC column totals of the last pass that ran the MC tiles
  unsigned* counter;     // blocks finished; returned to 0 by the last block
  int* err;              // bounded-wait failures; read and cleared by the last block
  double* rates;         // optional: e^{-Gamma t} B per data event
  double* result;        // [nll, N, n_bad or status, sum ln B, grad...]
  double sum_t;
  double inv_sum_w;           // 1 / sum of MC weights (the MC event count when unweighted)
  unsigned long long* trace;  // optional: per block kTracePhases globaltimer stamps (ns)
  const int64_t* mc_ranges;   // [grid + 1]: block b takes MC tiles [mc_ranges[b], mc_ranges[b + 1])
};

// Phases stamped by the evaluation kernel when tracing is on: start,
// constants ready, data tiles done, MC tiles done, partials written, and in
// the last block: column totals formed, result written; end.
constexpr int kTracePhases = 8;

// Relative cost of one data tile in units of one MC tile (used to balance
// the static assignment of tiles to blocks).
constexpr int kDataTileCostF32 = 4;
constexpr int kDataTileCostF64 = 1;

constexpr int kServeMaxChunks = 256;     // chunks per request at most
constexpr int kServeMaxRequests = 1024;  // requests per batch at most

// One request of a serving batch (see serve.cuh).
struct ServeReq {
  const void* cache;     // [2U][pitch] components (working precision)
  const double* t;       // [pitch] decay times
  int64_t n, pitch;
  int32_t chunk_begin;   // first row of this request in the partial array
  int32_t n_chunks;
  int32_t chunk_tiles;   // tiles per chunk (the last chunk may have fewer)
  int32_t n_tiles;
  double sum_t;
};

struct ServeArgs {
  const ServeReq* reqs;
  int n_req;
  int total_chunks;
  const double* params;     // [n_req][n_params]
  const DevModel* dm;
  const int* floating;
  const double* mc_cols;    // MC column totals of the fixed model
  double inv_sum_w;
  void* part;               // float2 [total_chunks][WD] chunk partials
  unsigned* counters;       // [n_req] chunks finished (returned to 0)
  double* results;          // [n_req][kResHeader + n_params]
  int* err;
};

// Result vector written by the evaluation kernel: [nll, N, n_bad or status, sum ln B, grad...]
constexpr int kResHeader = 4;

}  // namespace tdmix
