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
  // lineshape structure, read by the runtime-table (generic) evaluation:
  // Breit-Wigner instances of each term (-1: none) and, per instance, its
  // resonance, invariant plane and width plane (-1: constant width)
  int term_bw[kMaxTerms][2];
  int bw_res[kMaxBW], bw_splane[kMaxBW], bw_xplane[kMaxBW];
};

// Model constants the likelihood kernels read, passed by value in the
// kernel parameters (constant bank): the fields of the model that enter the
// per-evaluation constants and the epilogue.
constexpr int kMaxParams = 2 * kMaxChains + 2 * kMaxRes + 2;
struct ModelConst {
  int n_chains, n_params;
  double r_res, gamma, tau;  // tau = 1 / gamma
  double sigma_t;            // Gaussian decay-time resolution (0: none; generic evaluation only)
  double bkg_fraction, bkg_tau;  // background fraction (0: none) and lifetime (generic evaluation only)
  double res_ma[kMaxRes], res_mb[kMaxRes];
  int8_t res_shape[kMaxRes], res_L[kMaxRes];
  int8_t chain_comp[kMaxChains], chain_amp[kMaxChains];
  uint8_t floating[kMaxParams];
};

// Largest |x| Gamma sigma_t / sqrt 2 the folded rate accepts (the real part
// of the Faddeeva argument; the evaluation is verified up to 0.3).
constexpr double kMaxResolutionMix = 0.25;

// Blocks per SM of the cached pass (component cache in, no MC tiles): its
// registers (~113 per thread) and a ring of at most 88 KiB allow two, which
// doubles the warps that hide the latency of its short per-event work.
constexpr int kCachedBlocksPerSM = 2;

// Events per tile: the unit of every bulk copy and of the static work
// assignment; one event per consumer thread.
constexpr int kTileEvents = 256;

// Device view of one event sample (data or phase-space MC), tile-major: tile
// q (events 256 q .. 256 q + 255) is one contiguous block, so one bulk copy
// moves a whole tile.
//   planes: per tile the precomputed event planes [NPL][256] in the working
//           precision T (invariants: fp64 [NS]; fp32 hi [NS] then lo [NS];
//           width factors X [NX]; spin x barrier factors K [U*NO]), then the
//           256 decay times (f64, data) or the 256 weights (T, weighted MC)
//   cache:  (data) per tile the components [2U][256] (T: re planes, then im
//           planes), then the 256 decay times (f64)
//   lo:     (data, fp32 path) per tile the rounding residuals (value minus
//           its float) of the width factors and spin x barrier factors,
//           [NX + U*NO][256] floats; read only for the ill-conditioned
//           events that are recomputed in double-float
// The event slots of the last tile beyond n are zero.
struct SampleDev {
  int64_t n, n_tiles;
  const void* planes;
  int64_t tile_bytes;
  void* cache;
  int64_t cache_tile_bytes;
  const float* lo;
  int weighted;
};

// Arguments of the fused evaluation kernel (passed as a grid constant).
struct EvalArgs {
  SampleDev data, mc;
  ModelConst km;
  const double* params;       // device parameter vector, or null: hp holds it
  double hp[kMaxParams];      // parameter vector by value (host callers)
  void* part;            // float2 [ld][width] double-float block partial rows (MC columns, then data columns)
  int64_t ld;            // rows of part (>= grid)
  double* gram_store;    // MC column totals of the last pass that ran the MC tiles
  unsigned* counter;     // blocks finished (low 16 bits) and blocks that timed out
                         // (high bits); returned to 0 by the last block
  double* rates;         // optional: e^{-Gamma t} B per data event
  double* result;        // [nll, N, n_bad or status, sum ln B, n recomputed, grad...]
  double* out_nll;       // optional second destination of the NLL
  double* out_grad;      // optional second destination of the gradient
  double sum_t;
  double inv_sum_w;           // 1 / sum of MC weights (the MC event count when unweighted)
  unsigned long long* trace;  // optional: per block kTracePhases globaltimer stamps (ns)
  const int64_t* mc_ranges;   // [grid + 1]: block b takes MC tiles [mc_ranges[b], mc_ranges[b + 1])
  const void* logtab;         // logarithm table: double2 {1/F, ln F}, F = 1 + j/128, j = 0..128
  int withhold_first_copy;    // test hook: block 0 does not issue its first tile copy, so its
                              // bounded wait for that tile runs out (TDMIX_ERR_TIMEOUT)
  int gram_pref;              // how to accumulate the MC normalisation matrix (TDMIX_GRAM_*)
  const DevModel* dm;         // structure tables (read by the generic evaluation only)
  const void* derived;        // per-evaluation constants derived for a batch (k_derive), or null:
                              // every block derives them from the parameters
};

// Phases stamped by the evaluation kernel when tracing is on: start,
// constants ready, MC tiles done, data tiles done, partials written, and in
// the last block: column totals formed, result written; end.
constexpr int kTracePhases = 8;

// Relative cost of one data tile and one MC tile, in common units (used to
// balance the static assignment of tiles to blocks).  fp32: a data tile
// (double-float Eq. (mix), its adjoint and the component-cache write) takes
// about 5/3 of an MC tile, measured per block with the trace stamps (2.2 us
// against 1.34 us on GB300); fp64: about equal.
constexpr int kDataTileCostF32 = 5, kMcTileCostF32 = 3;
constexpr int kDataTileCostF64 = 1, kMcTileCostF64 = 1;

// Result vector written by the evaluation kernel:
// [nll, N, n_bad or status, sum ln B, data events recomputed in double-float, grad...]
constexpr int kResHeader = 5;

constexpr int kServeMaxChunks = 256;     // chunks per request at most
constexpr int kServeMaxSlots = 1024;     // requests in flight at most
constexpr int kServeRingCap = 1 << 16;   // ring entries per launch of the serving loop

// One request slot of the serving loop (mapped, page-locked host memory;
// written by the host before the request is published, read by the device;
// the device writes the result and then `done`).  A slot is reused only
// after its request finished.
struct ServeSlot {
  const void* cache;     // tile-major component cache with decay times (SampleDev::cache)
  int64_t n;
  int64_t tile_bytes;    // bytes of one cache tile
  int32_t n_chunks;
  int32_t chunk_tiles;   // tiles per chunk (the last chunk may have fewer)
  int32_t n_tiles;
  int32_t pad;
  double sum_t;
  double params[kMaxParams];
  double result[kResHeader + kMaxParams];  // [nll, N, n_bad or status, sum ln B, n recomputed, grad...]
  unsigned long long done;            // ring entry + 1 of the last request finished in this slot
};

// Ring of the serving loop (mapped host memory): entry e of a launch is
// slot[e - head]; the host publishes entries by a release store of `tail`
// and stops the loop with `stop`.
struct ServeRing {
  unsigned long long tail;
  unsigned stop;
  unsigned pad;
  int32_t slot[kServeRingCap];
};

// Arguments of the persistent serving loop (grid constant).
struct ServeLoopArgs {
  ServeRing* ring;            // mapped
  ServeSlot* slots;           // mapped, [kServeMaxSlots]
  unsigned* claimed;          // device, [kServeRingCap]: chunks claimed per entry (zero at launch)
  unsigned* finished;         // device, [kServeRingCap]: chunks finished per entry (zero at launch)
  unsigned long long* low;    // device: the oldest entry with unclaimed chunks (head at launch)
  unsigned long long head;    // first entry of this launch
  ModelConst km;
  const double* mc_cols;      // MC column totals of the fixed model
  double inv_sum_w;
  void* part;                 // float2 [kServeMaxSlots][kServeMaxChunks][row stride] chunk partials
  int* status;                // device: 1 if a bounded wait gave up, 2 if the loop idled out
  const void* logtab;         // logarithm table (as in EvalArgs)
  unsigned long long idle_ns; // bound of one wait for new work
};



}  // namespace tdmix
