// C ABI of the library: context, event loading, evaluation orchestration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/tdmix.h"
#include "device_tables.hpp"
#include "generate.cuh"
#include "kernels.hpp"
#include "model.hpp"

namespace tdmix {
const ShapeOps* find_shape_ops_f64(const std::string& sig);
const ShapeOps* find_shape_ops_f32(const std::string& sig);
const ShapeOps* find_shape_ops(const std::string& sig, bool f32) {
  return f32 ? find_shape_ops_f32(sig) : find_shape_ops_f64(sig);
}
}  // namespace tdmix

using namespace tdmix;

namespace {


struct Sample {
  SampleDev dev{};
  std::vector<void*> owned;
  double* rates = nullptr;  // data: per-event rate scratch
  bool loaded = false;
};

}  // namespace

struct tdmix_ctx {
  CompiledModel model;
  bool f32 = false;
  const ShapeOps* ops = nullptr;
  bool generic = false;   // runtime-table evaluation (no compiled specialisation of the structure)
  ShapeOps generic_ops{};  // ops of the generic path (ops points here when generic)
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  DevModel* d_model = nullptr;  // structure tables of the kinematic precompute
  ModelConst km{};               // model constants passed to the likelihood kernels by value
  double* d_result = nullptr;
  double* d_gram = nullptr;
  double* d_sumt = nullptr;
  unsigned long long* d_trace = nullptr;  // per-block phase stamps of the last evaluation (tracing on)
  int64_t* d_ranges = nullptr;            // per-block MC tile ranges [num_sms + 1]
  int64_t* d_zero_ranges = nullptr;       // [num_sms + 1] zeros: no MC tiles (data-only passes)
  double* d_logtab = nullptr;             // logarithm table of the kernels ({1/F, ln F} pairs)
  int64_t ranges_key[3] = {-1, -1, -1};   // (data tiles, MC tiles, grid) the ranges were made for
  double* last_result = nullptr;   // result vector the last evaluation wrote (d_result or d_result_map)
  double* h_result = nullptr;      // pinned, mapped: written by the kernel for host callers
  double* d_result_map = nullptr;  // device address of h_result
  void* d_part = nullptr;         // block partials of the evaluation kernel (float2 [num_sms][width])
  unsigned* d_counter = nullptr;  // blocks finished (returned to 0 by the kernel)
  void* d_derived = nullptr;      // per-evaluation constants of a batch (k_derive records)
  int64_t derived_cap = 0;        // records d_derived holds
  Sample data, mc;
  double sum_t = 0;
  double inv_sum_w = 1.0;  // 1 / sum of MC weights
  std::vector<int> floating;
  std::vector<double> last_res;
  bool cache_valid = false, gram_valid = false;
  bool withhold_first_copy = false;  // test hook (tdmix_test_withhold_copy)
  int gram_pref = TDMIX_GRAM_AUTO;   // normalisation-matrix accumulation (tdmix_set_gram)
  std::string err;
  // kernel profiling: CUDA event pairs per kernel class, recorded on the stream
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev[TDMIX_PROF_CLASSES][2];
  std::vector<int64_t> prof_count[TDMIX_PROF_CLASSES];  // launches between the events of each pair
  int prof_used[TDMIX_PROF_CLASSES] = {};
  double prof_ms[TDMIX_PROF_CLASSES] = {};
  int64_t prof_n[TDMIX_PROF_CLASSES] = {};
};

namespace {

int fail(tdmix_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define TDMIX_CK(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TDMIX_ERR_NOMEM : TDMIX_ERR_CUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Event buffers come from the stream-ordered allocator (cudaMallocAsync /
// cudaFreeAsync on the context's stream): unlike cudaMalloc / cudaFree they
// never wait for the whole device, so samples can be loaded and released
// while a persistent kernel (the serving loop) runs.
void free_sample(Sample& s, cudaStream_t st) {
  for (void* p : s.owned) cudaFreeAsync(p, st);
  s.owned.clear();
  s = Sample{};
}

int dalloc(tdmix_ctx* ctx, Sample& s, void** p, size_t bytes) {
  TDMIX_CK(cudaMallocAsync(p, bytes < 16 ? 16 : bytes, ctx->stream));
  s.owned.push_back(*p);
  return TDMIX_OK;
}

DevModel make_dev_model(const CompiledModel& m) {
  DevModel d;
  std::memset(&d, 0, sizeof d);
  d.U = m.U;
  d.NO = m.NO;
  d.NB = m.NB();
  d.NR = m.NR();
  d.NS = m.NS();
  d.NX = m.NX();
  d.n_chains = int(m.chains.size());
  d.n_params = m.n_params();
  for (size_t c = 0; c < m.chains.size(); ++c) {
    d.chain_comp[c] = m.chain_comp[c];
    d.chain_amp[c] = m.chains[c].amp;
  }
  for (size_t r = 0; r < m.res.size(); ++r) {
    d.res_shape[r] = m.res[r].shape;
    d.res_L[r] = m.res[r].L;
    d.res_ma[r] = m.res[r].ma;
    d.res_mb[r] = m.res[r].mb;
  }
  d.r_res = m.r_res;
  d.r_parent = m.r_parent;
  d.gamma = 1.0 / m.tau;
  for (size_t t = 0; t < m.terms.size(); ++t) {
    d.term_spin[t] = m.terms[t].spin;
    for (int k = 0; k < 4; ++k) d.term_parts[t][k] = m.terms[t].parts[k];
    d.term_bw[t][0] = m.terms[t].b[0];
    d.term_bw[t][1] = m.terms[t].b[1];
  }
  for (size_t b = 0; b < m.bws.size(); ++b) {
    d.bw_res[b] = m.bws[b].res;
    d.bw_splane[b] = m.bws[b].splane;
    d.bw_xplane[b] = m.bws[b].xplane;
  }
  for (int s = 0; s < m.NS(); ++s) d.splane_mask[s] = m.splane_mask[s];
  for (int x = 0; x < m.NX(); ++x) {
    d.xplane_s[x] = m.xplanes[x].splane;
    d.xplane_L[x] = m.xplanes[x].L;
    d.xplane_ma[x] = m.xplanes[x].ma;
    d.xplane_mb[x] = m.xplanes[x].mb;
  }
  return d;
}

ModelConst make_model_const(const CompiledModel& m, const std::vector<int>& floating) {
  ModelConst k;
  std::memset(&k, 0, sizeof k);
  k.n_chains = int(m.chains.size());
  k.n_params = m.n_params();
  k.r_res = m.r_res;
  k.gamma = 1.0 / m.tau;
  k.tau = m.tau;
  k.sigma_t = m.sigma_t;
  k.bkg_fraction = m.bkg_fraction;
  k.bkg_tau = m.bkg_tau;
  for (size_t r = 0; r < m.res.size(); ++r) {
    k.res_ma[r] = m.res[r].ma;
    k.res_mb[r] = m.res[r].mb;
    k.res_shape[r] = int8_t(m.res[r].shape);
    k.res_L[r] = int8_t(m.res[r].L);
  }
  for (size_t c = 0; c < m.chains.size(); ++c) {
    k.chain_comp[c] = int8_t(m.chain_comp[c]);
    k.chain_amp[c] = int8_t(m.chains[c].amp);
  }
  for (int q = 0; q < m.n_params(); ++q) k.floating[q] = floating[q] ? 1 : 0;
  return k;
}

cudaError_t generic_serve(int, cudaStream_t, const ServeLoopArgs&) { return cudaErrorNotSupported; }

// Layout of the generic path: fp64 planes of the kinematic precompute.
ShapeOps make_generic_ops(const CompiledModel& m) {
  ShapeOps o{};
  const int U = m.U, NR = m.NR();
  const int npl = m.NS() + m.NX() + U * m.NO;
  const int64_t plane_bytes = int64_t(npl) * kTileEvents * sizeof(double), extra = kTileEvents * sizeof(double);
  o.signature = "generic";
  o.U = U;
  o.NR = NR;
  o.mc_width = 1 + U * (U + 1) / 2 + U * (U - 1) / 2 + 2 * NR;
  o.data_width = 5 + 4 * U + 2 * NR;
  o.n_planes = npl;
  o.data_tile_bytes = plane_bytes + extra;
  o.mc_tile_bytes = plane_bytes;
  o.mc_tile_bytes_weighted = plane_bytes + extra;
  o.cache_tile_bytes = int64_t(2 * U) * kTileEvents * sizeof(double) + extra;
  o.eval = &generic_eval;
  o.serve = &generic_serve;
  o.serve_row_stride = 0;
  o.derive = nullptr;
  o.derived_bytes = 0;
  o.cached_blocks = 1;
  return o;
}

}  // namespace

// Table of the kernels' logarithm: {1/F_j, ln F_j} for F_j = 1 + j/128,
// j = 0..128, each rounded once from extended precision.
std::vector<double> tdmix::make_log_table() {
  std::vector<double> t(2 * 129);
  for (int j = 0; j <= 128; ++j) {
    const long double F = 1.0L + (long double)j / 128.0L;
    t[2 * j] = double(1.0L / F);
    t[2 * j + 1] = double(std::log(F));
  }
  return t;
}

namespace {

// Host-side screening of a parameter vector (host pointer only).
int check_params(tdmix_ctx* ctx, const double* p) {
  const CompiledModel& m = ctx->model;
  const int np = m.n_params(), nc = int(m.chains.size());
  for (int k = 0; k < np; ++k)
    if (!std::isfinite(p[k])) return fail(ctx, TDMIX_ERR_NONFINITE, "parameter " + std::to_string(k) + " is not finite");
  for (int r = 0; r < m.NR(); ++r) {
    if (m.res[r].shape == SHAPE_NONE) continue;
    if (!(p[2 * nc + 2 * r] > 0) || !(p[2 * nc + 2 * r + 1] > 0))
      return fail(ctx, TDMIX_ERR_DOMAIN, "resonance '" + m.res[r].name + "' needs a positive mass and width");
  }
  if (!(std::fabs(p[np - 1]) < 1.0)) return fail(ctx, TDMIX_ERR_DOMAIN, "|y| must be below 1");
  if (m.sigma_t > 0 && !(std::fabs(p[np - 2]) * m.sigma_t / (m.tau * std::sqrt(2.0)) <= kMaxResolutionMix))
    return fail(ctx, TDMIX_ERR_DOMAIN, "|x| Gamma sigma_t / sqrt 2 must not exceed 0.25 with a decay-time resolution");
  return TDMIX_OK;
}

constexpr int kProfPool = 4096;

// Folds recorded event pairs into the accumulated times (synchronises).
int prof_drain(tdmix_ctx* ctx) {
  for (int c = 0; c < TDMIX_PROF_CLASSES; ++c) {
    for (int k = 0; k < ctx->prof_used[c]; ++k) {
      float ms = 0;
      TDMIX_CK(cudaEventSynchronize(ctx->prof_ev[c][1][k]));
      TDMIX_CK(cudaEventElapsedTime(&ms, ctx->prof_ev[c][0][k], ctx->prof_ev[c][1][k]));
      ctx->prof_ms[c] += ms;
      ctx->prof_n[c] += ctx->prof_count[c][k];
    }
    ctx->prof_used[c] = 0;
  }
  return TDMIX_OK;
}

// Records the start (phase 0) or end (phase 1) of `launches` consecutive
// kernels of class c.
int prof_mark(tdmix_ctx* ctx, int c, int phase, int64_t launches = 1) {
  if (!ctx->prof_on) return TDMIX_OK;
  if (phase == 0 && ctx->prof_used[c] == kProfPool) {
    int rc = prof_drain(ctx);
    if (rc) return rc;
  }
  const int k = ctx->prof_used[c];
  TDMIX_CK(cudaEventRecord(ctx->prof_ev[c][phase][k], ctx->stream));
  if (phase == 1) {
    ctx->prof_count[c][k] = launches;
    ctx->prof_used[c] = k + 1;
  }
  return TDMIX_OK;
}

// Copies one event sample to the device and runs the kinematic precompute
// into its tile-major planes (see SampleDev).
int load_sample(tdmix_ctx* ctx, const tdmix_events* ev, bool is_data, Sample& s) {
  if (ev->n < 1) return fail(ctx, TDMIX_ERR_ARG, "an event sample needs n >= 1");
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c)
      if (!ev->p[a][c]) return fail(ctx, TDMIX_ERR_ARG, "missing momentum plane");
  if (is_data && !ev->t) return fail(ctx, TDMIX_ERR_ARG, "the data sample needs decay times");
  free_sample(s, ctx->stream);
  const ShapeOps* ops = ctx->ops;
  const int64_t n = ev->n;
  const int64_t n_tiles = (n + kTileEvents - 1) / kTileEvents;
  cudaStream_t st = ctx->stream;
  int rc;
  Momenta mom;
  std::vector<void*> temps;
  auto cleanup = [&]() {
    for (void* p : temps) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
  };
  auto fail_clean = [&](int code, const std::string& msg) {
    cleanup();
    free_sample(s, st);
    return fail(ctx, code, msg);
  };
  // f64 device copy of a per-event host array (or the caller's device array)
  auto on_device = [&](const double* src, const double** out) -> int {
    if (ev->on_device) {
      *out = src;
      return TDMIX_OK;
    }
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, size_t(n) * sizeof(double), st) != cudaSuccess) return TDMIX_ERR_NOMEM;
    temps.push_back(buf);
    if (cudaMemcpyAsync(buf, src, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return TDMIX_ERR_CUDA;
    *out = static_cast<const double*>(buf);
    return TDMIX_OK;
  };
  if (ev->on_device) {
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) mom.p[a][c] = ev->p[a][c];
  } else {
    void* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, size_t(16) * n * sizeof(double), st);
    if (e != cudaSuccess) return fail(ctx, TDMIX_ERR_NOMEM, "momentum staging buffer");
    temps.push_back(buf);
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        double* dst = static_cast<double*>(buf) + size_t(a * 4 + c) * n;
        e = cudaMemcpyAsync(dst, ev->p[a][c], n * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail_clean(TDMIX_ERR_CUDA, std::string("momentum copy: ") + cudaGetErrorString(e));
        mom.p[a][c] = dst;
      }
  }
  const double* t_dev = nullptr;
  const double* w_dev = nullptr;
  if (is_data && (rc = on_device(ev->t, &t_dev))) return fail_clean(rc, "decay time staging");
  if (!is_data && ev->w && (rc = on_device(ev->w, &w_dev))) return fail_clean(rc, "weight staging");

  SampleDev& d = s.dev;
  d.n = n;
  d.n_tiles = n_tiles;
  d.weighted = w_dev ? 1 : 0;
  d.tile_bytes = is_data ? ops->data_tile_bytes : (w_dev ? ops->mc_tile_bytes_weighted : ops->mc_tile_bytes);
  void* planes = nullptr;
  if ((rc = dalloc(ctx, s, &planes, size_t(n_tiles) * d.tile_bytes))) return fail_clean(rc, ctx->err);
  d.planes = planes;
  cudaMemsetAsync(planes, 0, size_t(n_tiles) * d.tile_bytes, st);  // slots beyond n stay zero
  if (is_data) {
    d.cache_tile_bytes = ops->cache_tile_bytes;
    if ((rc = dalloc(ctx, s, &d.cache, size_t(n_tiles) * d.cache_tile_bytes)) ||
        (rc = dalloc(ctx, s, reinterpret_cast<void**>(&s.rates), size_t(n) * sizeof(double))))
      return fail_clean(rc, ctx->err);
    cudaMemsetAsync(d.cache, 0, size_t(n_tiles) * d.cache_tile_bytes, st);
    if (ctx->f32) {  // residuals of the width and spin x barrier factors (ill-conditioned events)
      const CompiledModel& m = ctx->model;
      void* lo = nullptr;
      if ((rc = dalloc(ctx, s, &lo, size_t(n_tiles) * (m.NX() + m.U * m.NO) * kTileEvents * sizeof(float))))
        return fail_clean(rc, ctx->err);
      d.lo = static_cast<const float*>(lo);
    }
  }
  int prc = prof_mark(ctx, TDMIX_PROF_PRECOMPUTE, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_clean(TDMIX_ERR_CUDA, std::string("before precompute: ") + cudaGetErrorString(e));
  launch_precompute(ctx->f32, mom, n, ctx->d_model, planes, d.tile_bytes, ops->n_planes, t_dev, w_dev, d.cache,
                    d.cache_tile_bytes, const_cast<float*>(d.lo), st);
  e = cudaGetLastError();
  if (!prc) prc = prof_mark(ctx, TDMIX_PROF_PRECOMPUTE, 1);
  if (prc) {
    cleanup();
    free_sample(s, st);
    return prc;
  }
  double sum = 0;
  if (e == cudaSuccess && (t_dev || w_dev)) {
    launch_sum(t_dev ? t_dev : w_dev, n, ctx->d_sumt, st);
    e = cudaMemcpyAsync(&sum, ctx->d_sumt, sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  cleanup();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_sample(s, st);
    return fail(ctx, TDMIX_ERR_CUDA, std::string("precompute: ") + cudaGetErrorString(e));
  }
  if (is_data) {
    ctx->sum_t = sum;
  } else if (w_dev) {
    if (!(sum > 0)) {
      free_sample(s, st);
      return fail(ctx, TDMIX_ERR_ARG, "MC weights must have a positive sum");
    }
    ctx->inv_sum_w = 1.0 / sum;
  } else {
    ctx->inv_sum_w = 1.0 / double(n);
  }
  s.loaded = true;
  return TDMIX_OK;
}

// One evaluation: enqueue everything, leave the result in ctx->d_result.
// `result` receives [nll, N, n_bad or status, sum ln B, grad...] (device
// or mapped host memory); out_nll / out_grad are optional second
// destinations (device memory).
// data_only: a full evaluation of the data tiles alone (components written to
// the cache); the MC tiles are skipped, so its NLL and stored normalisation
// are not meaningful (used to build component caches).
// pdl: may start while the evaluation before it in the stream finishes (only
// between evaluations of one batch); grid_cap: blocks at most (0: one per SM).
// prof: record profiling events around this launch.
int enqueue_eval(tdmix_ctx* ctx, const double* params, bool host_params, bool want_grad, double* rates,
                 double* result, double* out_nll = nullptr, double* out_grad = nullptr, bool data_only = false,
                 bool pdl = false, int grid_cap = 0, bool prof = true, const void* derived = nullptr) {
  const CompiledModel& m = ctx->model;
  const int np = m.n_params(), nc = int(m.chains.size());
  cudaStream_t st = ctx->stream;
  if (!ctx->data.loaded || !ctx->mc.loaded) return fail(ctx, TDMIX_ERR_STATE, "load data and MC events first");
  bool res_floating = false;
  for (int k = 2 * nc; k < 2 * nc + 2 * m.NR(); ++k) res_floating |= ctx->floating[k] != 0;
  // per-event rates always come from a full evaluation (the recomputation
  // of ill-conditioned events of the fp32 path runs there); the generic path
  // keeps no component cache
  bool full = data_only || rates != nullptr || !host_params || !ctx->cache_valid || (want_grad && res_floating) ||
              ctx->generic;
  if (host_params && !full) {
    for (int k = 0; k < 2 * m.NR(); ++k)
      if (params[2 * nc + k] != ctx->last_res[k]) full = true;
  }
  int rc;
  const int64_t items = ctx->data.dev.n_tiles + (full && !data_only ? ctx->mc.dev.n_tiles : 0);
  // the cached pass may run several blocks per SM (ShapeOps::cached_blocks)
  // when every block gets several tiles; on fewer tiles the per-block fixed
  // costs (constants, block sums, the last block's column sums over more
  // rows) outweigh the latency hidden by the extra warps
  const int per_sm = full || items < int64_t(4) * ctx->ops->cached_blocks * ctx->num_sms ? 1 : ctx->ops->cached_blocks;
  const int cap = grid_cap > 0 && grid_cap < per_sm * ctx->num_sms ? grid_cap : per_sm * ctx->num_sms;
  const int grid = int(items < cap ? items : cap);
  // parameters travel in the kernel arguments (host callers) or are read
  // from the caller's device array
  EvalArgs a;
  std::memset(&a, 0, sizeof a);
  a.data = ctx->data.dev;
  a.mc = ctx->mc.dev;
  a.km = ctx->km;
  if (host_params) std::memcpy(a.hp, params, np * sizeof(double));
  else a.params = params;
  a.part = ctx->d_part;
  // rows of the partial array the kernel may stage in shared memory: a full
  // evaluation reserves room for one per SM; a cached pass only for its grid
  a.ld = full ? ctx->num_sms : grid;
  a.gram_store = ctx->d_gram;
  a.counter = ctx->d_counter;
  a.rates = rates;
  a.result = result;
  a.out_nll = out_nll;
  a.out_grad = out_grad;
  a.logtab = ctx->d_logtab;
  a.withhold_first_copy = ctx->withhold_first_copy ? 1 : 0;
  a.gram_pref = ctx->gram_pref;
  a.dm = ctx->d_model;
  a.derived = derived;
  a.sum_t = ctx->sum_t;
  a.inv_sum_w = ctx->inv_sum_w;
  a.trace = ctx->d_trace;
  if (full && !data_only) {
    // Static, cost-balanced assignment of MC tiles to blocks: block q takes
    // data tiles q, q + grid, ... and MC tiles [range[q], range[q + 1]).
    const int64_t n_dt = ctx->data.dev.n_tiles, n_mt = ctx->mc.dev.n_tiles;
    if (ctx->ranges_key[0] != n_dt || ctx->ranges_key[1] != n_mt || ctx->ranges_key[2] != grid) {
      const int64_t Rd = ctx->f32 ? kDataTileCostF32 : kDataTileCostF64;
      const int64_t Rm = ctx->f32 ? kMcTileCostF32 : kMcTileCostF64;
      const int64_t total = Rd * n_dt + Rm * n_mt, G = grid;
      std::vector<int64_t> rg(G + 1, 0);
      int64_t run = 0, data_upto = 0;
      for (int64_t q = 0; q < G; ++q) {
        data_upto += n_dt > q ? (n_dt - 1 - q) / G + 1 : 0;  // data tiles of blocks <= q
        // MC tiles of blocks <= q: their share of the cost units, less their data tiles'
        int64_t e = ((q + 1) * total / G - Rd * data_upto + Rm / 2) / Rm;
        e = e < 0 ? 0 : (e > n_mt ? n_mt : e);
        run = e > run ? e : run;
        rg[q + 1] = q == G - 1 ? n_mt : run;
      }
      TDMIX_CK(cudaMemcpyAsync(ctx->d_ranges, rg.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
      TDMIX_CK(cudaStreamSynchronize(st));
      ctx->ranges_key[0] = n_dt;
      ctx->ranges_key[1] = n_mt;
      ctx->ranges_key[2] = grid;
    }
  }
  a.mc_ranges = data_only ? ctx->d_zero_ranges : ctx->d_ranges;

  if (prof && (rc = prof_mark(ctx, TDMIX_PROF_EVAL, 0))) return rc;
  ctx->last_result = result;
  TDMIX_CK(ctx->ops->eval(full, want_grad, grid, pdl, st, a));
  if (prof && (rc = prof_mark(ctx, TDMIX_PROF_EVAL, 1))) return rc;
  if (data_only) {
    ctx->gram_valid = ctx->cache_valid = false;
  } else if (full) {
    ctx->gram_valid = true;
    ctx->cache_valid = true;
    if (host_params) ctx->last_res.assign(params + 2 * nc, params + 2 * nc + 2 * m.NR());
    else ctx->cache_valid = false;  // parameter values unknown on the host
  }
  return TDMIX_OK;
}

int result_status(tdmix_ctx* ctx) {
  const double* r = ctx->h_result;
  if (r[2] < 0) {
    int st = int(r[2]);
    return fail(ctx, st, st == TDMIX_ERR_DOMAIN    ? "parameter outside its domain (|y| < 1, m0 > 0, Gamma0 > 0, "
                                                       "pole above the decay threshold)"
                         : st == TDMIX_ERR_TIMEOUT ? "a bounded device wait gave up (event tile copy did not arrive)"
                                                   : "non-finite parameter");
  }
  if (r[2] > 0)
    return fail(ctx, TDMIX_ERR_NONFINITE, std::to_string(int64_t(r[2])) + " data events have a rate <= 0 or not finite");
  if (!(r[1] > 0) || !std::isfinite(r[0])) return fail(ctx, TDMIX_ERR_NONFINITE, "normalisation <= 0 or NLL not finite");
  return TDMIX_OK;
}

}  // namespace

namespace tdmix {
namespace internal {

cudaStream_t stream_of(tdmix_ctx* ctx) { return ctx->stream; }
int num_sms_of(tdmix_ctx* ctx) { return ctx->num_sms; }
const CompiledModel& model_of(tdmix_ctx* ctx) { return ctx->model; }
const ShapeOps* ops_of(tdmix_ctx* ctx) { return ctx->ops; }
const ModelConst& model_const_of(tdmix_ctx* ctx) { return ctx->km; }
const void* log_table_of(tdmix_ctx* ctx) { return ctx->d_logtab; }
bool is_f32(tdmix_ctx* ctx) { return ctx->f32; }
bool is_generic(tdmix_ctx* ctx) { return ctx->generic; }
double inv_sum_w_of(tdmix_ctx* ctx) { return ctx->inv_sum_w; }
const double* gram_store_of(tdmix_ctx* ctx) { return ctx->d_gram; }
std::string& error_of(tdmix_ctx* ctx) { return ctx->err; }

// Computes the component cache of a data sample at host parameters `params`
// (one full evaluation with the loaded MC) and hands its device buffer to
// the caller: *cache (tile-major, SampleDev::cache), *tile_bytes per tile.
int take_component_cache(tdmix_ctx* ctx, const tdmix_events* ev, const double* params, void** cache,
                         int64_t* tile_bytes, double* sum_t) {
  int rc = load_sample(ctx, ev, true, ctx->data);
  if (rc) return rc;
  ctx->cache_valid = false;
  if ((rc = enqueue_eval(ctx, params, true, false, nullptr, ctx->d_result, nullptr, nullptr, true))) return rc;
  TDMIX_CK(cudaStreamSynchronize(ctx->stream));
  Sample& d = ctx->data;
  *cache = d.dev.cache;
  *tile_bytes = d.dev.cache_tile_bytes;
  *sum_t = ctx->sum_t;
  // keep the cache alive, free the planes and scratch
  for (void* p : d.owned)
    if (p != d.dev.cache) cudaFreeAsync(p, ctx->stream);
  d.owned.clear();
  d = Sample{};
  ctx->cache_valid = false;
  return TDMIX_OK;
}

// Runs one full evaluation at host `params` with a one-event stand-in data
// sample, leaving the MC column totals (normalisation sums) in the context.
int compute_mc_totals(tdmix_ctx* ctx, const double* params, const tdmix_events* one_event) {
  int rc = load_sample(ctx, one_event, true, ctx->data);
  if (rc) return rc;
  ctx->cache_valid = false;
  if ((rc = enqueue_eval(ctx, params, true, false, nullptr, ctx->d_result))) return rc;
  TDMIX_CK(cudaStreamSynchronize(ctx->stream));
  free_sample(ctx->data, ctx->stream);
  ctx->cache_valid = false;
  return TDMIX_OK;
}

}  // namespace internal
}  // namespace tdmix

extern "C" {

int tdmix_create(const char* model_json, int precision, tdmix_ctx** out) {
  if (!out || !model_json) return TDMIX_ERR_ARG;
  *out = nullptr;
  const bool force_generic = (precision & TDMIX_GENERIC) != 0;
  precision &= ~TDMIX_GENERIC;
  if (precision != TDMIX_FP64 && precision != TDMIX_FP32) return TDMIX_ERR_ARG;
  tdmix_ctx* ctx = new (std::nothrow) tdmix_ctx;
  if (!ctx) return TDMIX_ERR_NOMEM;
  try {
    ctx->model = compile_model(model_json);
  } catch (const std::exception& e) {
    // keep a context alive only to carry the message
    ctx->err = e.what();
    *out = ctx;
    return TDMIX_ERR_ARG;
  }
  ctx->f32 = precision == TDMIX_FP32;
  // a decay-time resolution and a background are evaluated by the runtime-table kernels only
  const bool extension = ctx->model.sigma_t > 0 || ctx->model.bkg_fraction > 0;
  ctx->ops = force_generic || extension ? nullptr : find_shape_ops(ctx->model.signature(), ctx->f32);
  *out = ctx;
  if (!ctx->ops) {
    // no specialisation of this structure: the runtime-table kernels, in fp64
    ctx->generic = true;
    ctx->f32 = false;
    ctx->generic_ops = make_generic_ops(ctx->model);
    ctx->ops = &ctx->generic_ops;
  }
  TDMIX_CK(cudaGetDevice(&ctx->device));
  TDMIX_CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int np = ctx->model.n_params();
  {
    const CompiledModel& m = ctx->model;
    const int npl = (ctx->f32 ? 2 : 1) * m.NS() + m.NX() + m.U * m.NO;
    if (npl != ctx->ops->n_planes || np > kMaxParams)
      return fail(ctx, TDMIX_ERR_UNSUPPORTED, "model tables do not match the compiled specialisation");
  }
  TDMIX_CK(cudaMalloc(&ctx->d_model, sizeof(DevModel)));
  TDMIX_CK(cudaMalloc(&ctx->d_result, (kResHeader + np) * sizeof(double)));
  TDMIX_CK(cudaMalloc(&ctx->d_gram, (1 + 2 * kMaxComp * kMaxComp + 2 * kMaxRes) * sizeof(double)));
  TDMIX_CK(cudaMalloc(&ctx->d_sumt, sizeof(double)));
  // block partial rows [num_sms][width] (+16 bytes: copied in whole 16-byte units)
  TDMIX_CK(cudaMalloc(&ctx->d_part, size_t(kCachedBlocksPerSM) * ctx->num_sms *
                                         (ctx->ops->mc_width + ctx->ops->data_width) * 8 + 16));
  TDMIX_CK(cudaMalloc(&ctx->d_counter, sizeof(unsigned)));
  TDMIX_CK(cudaMalloc(&ctx->d_ranges, (ctx->num_sms + 1) * sizeof(int64_t)));
  TDMIX_CK(cudaMalloc(&ctx->d_zero_ranges, (ctx->num_sms + 1) * sizeof(int64_t)));
  TDMIX_CK(cudaMemset(ctx->d_zero_ranges, 0, (ctx->num_sms + 1) * sizeof(int64_t)));
  {
    const std::vector<double> lt = make_log_table();
    TDMIX_CK(cudaMalloc(&ctx->d_logtab, lt.size() * sizeof(double)));
    TDMIX_CK(cudaMemcpy(ctx->d_logtab, lt.data(), lt.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  TDMIX_CK(cudaMemset(ctx->d_counter, 0, sizeof(unsigned)));
  TDMIX_CK(cudaHostAlloc(&ctx->h_result, (kResHeader + np) * sizeof(double), cudaHostAllocMapped));
  TDMIX_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->d_result_map), ctx->h_result, 0));
  DevModel dm = make_dev_model(ctx->model);
  TDMIX_CK(cudaMemcpy(ctx->d_model, &dm, sizeof dm, cudaMemcpyHostToDevice));
  ctx->floating = ctx->model.floating_mask();
  ctx->km = make_model_const(ctx->model, ctx->floating);
  return TDMIX_OK;
}

int tdmix_set_stream(tdmix_ctx* ctx, void* cuda_stream) {
  if (!ctx) return TDMIX_ERR_ARG;
  // work enqueued on the old stream completes before buffers are reused on the new one
  if (ctx->ops && ctx->stream != static_cast<cudaStream_t>(cuda_stream)) TDMIX_CK(cudaStreamSynchronize(ctx->stream));
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return TDMIX_OK;
}

int tdmix_num_params(const tdmix_ctx* ctx) { return ctx ? ctx->model.n_params() : TDMIX_ERR_ARG; }

int tdmix_kernel_path(const tdmix_ctx* ctx) {
  if (!ctx || !ctx->ops) return TDMIX_ERR_ARG;
  return ctx->generic ? TDMIX_PATH_GENERIC : (ctx->f32 ? TDMIX_PATH_FP32 : TDMIX_PATH_FP64);
}

int tdmix_num_components(const tdmix_ctx* ctx) { return ctx ? ctx->model.U : TDMIX_ERR_ARG; }

int tdmix_chain_component(const tdmix_ctx* ctx, int chain) {
  if (!ctx || chain < 0 || chain >= int(ctx->model.chains.size())) return TDMIX_ERR_ARG;
  return ctx->model.chain_comp[chain];
}

int tdmix_default_params(const tdmix_ctx* ctx, double* out) {
  if (!ctx || !out) return TDMIX_ERR_ARG;
  std::vector<double> p = ctx->model.default_params();
  std::memcpy(out, p.data(), p.size() * sizeof(double));
  return TDMIX_OK;
}

int tdmix_set_floating(tdmix_ctx* ctx, const int* mask) {
  if (!ctx || !mask) return TDMIX_ERR_ARG;
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  const int np = ctx->model.n_params();
  for (int k = 0; k < np; ++k) ctx->floating[k] = mask[k] != 0;
  ctx->km = make_model_const(ctx->model, ctx->floating);
  return TDMIX_OK;
}

int tdmix_load_events(tdmix_ctx* ctx, const tdmix_events* data, const tdmix_events* mc) {
  if (!ctx) return TDMIX_ERR_ARG;
  cudaGetLastError();  // a failure left by earlier, unrelated work must not be reported here
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  int rc;
  if (data && (rc = load_sample(ctx, data, true, ctx->data))) return rc;
  if (mc && (rc = load_sample(ctx, mc, false, ctx->mc))) return rc;
  ctx->cache_valid = false;
  if (mc) ctx->gram_valid = false;
  return TDMIX_OK;
}

int tdmix_nll(tdmix_ctx* ctx, const double* params, double* nll_out, double* grad_out) {
  if (!ctx || !params || !nll_out) return fail(ctx, TDMIX_ERR_ARG, "null argument");
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  cudaGetLastError();  // a failure left by earlier, unrelated work must not be reported here
  const bool host_params = !is_device_ptr(params);
  const bool host_out = !is_device_ptr(nll_out);
  if (grad_out && is_device_ptr(grad_out) == host_out)
    return fail(ctx, TDMIX_ERR_ARG, "nll_out and grad_out must both be host or both be device memory");
  int rc;
  if (host_params && (rc = check_params(ctx, params))) return rc;
  cudaStream_t st = ctx->stream;
  const int np = ctx->model.n_params();
  if (host_out) {
    // the last block writes the result vector straight into mapped host memory
    if ((rc = enqueue_eval(ctx, params, host_params, grad_out != nullptr, nullptr, ctx->d_result_map))) return rc;
    TDMIX_CK(cudaStreamSynchronize(st));
    *nll_out = ctx->h_result[0];
    if (grad_out) std::memcpy(grad_out, ctx->h_result + kResHeader, np * sizeof(double));
    const int st = result_status(ctx);
    if (st == TDMIX_ERR_TIMEOUT) ctx->cache_valid = ctx->gram_valid = false;  // partial sums incomplete
    return st;
  }
  // device outputs: written by the kernel itself, nothing else is enqueued
  return enqueue_eval(ctx, params, host_params, grad_out != nullptr, nullptr, ctx->d_result, nll_out, grad_out);
}

int tdmix_nll_batch(tdmix_ctx* ctx, const double* params, int64_t n_points, double* nll_out, double* grad_out) {
  if (!ctx || !params || !nll_out || n_points < 1) return fail(ctx, TDMIX_ERR_ARG, "null argument or no points");
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  if (!is_device_ptr(params) || !is_device_ptr(nll_out) || (grad_out && !is_device_ptr(grad_out)))
    return fail(ctx, TDMIX_ERR_ARG, "a batch takes device parameters and device outputs");
  if (n_points > (int64_t(1) << 30)) return fail(ctx, TDMIX_ERR_ARG, "too many points in one batch");
  cudaGetLastError();
  const int np = ctx->model.n_params();
  // Consecutive evaluations overlap: each may start while the one before it
  // finishes.  One SM is left to the finishing evaluation's last block, so
  // that the next one's blocks all start at once.
  const int cap = n_points > 1 && ctx->num_sms > 1 ? ctx->num_sms - 1 : ctx->num_sms;
  int rc;
  if ((rc = prof_mark(ctx, TDMIX_PROF_EVAL, 0))) return rc;
  // the constants of every point are derived once, by one launch, before the evaluations
  const unsigned char* derived = nullptr;
  if (ctx->ops->derive && n_points > 1) {
    const int64_t rb = ctx->ops->derived_bytes;
    if (ctx->derived_cap < n_points) {
      if (ctx->d_derived) TDMIX_CK(cudaFreeAsync(ctx->d_derived, ctx->stream));
      ctx->d_derived = nullptr;
      ctx->derived_cap = 0;
      TDMIX_CK(cudaMallocAsync(&ctx->d_derived, size_t(n_points * rb), ctx->stream));
      ctx->derived_cap = n_points;
    }
    TDMIX_CK(ctx->ops->derive(int(n_points), params, np, ctx->km, ctx->d_derived, ctx->stream));
    derived = static_cast<const unsigned char*>(ctx->d_derived);
  }
  for (int64_t k = 0; k < n_points; ++k) {
    rc = enqueue_eval(ctx, params + k * np, false, grad_out != nullptr, nullptr, ctx->d_result, nll_out + k,
                      grad_out ? grad_out + k * np : nullptr, false, k > 0, cap, false,
                      derived ? derived + k * ctx->ops->derived_bytes : nullptr);
    if (rc) return rc;
  }
  return prof_mark(ctx, TDMIX_PROF_EVAL, 1, n_points);
}

int tdmix_event_rates(tdmix_ctx* ctx, const double* params, double* rates_out, double* norm_out) {
  if (!ctx || !params || !rates_out) return fail(ctx, TDMIX_ERR_ARG, "null argument");
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  const bool host_params = !is_device_ptr(params);
  const bool host_out = !is_device_ptr(rates_out);
  int rc;
  if (host_params && (rc = check_params(ctx, params))) return rc;
  if (!ctx->data.loaded) return fail(ctx, TDMIX_ERR_STATE, "load data and MC events first");
  double* rates = host_out ? ctx->data.rates : rates_out;
  if ((rc = enqueue_eval(ctx, params, host_params, false, rates, ctx->d_result))) return rc;
  cudaStream_t st = ctx->stream;
  const int64_t n = ctx->data.dev.n;
  if (host_out) {
    TDMIX_CK(cudaMemcpyAsync(ctx->h_result, ctx->d_result, kResHeader * sizeof(double), cudaMemcpyDeviceToHost, st));
    TDMIX_CK(cudaMemcpyAsync(rates_out, rates, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    TDMIX_CK(cudaStreamSynchronize(st));
    if (norm_out) *norm_out = ctx->h_result[1];
    if (ctx->h_result[2] < 0) return result_status(ctx);
    return TDMIX_OK;
  }
  if (norm_out) TDMIX_CK(cudaMemcpyAsync(norm_out, ctx->d_result + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return TDMIX_OK;
}

int tdmix_norm_matrix(tdmix_ctx* ctx, double* I_out) {
  if (!ctx || !I_out) return fail(ctx, TDMIX_ERR_ARG, "null argument");
  if (!ctx->gram_valid) return fail(ctx, TDMIX_ERR_STATE, "no evaluation has computed the normalisation matrix yet");
  const int U = ctx->model.U;
  const int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  std::vector<double> row(1 + NRE + NIM);
  TDMIX_CK(cudaMemcpyAsync(row.data(), ctx->d_gram, row.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TDMIX_CK(cudaStreamSynchronize(ctx->stream));
  const double sw = row[0];
  int ir = 0, ii = 0;
  for (int j = 0; j < U; ++j)
    for (int k = j; k < U; ++k) {
      const double re = row[1 + ir++] / sw;
      const double im = k > j ? row[1 + NRE + ii++] / sw : 0.0;
      I_out[2 * (j * U + k)] = re;
      I_out[2 * (j * U + k) + 1] = im;
      I_out[2 * (k * U + j)] = re;
      I_out[2 * (k * U + j) + 1] = -im;
    }
  return TDMIX_OK;
}

int tdmix_profile(tdmix_ctx* ctx, int enable) {
  if (!ctx) return TDMIX_ERR_ARG;
  if (enable && ctx->prof_ev[0][0].empty()) {
    for (int c = 0; c < TDMIX_PROF_CLASSES; ++c)
      for (int ph = 0; ph < 2; ++ph) {
        ctx->prof_ev[c][ph].resize(kProfPool);
        ctx->prof_count[c].assign(kProfPool, 1);
        for (auto& e : ctx->prof_ev[c][ph]) TDMIX_CK(cudaEventCreate(&e));
      }
  }
  if (!enable) {
    int rc = prof_drain(ctx);
    if (rc) return rc;
  }
  ctx->prof_on = enable != 0;
  return TDMIX_OK;
}

int tdmix_profile_read(tdmix_ctx* ctx, double* ms_out, int64_t* launches_out, int reset) {
  if (!ctx || !ms_out || !launches_out) return fail(ctx, TDMIX_ERR_ARG, "null argument");
  int rc = prof_drain(ctx);
  if (rc) return rc;
  for (int c = 0; c < TDMIX_PROF_CLASSES; ++c) {
    ms_out[c] = ctx->prof_ms[c];
    launches_out[c] = ctx->prof_n[c];
    if (reset) {
      ctx->prof_ms[c] = 0;
      ctx->prof_n[c] = 0;
    }
  }
  return TDMIX_OK;
}

int tdmix_generate(tdmix_ctx* ctx, const double* params, int64_t n, uint64_t seed, uint32_t stream, int flags,
                   double* p_out, double* t_out, double* info) {
  const bool flat = (flags & TDMIX_GEN_FLAT) != 0;
  if (!ctx || n < 1 || !p_out || (!flat && !params)) return fail(ctx, TDMIX_ERR_ARG, "bad argument");
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  cudaGetLastError();  // a failure left by earlier, unrelated work must not be reported here
  if (!is_device_ptr(p_out) || (t_out && !is_device_ptr(t_out)))
    return fail(ctx, TDMIX_ERR_ARG, "p_out and t_out must be device memory");
  const GenOps* g = find_gen_ops(ctx->model.signature());
  if (!g) return fail(ctx, TDMIX_ERR_UNSUPPORTED, "no generator compiled for this model structure");
  int rc;
  if (!flat && (rc = check_params(ctx, params))) return rc;
  const CompiledModel& m = ctx->model;
  GenArgs a;
  std::memset(&a, 0, sizeof a);
  a.km = ctx->km;
  if (!flat) std::memcpy(a.hp, params, m.n_params() * sizeof(double));
  a.dm = ctx->d_model;
  a.mD = m.parent_mass;
  double msum = 0, cum[4];
  for (int i = 0; i < 4; ++i) {
    a.m[i] = m.masses[i];
    msum += m.masses[i];
    cum[i] = msum;
  }
  a.tecm = a.mD - msum;
  if (!(a.tecm > 0)) return fail(ctx, TDMIX_ERR_ARG, "decay below threshold");
  // GENBOD's bound of the product of breakup momenta: each at the largest
  // parent and smallest subsystem mass
  auto q = [](double M, double x, double y) {
    const double l = (M * M - (x + y) * (x + y)) * (M * M - (x - y) * (x - y));
    return l > 0 ? std::sqrt(l) / (2 * M) : 0.0;
  };
  double wtmax = 1.0;
  for (int j = 1; j < 4; ++j) wtmax *= q(a.tecm + cum[j], cum[j - 1], m.masses[j]);
  a.inv_wtmax = 1.0 / wtmax;
  const double y = flat ? 0.0 : params[m.n_params() - 1];
  a.lambda = (1.0 - std::fabs(y)) / m.tau;
  a.key0 = uint32_t(seed);
  a.key1 = uint32_t(seed >> 32);
  a.flat = flat ? 1 : 0;
  a.prescreen = (flags & TDMIX_GEN_FP64_ONLY) ? 0 : 1;
  a.p_out = p_out;
  a.t_out = t_out;
  a.ld = n;
  a.out_end = n;
  cudaStream_t st = ctx->stream;
  const int grid = 1024;
  const int64_t batch = int64_t(grid) * kGenPerBlock;
  std::vector<void*> bufs;
  auto cleanup = [&]() {
    for (void* p : bufs) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
  };
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMallocAsync(p, bytes, st) != cudaSuccess) return false;
    bufs.push_back(*p);
    return true;
  };
  int64_t* d_pos = nullptr;
  if (!alloc(reinterpret_cast<void**>(&a.mask), batch / 32 * sizeof(uint32_t)) ||
      !alloc(reinterpret_cast<void**>(&a.block_count), grid * sizeof(uint32_t)) ||
      !alloc(reinterpret_cast<void**>(&a.wmax), sizeof(unsigned long long)) ||
      !alloc(reinterpret_cast<void**>(&d_pos), grid * sizeof(int64_t))) {
    cleanup();
    return fail(ctx, TDMIX_ERR_NOMEM, "generator buffers");
  }
  a.block_pos = d_pos;
  std::vector<uint32_t> counts(grid);
  std::vector<int64_t> pos(grid);
  unsigned long long wbits = 0;
  auto pass1 = [&](double* wmax_out) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(a.wmax, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = g->pass1(grid, st, a);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts.data(), a.block_count, grid * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&wbits, a.wmax, sizeof wbits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    double w;
    std::memcpy(&w, &wbits, sizeof w);
    *wmax_out = w;
    return e;
  };
  // pilot (model events): the envelope is 1.5 x the largest weight of one
  // batch (4.2M candidates) drawn from a separate stream; the weight
  // R e^{lambda t} has a long tail (narrow resonances), so a tighter
  // headroom makes later batches exceed it and the sample be redrawn
  double env = 0, wmax = 0;
  cudaError_t e = cudaSuccess;
  const int prescreen = a.prescreen;
  if (!flat && info && info[0] > 0) {  // the caller's envelope (from an earlier call at the same parameters)
    env = info[0];
  } else if (!flat) {
    a.stream = stream ^ 0x80000000u;
    a.env = 0.0;
    a.cand0 = 0;
    a.prescreen = 0;  // exact weights: the envelope is the same with and without the pre-screen
    if ((e = pass1(&wmax)) != cudaSuccess) {
      cleanup();
      return fail(ctx, TDMIX_ERR_CUDA, std::string("generator pilot: ") + cudaGetErrorString(e));
    }
    if (!(wmax > 0) || !std::isfinite(wmax)) {
      cleanup();
      return fail(ctx, TDMIX_ERR_NONFINITE, "generator pilot: no positive finite weight");
    }
    env = 1.5 * wmax;
  }
  a.stream = stream;
  a.prescreen = prescreen;
  int64_t have = 0, proposed = 0;
  int restarts = 0;
  while (have < n) {
    a.env = env;
    a.cand0 = proposed;
    if ((e = pass1(&wmax)) != cudaSuccess) break;
    if (!flat && wmax > env) {  // the envelope was exceeded: raise it and start again
      if (++restarts > 4) {
        cleanup();
        return fail(ctx, TDMIX_ERR_NONFINITE, "generator envelope kept being exceeded");
      }
      env = 1.5 * wmax;
      have = proposed = 0;
      continue;
    }
    int64_t run = have;
    for (int b = 0; b < grid; ++b) {
      pos[b] = run;
      run += counts[b];
    }
    if ((e = cudaMemcpyAsync(d_pos, pos.data(), grid * sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess)
      break;
    if ((e = g->pass2(grid, st, a)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;  // pos[] is reused by the next batch
    have = run;
    proposed += batch;
  }
  cleanup();
  if (e != cudaSuccess) return fail(ctx, TDMIX_ERR_CUDA, std::string("generator: ") + cudaGetErrorString(e));
  if (info) {
    info[0] = env;
    info[1] = double(proposed);
    info[2] = double(n) / double(proposed);
    info[3] = restarts;
  }
  return TDMIX_OK;
}

int tdmix_set_gram(tdmix_ctx* ctx, int mode) {
  if (!ctx) return TDMIX_ERR_ARG;
  if (!ctx->ops) return fail(ctx, TDMIX_ERR_STATE, "context has no compiled model");
  if (mode != TDMIX_GRAM_AUTO && mode != TDMIX_GRAM_REGISTERS && mode != TDMIX_GRAM_TENSOR)
    return fail(ctx, TDMIX_ERR_ARG, "unknown normalisation-matrix mode");
  if (ctx->generic && mode != TDMIX_GRAM_AUTO)
    return fail(ctx, TDMIX_ERR_UNSUPPORTED, "the generic evaluation has one normalisation-matrix mode");
  if (mode == TDMIX_GRAM_TENSOR && !ctx->f32)
    return fail(ctx, TDMIX_ERR_UNSUPPORTED, "the tensor-core normalisation matrix runs on the fp32 path");
  if (mode == TDMIX_GRAM_REGISTERS && ctx->model.U > 8)
    return fail(ctx, TDMIX_ERR_UNSUPPORTED, "register accumulation of the normalisation matrix holds up to 8 components");
  ctx->gram_pref = mode;
  ctx->gram_valid = false;  // the stored normalisation sums came from the other mode
  ctx->cache_valid = false;
  return TDMIX_OK;
}

int tdmix_recomputed_events(tdmix_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return fail(ctx, TDMIX_ERR_ARG, "null argument");
  if (!ctx->last_result) return fail(ctx, TDMIX_ERR_STATE, "no evaluation yet");
  TDMIX_CK(cudaStreamSynchronize(ctx->stream));
  double v = 0;
  if (ctx->last_result == ctx->d_result_map) v = ctx->h_result[4];
  else TDMIX_CK(cudaMemcpy(&v, ctx->last_result + 4, sizeof(double), cudaMemcpyDeviceToHost));
  *n = int64_t(v);
  return TDMIX_OK;
}

int tdmix_test_withhold_copy(tdmix_ctx* ctx, int enable) {
  if (!ctx) return TDMIX_ERR_ARG;
  ctx->withhold_first_copy = enable != 0;
  return TDMIX_OK;
}

int tdmix_trace(tdmix_ctx* ctx, int enable) {
  if (!ctx) return TDMIX_ERR_ARG;
  if (enable && !ctx->d_trace) {
    // room for every block of a cached pass (kCachedBlocksPerSM per SM); the first num_sms are read back
    const size_t n = size_t(kCachedBlocksPerSM) * ctx->num_sms * kTracePhases;
    TDMIX_CK(cudaMalloc(&ctx->d_trace, n * sizeof(unsigned long long)));
    TDMIX_CK(cudaMemset(ctx->d_trace, 0, n * sizeof(unsigned long long)));
  } else if (!enable && ctx->d_trace) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_trace);
    ctx->d_trace = nullptr;
  }
  return TDMIX_OK;
}

int tdmix_trace_read(tdmix_ctx* ctx, unsigned long long* stamps, int* n_blocks) {
  if (!ctx || !stamps || !n_blocks) return fail(ctx, TDMIX_ERR_ARG, "null argument");
  if (!ctx->d_trace) return fail(ctx, TDMIX_ERR_STATE, "tracing is off");
  TDMIX_CK(cudaStreamSynchronize(ctx->stream));
  TDMIX_CK(cudaMemcpy(stamps, ctx->d_trace, size_t(ctx->num_sms) * kTracePhases * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
  *n_blocks = ctx->num_sms;
  return TDMIX_OK;
}

const char* tdmix_last_error(const tdmix_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void tdmix_destroy(tdmix_ctx* ctx) {
  if (!ctx) return;
  if (ctx->ops) cudaStreamSynchronize(ctx->stream);
  free_sample(ctx->data, ctx->stream);
  free_sample(ctx->mc, ctx->stream);
  if (ctx->d_derived) cudaFreeAsync(ctx->d_derived, ctx->stream);
  if (ctx->ops) cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_model);
  cudaFree(ctx->d_result);
  cudaFree(ctx->d_gram);
  cudaFree(ctx->d_sumt);
  cudaFree(ctx->d_counter);
  cudaFree(ctx->d_part);
  cudaFree(ctx->d_trace);
  cudaFree(ctx->d_ranges);
  cudaFree(ctx->d_zero_ranges);
  cudaFree(ctx->d_logtab);
  if (ctx->h_result) cudaFreeHost(ctx->h_result);
  for (int c = 0; c < TDMIX_PROF_CLASSES; ++c)
    for (int ph = 0; ph < 2; ++ph)
      for (auto& e : ctx->prof_ev[c][ph]) cudaEventDestroy(e);
  delete ctx;
}

}  // extern "C"
