// Serving: many concurrent minimisers submit (sample, parameters) requests;
// a scheduler thread batches whatever is pending into one persistent kernel
// launch (continuous batching: requests that arrive while a batch runs join
// the next one), admits samples into device memory by footprint (least
// recently used samples without pending requests are evicted when the
// budget binds), and completes tickets that clients wait on.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tdmix.h"
#include "device_tables.hpp"
#include "kernels.hpp"
#include "model.hpp"

namespace tdmix {
namespace internal {
cudaStream_t stream_of(tdmix_ctx* ctx);
int num_sms_of(tdmix_ctx* ctx);
const CompiledModel& model_of(tdmix_ctx* ctx);
const ShapeOps* ops_of(tdmix_ctx* ctx);
const ModelConst& model_const_of(tdmix_ctx* ctx);
const void* log_table_of(tdmix_ctx* ctx);
bool is_f32(tdmix_ctx* ctx);
double inv_sum_w_of(tdmix_ctx* ctx);
const double* gram_store_of(tdmix_ctx* ctx);
std::string& error_of(tdmix_ctx* ctx);
int take_component_cache(tdmix_ctx* ctx, const tdmix_events* ev, const double* params, void** cache,
                         int64_t* tile_bytes, double* sum_t);
int compute_mc_totals(tdmix_ctx* ctx, const double* params, const tdmix_events* one_event);
}  // namespace internal
}  // namespace tdmix

using namespace tdmix;
using Clock = std::chrono::steady_clock;

namespace {

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// Page-locked host array (cudaMallocHost), so that the copies of a sample at
// each (re-)admission run at the full rate of the host link.
struct PinnedDoubles {
  double* p = nullptr;
  PinnedDoubles() = default;
  PinnedDoubles(const PinnedDoubles&) = delete;
  PinnedDoubles& operator=(const PinnedDoubles&) = delete;
  PinnedDoubles(PinnedDoubles&& o) noexcept : p(o.p) { o.p = nullptr; }
  PinnedDoubles& operator=(PinnedDoubles&& o) noexcept {
    if (this != &o) {
      reset();
      p = o.p;
      o.p = nullptr;
    }
    return *this;
  }
  ~PinnedDoubles() { reset(); }
  cudaError_t alloc(size_t count) {
    reset();
    void* q = nullptr;
    const cudaError_t e = cudaMallocHost(&q, count * sizeof(double));
    if (e == cudaSuccess) p = static_cast<double*>(q);
    return e;
  }
  void reset() {
    if (p) cudaFreeHost(p);
    p = nullptr;
  }
  double* data() { return p; }
};

struct SampleRec {
  int64_t n = 0;
  PinnedDoubles planes;  // host copy [16][n] for (re-)admission
  PinnedDoubles t;
  bool resident = false;
  void* cache = nullptr;   // tile-major components and decay times
  int64_t tile_bytes = 0;
  double sum_t = 0;
  size_t bytes = 0;
  uint64_t last_used = 0;
  int pending = 0;
};

struct Request {
  uint64_t ticket;
  int sample;
  std::vector<double> params;
  double t_submit;
};

struct Done {
  int status;
  std::vector<double> result;  // [nll, N, n_bad, sum ln B, grad...]
  double latency_s;
};

}  // namespace

struct tdmix_server {
  tdmix_ctx* ctx = nullptr;
  int device = 0;
  int np = 0, nc = 0, nr = 0;
  size_t budget = 0, resident_bytes = 0;
  int max_slots = 0;
  std::vector<double> fixed;  // masses and widths of the fixed model
  std::vector<double> defaults;
  bool have_mc = false;
  std::vector<double> mc_cols;  // host copy of the MC totals
  double* d_mc_cols = nullptr;
  double inv_sum_w = 1.0;
  // batch buffers
  ServeReq* d_reqs = nullptr;
  ServeReq* h_reqs = nullptr;     // pinned
  double* d_params = nullptr;
  double* h_params = nullptr;     // pinned
  double* d_results = nullptr;
  double* h_results = nullptr;    // pinned
  void* d_part = nullptr;
  unsigned* d_counters = nullptr;
  int* d_err = nullptr;
  // state shared with clients
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Done> done;
  std::map<int, SampleRec> samples;
  uint64_t next_ticket = 1;
  int next_sample = 0;
  bool stop = false;
  std::thread worker;
  std::vector<double> latencies;
  double t_first = 0, t_last = 0;
  uint64_t n_done = 0, use_clock = 0;
  std::string err;
  int worker_status = TDMIX_OK;
};

namespace {

int sfail(tdmix_server* s, int code, const std::string& m) {
  if (s) s->err = m;
  return code;
}

#define SV_CK(call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return sfail(s, TDMIX_ERR_CUDA, std::string(#call) + ": " + \
                                                               cudaGetErrorString(e_)); \
  } while (0)

// Admits sample `id` (component cache on the device), evicting least recently
// used samples without pending requests while the budget is exceeded.
// Returns TDMIX_ERR_NOMEM if the sample cannot fit now (it stays queued).
int admit(tdmix_server* s, int id) {
  SampleRec& rec = s->samples[id];
  if (rec.resident) return TDMIX_OK;
  const size_t need = size_t((rec.n + kTileEvents - 1) / kTileEvents) * internal::ops_of(s->ctx)->cache_tile_bytes;
  while (s->resident_bytes + need > s->budget) {
    int victim = -1;
    uint64_t oldest = UINT64_MAX;
    for (auto& kv : s->samples)
      if (kv.second.resident && kv.second.pending == 0 && kv.second.last_used < oldest) {
        oldest = kv.second.last_used;
        victim = kv.first;
      }
    if (victim < 0) return TDMIX_ERR_NOMEM;
    SampleRec& v = s->samples[victim];
    cudaFree(v.cache);
    v.cache = nullptr;
    v.resident = false;
    s->resident_bytes -= v.bytes;
  }
  tdmix_events ev{};
  ev.n = rec.n;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) ev.p[a][c] = rec.planes.data() + size_t(a * 4 + c) * rec.n;
  ev.t = rec.t.data();
  ev.on_device = 0;
  int rc = internal::take_component_cache(s->ctx, &ev, s->defaults.data(), &rec.cache, &rec.tile_bytes,
                                          &rec.sum_t);
  if (rc) return sfail(s, rc, "admission: " + internal::error_of(s->ctx));
  rec.bytes = need;
  rec.resident = true;
  s->resident_bytes += need;
  return TDMIX_OK;
}

// Device view of a resident sample, copied out of the sample table while
// the server mutex is held, so that the batch never reads the table (which
// other threads insert into) without the lock.
struct ResidentView {
  const void* cache;
  int64_t n, tile_bytes;
  double sum_t;
};

// Evaluates one batch (worker thread, mutex not held).
int run_batch(tdmix_server* s, std::vector<Request>& batch, const std::vector<ResidentView>& views,
              std::vector<Done>& out) {
  const ShapeOps* ops = internal::ops_of(s->ctx);
  cudaStream_t st = internal::stream_of(s->ctx);
  const int nb = int(batch.size());
  int chunks = 0;
  for (int r = 0; r < nb; ++r) {
    const ResidentView& rec = views[r];
    const int n_tiles = int((rec.n + kTileEvents - 1) / kTileEvents);
    const int ct = std::max(1, (n_tiles + kServeMaxChunks - 1) / kServeMaxChunks);
    ServeReq& q = s->h_reqs[r];
    q.cache = rec.cache;
    q.n = rec.n;
    q.tile_bytes = rec.tile_bytes;
    q.chunk_begin = chunks;
    q.chunk_tiles = ct;
    q.n_tiles = n_tiles;
    q.n_chunks = (n_tiles + ct - 1) / ct;
    q.sum_t = rec.sum_t;
    chunks += q.n_chunks;
    std::memcpy(s->h_params + size_t(r) * s->np, batch[r].params.data(), s->np * sizeof(double));
  }
  SV_CK(cudaMemcpyAsync(s->d_reqs, s->h_reqs, nb * sizeof(ServeReq), cudaMemcpyHostToDevice, st));
  SV_CK(cudaMemcpyAsync(s->d_params, s->h_params, size_t(nb) * s->np * sizeof(double), cudaMemcpyHostToDevice, st));
  ServeArgs a{};
  a.reqs = s->d_reqs;
  a.n_req = nb;
  a.total_chunks = chunks;
  a.params = s->d_params;
  a.km = internal::model_const_of(s->ctx);
  a.logtab = internal::log_table_of(s->ctx);
  a.mc_cols = s->d_mc_cols;
  a.inv_sum_w = s->inv_sum_w;
  a.part = s->d_part;
  a.counters = s->d_counters;
  a.results = s->d_results;
  a.err = s->d_err;
  const int grid = std::min(chunks, internal::num_sms_of(s->ctx));
  SV_CK(ops->serve(true, grid, st, a));
  const int rw = kResHeader + s->np;
  SV_CK(cudaMemcpyAsync(s->h_results, s->d_results, size_t(nb) * rw * sizeof(double), cudaMemcpyDeviceToHost, st));
  SV_CK(cudaStreamSynchronize(st));
  const double t_end = now_s();
  out.resize(nb);
  for (int r = 0; r < nb; ++r) {
    Done& d = out[r];
    const double* res = s->h_results + size_t(r) * rw;
    d.result.assign(res, res + rw);
    d.status = res[2] < 0 ? int(res[2]) : ((res[2] > 0 || !std::isfinite(res[0])) ? TDMIX_ERR_NONFINITE : TDMIX_OK);
    d.latency_s = t_end - batch[r].t_submit;
  }
  return TDMIX_OK;
}

void worker_loop(tdmix_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    if (s->stop) break;
    // take up to max_slots pending requests whose samples are or can be made resident
    std::vector<Request> batch;
    std::deque<Request> later;
    while (!s->queue.empty() && int(batch.size()) < s->max_slots) {
      Request q = std::move(s->queue.front());
      s->queue.pop_front();
      int rc = admit(s, q.sample);
      if (rc == TDMIX_ERR_NOMEM && !batch.empty()) {
        later.push_back(std::move(q));  // memory frees up when this batch completes
        continue;
      }
      if (rc) {
        Done d{rc, std::vector<double>(kResHeader + s->np, NAN), now_s() - q.t_submit};
        s->samples[q.sample].pending--;
        s->done[q.ticket] = std::move(d);
        continue;
      }
      s->samples[q.sample].last_used = ++s->use_clock;
      batch.push_back(std::move(q));
    }
    for (auto it = later.rbegin(); it != later.rend(); ++it) s->queue.push_front(std::move(*it));
    if (batch.empty()) {
      s->cv_done.notify_all();
      continue;
    }
    std::vector<ResidentView> views;
    views.reserve(batch.size());
    for (const Request& q : batch) {
      const SampleRec& rec = s->samples.at(q.sample);
      views.push_back(ResidentView{rec.cache, rec.n, rec.tile_bytes, rec.sum_t});
    }
    lk.unlock();
    std::vector<Done> out;
    int rc = run_batch(s, batch, views, out);
    lk.lock();
    for (size_t r = 0; r < batch.size(); ++r) {
      Done d = rc ? Done{rc, std::vector<double>(kResHeader + s->np, NAN), now_s() - batch[r].t_submit} : out[r];
      s->samples[batch[r].sample].pending--;
      s->latencies.push_back(d.latency_s);
      if (s->n_done == 0) s->t_first = batch[r].t_submit;
      s->t_last = now_s();
      s->n_done++;
      s->done[batch[r].ticket] = std::move(d);
    }
    if (rc) s->worker_status = rc;
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int tdmix_server_create(const char* model_json, int precision, size_t hbm_budget_bytes, int max_slots,
                        tdmix_server** out) {
  if (!out) return TDMIX_ERR_ARG;
  *out = nullptr;
  if (max_slots < 1 || max_slots > kServeMaxRequests || hbm_budget_bytes == 0) return TDMIX_ERR_ARG;
  tdmix_server* s = new tdmix_server;
  *out = s;
  if (cudaGetDevice(&s->device) != cudaSuccess) return sfail(s, TDMIX_ERR_CUDA, "no CUDA device");
  int rc = tdmix_create(model_json, precision, &s->ctx);
  if (rc) return sfail(s, rc, s->ctx ? tdmix_last_error(s->ctx) : "model");
  cudaStream_t st;
  SV_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  tdmix_set_stream(s->ctx, st);
  const CompiledModel& m = internal::model_of(s->ctx);
  s->np = m.n_params();
  s->nc = int(m.chains.size());
  s->nr = m.NR();
  s->defaults = m.default_params();
  s->fixed.assign(s->defaults.begin() + 2 * s->nc, s->defaults.begin() + 2 * s->nc + 2 * s->nr);
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  // serving keeps the model fixed: only coefficients and x, y float
  std::vector<int> mask = m.floating_mask();
  for (int k = 2 * s->nc; k < 2 * s->nc + 2 * s->nr; ++k) mask[k] = 0;
  tdmix_set_floating(s->ctx, mask.data());
  const int rw = kResHeader + s->np;
  const ShapeOps* ops = internal::ops_of(s->ctx);
  const int wd = ops->data_width;
  SV_CK(cudaMalloc(&s->d_reqs, max_slots * sizeof(ServeReq)));
  SV_CK(cudaMallocHost(&s->h_reqs, max_slots * sizeof(ServeReq)));
  SV_CK(cudaMalloc(&s->d_params, size_t(max_slots) * s->np * sizeof(double)));
  SV_CK(cudaMallocHost(&s->h_params, size_t(max_slots) * s->np * sizeof(double)));
  SV_CK(cudaMalloc(&s->d_results, size_t(max_slots) * rw * sizeof(double)));
  SV_CK(cudaMallocHost(&s->h_results, size_t(max_slots) * rw * sizeof(double)));
  // chunk-partial rows with an even stride (16-byte aligned rows, see k_serve)
  SV_CK(cudaMalloc(&s->d_part, size_t(max_slots) * kServeMaxChunks * ((wd + 1) & ~1) * 8));
  SV_CK(cudaMalloc(&s->d_counters, max_slots * sizeof(unsigned)));
  SV_CK(cudaMemset(s->d_counters, 0, max_slots * sizeof(unsigned)));
  SV_CK(cudaMalloc(&s->d_err, sizeof(int)));
  SV_CK(cudaMemset(s->d_err, 0, sizeof(int)));
  SV_CK(cudaMalloc(&s->d_mc_cols, ops->mc_width * sizeof(double)));
  s->worker = std::thread(worker_loop, s);
  return TDMIX_OK;
}

int tdmix_server_add_mc(tdmix_server* s, const tdmix_events* mc) {
  if (!s || !mc || !s->ctx) return sfail(s, TDMIX_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int rc = tdmix_load_events(s->ctx, nullptr, mc);
  if (rc) return sfail(s, rc, tdmix_last_error(s->ctx));
  // one stand-in data event (the first MC event at t = 0) to run the MC pass
  std::vector<double> one(16);
  double t0 = 0.0;
  tdmix_events ev{};
  ev.n = 1;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) {
      if (mc->on_device) SV_CK(cudaMemcpy(&one[a * 4 + c], mc->p[a][c], sizeof(double), cudaMemcpyDeviceToHost));
      else one[a * 4 + c] = mc->p[a][c][0];
      ev.p[a][c] = &one[a * 4 + c];
    }
  ev.t = &t0;
  rc = internal::compute_mc_totals(s->ctx, s->defaults.data(), &ev);
  if (rc) return sfail(s, rc, tdmix_last_error(s->ctx));
  const ShapeOps* ops = internal::ops_of(s->ctx);
  SV_CK(cudaMemcpy(s->d_mc_cols, internal::gram_store_of(s->ctx), ops->mc_width * sizeof(double),
                   cudaMemcpyDeviceToDevice));
  s->inv_sum_w = internal::inv_sum_w_of(s->ctx);
  s->have_mc = true;
  return TDMIX_OK;
}

int tdmix_server_add_sample(tdmix_server* s, const tdmix_events* data, int* sample_id) {
  if (!s || !data || !sample_id || data->n < 1 || !data->t) return sfail(s, TDMIX_ERR_ARG, "bad sample");
  SampleRec rec;
  rec.n = data->n;
  SV_CK(rec.planes.alloc(size_t(16) * data->n));
  SV_CK(rec.t.alloc(size_t(data->n)));
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) {
      double* dst = rec.planes.data() + size_t(a * 4 + c) * data->n;
      if (data->on_device) SV_CK(cudaMemcpy(dst, data->p[a][c], data->n * sizeof(double), cudaMemcpyDeviceToHost));
      else std::memcpy(dst, data->p[a][c], data->n * sizeof(double));
    }
  if (data->on_device) SV_CK(cudaMemcpy(rec.t.data(), data->t, data->n * sizeof(double), cudaMemcpyDeviceToHost));
  else std::memcpy(rec.t.data(), data->t, data->n * sizeof(double));
  std::lock_guard<std::mutex> lk(s->mu);
  *sample_id = s->next_sample++;
  s->samples[*sample_id] = std::move(rec);
  return TDMIX_OK;
}

int tdmix_server_submit(tdmix_server* s, int sample_id, const double* params, uint64_t* ticket) {
  if (!s || !params || !ticket) return sfail(s, TDMIX_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->have_mc) return sfail(s, TDMIX_ERR_STATE, "add the MC sample first");
  auto it = s->samples.find(sample_id);
  if (it == s->samples.end()) return sfail(s, TDMIX_ERR_ARG, "unknown sample id");
  for (int k = 0; k < 2 * s->nr; ++k)
    if (params[2 * s->nc + k] != s->fixed[k])
      return sfail(s, TDMIX_ERR_ARG, "serving keeps resonance masses and widths at the model's values");
  Request q{s->next_ticket++, sample_id, std::vector<double>(params, params + s->np), now_s()};
  *ticket = q.ticket;
  it->second.pending++;
  s->queue.push_back(std::move(q));
  s->cv_work.notify_one();
  return TDMIX_OK;
}

int tdmix_server_wait(tdmix_server* s, uint64_t ticket, double* nll, double* grad, double timeout_s) {
  if (!s || !nll) return sfail(s, TDMIX_ERR_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0);
  while (s->done.find(ticket) == s->done.end()) {
    if (ticket == 0 || ticket >= s->next_ticket) return sfail(s, TDMIX_ERR_ARG, "unknown ticket");
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->done.find(ticket) == s->done.end())
      return sfail(s, TDMIX_ERR_TIMEOUT, "request not finished within the timeout");
  }
  Done d = std::move(s->done[ticket]);
  s->done.erase(ticket);
  *nll = d.result[0];
  if (grad) std::memcpy(grad, d.result.data() + kResHeader, s->np * sizeof(double));
  if (d.status) return sfail(s, d.status, "request failed (status " + std::to_string(d.status) + ")");
  return TDMIX_OK;
}

int tdmix_server_stats(tdmix_server* s, double* p50_us, double* p99_us, double* evals_per_s) {
  if (!s) return TDMIX_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = s->latencies;
  if (l.empty()) return sfail(s, TDMIX_ERR_STATE, "no completed requests");
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) { return l[std::min(l.size() - 1, size_t(q * (l.size() - 1) + 0.5))] * 1e6; };
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  if (evals_per_s) *evals_per_s = s->t_last > s->t_first ? double(s->n_done) / (s->t_last - s->t_first) : 0.0;
  return TDMIX_OK;
}

int tdmix_server_reset_stats(tdmix_server* s) {
  if (!s) return TDMIX_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->n_done = 0;
  s->t_first = s->t_last = 0;
  return TDMIX_OK;
}

int tdmix_server_resident_bytes(tdmix_server* s, size_t* bytes) {
  if (!s || !bytes) return TDMIX_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *bytes = s->resident_bytes;
  return TDMIX_OK;
}

const char* tdmix_server_last_error(const tdmix_server* s) { return s ? s->err.c_str() : "null server"; }

void tdmix_server_destroy(tdmix_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->samples) {
    cudaFree(kv.second.cache);
  }
  cudaStream_t st = s->ctx ? internal::stream_of(s->ctx) : nullptr;
  cudaFree(s->d_reqs);
  cudaFreeHost(s->h_reqs);
  cudaFree(s->d_params);
  cudaFreeHost(s->h_params);
  cudaFree(s->d_results);
  cudaFreeHost(s->h_results);
  cudaFree(s->d_part);
  cudaFree(s->d_counters);
  cudaFree(s->d_err);
  cudaFree(s->d_mc_cols);
  if (s->ctx) tdmix_destroy(s->ctx);
  if (st) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
