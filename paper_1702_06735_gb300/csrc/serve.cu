// Serving: many concurrent minimisers submit (sample, parameters) requests
// to a device-resident loop (serve.cuh).
//
// Host side, three parts sharing one mutex:
//   * client calls (submit, wait, stats) only touch host queues;
//   * the admission thread makes samples resident: it evicts least recently
//     used samples without pending requests while the device-memory budget
//     binds, then (without the mutex) regenerates or uploads the sample's
//     events and builds its component cache on its own stream, with the
//     stream-ordered allocator, so that it runs while the loop serves other
//     requests;
//   * the dispatcher thread writes requests whose samples are resident into
//     free slots of mapped memory and publishes them as ring entries,
//     launches the persistent loop when it is not running, polls the slots'
//     completion flags, and stops the loop when nothing is in flight (or the
//     ring is used up; the next request relaunches it).
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
double inv_sum_w_of(tdmix_ctx* ctx);
const double* gram_store_of(tdmix_ctx* ctx);
std::string& error_of(tdmix_ctx* ctx);
bool is_generic(tdmix_ctx* ctx);
int take_component_cache(tdmix_ctx* ctx, const tdmix_events* ev, const double* params, void** cache,
                         int64_t* tile_bytes, double* sum_t);
int compute_mc_totals(tdmix_ctx* ctx, const double* params, const tdmix_events* one_event);
}  // namespace internal
}  // namespace tdmix

using namespace tdmix;
using Clock = std::chrono::steady_clock;

namespace {

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr int kReservedSMs = 16;                 // left to admission and generation kernels
constexpr unsigned long long kIdleNs = 2000000000ull;  // bound of the loop's wait for work (2 s)
constexpr double kLoopIdleStop = 0.02;           // stop the loop after 20 ms with nothing in flight

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
  // host-registered sample: page-locked copy for (re-)admission
  PinnedDoubles planes;  // [16][n]
  PinnedDoubles t;
  // generated sample: regenerated on the device at each admission
  bool generated = false;
  std::vector<double> gen_params;
  uint64_t seed = 0;
  uint32_t stream = 0;
  bool resident = false, admitting = false;
  void* cache = nullptr;  // tile-major components and decay times
  int64_t tile_bytes = 0;
  double sum_t = 0;
  size_t bytes = 0;
  uint64_t last_used = 0;
  int pending = 0;  // submitted and not completed
};

struct Request {
  uint64_t ticket;
  int sample;
  std::vector<double> params;
  double t_submit;
  bool admitted = false;  // its sample was not resident at submission
};

struct Done {
  int status;
  std::vector<double> result;  // [header..., grad...]
  double latency_s;
};

struct InFlight {
  Request req;
  unsigned long long entry;
};

}  // namespace

struct tdmix_server {
  tdmix_ctx* ctx = nullptr;  // model context; its stream is the admission stream
  int device = 0, np = 0, nc = 0, nr = 0, grid = 0;
  size_t budget = 0, resident_bytes = 0;
  int max_slots = 0;
  std::vector<double> fixed;  // masses and widths of the fixed model
  std::vector<double> defaults;
  bool have_mc = false;
  double* d_mc_cols = nullptr;
  double inv_sum_w = 1.0;
  // the device-resident loop
  cudaStream_t loop_stream = nullptr;
  cudaEvent_t loop_done = nullptr;
  ServeRing* h_ring = nullptr;
  ServeRing* d_ring = nullptr;
  ServeSlot* h_slots = nullptr;
  ServeSlot* d_slots = nullptr;
  unsigned* d_claimed = nullptr;
  unsigned* d_finished = nullptr;
  unsigned long long* d_low = nullptr;
  unsigned long long h_low = 0;  // source of the reset copy of d_low
  int* d_status = nullptr;
  void* d_part = nullptr;
  bool loop_running = false;
  unsigned long long head = 0, next_entry = 0;
  double last_activity = 0;
  int launches = 0, abnormal_exits = 0;
  int last_exit_status = 0;       // status bits of the last launch that ended on its own
  double launched_at = 0, last_exit_after = 0;
  std::vector<int> free_slots;
  std::unordered_map<int, InFlight> in_flight;  // slot -> request
  // state shared with clients
  std::mutex mu;
  std::condition_variable cv_dispatch, cv_admit, cv_done;
  std::deque<Request> waiting;  // sample not resident yet
  std::deque<Request> ready;    // sample resident, not published yet
  std::unordered_map<uint64_t, Done> done;
  std::map<int, SampleRec> samples;
  uint64_t next_ticket = 1;
  int next_sample = 0;
  bool stop = false;
  std::thread dispatcher, admitter;
  // envelope of the generator at the last generating parameters (pilot once)
  std::vector<double> env_params;
  double env_value = 0;
  std::vector<double> latencies;
  std::vector<double> latencies_by_kind[2];  // resident at submission, admitted for the request
  double t_first = 0, t_last = 0;
  uint64_t n_done = 0, use_clock = 0;
  std::string err;
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

size_t footprint(tdmix_server* s, int64_t n) {
  return size_t((n + kTileEvents - 1) / kTileEvents) * internal::ops_of(s->ctx)->cache_tile_bytes;
}

// ---- the loop (dispatcher thread, mutex held)

cudaError_t launch_loop(tdmix_server* s) {
  cudaStream_t st = s->loop_stream;
  s->head = s->next_entry;
  s->h_low = s->head;
  cudaError_t e = cudaMemsetAsync(s->d_claimed, 0, kServeRingCap * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_finished, 0, kServeRingCap * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_low, &s->h_low, sizeof s->h_low, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // h_low is read by the copy
  if (e != cudaSuccess) return e;
  __atomic_store_n(&s->h_ring->stop, 0u, __ATOMIC_RELEASE);
  ServeLoopArgs a{};
  a.ring = s->d_ring;
  a.slots = s->d_slots;
  a.claimed = s->d_claimed;
  a.finished = s->d_finished;
  a.low = s->d_low;
  a.head = s->head;
  a.km = internal::model_const_of(s->ctx);
  a.mc_cols = s->d_mc_cols;
  a.inv_sum_w = s->inv_sum_w;
  a.part = s->d_part;
  a.status = s->d_status;
  a.logtab = internal::log_table_of(s->ctx);
  a.idle_ns = kIdleNs;
  e = internal::ops_of(s->ctx)->serve(s->grid, st, a);
  if (e == cudaSuccess) e = cudaEventRecord(s->loop_done, st);
  if (e == cudaSuccess) {
    s->loop_running = true;
    s->launches++;
    s->launched_at = now_s();
  }
  return e;
}

void stop_loop(tdmix_server* s) {
  if (!s->loop_running) return;
  __atomic_store_n(&s->h_ring->stop, 1u, __ATOMIC_RELEASE);
  cudaEventSynchronize(s->loop_done);
  s->loop_running = false;
}

void complete(tdmix_server* s, int slot, InFlight& inf, int status, const double* result) {
  const int rw = kResHeader + s->np;
  Done d{status, result ? std::vector<double>(result, result + rw) : std::vector<double>(rw, NAN),
         now_s() - inf.req.t_submit};
  auto it = s->samples.find(inf.req.sample);
  if (it != s->samples.end()) it->second.pending--;
  s->latencies.push_back(d.latency_s);
  s->latencies_by_kind[inf.req.admitted ? 1 : 0].push_back(d.latency_s);
  if (s->n_done == 0) s->t_first = inf.req.t_submit;
  s->t_last = now_s();
  s->n_done++;
  s->done[inf.req.ticket] = std::move(d);
  s->free_slots.push_back(slot);
}

void dispatcher_loop(tdmix_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // (1) publish ready requests into free slots
    bool published = false;
    while (!s->ready.empty() && !s->free_slots.empty() && s->next_entry - s->head < kServeRingCap) {
      if (!s->loop_running) {
        const cudaError_t e = launch_loop(s);
        if (e != cudaSuccess) {  // the request fails with the launch's error
          s->err = std::string("serving loop launch: ") + cudaGetErrorString(e);
          Request q = std::move(s->ready.front());
          s->ready.pop_front();
          InFlight inf{std::move(q), 0};
          const int slot = s->free_slots.back();
          s->free_slots.pop_back();
          complete(s, slot, inf, TDMIX_ERR_CUDA, nullptr);
          s->cv_done.notify_all();
          continue;
        }
      }
      Request q = std::move(s->ready.front());
      s->ready.pop_front();
      const int slot = s->free_slots.back();
      s->free_slots.pop_back();
      SampleRec& rec = s->samples.at(q.sample);
      const int n_tiles = int((rec.n + kTileEvents - 1) / kTileEvents);
      const int ct = std::max(1, (n_tiles + kServeMaxChunks - 1) / kServeMaxChunks);
      ServeSlot& sl = s->h_slots[slot];
      sl.cache = rec.cache;
      sl.n = rec.n;
      sl.tile_bytes = rec.tile_bytes;
      sl.chunk_tiles = ct;
      sl.n_tiles = n_tiles;
      sl.n_chunks = (n_tiles + ct - 1) / ct;
      sl.sum_t = rec.sum_t;
      std::memcpy(sl.params, q.params.data(), s->np * sizeof(double));
      const unsigned long long e = s->next_entry++;
      s->h_ring->slot[e - s->head] = slot;
      __atomic_store_n(&s->h_ring->tail, e + 1, __ATOMIC_RELEASE);  // publishes the slot and the entry
      rec.last_used = ++s->use_clock;
      s->in_flight.emplace(slot, InFlight{std::move(q), e});
      published = true;
    }
    if (published) s->last_activity = now_s();
    // (2) completions
    bool completed = false;
    for (auto it = s->in_flight.begin(); it != s->in_flight.end();) {
      const int slot = it->first;
      const unsigned long long d = __atomic_load_n(&s->h_slots[slot].done, __ATOMIC_ACQUIRE);
      if (d == it->second.entry + 1) {
        const double* r = s->h_slots[slot].result;
        const int status = r[2] < 0 ? int(r[2]) : ((r[2] > 0 || !std::isfinite(r[0])) ? TDMIX_ERR_NONFINITE : TDMIX_OK);
        complete(s, slot, it->second, status, r);
        it = s->in_flight.erase(it);
        completed = true;
      } else {
        ++it;
      }
    }
    if (completed) {
      s->last_activity = now_s();
      s->cv_done.notify_all();
      s->cv_admit.notify_all();  // samples may have become evictable
    }
    // (3) the loop's lifetime
    if (s->loop_running && cudaEventQuery(s->loop_done) == cudaSuccess) {
      // the loop left by itself (a bounded wait gave up): requests it did not
      // finish run again in the next launch
      s->loop_running = false;
      s->abnormal_exits++;
      int status = -1;
      if (cudaMemcpy(&status, s->d_status, sizeof status, cudaMemcpyDeviceToHost) == cudaSuccess)
        s->last_exit_status = status;
      s->last_exit_after = now_s() - s->launched_at;
      std::vector<int> slots;
      for (auto& kv : s->in_flight) slots.push_back(kv.first);
      std::sort(slots.begin(), slots.end(), [&](int x, int y) { return s->in_flight[x].entry > s->in_flight[y].entry; });
      for (int sl : slots) {
        s->ready.push_front(std::move(s->in_flight[sl].req));
        s->free_slots.push_back(sl);
      }
      s->in_flight.clear();
      continue;
    }
    if (s->loop_running && s->in_flight.empty()) {
      const bool ring_used_up = s->next_entry - s->head >= kServeRingCap;
      if (ring_used_up || (s->ready.empty() && now_s() - s->last_activity > kLoopIdleStop)) stop_loop(s);
    }
    // (4) wait: poll while requests are in flight
    if (!s->in_flight.empty()) {
      lk.unlock();
      std::this_thread::yield();  // poll the completion flags again soon
      lk.lock();
    } else if (s->loop_running) {
      s->cv_dispatch.wait_for(lk, std::chrono::milliseconds(5));
    } else {
      s->cv_dispatch.wait(lk, [&] { return s->stop || !s->ready.empty(); });
    }
  }
  stop_loop(s);
}

// ---- admission (admission thread)

void admitter_loop(tdmix_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // the first waiting request whose sample is neither resident nor being admitted
    int id = -1;
    for (const Request& q : s->waiting) {
      const SampleRec& r = s->samples.at(q.sample);
      if (!r.resident && !r.admitting) {
        id = q.sample;
        break;
      }
    }
    if (id < 0) {
      s->cv_admit.wait(lk);
      continue;
    }
    SampleRec& rec = s->samples.at(id);
    const size_t need = footprint(s, rec.n);
    bool room = true;
    while (s->resident_bytes + need > s->budget) {
      int victim = -1;
      uint64_t oldest = UINT64_MAX;
      for (auto& kv : s->samples)
        if (kv.second.resident && kv.second.pending == 0 && kv.second.last_used < oldest) {
          oldest = kv.second.last_used;
          victim = kv.first;
        }
      if (victim < 0) {
        room = false;
        break;
      }
      SampleRec& v = s->samples.at(victim);
      cudaFreeAsync(v.cache, internal::stream_of(s->ctx));  // no request uses it (pending == 0)
      v.cache = nullptr;
      v.resident = false;
      s->resident_bytes -= v.bytes;
    }
    if (!room) {  // memory frees up as requests complete
      s->cv_admit.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    rec.admitting = true;
    // inputs of the admission, used without the mutex (the record is not
    // erased while admitting)
    const bool generated = rec.generated;
    const int64_t n = rec.n;
    double gen_info[4] = {generated && rec.gen_params == s->env_params ? s->env_value : 0.0, 0, 0, 0};
    lk.unlock();
    void* cache = nullptr;
    int64_t tile_bytes = 0;
    double sum_t = 0;
    int rc = TDMIX_OK;
    cudaStream_t st = internal::stream_of(s->ctx);
    if (generated) {
      double* p = nullptr;
      double* t = nullptr;
      if (cudaMallocAsync(reinterpret_cast<void**>(&p), size_t(16) * n * sizeof(double), st) != cudaSuccess ||
          cudaMallocAsync(reinterpret_cast<void**>(&t), size_t(n) * sizeof(double), st) != cudaSuccess) {
        rc = TDMIX_ERR_NOMEM;
      } else {
        rc = tdmix_generate(s->ctx, rec.gen_params.data(), n, rec.seed, rec.stream, 0, p, t, gen_info);
        if (rc == TDMIX_OK) {
          tdmix_events ev{};
          ev.n = n;
          for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 4; ++c) ev.p[a][c] = p + size_t(a * 4 + c) * n;
          ev.t = t;
          ev.on_device = 1;
          rc = internal::take_component_cache(s->ctx, &ev, s->defaults.data(), &cache, &tile_bytes, &sum_t);
        }
      }
      if (p) cudaFreeAsync(p, st);
      if (t) cudaFreeAsync(t, st);
      cudaStreamSynchronize(st);
    } else {
      tdmix_events ev{};
      ev.n = n;
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) ev.p[a][c] = rec.planes.data() + size_t(a * 4 + c) * n;
      ev.t = rec.t.data();
      ev.on_device = 0;
      rc = internal::take_component_cache(s->ctx, &ev, s->defaults.data(), &cache, &tile_bytes, &sum_t);
    }
    std::string msg = rc ? internal::error_of(s->ctx) : std::string();
    lk.lock();
    rec.admitting = false;
    if (generated && rc == TDMIX_OK) {
      s->env_params = rec.gen_params;
      s->env_value = gen_info[0];
    }
    if (rc) {
      // every waiting request of this sample fails with the admission's status
      s->err = "admission: " + msg;
      for (auto it = s->waiting.begin(); it != s->waiting.end();) {
        if (it->sample == id) {
          Done d{rc, std::vector<double>(kResHeader + s->np, NAN), now_s() - it->t_submit};
          rec.pending--;
          s->done[it->ticket] = std::move(d);
          it = s->waiting.erase(it);
        } else {
          ++it;
        }
      }
      s->cv_done.notify_all();
      continue;
    }
    rec.cache = cache;
    rec.tile_bytes = tile_bytes;
    rec.sum_t = sum_t;
    rec.bytes = need;
    rec.resident = true;
    s->resident_bytes += need;
    for (auto it = s->waiting.begin(); it != s->waiting.end();) {
      if (it->sample == id) {
        s->ready.push_back(std::move(*it));
        it = s->waiting.erase(it);
      } else {
        ++it;
      }
    }
    s->cv_dispatch.notify_all();
  }
}

int new_sample(tdmix_server* s, SampleRec&& rec, int* sample_id) {
  std::lock_guard<std::mutex> lk(s->mu);
  *sample_id = s->next_sample++;
  s->samples.emplace(*sample_id, std::move(rec));
  return TDMIX_OK;
}

}  // namespace

extern "C" {

int tdmix_server_create(const char* model_json, int precision, size_t hbm_budget_bytes, int max_slots,
                        tdmix_server** out) {
  if (!out) return TDMIX_ERR_ARG;
  *out = nullptr;
  if (max_slots < 1 || max_slots > kServeMaxSlots || hbm_budget_bytes == 0) return TDMIX_ERR_ARG;
  tdmix_server* s = new tdmix_server;
  *out = s;
  if (cudaGetDevice(&s->device) != cudaSuccess) return sfail(s, TDMIX_ERR_CUDA, "no CUDA device");
  int rc = tdmix_create(model_json, precision, &s->ctx);
  if (rc) return sfail(s, rc, s->ctx ? tdmix_last_error(s->ctx) : "model");
  if (internal::is_generic(s->ctx))
    return sfail(s, TDMIX_ERR_UNSUPPORTED,
                 "serving needs a model structure compiled into the library (the generic evaluation keeps no "
                 "component cache)");
  cudaStream_t st;
  SV_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  tdmix_set_stream(s->ctx, st);
  SV_CK(cudaStreamCreateWithFlags(&s->loop_stream, cudaStreamNonBlocking));
  SV_CK(cudaEventCreateWithFlags(&s->loop_done, cudaEventDisableTiming));
  const CompiledModel& m = internal::model_of(s->ctx);
  s->np = m.n_params();
  s->nc = int(m.chains.size());
  s->nr = m.NR();
  s->defaults = m.default_params();
  s->fixed.assign(s->defaults.begin() + 2 * s->nc, s->defaults.begin() + 2 * s->nc + 2 * s->nr);
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->grid = std::max(1, internal::num_sms_of(s->ctx) - kReservedSMs);
  // serving keeps the model fixed: only coefficients and x, y float
  std::vector<int> mask = m.floating_mask();
  for (int k = 2 * s->nc; k < 2 * s->nc + 2 * s->nr; ++k) mask[k] = 0;
  tdmix_set_floating(s->ctx, mask.data());
  const ShapeOps* ops = internal::ops_of(s->ctx);
  SV_CK(cudaHostAlloc(reinterpret_cast<void**>(&s->h_ring), sizeof(ServeRing), cudaHostAllocMapped));
  SV_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_ring), s->h_ring, 0));
  std::memset(s->h_ring, 0, sizeof(ServeRing));
  SV_CK(cudaHostAlloc(reinterpret_cast<void**>(&s->h_slots), kServeMaxSlots * sizeof(ServeSlot), cudaHostAllocMapped));
  SV_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_slots), s->h_slots, 0));
  std::memset(s->h_slots, 0, kServeMaxSlots * sizeof(ServeSlot));
  SV_CK(cudaMalloc(&s->d_claimed, kServeRingCap * sizeof(unsigned)));
  SV_CK(cudaMalloc(&s->d_finished, kServeRingCap * sizeof(unsigned)));
  SV_CK(cudaMalloc(&s->d_low, sizeof(unsigned long long)));
  SV_CK(cudaMalloc(&s->d_status, sizeof(int)));
  // chunk-partial rows per slot (16-byte aligned rows of an even stride)
  SV_CK(cudaMalloc(&s->d_part, size_t(max_slots) * kServeMaxChunks * ops->serve_row_stride * 8));
  SV_CK(cudaMalloc(&s->d_mc_cols, ops->mc_width * sizeof(double)));
  for (int k = max_slots - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->dispatcher = std::thread(dispatcher_loop, s);
  s->admitter = std::thread(admitter_loop, s);
  return TDMIX_OK;
}

int tdmix_server_add_mc(tdmix_server* s, const tdmix_events* mc) {
  if (!s || !mc || !s->ctx) return sfail(s, TDMIX_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->have_mc) return sfail(s, TDMIX_ERR_STATE, "the MC sample is already set");
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
  return new_sample(s, std::move(rec), sample_id);
}

int tdmix_server_add_generated_sample(tdmix_server* s, const double* params, int64_t n, uint64_t seed,
                                      uint32_t stream, int* sample_id) {
  if (!s || !params || !sample_id || n < 1) return sfail(s, TDMIX_ERR_ARG, "bad sample");
  for (int k = 0; k < s->np; ++k)
    if (!std::isfinite(params[k])) return sfail(s, TDMIX_ERR_NONFINITE, "generating parameters are not finite");
  if (!(std::fabs(params[s->np - 1]) < 1.0)) return sfail(s, TDMIX_ERR_DOMAIN, "|y| must be below 1");
  SampleRec rec;
  rec.n = n;
  rec.generated = true;
  rec.gen_params.assign(params, params + s->np);
  rec.seed = seed;
  rec.stream = stream;
  return new_sample(s, std::move(rec), sample_id);
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
  for (int k = 0; k < s->np; ++k)
    if (!std::isfinite(params[k])) return sfail(s, TDMIX_ERR_NONFINITE, "parameter is not finite");
  if (!(std::fabs(params[s->np - 1]) < 1.0)) return sfail(s, TDMIX_ERR_DOMAIN, "|y| must be below 1");
  Request q{s->next_ticket++, sample_id, std::vector<double>(params, params + s->np), now_s()};
  *ticket = q.ticket;
  it->second.pending++;
  if (it->second.resident) {
    it->second.last_used = ++s->use_clock;
    s->ready.push_back(std::move(q));
    s->cv_dispatch.notify_all();
  } else {
    q.admitted = true;
    s->waiting.push_back(std::move(q));
    s->cv_admit.notify_all();
  }
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

namespace {

// nearest-rank percentile q of the latencies l (sorted in place), microseconds
double percentile_us(std::vector<double>& l, double q) {
  std::sort(l.begin(), l.end());
  return l[std::min(l.size() - 1, size_t(q * (l.size() - 1) + 0.5))] * 1e6;
}

}  // namespace

int tdmix_server_stats(tdmix_server* s, double* p50_us, double* p99_us, double* evals_per_s) {
  if (!s) return TDMIX_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = s->latencies;
  if (l.empty()) return sfail(s, TDMIX_ERR_STATE, "no completed requests");
  if (p50_us) *p50_us = percentile_us(l, 0.50);
  if (p99_us) *p99_us = percentile_us(l, 0.99);
  if (evals_per_s) *evals_per_s = s->t_last > s->t_first ? double(s->n_done) / (s->t_last - s->t_first) : 0.0;
  return TDMIX_OK;
}

int tdmix_server_latency(tdmix_server* s, int kind, double* p50_us, double* p99_us, int64_t* count) {
  if (!s || kind < TDMIX_LATENCY_ALL || kind > TDMIX_LATENCY_ADMITTED) return sfail(s, TDMIX_ERR_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = kind == TDMIX_LATENCY_ALL ? s->latencies : s->latencies_by_kind[kind - 1];
  if (count) *count = int64_t(l.size());
  if (l.empty()) {
    if (p50_us) *p50_us = NAN;
    if (p99_us) *p99_us = NAN;
    return TDMIX_OK;
  }
  if (p50_us) *p50_us = percentile_us(l, 0.50);
  if (p99_us) *p99_us = percentile_us(l, 0.99);
  return TDMIX_OK;
}

int tdmix_server_reset_stats(tdmix_server* s) {
  if (!s) return TDMIX_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->latencies_by_kind[0].clear();
  s->latencies_by_kind[1].clear();
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

int tdmix_server_loop_info(tdmix_server* s, int64_t* info) {
  if (!s || !info) return TDMIX_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  info[0] = s->launches;
  info[1] = s->abnormal_exits;
  info[2] = int64_t(s->next_entry);
  info[3] = s->loop_running ? 1 : 0;
  info[4] = s->last_exit_status;
  info[5] = int64_t(s->last_exit_after * 1e6);
  return TDMIX_OK;
}

const char* tdmix_server_last_error(const tdmix_server* s) { return s ? s->err.c_str() : "null server"; }

void tdmix_server_destroy(tdmix_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_dispatch.notify_all();
  s->cv_admit.notify_all();
  s->cv_done.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  if (s->admitter.joinable()) s->admitter.join();
  cudaStream_t st = s->ctx ? internal::stream_of(s->ctx) : nullptr;
  for (auto& kv : s->samples)
    if (kv.second.cache) cudaFreeAsync(kv.second.cache, st);
  if (st) cudaStreamSynchronize(st);
  cudaFree(s->d_claimed);
  cudaFree(s->d_finished);
  cudaFree(s->d_low);
  cudaFree(s->d_status);
  cudaFree(s->d_part);
  cudaFree(s->d_mc_cols);
  if (s->h_ring) cudaFreeHost(s->h_ring);
  if (s->h_slots) cudaFreeHost(s->h_slots);
  if (s->loop_done) cudaEventDestroy(s->loop_done);
  if (s->loop_stream) cudaStreamDestroy(s->loop_stream);
  if (s->ctx) tdmix_destroy(s->ctx);
  if (st) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
