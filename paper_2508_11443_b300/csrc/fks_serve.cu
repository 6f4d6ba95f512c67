// fks_serve.cu -- the serving loop: resident maps under a memory budget,
// build and lookup requests that arrive over time, continuous batching of
// lookups into one launch, and latency statistics.
//
// Threads:
//   clients     fks_server_submit (any thread) appends to the arrival queue
//   scheduler   applies arrivals in order (admission + LRU eviction for
//               builds, routing for lookups), launches coalesced lookup
//               batches on its stream, observes their completion events
//   workers     run builds (each blocks on its own stream until the build's
//               status is known) and hand the finished map back
// In FKS_SERVE_PER_CALL mode the scheduler itself runs each request alone,
// in arrival order, with a synchronisation after each (the comparison point).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "fks.h"
#include "fks_internal.cuh"
#include "fks_testing.h"

using namespace fks;

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Accounted bytes of a map (the allocation of its tables).
uint64_t map_bytes(uint32_t kind, uint64_t n, uint64_t ctx_bytes) {
  return kind == FKS_KEY_BYTES ? 136 * n + ctx_bytes : 72 * n;
}

struct Req {
  fks_request r{};
  uint64_t ticket = 0;
  double t_arrive = 0, t_done = 0;
  fks_status status = FKS_OK;
  bool done = false;
  fks_map_t built = nullptr;  // build result, handed from a worker
};

enum MapState { kEmpty = 0, kBuilding, kReady, kEvicted };

struct MapSlot {
  fks_map_t map = nullptr;
  MapState state = kEmpty;
  uint64_t bytes = 0;
  uint64_t lru = 0;
  uint32_t inflight = 0;       // lookups routed to the map and not yet complete
  bool free_when_idle = false; // evicted while lookups were in flight
  bool discard = false;        // evicted while its build was running
  std::vector<Req*> parked;    // lookups waiting for the map's build
  LookupMap view{};
  int strings = 0, out_i64 = 1;
};

struct Batch {
  cudaEvent_t ev = nullptr;
  cudaError_t err = cudaSuccess;  // a failed upload or launch: the batch's requests fail
  std::vector<Req*> reqs;
  LookupReq* h_reqs = nullptr;  // pinned
  uint64_t* h_begins = nullptr;
  LookupReq* d_reqs = nullptr;
  uint64_t* d_begins = nullptr;
};

}  // namespace

struct fks_server {
  fks_server_opts opts{};
  std::mutex mu;                 // arrivals, completions, build results
  std::condition_variable cv;    // wakes the scheduler
  std::condition_variable done_cv;
  std::deque<Req*> arrivals;
  std::deque<Req*> build_results;
  std::atomic<uint64_t> posted{0};  // arrivals + build results ever queued (lets a busy scheduler skip mu)
  std::vector<Req*> all;         // every request, by ticket - 1
  std::atomic<bool> stop{false};
  // scheduler state
  std::vector<MapSlot> maps;
  std::set<std::pair<uint64_t, uint32_t>> lru;  // (last use, id) of resident maps (ready or building)
  uint64_t used = 0, peak = 0, seq = 0;
  uint64_t evictions = 0, rejected = 0, batches = 0;
  std::vector<Req*> ready;       // lookups ready for the next batch
  std::deque<Batch*> inflight;
  std::vector<Batch*> idle_batches;
  cudaStream_t stream = nullptr;
  int sms = 148;
  // builds
  std::mutex bmu;
  std::condition_variable bcv;
  std::deque<Req*> build_queue;
  std::vector<std::thread> workers;
  std::thread sched;
};

namespace {

void complete(fks_server* S, Req* q, fks_status st) {
  q->status = st;
  q->t_done = now_us();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->done = true;
  }
  S->done_cv.notify_all();
}

void touch(fks_server* S, uint32_t id) {
  MapSlot& m = S->maps[id];
  const bool resident = m.state == kReady || m.state == kBuilding;
  if (resident) S->lru.erase({m.lru, id});
  m.lru = ++S->seq;
  if (resident) S->lru.insert({m.lru, id});
}

void release_map(fks_server* S, uint32_t id) {
  MapSlot& m = S->maps[id];
  if (m.map) fks_map_destroy(m.map);
  m.map = nullptr;
  m.free_when_idle = false;
  m.state = kEvicted;
  (void)S;
}

// Evict least-recently-used resident maps until `need` more bytes fit.  A
// map still being built is evicted all the same (residency follows arrival
// order exactly); its result is discarded when the build finishes.
bool admit(fks_server* S, uint64_t need) {
  while (S->used + need > S->opts.memory_budget && !S->lru.empty()) {
    const uint32_t id = S->lru.begin()->second;
    S->lru.erase(S->lru.begin());
    MapSlot& m = S->maps[id];
    S->used -= m.bytes;
    m.bytes = 0;
    ++S->evictions;
    if (m.state == kBuilding) {
      m.discard = true;
      m.state = kEvicted;
      continue;
    }
    m.state = kEvicted;
    if (m.inflight == 0) release_map(S, id);
    else m.free_when_idle = true;  // freed once its in-flight lookups finish
  }
  return S->used + need <= S->opts.memory_budget;
}

void worker_main(fks_server* S) {
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Req* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->bmu);
      S->bcv.wait(lk, [&] { return S->stop.load() || !S->build_queue.empty(); });
      if (S->build_queue.empty()) break;
      q = S->build_queue.front();
      S->build_queue.pop_front();
    }
    const fks_request& r = q->r;
    fks_map_t m = nullptr;
    fks_status st_ = r.key_kind == FKS_KEY_BYTES
                         ? fks_build_bytes(r.ctx, r.offs, r.vals, fks_val_type(r.val_type), r.n, r.seed, nullptr,
                                           nullptr, reinterpret_cast<fks_stream_t>(st), &m)
                         : fks_build_u64(r.keys, r.vals, fks_val_type(r.val_type), r.n, r.seed, nullptr, nullptr,
                                         reinterpret_cast<fks_stream_t>(st), &m);
    q->built = m;
    q->status = st_;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->build_results.push_back(q);
      S->posted.fetch_add(1, std::memory_order_release);
    }
    S->cv.notify_one();
  }
  cudaStreamDestroy(st);
}

// Route a lookup; returns false if it completed at once (unknown map).
void route_lookup(fks_server* S, Req* q) {
  const uint32_t id = q->r.map_id;
  MapSlot& m = S->maps[id];
  touch(S, id);
  if (m.state == kReady) {
    ++m.inflight;
    S->ready.push_back(q);
  } else if (m.state == kBuilding) {
    ++m.inflight;
    m.parked.push_back(q);
  } else {
    complete(S, q, FKS_ERR_EVICTED);
  }
}

void lookup_done(fks_server* S, Req* q) {
  MapSlot& m = S->maps[q->r.map_id];
  if (--m.inflight == 0 && m.free_when_idle) release_map(S, q->r.map_id);
}

void apply_arrival(fks_server* S, Req* q) {
  const fks_request& r = q->r;
  if (r.type == FKS_REQ_LOOKUP) {
    route_lookup(S, q);
    return;
  }
  MapSlot& m = S->maps[r.map_id];
  if (m.state == kReady || m.state == kBuilding || m.free_when_idle || m.discard) {  // the id is taken
    complete(S, q, FKS_ERR_INVALID_ARG);
    return;
  }
  const uint64_t need = map_bytes(r.key_kind, r.n, r.ctx_bytes);
  if (!admit(S, need)) {
    ++S->rejected;
    complete(S, q, FKS_ERR_OUT_OF_MEMORY);
    return;
  }
  S->used += need;
  S->peak = std::max(S->peak, S->used);
  m.state = kBuilding;
  m.bytes = need;
  m.map = nullptr;
  m.lru = ++S->seq;
  S->lru.insert({m.lru, r.map_id});
  {
    std::lock_guard<std::mutex> lk(S->bmu);
    S->build_queue.push_back(q);
  }
  S->bcv.notify_one();
}

void apply_build_result(fks_server* S, Req* q) {
  MapSlot& m = S->maps[q->r.map_id];
  std::vector<Req*> parked;
  parked.swap(m.parked);
  if (m.discard) {
    // Evicted while building.  Lookups that arrived before the eviction are
    // still served; the map is freed once they finish.
    m.discard = false;
    if (q->status == FKS_OK && !parked.empty()) {
      m.map = q->built;
      fks::lookup_view_of(m.map, &m.view, &m.strings, &m.out_i64);
      m.free_when_idle = true;
      for (Req* l : parked) S->ready.push_back(l);
    } else {
      if (q->built) fks_map_destroy(q->built);
      for (Req* l : parked) {
        --m.inflight;
        complete(S, l, q->status == FKS_OK ? FKS_ERR_EVICTED : q->status);
      }
    }
  } else if (q->status == FKS_OK) {
    m.map = q->built;
    m.state = kReady;
    fks::lookup_view_of(m.map, &m.view, &m.strings, &m.out_i64);
    for (Req* l : parked) S->ready.push_back(l);
  } else {
    S->lru.erase({m.lru, q->r.map_id});
    S->used -= m.bytes;
    m.bytes = 0;
    m.state = kEmpty;
    for (Req* l : parked) {
      lookup_done(S, l);
      complete(S, l, q->status);
    }
  }
  complete(S, q, q->status);
}

// failure injection (fks_testing.h): lookup batches left to fail at launch
std::atomic<int> g_fail_serve_launches{0};

bool inject_launch_failure() {
  int n = g_fail_serve_launches.load();
  while (n > 0 && !g_fail_serve_launches.compare_exchange_weak(n, n - 1)) {
  }
  return n > 0;
}

void launch_batches(fks_server* S) {
  while (!S->ready.empty() && S->inflight.size() < S->opts.max_inflight_batches && !S->idle_batches.empty()) {
    Batch* b = S->idle_batches.back();
    S->idle_batches.pop_back();
    const size_t take = std::min<size_t>(S->ready.size(), S->opts.max_batch_requests);
    b->reqs.assign(S->ready.begin(), S->ready.begin() + take);
    S->ready.erase(S->ready.begin(), S->ready.begin() + take);
    uint64_t total = 0;
    for (size_t i = 0; i < take; ++i) {
      const Req* q = b->reqs[i];
      const MapSlot& m = S->maps[q->r.map_id];
      LookupReq& L = b->h_reqs[i];
      L.M = m.view;
      L.q = q->r.q;
      L.qctx = q->r.qctx;
      L.qoffs = q->r.qoffs;
      L.out = q->r.out_vals;
      L.found = q->r.out_found;
      L.absent = q->r.absent;
      L.begin = total;
      L.strings = uint32_t(m.strings);
      L.out_i64 = uint32_t(m.out_i64);
      b->h_begins[i] = total;
      total += q->r.nq;
    }
    b->h_begins[take] = total;
    cudaError_t e = cudaMemcpyAsync(b->d_reqs, b->h_reqs, sizeof(LookupReq) * take, cudaMemcpyHostToDevice,
                                    S->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_begins, b->h_begins, sizeof(uint64_t) * (take + 1), cudaMemcpyHostToDevice,
                          S->stream);
    if (e == cudaSuccess)
      e = inject_launch_failure() ? cudaErrorLaunchFailure
                                  : launch_lookup_requests(b->d_reqs, b->d_begins, uint32_t(take), total, S->sms,
                                                           S->stream);
    const cudaError_t er = cudaEventRecord(b->ev, S->stream);
    b->err = e != cudaSuccess ? e : er;
    S->inflight.push_back(b);
    ++S->batches;
  }
}

void poll_batches(fks_server* S) {
  while (!S->inflight.empty()) {
    Batch* b = S->inflight.front();
    const cudaError_t e = b->err != cudaSuccess ? b->err : cudaEventQuery(b->ev);
    if (e == cudaErrorNotReady) break;
    const fks_status st = e == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
    if (b->err != cudaSuccess) cudaStreamSynchronize(S->stream);  // nothing of the batch still reads its buffers
    b->err = cudaSuccess;
    for (Req* q : b->reqs) {
      lookup_done(S, q);
      complete(S, q, st);
    }
    b->reqs.clear();
    S->inflight.pop_front();
    S->idle_batches.push_back(b);
  }
}

// Per-call mode: one request at a time, each fully completed before the next.
void run_one_per_call(fks_server* S, Req* q) {
  const fks_request& r = q->r;
  if (r.type == FKS_REQ_BUILD) {
    MapSlot& m = S->maps[r.map_id];
    if (m.state == kReady || m.state == kBuilding) {
      complete(S, q, FKS_ERR_INVALID_ARG);
      return;
    }
    const uint64_t need = map_bytes(r.key_kind, r.n, r.ctx_bytes);
    if (!admit(S, need)) {
      ++S->rejected;
      complete(S, q, FKS_ERR_OUT_OF_MEMORY);
      return;
    }
    S->used += need;
    S->peak = std::max(S->peak, S->used);
    m.lru = ++S->seq;
    fks_map_t h = nullptr;
    const fks_status st = r.key_kind == FKS_KEY_BYTES
                              ? fks_build_bytes(r.ctx, r.offs, r.vals, fks_val_type(r.val_type), r.n, r.seed,
                                                nullptr, nullptr, reinterpret_cast<fks_stream_t>(S->stream), &h)
                              : fks_build_u64(r.keys, r.vals, fks_val_type(r.val_type), r.n, r.seed, nullptr,
                                              nullptr, reinterpret_cast<fks_stream_t>(S->stream), &h);
    if (st == FKS_OK) {
      m.map = h;
      m.state = kReady;
      m.bytes = need;
      fks::lookup_view_of(h, &m.view, &m.strings, &m.out_i64);
      S->lru.insert({m.lru, r.map_id});
    } else {
      S->used -= need;
      m.state = kEmpty;
    }
    complete(S, q, st);
    return;
  }
  MapSlot& m = S->maps[r.map_id];
  touch(S, r.map_id);
  if (m.state != kReady) {
    complete(S, q, FKS_ERR_EVICTED);
    return;
  }
  const fks_status st = m.strings
                            ? fks_lookup_bytes(m.map, r.qctx, r.qoffs, r.nq, r.out_vals, r.out_found, r.absent,
                                               reinterpret_cast<fks_stream_t>(S->stream))
                            : fks_lookup_u64(m.map, r.q, r.nq, r.out_vals, r.out_found, r.absent,
                                             reinterpret_cast<fks_stream_t>(S->stream));
  const cudaError_t e = cudaStreamSynchronize(S->stream);
  complete(S, q, st != FKS_OK ? st : (e == cudaSuccess ? FKS_OK : FKS_ERR_CUDA));
}

void scheduler_main(fks_server* S) {
  std::vector<Req*> arrivals, results;
  uint64_t seen = 0;  // posted requests already taken from the queues
  for (;;) {
    const bool busy = !S->inflight.empty();
    arrivals.clear();
    results.clear();
    // With batches in flight the loop polls their events without sleeping
    // (a timed wait would add the kernel's timer slack, tens of
    // microseconds, to every completion) and takes the lock only when
    // something was queued; idle, it sleeps until work arrives.
    if (!busy || S->posted.load(std::memory_order_acquire) != seen) {
      std::unique_lock<std::mutex> lk(S->mu);
      auto have_work = [&] { return S->stop.load() || !S->arrivals.empty() || !S->build_results.empty(); };
      if (!busy) S->cv.wait(lk, have_work);
      seen = S->posted.load(std::memory_order_relaxed);  // everything up to here is in the queues
      arrivals.assign(S->arrivals.begin(), S->arrivals.end());
      S->arrivals.clear();
      results.assign(S->build_results.begin(), S->build_results.end());
      S->build_results.clear();
      if (S->stop.load() && arrivals.empty() && results.empty() && S->inflight.empty()) break;
    }
    if (S->opts.mode == FKS_SERVE_PER_CALL) {
      for (Req* q : arrivals) run_one_per_call(S, q);
      continue;
    }
    for (Req* q : results) apply_build_result(S, q);
    for (Req* q : arrivals) apply_arrival(S, q);
    const size_t before = S->inflight.size();
    poll_batches(S);
    launch_batches(S);
    if (arrivals.empty() && results.empty() && S->inflight.size() == before && !S->inflight.empty())
      std::this_thread::yield();  // nothing changed: let other threads run before the next poll
  }
}

}  // namespace

extern "C" {

void fks_test_fail_serve_launches(int n) { g_fail_serve_launches.store(n > 0 ? n : 0); }

fks_status fks_server_create(const fks_server_opts* o, fks_server_t* out) {
  if (!out || !o || o->struct_size < sizeof(fks_server_opts) || o->max_maps == 0 || o->memory_budget == 0 ||
      o->mode > FKS_SERVE_PER_CALL)
    return FKS_ERR_INVALID_ARG;
  *out = nullptr;
  fks_server* S = new fks_server();
  S->opts = *o;
  if (!S->opts.build_workers) S->opts.build_workers = 2;
  if (!S->opts.max_batch_requests) S->opts.max_batch_requests = 4096;
  if (!S->opts.max_inflight_batches) S->opts.max_inflight_batches = 2;
  S->maps.resize(o->max_maps);
  S->sms = fks::device_sm_count();
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete S;
    return FKS_ERR_CUDA;
  }
  const uint32_t nb = S->opts.max_inflight_batches, per = S->opts.max_batch_requests;
  for (uint32_t i = 0; i < nb; ++i) {
    Batch* b = new Batch();
    bool ok = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMallocHost(&b->h_reqs, sizeof(LookupReq) * per) == cudaSuccess;
    ok = ok && cudaMallocHost(&b->h_begins, sizeof(uint64_t) * (per + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_reqs, sizeof(LookupReq) * per) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_begins, sizeof(uint64_t) * (per + 1)) == cudaSuccess;
    S->idle_batches.push_back(b);
    if (!ok) {
      fks_server_destroy(S);
      return FKS_ERR_OUT_OF_MEMORY;
    }
  }
  if (S->opts.mode == FKS_SERVE_BATCHED)
    for (uint32_t i = 0; i < S->opts.build_workers; ++i) S->workers.emplace_back(worker_main, S);
  S->sched = std::thread(scheduler_main, S);
  *out = S;
  return FKS_OK;
}

fks_status fks_server_submit(fks_server_t S, const fks_request* r, uint64_t* h_ticket) {
  if (!S || !r || r->struct_size < sizeof(fks_request) || r->map_id >= S->opts.max_maps) return FKS_ERR_INVALID_ARG;
  if (r->type == FKS_REQ_BUILD ? (r->n == 0 || !r->vals || (r->key_kind == FKS_KEY_BYTES ? (!r->ctx || !r->offs) : !r->keys))
                               : (r->type != FKS_REQ_LOOKUP || (r->nq && (r->key_kind == FKS_KEY_BYTES ? (!r->qctx || !r->qoffs) : !r->q))))
    return FKS_ERR_INVALID_ARG;
  Req* q = new Req();
  q->r = *r;
  q->t_arrive = now_us();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->all.push_back(q);
    q->ticket = S->all.size();
    S->arrivals.push_back(q);
    S->posted.fetch_add(1, std::memory_order_release);
  }
  if (h_ticket) *h_ticket = q->ticket;
  S->cv.notify_one();
  return FKS_OK;
}

fks_status fks_server_replay(fks_server_t S, const fks_request* reqs, const double* h_arrival_us, uint64_t count,
                             uint64_t* h_tickets) {
  if (!S || (count && (!reqs || !h_arrival_us))) return FKS_ERR_INVALID_ARG;
  const double t0 = now_us();
  for (uint64_t i = 0; i < count; ++i) {
    const double due = t0 + h_arrival_us[i];
    while (now_us() < due) {
    }
    const fks_status st = fks_server_submit(S, reqs + i, h_tickets ? h_tickets + i : nullptr);
    if (st != FKS_OK) return st;
  }
  return FKS_OK;
}

fks_status fks_server_wait(fks_server_t S, uint64_t ticket, fks_status* h_result, double* h_latency_us) {
  if (!S || ticket == 0) return FKS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket > S->all.size()) return FKS_ERR_INVALID_ARG;
  Req* q = S->all[ticket - 1];
  S->done_cv.wait(lk, [&] { return q->done; });
  if (h_result) *h_result = q->status;
  if (h_latency_us) *h_latency_us = q->t_done - q->t_arrive;
  return FKS_OK;
}

fks_status fks_server_drain(fks_server_t S) {
  if (!S) return FKS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  S->done_cv.wait(lk, [&] {
    for (const Req* q : S->all)
      if (!q->done) return false;
    return true;
  });
  return FKS_OK;
}

static double pct(std::vector<double>& v, double p) {
  if (v.empty()) return 0;
  const size_t k = std::min(v.size() - 1, size_t(p * (v.size() - 1) + 0.5));
  std::nth_element(v.begin(), v.begin() + k, v.end());
  return v[k];
}

fks_status fks_server_stats(fks_server_t S, fks_server_stats_t* o) {
  if (!S || !o) return FKS_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  std::vector<double> all, lk_, bd;
  double t0 = 1e300, t1 = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    o->submitted = S->all.size();
    for (const Req* q : S->all) {
      if (!q->done) continue;
      ++o->completed;
      const double l = q->t_done - q->t_arrive;
      all.push_back(l);
      t0 = std::min(t0, q->t_arrive);
      t1 = std::max(t1, q->t_done);
      if (q->r.type == FKS_REQ_BUILD) {
        ++o->builds;
        bd.push_back(l);
      } else {
        ++o->lookups;
        o->queries += q->r.nq;
        lk_.push_back(l);
      }
    }
    o->batches = S->batches;
    o->evictions = S->evictions;
    o->rejected = S->rejected;
    o->resident_bytes = S->used;
    o->peak_resident_bytes = S->peak;
  }
  o->span_s = t1 > t0 ? (t1 - t0) * 1e-6 : 0;
  o->p50_us = pct(all, 0.50);
  o->p99_us = pct(all, 0.99);
  o->p999_us = pct(all, 0.999);
  o->lookup_p50_us = pct(lk_, 0.50);
  o->lookup_p99_us = pct(lk_, 0.99);
  o->build_p50_us = pct(bd, 0.50);
  o->build_p99_us = pct(bd, 0.99);
  return FKS_OK;
}

fks_map_t fks_server_map(fks_server_t S, uint32_t id) {
  if (!S || id >= S->opts.max_maps) return nullptr;
  fks_server_drain(S);
  return S->maps[id].state == kReady ? S->maps[id].map : nullptr;
}

void fks_server_destroy(fks_server_t S) {
  if (!S) return;
  if (S->sched.joinable()) fks_server_drain(S);
  S->stop.store(true);
  S->cv.notify_all();
  S->bcv.notify_all();
  if (S->sched.joinable()) S->sched.join();
  for (auto& w : S->workers)
    if (w.joinable()) w.join();
  if (S->stream) cudaStreamSynchronize(S->stream);
  for (auto& m : S->maps)
    if (m.map) fks_map_destroy(m.map);
  for (Batch* b : S->idle_batches) {
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->h_reqs) cudaFreeHost(b->h_reqs);
    if (b->h_begins) cudaFreeHost(b->h_begins);
    if (b->d_reqs) cudaFree(b->d_reqs);
    if (b->d_begins) cudaFree(b->d_begins);
    delete b;
  }
  for (Req* q : S->all) delete q;
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
