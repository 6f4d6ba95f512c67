// fks_api.cu -- host side of the C ABI declared in include/fks.h.
//
// A build runs level-one rounds (Sec. 2.3 make_1: a fresh const per round)
// until every map of the call satisfies the space bound and every bucket
// found collision-free level-two constants (make_2).  One round of all
// still-unfinished maps is one "pass" of the device pipeline in
// fks_build.cu; after each pass the per-map status words are read back (one
// stream synchronisation) and the maps that must redraw are re-run together.
// A per-call build is the one-map case of the same code.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fks.h"
#include "fks_internal.cuh"

using namespace fks;

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

static fks_status fail(fks_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
static fks_status cuda_fail(cudaError_t e, const char* where) {
  return fail(FKS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define FKS_CUDA(call)                                       \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
  } while (0)

// ---------------------------------------------------------------- metrics
#include <atomic>
static std::atomic<uint64_t> g_launches{0};
void fks::note_launches(uint32_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local int g_profile = 0;
static thread_local fks_build_profile g_last_profile{};

struct ProfileEvents {
  PassEvents pe{};
  cudaEvent_t fp0 = nullptr, fp1 = nullptr;
  bool ok = false;
  ProfileEvents() {
    if (!g_profile) return;
    ok = true;
    for (auto& e : pe.ev) ok &= cudaEventCreate(&e) == cudaSuccess;
    ok &= cudaEventCreate(&fp0) == cudaSuccess && cudaEventCreate(&fp1) == cudaSuccess;
  }
  ~ProfileEvents() {
    for (auto& e : pe.ev)
      if (e) cudaEventDestroy(e);
    if (fp0) cudaEventDestroy(fp0);
    if (fp1) cudaEventDestroy(fp1);
  }
  // after the pass has been synchronised
  void accumulate(fks_build_profile* p, bool strings) const {
    if (!ok) return;
    float ms = 0;
    if (p->grouping_levels == 2) {
      if (cudaEventElapsedTime(&ms, pe.ev[0], pe.ev[3]) == cudaSuccess) p->group_ms += ms;
    } else {
      if (cudaEventElapsedTime(&ms, pe.ev[0], pe.ev[1]) == cudaSuccess) p->count_ms += ms;
      if (cudaEventElapsedTime(&ms, pe.ev[1], pe.ev[2]) == cudaSuccess) p->scan_ms += ms;
      if (cudaEventElapsedTime(&ms, pe.ev[2], pe.ev[3]) == cudaSuccess) p->scatter_ms += ms;
    }
    if (cudaEventElapsedTime(&ms, pe.ev[3], pe.ev[4]) == cudaSuccess) p->part_build_ms += ms;
    if (strings && cudaEventElapsedTime(&ms, fp0, fp1) == cudaSuccess) p->fingerprint_ms += ms;
    p->passes += 1;
  }
};

// ---------------------------------------------------------------- device facts
static int sm_count() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // keep freed blocks in the stream-ordered pool instead of returning them
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    // Lookups are random 8 B / 16 B reads: ask L2 to fetch single 32-byte
    // sectors on a miss instead of larger promoted blocks (a per-context
    // hint that ends with the process; FKS_L2_FETCH overrides it).
    size_t gran = 32;
    if (const char* env = getenv("FKS_L2_FETCH")) gran = size_t(atoi(env));
    if (gran) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, gran);
    cudaGetLastError();
    if (sms <= 0) sms = 148;
  });
  return sms;
}

// ---------------------------------------------------------------- memory
struct Alloc {
  fks_allocator hook{};
  bool user = false;
  explicit Alloc(const fks_allocator* a) {
    if (a && a->struct_size >= sizeof(fks_allocator) && a->alloc && a->free) {
      hook = *a;
      user = true;
    }
  }
  void* get(size_t bytes, cudaStream_t s) const {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (user) return hook.alloc(bytes, reinterpret_cast<fks_stream_t>(s), hook.user);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t bytes, cudaStream_t s) const {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (user) hook.free(p, bytes, reinterpret_cast<fks_stream_t>(s), hook.user);
    else cudaFreeAsync(p, s);
  }
};

// Bump carving of one allocation into 256-byte aligned pieces.
struct Carve {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t at = off;
    off += (count * sizeof(T) + 255) & ~size_t(255);
    return at;
  }
};

// Pinned host staging for small control transfers (per thread).
struct Pinned {
  void* p = nullptr;
  size_t cap = 0;
  void* get(size_t bytes) {
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      cap = std::max<size_t>(bytes, 1 << 16);
      if (cudaMallocHost(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        cap = 0;
      }
    }
    return p;
  }
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
static thread_local Pinned g_pin_up, g_pin_down;

// ---------------------------------------------------------------- handles
// A build started by fks_build_*_async: the host thread running it, and
// what it reports.  Every use of the handle joins the thread first.
struct AsyncBuild {
  std::mutex mu;
  std::thread worker;
  bool joined = false;
  fks_status status = FKS_OK;
  std::string msg;
  int64_t seg[2] = {0, 0};  // the call's own copies of its small host arguments
  uint64_t seed = 0;
  fks_build_opts opts{};
  bool has_opts = false;
  fks_allocator alloc{};
  bool has_alloc = false;
};

struct fks_map {
  fks_key_kind kind = FKS_KEY_U64;
  fks_val_type vt = FKS_VAL_I64;
  uint64_t n = 0, seed = 0, S = 0, slot_cap = 0, att_sum = 0, ctx_bytes = 0, bytes = 0;
  uint64_t nonempty = 0;
  uint64_t nb = 0;          // level-one buckets (= descriptors)
  uint32_t lambda = 1;      // keys per bucket of the level-one draw
  uint32_t round = 0, max_s = 0, max_att = 0, overflow = 0;
  HashConsts c1{};
  uint64_t fpb = 0;
  uint64_t* desc = nullptr;
  uint64_t* slots = nullptr;
  uint64_t* rec = nullptr;  // inline-singleton records, or null
  uint8_t* ctx = nullptr;
  // ownership (null for maps borrowed from a set)
  void* block = nullptr;
  size_t block_bytes = 0;
  Alloc alloc{nullptr};
  AsyncBuild* async = nullptr;  // set for handles of fks_build_*_async
};

// Wait for the build of an asynchronous handle; its status (FKS_OK for
// synchronous handles).  A failed build leaves an empty handle.
static fks_status settle(fks_map* m) {
  if (!m || !m->async) return FKS_OK;
  AsyncBuild* a = m->async;
  std::lock_guard<std::mutex> lock(a->mu);
  if (!a->joined) {
    a->worker.join();
    a->joined = true;
  }
  if (a->status != FKS_OK) g_last_error = a->msg;
  return a->status;
}

struct fks_mapset {
  fks_key_kind kind = FKS_KEY_U64;
  fks_val_type vt = FKS_VAL_I64;
  std::vector<fks_map> maps;
  LookupMap* d_table = nullptr;  // device copy for batched lookups
  void* block = nullptr;
  size_t block_bytes = 0;
  Alloc alloc{nullptr};
  bool borrowed = false;  // the set of a recorded build: freed with it
};

struct fks_sortmap {
  fks_val_type vt = FKS_VAL_I64;
  uint64_t n = 0;
  int eytzinger = 0;         // 0: sorted order; 1: Eytzinger order, 1-based (n + 1 words)
  uint64_t* keys = nullptr;
  uint64_t* vals = nullptr;  // int64 words
  void* block = nullptr;
  size_t block_bytes = 0;
  Alloc alloc{nullptr};
};

static LookupMap lookup_view(const fks_map& m) {
  LookupMap L;
  L.desc = m.desc;
  L.slots = m.slots;
  L.ctx = m.ctx;
  L.c1 = m.c1;
  L.seed = m.seed;
  L.fpb = m.fpb;
  L.nb = uint32_t(m.nb);
  L.round = m.round;
  return L;
}

// ---------------------------------------------------------------- options
struct Opts {
  uint32_t bound = 4, attempt_cap = 4095, round_cap = 32, reject = 0, spin = 1u << 20, hold = 0;
  uint32_t lambda = 1;  // keys per level-one bucket
  uint32_t dedup = 0;   // from_array: first occurrence of equal keys wins
  uint32_t inline1 = 0; // inline-singleton records (one-map u64 builds at lambda 1)
};

// Options of the older, shorter layout (without keys_per_bucket) are accepted.
static bool read_opts(const fks_build_opts* o, Opts* out) {
  if (!o) return true;
  if (o->struct_size < offsetof(fks_build_opts, spin_limit) + sizeof(uint32_t)) return false;
  if (o->struct_size >= offsetof(fks_build_opts, keys_per_bucket) + sizeof(uint32_t) && o->keys_per_bucket)
    out->lambda = o->keys_per_bucket;
  if (o->struct_size >= offsetof(fks_build_opts, dedup) + sizeof(uint32_t)) {
    if (o->dedup > 1) return false;
    out->dedup = o->dedup;
  }
  if (o->struct_size >= offsetof(fks_build_opts, inline_singletons) + sizeof(uint32_t)) {
    if (o->inline_singletons > 1) return false;
    out->inline1 = o->inline_singletons;
  }
  if (out->lambda != 1 && out->lambda != 2 && out->lambda != 4 && out->lambda != 8 && out->lambda != 16)
    return false;
  if (out->inline1 && out->lambda != 1) return false;
  out->bound = 2 * (1 + out->lambda);  // E[sum s^2] < (1 + lambda) n: bound = twice that
  if (o->bound_factor) out->bound = o->bound_factor;
  if (o->attempt_cap) out->attempt_cap = o->attempt_cap;
  if (o->round_cap) out->round_cap = o->round_cap;
  out->reject = o->reject_attempts;
  if (o->spin_limit) out->spin = o->spin_limit;
  if (out->attempt_cap > 4095 || out->round_cap > 65535 || out->bound < 1 || out->bound > 64)
    return false;
  return true;
}

// Slot offsets are 32-bit descriptor fields: bound * n must stay below 2^32.
static bool sizes_fit(const Opts& o, uint64_t n) { return uint64_t(o.bound) * n <= 0xFFFFFFFFull; }

// test hook (not in the public header): make partition 0 never publish its
// slot prefix so that the bounded wait of partition 1 runs out.
static thread_local int g_hold_first_partition = 0;
extern "C" void fks_test_hold_first_partition(int on) { g_hold_first_partition = on; }

// ---------------------------------------------------------------- the build

struct BuildIn {
  fks_key_kind kind;
  const uint64_t* keys;  // u64 keys (input numbering)
  const uint8_t* ctx;    // string maps
  const int64_t* offs;
  const void* vals;
  fks_val_type vt;
  uint32_t m;
  const int64_t* seg;     // host [m+1]
  const uint64_t* seeds;  // host [m]
};

struct SetMem {
  uint64_t* desc = nullptr;
  uint64_t* slots = nullptr;
  uint64_t* rec = nullptr;  // inline-singleton records (2 words per bucket), or null
  uint8_t* ctx = nullptr;
  std::vector<uint64_t> slot_base;  // per map
  std::vector<uint64_t> desc_base;  // per map
};

// A build of m maps over one input.  init allocates the set's tables and the
// scratch of its passes once; enqueue_pass puts one pass of the device
// pipeline on a stream -- pass-table upload, kernels, status download --
// with no host synchronisation in it, so that a pass can be recorded as a
// CUDA graph; run is the host loop over level-one rounds: after each pass
// the per-map status words decide which maps are done and which redraw.
struct GraphPass;

struct SetBuild {
  BuildIn in{};
  Opts o{};
  Alloc A{nullptr};
  uint32_t m = 0;
  bool str = false;
  int PW = 1, W = 2;
  uint64_t total = 0;
  uint32_t logB = 0;
  uint64_t B = 0;
  std::vector<uint64_t> nbs;
  uint64_t ctx_bytes = 0;
  uint8_t* block = nullptr;  // the set's tables (desc, slots, context)
  size_t block_bytes = 0;
  uint8_t* scr = nullptr;    // scratch of the passes
  size_t scr_bytes = 0;
  SetMem mem;
  PassDev p{};
  MapDev* d_maps = nullptr;
  uint64_t* d_pseg = nullptr;
  uint32_t* d_qseg = nullptr;
  MapStatus* d_stat = nullptr;
  uint64_t* fps = nullptr;
  BuildShape bs{};  // launch shape (fks_tune.cu)
  SplitShape shape{};
  bool use_split = false;
  size_t hist_words = 0;
  size_t s_ka = 0, s_pa = 0, s_ga = 0, s_hist = 0, s_sums = 0, s_sa = 0, s_tb = 0;
  uint64_t* ovf_key = nullptr;
  size_t ovf_bytes = 0;
  int sms = 0;
  uint32_t levels = 1;  // grouping levels of the last pass
  // outcome of the last run
  std::vector<uint32_t> round;
  std::vector<fks_status> per_map;
  std::vector<fks_map> maps;
  fks_build_profile profile{};

  // pinned pass tables: MapDev[ma] | pass offsets u64[ma+1] | partition offsets u32[ma+1]
  static size_t up_bytes(uint32_t ma) {
    return sizeof(MapDev) * ma + sizeof(uint64_t) * (ma + 1) + sizeof(uint32_t) * (ma + 1);
  }
  // pinned status: MapStatus[ma] | overflow count
  static size_t down_bytes(uint32_t ma) { return sizeof(MapStatus) * ma + 16; }

  fks_status init(const BuildIn& in_, const Opts& o_, const Alloc& A_, cudaStream_t st);
  uint32_t fill_tables(const std::vector<uint32_t>& active, uint8_t* up);
  cudaError_t enqueue_pass(uint32_t ma, const uint8_t* up, uint8_t* down, bool copy_ctx, ProfileEvents* prof,
                           cudaStream_t st);
  fks_status run(cudaStream_t st, GraphPass* g);
  void free_scratch(cudaStream_t st) {
    if (ovf_key) A.put(ovf_key, ovf_bytes, st);
    ovf_key = nullptr;
    if (scr) A.put(scr, scr_bytes, st);
    scr = nullptr;
  }
  void free_tables(cudaStream_t st) {
    if (block) A.put(block, block_bytes, st);
    block = nullptr;
  }
};

// A pass recorded as a CUDA graph: its tables are read from, and its status
// written to, pinned buffers owned here, so that a launch of the graph
// builds from whatever the host put there.
struct GraphPass {
  cudaGraphExec_t exec = nullptr;
  uint8_t* up = nullptr;
  uint8_t* down = nullptr;
  uint32_t kernels = 0;  // kernel nodes of the graph
};

fks_status SetBuild::init(const BuildIn& in_, const Opts& o_, const Alloc& A_, cudaStream_t st) {
  in = in_;
  o = o_;
  A = A_;
  m = in.m;
  str = in.kind == FKS_KEY_BYTES;
  PW = str ? 2 : 1;
  W = str ? 4 : 2;  // words per slot
  total = uint64_t(in.seg[m]);
  logB = part_log_buckets(o.lambda);
  B = 1ull << logB;
  sms = sm_count();
  bs = build_shape_for(int(in.kind), o.lambda);
  uint64_t slot_total = 0, desc_total = 0;
  std::vector<uint64_t> slot_base(m), desc_base(m);
  nbs.assign(m, 0);
  for (uint32_t j = 0; j < m; ++j) {
    const uint64_t n = uint64_t(in.seg[j + 1] - in.seg[j]);
    if (!sizes_fit(o, n)) return fail(FKS_ERR_INVALID_ARG, "bound_factor * n does not fit 32-bit slot offsets");
    slot_base[j] = slot_total;
    slot_total += uint64_t(o.bound) * n;
    nbs[j] = level1_buckets(n, o.lambda);
    desc_base[j] = desc_total;
    desc_total += nbs[j];
  }
  // context bytes: offs[total] from the device
  if (str) {
    int64_t last = 0;
    FKS_CUDA(cudaMemcpyAsync(&last, in.offs + total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FKS_CUDA(cudaStreamSynchronize(st));
    if (last < 0 || last >= (int64_t(1) << 40)) return fail(FKS_ERR_INVALID_ARG, "offsets out of range");
    ctx_bytes = uint64_t(last);
  }
  // the set's own memory: descriptors, slots, context copy
  Carve cm;
  const size_t o_desc = cm.take<uint64_t>(desc_total);
  const size_t o_slots = cm.take<uint64_t>(slot_total * W);
  const size_t o_ctx = cm.take<uint8_t>(str ? ctx_bytes + 16 : 0);
  const bool with_rec = o.inline1 && !str && m == 1;
  const size_t o_rec = cm.take<uint64_t>(with_rec ? 2 * desc_total : 0);
  block = static_cast<uint8_t*>(A.get(cm.off, st));
  if (!block) return fail(FKS_ERR_OUT_OF_MEMORY, "allocation of map tables failed");
  block_bytes = cm.off;
  mem.desc = reinterpret_cast<uint64_t*>(block + o_desc);
  mem.slots = reinterpret_cast<uint64_t*>(block + o_slots);
  mem.ctx = str ? block + o_ctx : nullptr;
  mem.rec = with_rec ? reinterpret_cast<uint64_t*>(block + o_rec) : nullptr;
  mem.slot_base = slot_base;
  mem.desc_base = desc_base;
  // scratch for the largest pass (the first one holds every map)
  uint64_t P_all = 0;
  for (uint32_t j = 0; j < m; ++j) P_all += (nbs[j] + B - 1) / B;
  Carve cs;
  const size_t s_cnt = cs.take<uint32_t>(P_all + 1);
  const size_t s_start = cs.take<uint32_t>(P_all + 1);
  const size_t s_cursor = cs.take<uint32_t>(P_all + 1);
  const size_t s_lb = cs.take<uint64_t>(P_all + 1);
  const size_t s_ticket = cs.take<uint32_t>(4);
  const size_t s_ovl = cs.take<uint32_t>(P_all + 1);
  const size_t s_ove = cs.take<uint64_t>(P_all + 1);
  const size_t s_skey = cs.take<uint64_t>(total + 2);  // +2: 16-byte rounded bulk copies
  const size_t s_spay = cs.take<uint64_t>((total + 2) * PW);
  const size_t s_maps = cs.take<MapDev>(m);
  const size_t s_pseg = cs.take<uint64_t>(m + 1);
  const size_t s_qseg = cs.take<uint32_t>(m + 1);
  const size_t s_stat = cs.take<MapStatus>(m);
  const size_t s_fps = cs.take<uint64_t>(str ? total + 1 : 0);
  // two-level grouping for large builds
  shape = split_shape(uint32_t(P_all), total);
  use_split = total >= (1ull << bs.split_min_log2) && shape.ok;
  if (use_split) {
    hist_words = split_hist_words(shape);
    s_ka = cs.take<uint64_t>(total);
    s_pa = cs.take<uint64_t>(total * PW);
    s_ga = cs.take<uint32_t>(total);
    s_hist = cs.take<uint32_t>(hist_words);
    s_sums = cs.take<uint32_t>(split_sum_words(shape));
    s_sa = cs.take<uint64_t>(shape.binsA + 1);
    s_tb = cs.take<uint32_t>(shape.binsA + 1);
  }
  scr = static_cast<uint8_t*>(A.get(cs.off, st));
  if (!scr) {
    free_tables(st);
    return fail(FKS_ERR_OUT_OF_MEMORY, "allocation of build scratch failed");
  }
  scr_bytes = cs.off;
  p = PassDev{};
  p.part_cnt = reinterpret_cast<uint32_t*>(scr + s_cnt);
  p.part_start = reinterpret_cast<uint32_t*>(scr + s_start);
  p.part_cursor = reinterpret_cast<uint32_t*>(scr + s_cursor);
  p.lookback = reinterpret_cast<uint64_t*>(scr + s_lb);
  p.ticket = reinterpret_cast<uint32_t*>(scr + s_ticket);
  p.ovf_count = p.ticket + 1;
  p.ovf_list = reinterpret_cast<uint32_t*>(scr + s_ovl);
  p.ovf_excl = reinterpret_cast<uint64_t*>(scr + s_ove);
  p.stage_key = reinterpret_cast<uint64_t*>(scr + s_skey);
  p.stage_pay = reinterpret_cast<uint64_t*>(scr + s_spay);
  d_maps = reinterpret_cast<MapDev*>(scr + s_maps);
  d_pseg = reinterpret_cast<uint64_t*>(scr + s_pseg);
  d_qseg = reinterpret_cast<uint32_t*>(scr + s_qseg);
  d_stat = reinterpret_cast<MapStatus*>(scr + s_stat);
  fps = str ? reinterpret_cast<uint64_t*>(scr + s_fps) : nullptr;
  p.maps = d_maps;
  p.status = d_stat;
  p.pass_seg = d_pseg;
  p.part_seg = d_qseg;
  p.hkeys = str ? fps : in.keys;
  p.vals = in.vals;
  p.vals_i64 = in.vt == FKS_VAL_I64;
  p.offs = in.offs;
  p.ctx = mem.ctx;
  p.desc = mem.desc;
  p.slots = mem.slots;
  p.rec = mem.rec;
  p.logB = logB;
  p.cfg.attempt_cap = o.attempt_cap;
  p.cfg.reject = o.reject;
  p.cfg.spin_limit = o.spin;
  p.cfg.hold_first = uint32_t(g_hold_first_partition);
  p.cfg.thread_max = bs.thread_max;
  p.cfg.prefetch = bs.prefetch;
  return FKS_OK;
}

// Pass tables of the `active` maps at their current rounds into `up`; sets
// the pass geometry (p.m, p.P, p.total).
uint32_t SetBuild::fill_tables(const std::vector<uint32_t>& active, uint8_t* up) {
  const uint32_t ma = uint32_t(active.size());
  MapDev* h_maps = reinterpret_cast<MapDev*>(up);
  uint64_t* h_pseg = reinterpret_cast<uint64_t*>(up + sizeof(MapDev) * ma);
  uint32_t* h_qseg = reinterpret_cast<uint32_t*>(up + sizeof(MapDev) * ma + sizeof(uint64_t) * (ma + 1));
  uint64_t pe = 0;
  uint32_t pp = 0;
  for (uint32_t a = 0; a < ma; ++a) {
    const uint32_t j = active[a];
    const uint64_t n = uint64_t(in.seg[j + 1] - in.seg[j]);
    MapDev& M = h_maps[a];
    M.key_begin = uint64_t(in.seg[j]);
    M.pass_begin = pe;
    M.desc_base = mem.desc_base[j];
    M.slot_base = mem.slot_base[j];
    M.seed = in.seeds[j];
    M.round = round[j];
    M.c1 = derive(M.seed, M.round, kTagLevel1, 0);
    M.fpb = fp_base(M.seed, M.round);
    M.n = uint32_t(n);
    M.nb = uint32_t(nbs[j]);
    M.slot_cap = uint32_t(uint64_t(o.bound) * n);
    M.part_begin = pp;
    if (mem.rec) {  // this round's key for the descriptor record of bucket g(0)
      p.rec_g0 = reduce32(hash32(M.c1, 0), M.nb);
      uint64_t x = 1;
      while (M.nb > 1 && x < (1u << 16) && reduce32(hash32(M.c1, x), M.nb) == p.rec_g0) ++x;
      p.rec_x1 = x;
    }
    h_pseg[a] = pe;
    h_qseg[a] = pp;
    pe += n;
    pp += uint32_t((nbs[j] + B - 1) / B);
  }
  h_pseg[ma] = pe;
  h_qseg[ma] = pp;
  p.m = ma;
  p.P = pp;
  p.total = pe;
  return ma;
}

cudaError_t SetBuild::enqueue_pass(uint32_t ma, const uint8_t* up, uint8_t* down, bool copy_ctx,
                                   ProfileEvents* prof, cudaStream_t st) {
  cudaError_t e;
#define FKS_STEP(call) \
  if ((e = (call)) != cudaSuccess) return e;
  if (copy_ctx && str && ctx_bytes)
    FKS_STEP(cudaMemcpyAsync(mem.ctx, in.ctx, ctx_bytes, cudaMemcpyDeviceToDevice, st));
  FKS_STEP(cudaMemcpyAsync(d_maps, up, sizeof(MapDev) * ma, cudaMemcpyHostToDevice, st));
  FKS_STEP(cudaMemcpyAsync(d_pseg, up + sizeof(MapDev) * ma, sizeof(uint64_t) * (ma + 1), cudaMemcpyHostToDevice, st));
  FKS_STEP(cudaMemcpyAsync(d_qseg, up + sizeof(MapDev) * ma + sizeof(uint64_t) * (ma + 1),
                           sizeof(uint32_t) * (ma + 1), cudaMemcpyHostToDevice, st));
  FKS_STEP(cudaMemsetAsync(d_stat, 0, sizeof(MapStatus) * ma, st));
  if (prof && str) cudaEventRecord(prof->fp0, st);
  if (str) FKS_STEP(launch_fingerprints(in.ctx, in.offs, total, d_maps, d_pseg, ma, p.total, fps, d_stat, st));
  if (prof && str) cudaEventRecord(prof->fp1, st);
  const SplitShape sh = split_shape(p.P, p.total);
  const bool split_pass = use_split && sh.ok && split_hist_words(sh) <= hist_words && sh.binsA <= shape.binsA &&
                          p.total >= (1ull << bs.split_min_log2);
  if (split_pass) {
    SplitDev sd{};
    sd.binsA = sh.binsA;
    sd.binsB = sh.binsB;
    sd.shiftB = sh.shiftB;
    sd.tilesA = sh.tilesA;
    sd.tilesB_max = sh.tilesB_max;
    sd.histA = sd.histB = reinterpret_cast<uint32_t*>(scr + s_hist);
    sd.sums = reinterpret_cast<uint32_t*>(scr + s_sums);
    sd.startA = reinterpret_cast<uint64_t*>(scr + s_sa);
    sd.tstartB = reinterpret_cast<uint32_t*>(scr + s_tb);
    sd.keyA = reinterpret_cast<uint64_t*>(scr + s_ka);
    sd.payA = reinterpret_cast<uint64_t*>(scr + s_pa);
    sd.gpA = reinterpret_cast<uint32_t*>(scr + s_ga);
    levels = 2;
    FKS_STEP(launch_pass_split(p, sd, str, sms, bs, st, prof ? &prof->pe : nullptr));
  } else {
    levels = 1;
    FKS_STEP(launch_pass(p, str, sms, bs, st, prof ? &prof->pe : nullptr));
  }
  MapStatus* h_stat = reinterpret_cast<MapStatus*>(down);
  uint32_t* h_ovf = reinterpret_cast<uint32_t*>(down + sizeof(MapStatus) * ma);
  FKS_STEP(cudaMemcpyAsync(h_stat, d_stat, sizeof(MapStatus) * ma, cudaMemcpyDeviceToHost, st));
  FKS_STEP(cudaMemcpyAsync(h_ovf, p.ovf_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
#undef FKS_STEP
  return cudaSuccess;
}

fks_status SetBuild::run(cudaStream_t st, GraphPass* g) {
  round.assign(m, 0);
  std::vector<uint32_t> active(m);
  for (uint32_t j = 0; j < m; ++j) active[j] = j;
  per_map.assign(m, FKS_OK);
  maps.assign(m, fks_map());
  profile = fks_build_profile{};
  std::vector<uint32_t> exhausted;  // maps whose rounds all failed
  fks_status hard = FKS_OK;         // a failure of the whole call
  std::string hard_msg;
  ProfileEvents prof;
  bool first = true;

  while (!active.empty() && hard == FKS_OK) {
    const uint32_t ma = uint32_t(active.size());
    NvtxRange pass_range(first ? "level-one pass" : "level-one pass (redraw)");
    // the first pass of a recorded build is a launch of its graph
    const bool replay = first && g != nullptr;
    uint8_t* up = replay ? g->up : static_cast<uint8_t*>(g_pin_up.get(up_bytes(ma)));
    uint8_t* down = replay ? g->down : static_cast<uint8_t*>(g_pin_down.get(down_bytes(ma)));
    if (!up || !down) {
      hard = FKS_ERR_CUDA;
      hard_msg = "pinned staging";
      break;
    }
    fill_tables(active, up);
    cudaError_t e;
#define FKS_PASS(call)                                          \
  if ((e = (call)) != cudaSuccess) {                            \
    hard = FKS_ERR_CUDA;                                        \
    hard_msg = std::string(#call ": ") + cudaGetErrorString(e); \
    break;                                                      \
  }
    if (replay) {
      FKS_PASS(cudaGraphLaunch(g->exec, st));
      note_launches(g->kernels);
    } else {
      FKS_PASS(enqueue_pass(ma, up, down, first, prof.ok ? &prof : nullptr, st));
    }
    FKS_PASS(cudaStreamSynchronize(st));
    if (!replay) {
      profile.grouping_levels = levels;
      prof.accumulate(&profile, str);
    }
    first = false;
    MapStatus* h_stat = reinterpret_cast<MapStatus*>(down);
    const uint32_t h_ovf = *reinterpret_cast<uint32_t*>(down + sizeof(MapStatus) * ma);
    if (h_ovf) {
      if (!ovf_key) {
        ovf_bytes = sizeof(uint64_t) * (total * (1 + PW) + 2);
        ovf_key = static_cast<uint64_t*>(A.get(ovf_bytes, st));
        if (!ovf_key) {
          hard = FKS_ERR_OUT_OF_MEMORY;
          hard_msg = "overflow buffer";
          break;
        }
      }
      p.ovf_key = ovf_key;
      p.ovf_pay = ovf_key + total;
      FKS_PASS(launch_overflow(p, str, h_ovf, st));
      FKS_PASS(cudaMemcpyAsync(h_stat, d_stat, sizeof(MapStatus) * ma, cudaMemcpyDeviceToHost, st));
      FKS_PASS(cudaStreamSynchronize(st));
    }
#undef FKS_PASS
    // ---- decide per map
    const MapDev* h_maps = reinterpret_cast<const MapDev*>(up);
    std::vector<uint32_t> next;
    for (uint32_t a = 0; a < ma; ++a) {
      const uint32_t j = active[a];
      const MapStatus& S = h_stat[a];
      if (S.invalid) {
        per_map[j] = FKS_ERR_INVALID_ARG;
        continue;
      }
      if (S.timeout) {
        per_map[j] = FKS_ERR_TIMEOUT;
        continue;
      }
      bool redo = false;
      if (S.reseed) redo = true;
      else if (S.dup) {
        per_map[j] = FKS_ERR_DUPLICATE_KEY;
        continue;
      } else if (S.next_round) redo = true;
      if (redo) {
        if (round[j] + 1 >= o.round_cap) exhausted.push_back(j);
        else {
          round[j] += 1;
          next.push_back(j);
        }
        continue;
      }
      fks_map& M = maps[j];
      M.kind = in.kind;
      M.vt = in.vt;
      M.n = uint64_t(in.seg[j + 1] - in.seg[j]);
      M.seed = in.seeds[j];
      M.round = round[j];
      M.c1 = h_maps[a].c1;
      M.fpb = h_maps[a].fpb;
      M.S = S.S;
      M.slot_cap = uint64_t(o.bound) * M.n;
      M.att_sum = S.att_sum;
      M.max_s = S.max_s;
      M.max_att = S.max_att;
      M.overflow = S.overflow;
      M.nonempty = S.nonempty;
      M.nb = nbs[j];
      M.lambda = o.lambda;
      M.desc = mem.desc + mem.desc_base[j];
      M.slots = mem.slots + mem.slot_base[j] * W;
      M.rec = mem.rec;
      M.ctx = mem.ctx;
      M.ctx_bytes = ctx_bytes;
      M.bytes = sizeof(uint64_t) * (M.nb * (mem.rec ? 3 : 1) + W * M.slot_cap);
    }
    active.swap(next);
  }
  // ---- maps whose every round failed: exact duplicate test
  for (uint32_t j : exhausted) {
    if (hard != FKS_OK) break;
    const uint64_t n = uint64_t(in.seg[j + 1] - in.seg[j]);
    uint64_t size = 1;
    while (size < 2 * n) size <<= 1;
    const size_t tb = sizeof(uint64_t) * size + (str ? sizeof(uint32_t) * size : 0) + 64;
    uint8_t* tbl = static_cast<uint8_t*>(A.get(tb, st));
    if (!tbl) {
      hard = FKS_ERR_OUT_OF_MEMORY;
      hard_msg = "duplicate test table";
      break;
    }
    uint64_t* table = reinterpret_cast<uint64_t*>(tbl);
    uint32_t* tidx = str ? reinterpret_cast<uint32_t*>(tbl + sizeof(uint64_t) * size) : nullptr;
    uint32_t* flags = reinterpret_cast<uint32_t*>(tbl + tb - 64);
    const uint64_t* hk = str ? fps + in.seg[j] : in.keys + in.seg[j];
    cudaError_t e = launch_dupcheck(hk, str ? in.offs + in.seg[j] : nullptr, in.ctx, n, table, tidx, size, flags,
                                    o.spin, st);
    uint32_t hf[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    A.put(tbl, tb, st);
    if (e != cudaSuccess) {
      hard = FKS_ERR_CUDA;
      hard_msg = std::string("duplicate test: ") + cudaGetErrorString(e);
      break;
    }
    per_map[j] = hf[2] ? FKS_ERR_TIMEOUT : (hf[0] ? FKS_ERR_DUPLICATE_KEY : FKS_ERR_BUILD_FAILED);
  }
  if (prof.ok) g_last_profile = profile;
  if (hard != FKS_OK) return fail(hard, hard_msg);
  return FKS_OK;
}

// One-shot build of a set: init, the rounds, scratch released; the tables
// are handed to the caller.
static fks_status build_impl(const BuildIn& in, const Opts& o, const Alloc& A, cudaStream_t st,
                             void** out_block, size_t* out_block_bytes, SetMem* mem,
                             std::vector<fks_map>* maps_out, std::vector<fks_status>* per_map) {
  SetBuild b;
  fks_status s = b.init(in, o, A, st);
  if (s != FKS_OK) return s;
  s = b.run(st, nullptr);
  b.free_scratch(st);
  if (s != FKS_OK) {
    b.free_tables(st);
    return s;
  }
  *out_block = b.block;
  *out_block_bytes = b.block_bytes;
  *mem = b.mem;
  *maps_out = std::move(b.maps);
  *per_map = std::move(b.per_map);
  return FKS_OK;
}

static const char* status_name(fks_status s) {
  switch (s) {
    case FKS_OK: return "ok";
    case FKS_ERR_INVALID_ARG: return "invalid argument";
    case FKS_ERR_DUPLICATE_KEY: return "duplicate key";
    case FKS_ERR_OUT_OF_MEMORY: return "out of memory";
    case FKS_ERR_BUILD_FAILED: return "build failed";
    case FKS_ERR_TIMEOUT: return "device wait timed out";
    case FKS_ERR_CUDA: return "CUDA error";
    case FKS_ERR_EVICTED: return "map evicted";
  }
  return "unknown status";
}

// ---------------------------------------------------------------- from_array
// The deduplicated inputs of a build (kept pairs in input order) and the
// block that holds them until the build has read them.
struct DedupOut {
  uint8_t* block = nullptr;
  size_t bytes = 0;
  BuildIn in{};
  std::vector<int64_t> seg;
};

static fks_status dedup_inputs(const BuildIn& in, const Alloc& A, cudaStream_t st, DedupOut* out) {
  NvtxRange range("from_array: deduplication");
  const bool str = in.kind == FKS_KEY_BYTES;
  const uint32_t m = in.m;
  const uint64_t u = uint64_t(in.seg[m]);
  const int sms = sm_count();
  uint64_t ctx_bytes = 0;
  if (str) {
    int64_t last = 0;
    FKS_CUDA(cudaMemcpyAsync(&last, in.offs + u, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FKS_CUDA(cudaStreamSynchronize(st));
    if (last < 0 || last >= (int64_t(1) << 40)) return fail(FKS_ERR_INVALID_ARG, "offsets out of range");
    ctx_bytes = uint64_t(last);
  }
  const size_t tw = dedup_table_words(u);
  Carve c;
  const size_t o_tab = c.take<uint64_t>(tw);
  const size_t o_pos = c.take<uint32_t>(u + 1);
  const size_t o_sum = c.take<uint64_t>(scan_sum_words(u + 1));
  const size_t o_flag = c.take<uint32_t>(4);
  const size_t o_seg = c.take<int64_t>(m > 1 ? m + 1 : 0);
  const size_t o_oseg = c.take<int64_t>(m + 1);
  const size_t o_keys = c.take<uint64_t>(str ? 0 : u);
  const size_t o_vals = c.take<int64_t>(u);
  const size_t o_offs = c.take<int64_t>(str ? u + 1 : 0);
  const size_t o_lens = c.take<uint64_t>(str ? u + 1 : 0);
  const size_t o_ctx = c.take<uint8_t>(str ? ctx_bytes + 16 : 0);
  uint8_t* b = static_cast<uint8_t*>(A.get(c.off, st));
  if (!b) return fail(FKS_ERR_OUT_OF_MEMORY, "allocation of the deduplication buffers failed");
  out->block = b;
  out->bytes = c.off;
  uint32_t* pos = reinterpret_cast<uint32_t*>(b + o_pos);
  uint32_t* flags = reinterpret_cast<uint32_t*>(b + o_flag);
  int64_t* d_seg = m > 1 ? reinterpret_cast<int64_t*>(b + o_seg) : nullptr;
  int64_t* oseg = reinterpret_cast<int64_t*>(b + o_oseg);
  if (d_seg) FKS_CUDA(cudaMemcpyAsync(d_seg, in.seg, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, st));
  FKS_CUDA(launch_dedup_mark(str ? nullptr : in.keys, in.ctx, in.offs, d_seg, m, u,
                             reinterpret_cast<uint64_t*>(b + o_tab), tw, pos, flags, sms, st));
  FKS_CUDA(scan_exclusive<uint32_t>(pos, u + 1, reinterpret_cast<uint32_t*>(b + o_sum), st));
  uint32_t h[3] = {0, 0, 0};
  FKS_CUDA(cudaMemcpyAsync(h, flags, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, st));
  FKS_CUDA(cudaMemcpyAsync(h + 2, pos + u, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  FKS_CUDA(cudaStreamSynchronize(st));
  if (h[0]) return fail(FKS_ERR_INVALID_ARG, "bad string offsets");
  if (h[1]) return fail(FKS_ERR_CUDA, "deduplication table probe limit reached");
  const int i64 = in.vt == FKS_VAL_I64;
  void* ovals = b + o_vals;
  BuildIn r = in;
  r.vals = ovals;
  if (!str) {
    uint64_t* okeys = reinterpret_cast<uint64_t*>(b + o_keys);
    FKS_CUDA(launch_dedup_pack_u64(in.keys, in.vals, i64, u, pos, okeys, ovals, sms, st));
    r.keys = okeys;
  } else {
    uint64_t* lens = reinterpret_cast<uint64_t*>(b + o_lens);
    int64_t* ooffs = reinterpret_cast<int64_t*>(b + o_offs);
    uint8_t* octx = b + o_ctx;
    FKS_CUDA(launch_dedup_lengths(in.offs, u, pos, lens, sms, st));
    FKS_CUDA(scan_exclusive<uint64_t>(lens, u + 1, reinterpret_cast<uint64_t*>(b + o_sum), st));
    FKS_CUDA(launch_dedup_pack_bytes(in.ctx, in.offs, in.vals, i64, u, pos, lens, octx, ooffs, ovals, sms, st));
    r.ctx = octx;
    r.offs = ooffs;
  }
  out->seg.assign(m + 1, 0);
  if (m > 1) {
    FKS_CUDA(launch_dedup_segs(pos, d_seg, m, oseg, st));
    FKS_CUDA(cudaMemcpyAsync(out->seg.data(), oseg, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost, st));
    FKS_CUDA(cudaStreamSynchronize(st));
  } else {
    out->seg[1] = int64_t(h[2]);
  }
  r.seg = out->seg.data();
  out->in = r;
  return FKS_OK;
}

static fks_status build_single(const BuildIn& in, const fks_build_opts* opts,
                               const fks_allocator* alloc, cudaStream_t st, fks_map_t* out) {
  NvtxRange range("fks_build");
  Opts o;
  if (!read_opts(opts, &o)) return fail(FKS_ERR_INVALID_ARG, "bad build options");
  if (o.inline1 && in.kind != FKS_KEY_U64)
    return fail(FKS_ERR_INVALID_ARG, "inline_singletons: uint64 keys only");
  Alloc A(alloc);
  void* block = nullptr;
  size_t bb = 0;
  SetMem mem;
  std::vector<fks_map> maps;
  std::vector<fks_status> per;
  sm_count();
  DedupOut dd;
  if (o.dedup) {
    const fks_status ds = dedup_inputs(in, A, st, &dd);
    if (ds != FKS_OK) {
      if (dd.block) A.put(dd.block, dd.bytes, st);
      return ds;
    }
  }
  fks_status s = build_impl(o.dedup ? dd.in : in, o, A, st, &block, &bb, &mem, &maps, &per);
  if (dd.block) A.put(dd.block, dd.bytes, st);
  if (s != FKS_OK) return s;
  if (per[0] != FKS_OK) {
    A.put(block, bb, st);
    return fail(per[0], std::string("build: ") + status_name(per[0]));
  }
  fks_map* m = new fks_map(maps[0]);
  m->block = block;
  m->block_bytes = bb;
  m->alloc = A;
  m->bytes = bb;
  *out = m;
  return FKS_OK;
}

// The device table of a set for batched lookups (set->d_table, already
// allocated): maps that failed keep n = 0 and answer every needle with
// absent, their first descriptor made an empty bucket.  Synchronises.
static fks_status publish_set(fks_mapset* set, const SetMem& mem, const std::vector<fks_status>& per,
                              cudaStream_t st) {
  const uint32_t m = uint32_t(set->maps.size());
  std::vector<LookupMap> tab(m);
  for (uint32_t j = 0; j < m; ++j) {
    if (per[j] == FKS_OK) tab[j] = lookup_view(set->maps[j]);
    else {
      memset(&tab[j], 0, sizeof(LookupMap));
      tab[j].desc = mem.desc + mem.desc_base[j];
      tab[j].nb = 1;  // a single empty bucket
    }
  }
  for (uint32_t j = 0; j < m; ++j)
    if (per[j] != FKS_OK) FKS_CUDA(cudaMemsetAsync(mem.desc + mem.desc_base[j], 0, sizeof(uint64_t), st));
  FKS_CUDA(cudaMemcpyAsync(set->d_table, tab.data(), sizeof(LookupMap) * m, cudaMemcpyHostToDevice, st));
  FKS_CUDA(cudaStreamSynchronize(st));
  return FKS_OK;
}

// Lookup view of a map handle, for the serving loop (fks_serve.cu).
namespace fks {
bool lookup_view_of(fks_map_t m, LookupMap* out, int* strings, int* out_i64) {
  if (!m || settle(m) != FKS_OK || !m->desc) return false;
  *out = lookup_view(*m);
  *strings = m->kind == FKS_KEY_BYTES;
  *out_i64 = m->vt == FKS_VAL_I64;
  return true;
}
int device_sm_count() { return sm_count(); }
}  // namespace fks

// Arguments of a batched build; the segment offsets (host or device memory)
// are copied to *seg.
static fks_status check_batched(const char* who, fks_key_kind kind, const uint64_t* keys, const uint8_t* ctx,
                                const int64_t* offs, const int64_t* h_seg, uint32_t m, const void* vals,
                                fks_val_type val_type, std::vector<int64_t>* seg) {
  const std::string w(who);
  if (m == 0 || !h_seg || !vals || (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return fail(FKS_ERR_INVALID_ARG, w + ": bad arguments");
  seg->resize(size_t(m) + 1);
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, h_seg) == cudaSuccess &&
      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged)) {
    FKS_CUDA(cudaMemcpy(seg->data(), h_seg, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost));
  } else {
    memcpy(seg->data(), h_seg, sizeof(int64_t) * (m + 1));
  }
  cudaGetLastError();
  const int64_t* s = seg->data();
  if (kind == FKS_KEY_U64 ? !keys : (kind == FKS_KEY_BYTES ? (!ctx || !offs) : true))
    return fail(FKS_ERR_INVALID_ARG, w + ": bad key arguments");
  if (s[0] != 0) return fail(FKS_ERR_INVALID_ARG, w + ": h_seg[0] != 0");
  for (uint32_t j = 0; j < m; ++j) {
    const int64_t n = s[j + 1] - s[j];
    if (n <= 0 || n >= (int64_t(1) << 30)) return fail(FKS_ERR_INVALID_ARG, w + ": empty or oversized segment");
  }
  if (uint64_t(s[m]) >= (1ull << 32)) return fail(FKS_ERR_INVALID_ARG, w + ": 2^32 keys or more");
  return FKS_OK;
}

// ---------------------------------------------------------------- recorded builds
// A batched build whose first pass -- every map at level-one round 0 -- is
// recorded once as a CUDA graph over fixed input buffers and replayed by each
// run; maps that must redraw finish through the ordinary pass loop.
struct fks_build_graph {
  std::mutex mu;
  SetBuild b;
  GraphPass gp;
  cudaGraph_t graph = nullptr;
  std::vector<int64_t> seg;     // the graph's own copy of the segment offsets
  std::vector<uint64_t> seeds;  // seeds of the current run
  fks_mapset set;               // the maps of the last run; tables in b.block
};

static void graph_release(fks_build_graph* g) {
  if (g->gp.exec) cudaGraphExecDestroy(g->gp.exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->gp.up) cudaFreeHost(g->gp.up);
  if (g->gp.down) cudaFreeHost(g->gp.down);
  g->b.free_scratch(nullptr);
  g->b.free_tables(nullptr);
  if (g->set.d_table) g->b.A.put(g->set.d_table, sizeof(LookupMap) * g->b.m, nullptr);
  cudaDeviceSynchronize();
  delete g;
}

// Kernel nodes of a graph (what one launch of it runs).
static uint32_t graph_kernels(cudaGraph_t graph) {
  size_t count = 0;
  if (cudaGraphGetNodes(graph, nullptr, &count) != cudaSuccess || count == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(count);
  if (cudaGraphGetNodes(graph, nodes.data(), &count) != cudaSuccess) return 0;
  uint32_t k = 0;
  for (size_t i = 0; i < count; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// ================================================================ C ABI
extern "C" {

fks_status fks_build_u64(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                         uint64_t seed, const fks_build_opts* opts, const fks_allocator* alloc,
                         fks_stream_t stream, fks_map_t* out) {
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!keys || !vals || n == 0 || n >= (1ull << 30) ||
      (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return fail(FKS_ERR_INVALID_ARG, "fks_build_u64: bad keys, vals, n or val_type");
  const int64_t seg[2] = {0, int64_t(n)};
  BuildIn in{FKS_KEY_U64, keys, nullptr, nullptr, vals, val_type, 1, seg, &seed};
  return build_single(in, opts, alloc, reinterpret_cast<cudaStream_t>(stream), out);
}

fks_status fks_build_bytes(const uint8_t* ctx, const int64_t* offs, const void* vals,
                           fks_val_type val_type, uint64_t n, uint64_t seed,
                           const fks_build_opts* opts, const fks_allocator* alloc,
                           fks_stream_t stream, fks_map_t* out) {
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ctx || !offs || !vals || n == 0 || n >= (1ull << 30) ||
      (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return fail(FKS_ERR_INVALID_ARG, "fks_build_bytes: bad ctx, offs, vals, n or val_type");
  const int64_t seg[2] = {0, int64_t(n)};
  BuildIn in{FKS_KEY_BYTES, nullptr, ctx, offs, vals, val_type, 1, seg, &seed};
  return build_single(in, opts, alloc, reinterpret_cast<cudaStream_t>(stream), out);
}

// Start a build on a host thread of its own; the handle is returned at once.
static fks_status build_async(BuildIn in, const fks_build_opts* opts, const fks_allocator* alloc,
                              fks_stream_t stream, fks_map_t* out) {
  fks_map* shell = new fks_map();
  shell->kind = in.kind;
  shell->vt = in.vt;
  AsyncBuild* a = new AsyncBuild();
  shell->async = a;
  a->seg[1] = in.seg[1];
  a->seed = in.seeds[0];
  if (opts) {
    const size_t nb = opts->struct_size < sizeof(fks_build_opts) ? opts->struct_size : sizeof(fks_build_opts);
    memcpy(&a->opts, opts, nb);
    a->has_opts = true;
  }
  if (alloc) {
    a->alloc = *alloc;
    a->has_alloc = true;
  }
  in.seg = a->seg;
  in.seeds = &a->seed;
  int device = 0;
  cudaGetDevice(&device);  // the current device is per host thread
  try {
    a->worker = std::thread([shell, a, in, stream, device]() {
      cudaSetDevice(device);
      fks_map_t built = nullptr;
      const fks_status st = build_single(in, a->has_opts ? &a->opts : nullptr, a->has_alloc ? &a->alloc : nullptr,
                                         reinterpret_cast<cudaStream_t>(stream), &built);
      a->status = st;
      if (st != FKS_OK) {
        a->msg = g_last_error;  // this worker thread's message
        return;
      }
      *shell = *built;  // the built tables now belong to the shell
      shell->async = a;
      delete built;
    });
  } catch (...) {
    delete a;
    delete shell;
    return fail(FKS_ERR_OUT_OF_MEMORY, "could not start the build thread");
  }
  *out = shell;
  return FKS_OK;
}

fks_status fks_build_u64_async(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                               uint64_t seed, const fks_build_opts* opts, const fks_allocator* alloc,
                               fks_stream_t stream, fks_map_t* out) {
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!keys || !vals || n == 0 || n >= (1ull << 30) ||
      (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return fail(FKS_ERR_INVALID_ARG, "fks_build_u64_async: bad keys, vals, n or val_type");
  const int64_t seg[2] = {0, int64_t(n)};
  BuildIn in{FKS_KEY_U64, keys, nullptr, nullptr, vals, val_type, 1, seg, &seed};
  return build_async(in, opts, alloc, stream, out);
}

fks_status fks_build_bytes_async(const uint8_t* ctx, const int64_t* offs, const void* vals,
                                 fks_val_type val_type, uint64_t n, uint64_t seed,
                                 const fks_build_opts* opts, const fks_allocator* alloc,
                                 fks_stream_t stream, fks_map_t* out) {
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ctx || !offs || !vals || n == 0 || n >= (1ull << 30) ||
      (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return fail(FKS_ERR_INVALID_ARG, "fks_build_bytes_async: bad ctx, offs, vals, n or val_type");
  const int64_t seg[2] = {0, int64_t(n)};
  BuildIn in{FKS_KEY_BYTES, nullptr, ctx, offs, vals, val_type, 1, seg, &seed};
  return build_async(in, opts, alloc, stream, out);
}

static bool absent_fits(const fks_map* m, int64_t absent) {
  return m->vt == FKS_VAL_I64 || (absent >= INT32_MIN && absent <= INT32_MAX);
}

fks_status fks_lookup_u64(fks_map_t map, const uint64_t* q, uint64_t nq, void* out_vals,
                          uint8_t* out_found, int64_t absent, fks_stream_t stream) {
  NvtxRange range("fks_lookup_u64");
  if (!map) return fail(FKS_ERR_INVALID_ARG, "fks_lookup_u64: NULL map");
  if (const fks_status bs = settle(map)) return bs;
  if (map->kind != FKS_KEY_U64) return fail(FKS_ERR_INVALID_ARG, "fks_lookup_u64: not a u64 map");
  if (nq == 0) return FKS_OK;
  if (!q || !absent_fits(map, absent)) return fail(FKS_ERR_INVALID_ARG, "fks_lookup_u64: bad arguments");
  if (map->rec) {
    FKS_CUDA(launch_lookup_inline(lookup_view(*map), map->rec, q, nq, out_vals, map->vt == FKS_VAL_I64, out_found,
                                  absent, sm_count(), reinterpret_cast<cudaStream_t>(stream)));
    return FKS_OK;
  }
  FKS_CUDA(launch_lookup_u64(lookup_view(*map), q, nq, out_vals, map->vt == FKS_VAL_I64, out_found,
                             absent, sm_count(), lookup_shape_for(map->lambda), reinterpret_cast<cudaStream_t>(stream)));
  return FKS_OK;
}

fks_status fks_lookup_bytes(fks_map_t map, const uint8_t* qctx, const int64_t* qoffs, uint64_t nq,
                            void* out_vals, uint8_t* out_found, int64_t absent,
                            fks_stream_t stream) {
  NvtxRange range("fks_lookup_bytes");
  if (!map) return fail(FKS_ERR_INVALID_ARG, "fks_lookup_bytes: NULL map");
  if (const fks_status bs = settle(map)) return bs;
  if (map->kind != FKS_KEY_BYTES) return fail(FKS_ERR_INVALID_ARG, "fks_lookup_bytes: not a string map");
  if (nq == 0) return FKS_OK;
  if (!qctx || !qoffs || !absent_fits(map, absent))
    return fail(FKS_ERR_INVALID_ARG, "fks_lookup_bytes: bad arguments");
  FKS_CUDA(launch_lookup_bytes(lookup_view(*map), qctx, qoffs, nq, out_vals, map->vt == FKS_VAL_I64,
                               out_found, absent, sm_count(), reinterpret_cast<cudaStream_t>(stream)));
  return FKS_OK;
}

fks_status fks_build_batched(fks_key_kind kind, const uint64_t* keys, const uint8_t* ctx,
                             const int64_t* offs, const int64_t* h_seg, const uint64_t* h_seeds,
                             uint32_t m, const void* vals, fks_val_type val_type,
                             const fks_build_opts* opts, const fks_allocator* alloc,
                             fks_stream_t stream, fks_mapset_t* out, fks_status* h_status) {
  NvtxRange range("fks_build_batched");
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!h_seeds) return fail(FKS_ERR_INVALID_ARG, "fks_build_batched: bad arguments");
  std::vector<int64_t> seg_copy;
  if (const fks_status cs = check_batched("fks_build_batched", kind, keys, ctx, offs, h_seg, m, vals, val_type,
                                          &seg_copy))
    return cs;
  h_seg = seg_copy.data();
  Opts o;
  if (!read_opts(opts, &o)) return fail(FKS_ERR_INVALID_ARG, "bad build options");
  if (o.inline1) return fail(FKS_ERR_INVALID_ARG, "fks_build_batched: inline_singletons is for one-map builds");
  Alloc A(alloc);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BuildIn in{kind, keys, ctx, offs, vals, val_type, m, h_seg, h_seeds};
  void* block = nullptr;
  size_t bb = 0;
  SetMem mem;
  std::vector<fks_map> maps;
  std::vector<fks_status> per;
  sm_count();
  DedupOut dd;
  if (o.dedup) {
    const fks_status ds = dedup_inputs(in, A, st, &dd);
    if (ds != FKS_OK) {
      if (dd.block) A.put(dd.block, dd.bytes, st);
      return ds;
    }
  }
  fks_status s = build_impl(o.dedup ? dd.in : in, o, A, st, &block, &bb, &mem, &maps, &per);
  if (dd.block) A.put(dd.block, dd.bytes, st);
  if (s != FKS_OK) return s;
  fks_status worst = FKS_OK;
  for (uint32_t j = 0; j < m; ++j) {
    if (h_status) h_status[j] = per[j];
    if (per[j] != FKS_OK && worst == FKS_OK) worst = per[j];
  }
  fks_mapset* set = new fks_mapset();
  set->kind = kind;
  set->vt = val_type;
  set->maps = std::move(maps);
  set->block = block;
  set->block_bytes = bb;
  set->alloc = A;
  set->d_table = static_cast<LookupMap*>(A.get(sizeof(LookupMap) * m, st));
  if (!set->d_table) {
    fks_mapset_destroy(set);
    return fail(FKS_ERR_OUT_OF_MEMORY, "lookup table");
  }
  if (const fks_status ps = publish_set(set, mem, per, st)) {
    fks_mapset_destroy(set);
    return ps;
  }
  *out = set;
  if (worst != FKS_OK) g_last_error = std::string("fks_build_batched: ") + status_name(worst);
  return worst;
}

fks_status fks_lookup_batched(fks_mapset_t set, const uint32_t* map_ids, const uint64_t* q,
                              const uint8_t* qctx, const int64_t* qoffs, uint64_t nq,
                              void* out_vals, uint8_t* out_found, int64_t absent,
                              fks_stream_t stream) {
  NvtxRange range("fks_lookup_batched");
  if (!set) return fail(FKS_ERR_INVALID_ARG, "fks_lookup_batched: set is NULL");
  if (nq == 0) return FKS_OK;
  const bool str = set->kind == FKS_KEY_BYTES;
  if (!map_ids || (str ? (!qctx || !qoffs) : !q))
    return fail(FKS_ERR_INVALID_ARG, "fks_lookup_batched: bad arguments");
  if (set->vt == FKS_VAL_I32 && (absent < INT32_MIN || absent > INT32_MAX))
    return fail(FKS_ERR_INVALID_ARG, "fks_lookup_batched: absent does not fit int32");
  FKS_CUDA(launch_lookup_batched(set->d_table, uint32_t(set->maps.size()), str, map_ids, q, qctx,
                                 qoffs, nq, out_vals, set->vt == FKS_VAL_I64, out_found, absent,
                                 sm_count(), reinterpret_cast<cudaStream_t>(stream)));
  return FKS_OK;
}

fks_status fks_build_graph_create(fks_key_kind kind, const uint64_t* keys, const uint8_t* ctx,
                                  const int64_t* offs, const int64_t* h_seg, uint32_t m, const void* vals,
                                  fks_val_type val_type, const fks_build_opts* opts, const fks_allocator* alloc,
                                  fks_stream_t stream, fks_build_graph_t* out) {
  NvtxRange range("fks_build_graph_create");
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::vector<int64_t> seg;
  if (const fks_status cs = check_batched("fks_build_graph_create", kind, keys, ctx, offs, h_seg, m, vals,
                                          val_type, &seg))
    return cs;
  Opts o;
  if (!read_opts(opts, &o)) return fail(FKS_ERR_INVALID_ARG, "bad build options");
  if (o.dedup) return fail(FKS_ERR_INVALID_ARG, "fks_build_graph_create: dedup changes the sizes; not recordable");
  if (o.inline1) return fail(FKS_ERR_INVALID_ARG, "fks_build_graph_create: inline_singletons is for one-map builds");
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  sm_count();
  fks_build_graph* g = new fks_build_graph();
  g->seg = std::move(seg);
  g->seeds.assign(m, 0);
  const BuildIn in{kind, keys, ctx, offs, vals, val_type, m, g->seg.data(), g->seeds.data()};
  fks_status s = g->b.init(in, o, Alloc(alloc), st);
  if (s != FKS_OK) {
    delete g;
    return s;
  }
  SetBuild& b = g->b;
  g->set.kind = kind;
  g->set.vt = val_type;
  g->set.alloc = b.A;
  g->set.borrowed = true;
  g->set.maps.assign(m, fks_map());
  g->set.d_table = static_cast<LookupMap*>(b.A.get(sizeof(LookupMap) * m, st));
  if (!g->set.d_table || cudaMallocHost(&g->gp.up, SetBuild::up_bytes(m)) != cudaSuccess ||
      cudaMallocHost(&g->gp.down, SetBuild::down_bytes(m)) != cudaSuccess) {
    cudaGetLastError();
    graph_release(g);
    return fail(FKS_ERR_OUT_OF_MEMORY, "fks_build_graph_create: tables or pinned buffers");
  }
  // record the first pass on a stream of our own (the caller's may be the
  // legacy default stream, which cannot capture)
  b.round.assign(m, 0);
  std::vector<uint32_t> all(m);
  for (uint32_t j = 0; j < m; ++j) all[j] = j;
  b.fill_tables(all, g->gp.up);
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // allocations above are ordered on `st`
  if (e == cudaSuccess) {
    const uint64_t before = g_launches.load();
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      const cudaError_t ep = b.enqueue_pass(m, g->gp.up, g->gp.down, true, nullptr, cap);
      e = cudaStreamEndCapture(cap, &g->graph);
      if (ep != cudaSuccess) e = ep;
    }
    g_launches.fetch_sub(g_launches.load() - before);  // recorded, not launched
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->gp.exec, g->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    graph_release(g);
    return cuda_fail(e, "fks_build_graph_create: recording the first pass");
  }
  g->gp.kernels = graph_kernels(g->graph);
  *out = g;
  return FKS_OK;
}

fks_status fks_build_graph_run(fks_build_graph_t g, const uint64_t* h_seeds, fks_stream_t stream,
                               fks_status* h_status) {
  NvtxRange range("fks_build_graph_run");
  if (!g || !h_seeds) return fail(FKS_ERR_INVALID_ARG, "fks_build_graph_run: NULL argument");
  std::lock_guard<std::mutex> lock(g->mu);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SetBuild& b = g->b;
  const uint32_t m = b.m;
  memcpy(g->seeds.data(), h_seeds, sizeof(uint64_t) * m);
  fks_status s = b.run(st, &g->gp);
  if (s != FKS_OK) {
    for (uint32_t j = 0; j < m; ++j) g->set.maps[j] = fks_map();
    return s;
  }
  fks_status worst = FKS_OK;
  for (uint32_t j = 0; j < m; ++j) {
    g->set.maps[j] = b.maps[j];  // element-wise: handles from fks_mapset_get stay put
    if (h_status) h_status[j] = b.per_map[j];
    if (b.per_map[j] != FKS_OK && worst == FKS_OK) worst = b.per_map[j];
  }
  if (const fks_status ps = publish_set(&g->set, b.mem, b.per_map, st)) return ps;
  if (worst != FKS_OK) g_last_error = std::string("fks_build_graph_run: ") + status_name(worst);
  return worst;
}

fks_mapset_t fks_build_graph_mapset(fks_build_graph_t g) { return g ? &g->set : nullptr; }

uint32_t fks_build_graph_kernels(fks_build_graph_t g) { return g ? g->gp.kernels : 0u; }

void fks_build_graph_destroy(fks_build_graph_t g) {
  if (!g) return;
  { std::lock_guard<std::mutex> lock(g->mu); }  // a run on another thread finishes first
  graph_release(g);
}

uint32_t fks_mapset_size(fks_mapset_t set) { return set ? uint32_t(set->maps.size()) : 0u; }

fks_map_t fks_mapset_get(fks_mapset_t set, uint32_t j) {
  if (!set || j >= set->maps.size() || set->maps[j].n == 0) return nullptr;
  return &set->maps[j];
}

fks_status fks_map_info(fks_map_t map, fks_map_info_t* h_out) {
  if (!map || !h_out) return fail(FKS_ERR_INVALID_ARG, "fks_map_info: NULL argument");
  memset(h_out, 0, sizeof(*h_out));
  if (const fks_status bs = settle(map)) return bs;
  h_out->n = map->n;
  h_out->seed = map->seed;
  h_out->slots = map->S;
  h_out->slot_capacity = map->slot_cap;
  h_out->bytes = map->bytes;
  h_out->attempts_sum = map->att_sum;
  h_out->context_bytes = map->ctx_bytes;
  h_out->round = map->round;
  h_out->max_bucket = map->max_s;
  h_out->max_attempt = map->max_att;
  h_out->key_kind = map->kind;
  h_out->val_type = map->vt;
  h_out->overflow_partitions = map->overflow;
  h_out->nonempty_buckets = map->nonempty;
  h_out->buckets = map->nb;
  h_out->keys_per_bucket = map->lambda;
  h_out->inline_singletons = map->rec ? 1u : 0u;
  return FKS_OK;
}

fks_status fks_map_export_records(fks_map_t map, uint64_t* h_rec, fks_stream_t stream) {
  if (!map || !h_rec) return fail(FKS_ERR_INVALID_ARG, "fks_map_export_records: NULL argument");
  if (const fks_status bs = settle(map)) return bs;
  if (!map->rec) return fail(FKS_ERR_INVALID_ARG, "fks_map_export_records: the map has no inline records");
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  FKS_CUDA(cudaMemcpyAsync(h_rec, map->rec, 2 * sizeof(uint64_t) * map->nb, cudaMemcpyDeviceToHost, st));
  FKS_CUDA(cudaStreamSynchronize(st));
  return FKS_OK;
}

fks_status fks_map_export(fks_map_t map, uint64_t* h_desc, void* h_slots, uint8_t* h_ctx,
                          fks_stream_t stream) {
  if (!map) return fail(FKS_ERR_INVALID_ARG, "fks_map_export: NULL map");
  if (const fks_status bs = settle(map)) return bs;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int W = map->kind == FKS_KEY_BYTES ? 4 : 2;
  if (h_desc) FKS_CUDA(cudaMemcpyAsync(h_desc, map->desc, sizeof(uint64_t) * map->nb, cudaMemcpyDeviceToHost, st));
  if (h_slots && map->S)
    FKS_CUDA(cudaMemcpyAsync(h_slots, map->slots, sizeof(uint64_t) * W * map->S, cudaMemcpyDeviceToHost, st));
  if (h_ctx && map->kind == FKS_KEY_BYTES && map->ctx_bytes)
    FKS_CUDA(cudaMemcpyAsync(h_ctx, map->ctx, map->ctx_bytes, cudaMemcpyDeviceToHost, st));
  FKS_CUDA(cudaStreamSynchronize(st));
  return FKS_OK;
}

fks_status fks_map_import(const fks_map_info_t* h_info, const uint64_t* h_desc, const void* h_slots,
                          const uint8_t* h_ctx, const fks_allocator* alloc, fks_stream_t stream, fks_map_t* out) {
  NvtxRange range("fks_map_import");
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!h_info || !h_desc || !h_slots) return fail(FKS_ERR_INVALID_ARG, "fks_map_import: NULL argument");
  const fks_map_info_t& I = *h_info;
  const bool str = I.key_kind == FKS_KEY_BYTES;
  const uint32_t lam = I.keys_per_bucket ? I.keys_per_bucket : 1u;
  if ((I.key_kind != FKS_KEY_U64 && !str) || (I.val_type != FKS_VAL_I32 && I.val_type != FKS_VAL_I64) ||
      I.n == 0 || I.n >= (1ull << 30) || (lam != 1 && lam != 2 && lam != 4 && lam != 8 && lam != 16) ||
      I.buckets != level1_buckets(I.n, lam) || I.slots == 0 || I.slots > I.slot_capacity ||
      I.slot_capacity > 0xFFFFFFFFull || (str && (!h_ctx || I.context_bytes >= (1ull << 40))))
    return fail(FKS_ERR_INVALID_ARG, "fks_map_import: metadata out of range");
  // the descriptors must describe the slot array: every non-empty bucket's
  // s^2 slots inside it, sum s = n, sum s^2 = S, and the ranges in order
  uint64_t keys = 0, next = 0;
  for (uint64_t b = 0; b < I.buckets; ++b) {
    const uint64_t d = h_desc[b];
    const uint64_t s = desc_s(d);
    if (s == 0) continue;
    const uint64_t off = desc_off(d);
    if (off != next || off + s * s > I.slots)
      return fail(FKS_ERR_INVALID_ARG, "fks_map_import: descriptors do not match the slot array");
    next = off + s * s;
    keys += s;
  }
  if (keys != I.n || next != I.slots)
    return fail(FKS_ERR_INVALID_ARG, "fks_map_import: descriptors do not match n or the slot count");
  const int W = str ? 4 : 2;
  Alloc A(alloc);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Carve cm;
  const size_t o_desc = cm.take<uint64_t>(I.buckets);
  const size_t o_slots = cm.take<uint64_t>(I.slots * W);
  const size_t o_ctx = cm.take<uint8_t>(str ? I.context_bytes + 16 : 0);
  uint8_t* block = static_cast<uint8_t*>(A.get(cm.off, st));
  if (!block) return fail(FKS_ERR_OUT_OF_MEMORY, "fks_map_import: allocation");
  cudaError_t e = cudaMemcpyAsync(block + o_desc, h_desc, sizeof(uint64_t) * I.buckets, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(block + o_slots, h_slots, sizeof(uint64_t) * W * I.slots, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && str && I.context_bytes)
    e = cudaMemcpyAsync(block + o_ctx, h_ctx, I.context_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    A.put(block, cm.off, st);
    return cuda_fail(e, "fks_map_import: upload");
  }
  fks_map* m = new fks_map();
  m->kind = fks_key_kind(I.key_kind);
  m->vt = fks_val_type(I.val_type);
  m->n = I.n;
  m->seed = I.seed;
  m->round = I.round;
  m->c1 = derive(I.seed, I.round, kTagLevel1, 0);
  m->fpb = fp_base(I.seed, I.round);
  m->S = I.slots;
  m->slot_cap = I.slot_capacity;
  m->att_sum = I.attempts_sum;
  m->max_s = I.max_bucket;
  m->max_att = I.max_attempt;
  m->overflow = I.overflow_partitions;
  m->nonempty = I.nonempty_buckets;
  m->nb = I.buckets;
  m->lambda = lam;
  m->desc = reinterpret_cast<uint64_t*>(block + o_desc);
  m->slots = reinterpret_cast<uint64_t*>(block + o_slots);
  m->ctx = str ? block + o_ctx : nullptr;
  m->ctx_bytes = str ? I.context_bytes : 0;
  m->block = block;
  m->block_bytes = cm.off;
  m->alloc = A;
  m->bytes = cm.off;
  *out = m;
  return FKS_OK;
}

void fks_map_destroy(fks_map_t map) {
  if (!map) return;
  if (map->async) {  // an asynchronous handle: join its build, then free what it built
    settle(map);
    delete map->async;
    map->async = nullptr;
    if (map->block) map->alloc.put(map->block, map->block_bytes, nullptr);
    delete map;
    return;
  }
  if (!map->block) return;  // borrowed maps are freed with their set
  map->alloc.put(map->block, map->block_bytes, nullptr);
  delete map;
}

void fks_mapset_destroy(fks_mapset_t set) {
  if (!set || set->borrowed) return;
  if (set->d_table) set->alloc.put(set->d_table, sizeof(LookupMap) * set->maps.size(), nullptr);
  if (set->block) set->alloc.put(set->block, set->block_bytes, nullptr);
  delete set;
}

// Sorted (keys, values) of n pairs into a new map: layout 0 keeps the sorted
// order, layout 1 gathers it into Eytzinger order.
static fks_status sortmap_build(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                                int eytzinger, const fks_allocator* alloc, fks_stream_t stream, fks_sortmap_t* out,
                                const char* who) {
  if (!out) return fail(FKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!keys || !vals || n == 0 || n >= (1ull << 32) || (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return fail(FKS_ERR_INVALID_ARG, std::string(who) + ": bad arguments");
  sm_count();
  Alloc A(alloc);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t words = eytzinger ? n + 1 : n;
  const size_t bytes = 16 * words;
  uint8_t* block = static_cast<uint8_t*>(A.get(bytes, st));
  if (!block) return fail(FKS_ERR_OUT_OF_MEMORY, std::string(who) + ": tables");
  const size_t sorted_bytes = eytzinger ? 16 * n : 0;  // sorted pairs before the gather
  const size_t sbytes = sort_scratch_bytes(n) + (val_type == FKS_VAL_I32 ? 8 * n : 0) + sorted_bytes;
  uint8_t* scr = static_cast<uint8_t*>(A.get(sbytes, st));
  if (!scr) {
    A.put(block, bytes, st);
    return fail(FKS_ERR_OUT_OF_MEMORY, std::string(who) + ": scratch");
  }
  const uint64_t* v64 = static_cast<const uint64_t*>(vals);
  cudaError_t e = cudaSuccess;
  if (val_type == FKS_VAL_I32) {
    uint64_t* wide = reinterpret_cast<uint64_t*>(scr + sort_scratch_bytes(n));
    e = launch_widen_i32(static_cast<const int32_t*>(vals), n, wide, st);
    v64 = wide;
  }
  fks_sortmap* m = new fks_sortmap();
  m->vt = val_type;
  m->n = n;
  m->eytzinger = eytzinger;
  m->keys = reinterpret_cast<uint64_t*>(block);
  m->vals = m->keys + words;
  m->block = block;
  m->block_bytes = bytes;
  m->alloc = A;
  if (!eytzinger) {
    if (e == cudaSuccess) e = launch_sort_pairs(keys, v64, n, m->keys, m->vals, scr, st);
  } else {
    uint64_t* sk = reinterpret_cast<uint64_t*>(scr + sbytes - sorted_bytes);
    uint64_t* sv = sk + n;
    if (e == cudaSuccess) e = launch_sort_pairs(keys, v64, n, sk, sv, scr, st);
    if (e == cudaSuccess) e = launch_eytzinger_layout(sk, sv, n, m->keys, m->vals, sm_count(), st);
  }
  A.put(scr, sbytes, st);
  if (e != cudaSuccess) {
    fks_sortmap_destroy(m);
    return cuda_fail(e, who);
  }
  *out = m;
  return FKS_OK;
}

fks_status fks_sortmap_build(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                             const fks_allocator* alloc, fks_stream_t stream, fks_sortmap_t* out) {
  return sortmap_build(keys, vals, val_type, n, 0, alloc, stream, out, "fks_sortmap_build");
}

fks_status fks_eytzmap_build(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                             const fks_allocator* alloc, fks_stream_t stream, fks_sortmap_t* out) {
  return sortmap_build(keys, vals, val_type, n, 1, alloc, stream, out, "fks_eytzmap_build");
}

fks_status fks_sortmap_lookup(fks_sortmap_t map, const uint64_t* q, uint64_t nq, void* out_vals,
                              uint8_t* out_found, int64_t absent, fks_stream_t stream) {
  if (!map) return fail(FKS_ERR_INVALID_ARG, "fks_sortmap_lookup: NULL map");
  if (nq == 0) return FKS_OK;
  if (!q || (map->vt == FKS_VAL_I32 && (absent < INT32_MIN || absent > INT32_MAX)))
    return fail(FKS_ERR_INVALID_ARG, "fks_sortmap_lookup: bad arguments");
  if (map->eytzinger)
    FKS_CUDA(launch_eytzinger_search(map->keys, map->vals, map->n, q, nq, out_vals, map->vt == FKS_VAL_I64,
                                     out_found, absent, sm_count(), reinterpret_cast<cudaStream_t>(stream)));
  else
    FKS_CUDA(launch_sorted_search(map->keys, map->vals, map->n, q, nq, out_vals, map->vt == FKS_VAL_I64, out_found,
                                  absent, sm_count(), reinterpret_cast<cudaStream_t>(stream)));
  return FKS_OK;
}

fks_status fks_sortmap_export(fks_sortmap_t map, uint64_t* h_keys, int64_t* h_vals, fks_stream_t stream) {
  if (!map) return fail(FKS_ERR_INVALID_ARG, "fks_sortmap_export: NULL map");
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t first = map->eytzinger ? 1 : 0;  // Eytzinger slot 0 is unused
  if (h_keys) FKS_CUDA(cudaMemcpyAsync(h_keys, map->keys + first, 8 * map->n, cudaMemcpyDeviceToHost, st));
  if (h_vals) FKS_CUDA(cudaMemcpyAsync(h_vals, map->vals + first, 8 * map->n, cudaMemcpyDeviceToHost, st));
  FKS_CUDA(cudaStreamSynchronize(st));
  return FKS_OK;
}

void fks_sortmap_destroy(fks_sortmap_t map) {
  if (!map) return;
  map->alloc.put(map->block, map->block_bytes, nullptr);
  delete map;
}

const char* fks_status_str(fks_status status) { return status_name(status); }

const char* fks_last_error(void) { return g_last_error.c_str(); }

void fks_profile_enable(int on) {
  g_profile = on;
  if (on) g_last_profile = fks_build_profile{};
}

fks_status fks_last_build_profile(fks_build_profile* h_out) {
  if (!h_out) return fail(FKS_ERR_INVALID_ARG, "fks_last_build_profile: NULL");
  *h_out = g_last_profile;
  return FKS_OK;
}

uint64_t fks_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
