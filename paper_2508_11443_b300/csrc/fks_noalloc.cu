// fks_noalloc.cu -- fks_build_u64_noalloc: the uint64 build for callers that
// cannot allocate device memory.
//
// Some callers of this library must not allocate: a service whose device
// memory is all pre-reserved in its own pool or budget (an allocation by a
// library would bypass that accounting, or simply fail once the pool owns
// the whole device), or a latency-critical loop that cannot afford
// cudaMalloc / cudaFree, which may synchronise the whole device and stall
// other work.  Such callers pass the inputs and the output tables; the
// build's scratch comes from one fixed array compiled into this library.
//
// The scratch is a file-scope __device__ array of kNoAllocBytes.  Every GPU
// that loads the library holds it until the process exits.  Host code must
// not use the array's name as a pointer (on the host it is only a stand-in
// for the device symbol): its device address is looked up once per device
// with cudaGetSymbolAddress and passed to the kernels.
//
// All calls share the one array and it keeps the contents of the last call:
// everything that must start at zero is cleared on every call (the kernels'
// counters, cursors, look-back words and status words), and calls whose
// work overlaps on the GPU -- from two host threads, or on two streams --
// race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "fks.h"
#include "fks_internal.cuh"

using namespace fks;

namespace {

constexpr uint64_t kMaxKeys = FKS_NOALLOC_MAX_KEYS;
constexpr uint64_t kMaxParts = (kMaxKeys + kB - 1) / kB;
constexpr uint64_t kMaxTable = 2 * kMaxKeys;  // duplicate-test set size (power of two)

constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the pieces of the scratch array.
constexpr size_t kOffCnt = 0;
constexpr size_t kOffStart = kOffCnt + up256(4 * (kMaxParts + 1));
constexpr size_t kOffCursor = kOffStart + up256(4 * (kMaxParts + 1));
constexpr size_t kOffLookback = kOffCursor + up256(4 * (kMaxParts + 1));
constexpr size_t kOffTicket = kOffLookback + up256(8 * (kMaxParts + 1));
constexpr size_t kOffOvfList = kOffTicket + 256;
constexpr size_t kOffOvfExcl = kOffOvfList + up256(4 * (kMaxParts + 1));
constexpr size_t kOffMaps = kOffOvfExcl + up256(8 * (kMaxParts + 1));
constexpr size_t kOffPassSeg = kOffMaps + up256(sizeof(MapDev));
constexpr size_t kOffPartSeg = kOffPassSeg + 256;
constexpr size_t kOffStatus = kOffPartSeg + 256;
constexpr size_t kOffStageKey = kOffStatus + up256(sizeof(MapStatus));
constexpr size_t kOffStagePay = kOffStageKey + up256(8 * (kMaxKeys + 2));
// grouped buffers of oversized partitions; reused as the duplicate-test set
constexpr size_t kOffOvf = kOffStagePay + up256(8 * (kMaxKeys + 2));
constexpr size_t kOvfBytes = up256(8 * (2 * kMaxKeys + 2)) > up256(8 * kMaxTable + 64)
                                 ? up256(8 * (2 * kMaxKeys + 2))
                                 : up256(8 * kMaxTable + 64);
constexpr size_t kNoAllocBytes = kOffOvf + kOvfBytes;

static_assert((kMaxTable & (kMaxTable - 1)) == 0, "the duplicate-test set needs a power of two");

}  // namespace

// The scratch of every fks_build_u64_noalloc call (device memory).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// The reason is documented at each return; only the status code is reported.
fks_status noalloc_fail(fks_status st, const char* /*why*/) { return st; }

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
fks_status scratch_for_current_device(unsigned char** out, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(FKS_ERR_CUDA, "fks_build_u64_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return noalloc_fail(FKS_ERR_CUDA, "fks_build_u64_noalloc: cudaGetSymbolAddress of the scratch failed");
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    g_sms[dev] = n;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  *sms = g_sms[dev];
  return FKS_OK;
}

}  // namespace

extern "C" fks_status fks_build_u64_noalloc(const uint64_t* keys, const void* vals,
                                            fks_val_type val_type, uint64_t n, uint64_t seed,
                                            const fks_build_opts* opts, uint64_t* desc_out,
                                            void* slots_out, uint64_t slot_capacity,
                                            fks_map_info_t* h_info, fks_stream_t stream) {
  if (!keys || !vals || !desc_out || !slots_out || n == 0 ||
      (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return noalloc_fail(FKS_ERR_INVALID_ARG, "fks_build_u64_noalloc: bad keys, vals, outputs, n or val_type");
  if (n > kMaxKeys)
    return noalloc_fail(FKS_ERR_INVALID_ARG,
                        "fks_build_u64_noalloc: n exceeds FKS_NOALLOC_MAX_KEYS (262144)");
  uint32_t bound = 4, attempt_cap = 4095, round_cap = 32, reject = 0, spin = 1u << 20;
  if (opts) {
    if (opts->struct_size < offsetof(fks_build_opts, spin_limit) + sizeof(uint32_t))
      return noalloc_fail(FKS_ERR_INVALID_ARG, "fks_build_u64_noalloc: bad options");
    if (opts->bound_factor) bound = opts->bound_factor;
    if (opts->attempt_cap) attempt_cap = opts->attempt_cap;
    if (opts->round_cap) round_cap = opts->round_cap;
    reject = opts->reject_attempts;
    if (opts->spin_limit) spin = opts->spin_limit;
    if (attempt_cap > 4095 || round_cap > 65535 || bound < 1 || bound > 4)
      return noalloc_fail(FKS_ERR_INVALID_ARG, "fks_build_u64_noalloc: bad options");
    // the scratch array is sized for one level-one bucket per key
    if (opts->struct_size >= offsetof(fks_build_opts, keys_per_bucket) + sizeof(uint32_t) &&
        opts->keys_per_bucket > 1)
      return noalloc_fail(FKS_ERR_INVALID_ARG, "fks_build_u64_noalloc: keys_per_bucket must be 1");
    // the deduplicating pre-pass needs buffers of its own
    if (opts->struct_size >= offsetof(fks_build_opts, dedup) + sizeof(uint32_t) && opts->dedup)
      return noalloc_fail(FKS_ERR_INVALID_ARG, "fks_build_u64_noalloc: dedup is not available");
    if (opts->struct_size >= offsetof(fks_build_opts, inline_singletons) + sizeof(uint32_t) &&
        opts->inline_singletons)
      return noalloc_fail(FKS_ERR_INVALID_ARG, "fks_build_u64_noalloc: inline_singletons is not available");
  }
  if (slot_capacity < uint64_t(bound) * n)
    return noalloc_fail(FKS_ERR_INVALID_ARG,
                        "fks_build_u64_noalloc: slots_out holds fewer than bound_factor * n slots");
  unsigned char* base = nullptr;
  int sms = 0;
  fks_status st = scratch_for_current_device(&base, &sms);
  if (st != FKS_OK) return st;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t P = uint32_t((n + kB - 1) / kB);

  PassDev p{};
  p.part_cnt = reinterpret_cast<uint32_t*>(base + kOffCnt);
  p.part_start = reinterpret_cast<uint32_t*>(base + kOffStart);
  p.part_cursor = reinterpret_cast<uint32_t*>(base + kOffCursor);
  p.lookback = reinterpret_cast<uint64_t*>(base + kOffLookback);
  p.ticket = reinterpret_cast<uint32_t*>(base + kOffTicket);
  p.ovf_count = p.ticket + 1;
  p.ovf_list = reinterpret_cast<uint32_t*>(base + kOffOvfList);
  p.ovf_excl = reinterpret_cast<uint64_t*>(base + kOffOvfExcl);
  p.stage_key = reinterpret_cast<uint64_t*>(base + kOffStageKey);
  p.stage_pay = reinterpret_cast<uint64_t*>(base + kOffStagePay);
  p.ovf_key = reinterpret_cast<uint64_t*>(base + kOffOvf);
  p.ovf_pay = p.ovf_key + n;
  MapDev* d_maps = reinterpret_cast<MapDev*>(base + kOffMaps);
  uint64_t* d_pseg = reinterpret_cast<uint64_t*>(base + kOffPassSeg);
  uint32_t* d_qseg = reinterpret_cast<uint32_t*>(base + kOffPartSeg);
  MapStatus* d_stat = reinterpret_cast<MapStatus*>(base + kOffStatus);
  p.maps = d_maps;
  p.status = d_stat;
  p.pass_seg = d_pseg;
  p.part_seg = d_qseg;
  p.m = 1;
  p.P = P;
  p.total = n;
  p.logB = kLogB;
  p.hkeys = keys;
  p.vals = vals;
  p.vals_i64 = val_type == FKS_VAL_I64;
  p.desc = desc_out;
  p.slots = static_cast<uint64_t*>(slots_out);
  p.cfg.attempt_cap = attempt_cap;
  p.cfg.reject = reject;
  p.cfg.spin_limit = spin;
  p.cfg.hold_first = 0;
  p.cfg.thread_max = 3;
  p.cfg.prefetch = 1;

  // control words live on the host stack (pageable copies; nothing allocated)
  const uint64_t h_pseg[2] = {0, n};
  const uint32_t h_qseg[2] = {0, P};
  MapStatus h_stat;
  uint32_t h_ovf = 0;
#define NOALLOC_CUDA(call)                                                           \
  do {                                                                               \
    if ((call) != cudaSuccess) {                                                     \
      cudaGetLastError();                                                            \
      return noalloc_fail(FKS_ERR_CUDA, "fks_build_u64_noalloc: CUDA call failed: " #call); \
    }                                                                                \
  } while (0)
  NOALLOC_CUDA(cudaMemcpyAsync(d_pseg, h_pseg, sizeof(h_pseg), cudaMemcpyHostToDevice, s));
  NOALLOC_CUDA(cudaMemcpyAsync(d_qseg, h_qseg, sizeof(h_qseg), cudaMemcpyHostToDevice, s));
  for (uint32_t r = 0; r < round_cap; ++r) {
    MapDev M{};
    M.seed = seed;
    M.round = r;
    M.c1 = derive(seed, r, kTagLevel1, 0);
    M.n = uint32_t(n);
    M.nb = uint32_t(n);
    M.slot_cap = uint32_t(uint64_t(bound) * n);
    NOALLOC_CUDA(cudaMemcpyAsync(d_maps, &M, sizeof(M), cudaMemcpyHostToDevice, s));
    NOALLOC_CUDA(cudaMemsetAsync(d_stat, 0, sizeof(MapStatus), s));
    NOALLOC_CUDA(launch_pass(p, false, sms, default_build_shape(1), s, nullptr));
    NOALLOC_CUDA(cudaMemcpyAsync(&h_stat, d_stat, sizeof(h_stat), cudaMemcpyDeviceToHost, s));
    NOALLOC_CUDA(cudaMemcpyAsync(&h_ovf, p.ovf_count, sizeof(h_ovf), cudaMemcpyDeviceToHost, s));
    NOALLOC_CUDA(cudaStreamSynchronize(s));
    if (h_ovf) {
      NOALLOC_CUDA(launch_overflow(p, false, h_ovf, s));
      NOALLOC_CUDA(cudaMemcpyAsync(&h_stat, d_stat, sizeof(h_stat), cudaMemcpyDeviceToHost, s));
      NOALLOC_CUDA(cudaStreamSynchronize(s));
    }
    if (h_stat.timeout) return noalloc_fail(FKS_ERR_TIMEOUT, "fks_build_u64_noalloc: a device wait timed out");
    if (h_stat.reseed) continue;  // space bound failed: next level-one round
    if (h_stat.dup) return noalloc_fail(FKS_ERR_DUPLICATE_KEY, "fks_build_u64_noalloc: duplicate key");
    if (h_stat.next_round) continue;
    if (h_info) {
      memset(h_info, 0, sizeof(*h_info));
      h_info->n = n;
      h_info->seed = seed;
      h_info->slots = h_stat.S;
      h_info->slot_capacity = uint64_t(bound) * n;
      h_info->attempts_sum = h_stat.att_sum;
      h_info->round = r;
      h_info->max_bucket = h_stat.max_s;
      h_info->max_attempt = h_stat.max_att;
      h_info->key_kind = FKS_KEY_U64;
      h_info->val_type = val_type;
      h_info->overflow_partitions = h_stat.overflow;
      h_info->nonempty_buckets = h_stat.nonempty;
      h_info->buckets = n;
      h_info->keys_per_bucket = 1;
    }
    return FKS_OK;
  }
  // every round failed: exact duplicate test in the (now free) overflow area
  uint64_t size = 1;
  while (size < 2 * n) size <<= 1;
  uint64_t* table = reinterpret_cast<uint64_t*>(base + kOffOvf);
  uint32_t* flags = reinterpret_cast<uint32_t*>(base + kOffOvf + 8 * kMaxTable);
  uint32_t hf[4] = {0, 0, 0, 0};
  NOALLOC_CUDA(launch_dupcheck(keys, nullptr, nullptr, n, table, nullptr, size, flags, spin, s));
  NOALLOC_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  NOALLOC_CUDA(cudaStreamSynchronize(s));
#undef NOALLOC_CUDA
  if (hf[2]) return noalloc_fail(FKS_ERR_TIMEOUT, "fks_build_u64_noalloc: a device wait timed out");
  return hf[0] ? noalloc_fail(FKS_ERR_DUPLICATE_KEY, "fks_build_u64_noalloc: duplicate key")
               : noalloc_fail(FKS_ERR_BUILD_FAILED, "fks_build_u64_noalloc: every level-one round failed");
}
