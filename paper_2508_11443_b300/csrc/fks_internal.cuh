// fks_internal.cuh -- data structures shared by the kernels and the host side
// of the library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "fks_device.cuh"

struct fks_map;  // handle type of the C ABI (fks_api.cu)

namespace fks {

// Level-one buckets are processed in partitions of consecutive buckets,
// at most kB of them.  A partition's keys are grouped, searched and placed
// inside one CTA's shared memory.  With one bucket per key (the paper's
// construction) a partition is kB buckets, about kB keys and 2 kB slots.
constexpr int kLogB = 10;
constexpr uint32_t kB = 1u << kLogB;
constexpr uint32_t kCap = 2048;        // keys of a partition held in shared memory
constexpr uint32_t kOwnerCap = 8192;   // slots of a partition staged in shared memory

// Buckets per partition (log2) for lambda keys per bucket: kB / lambda, so
// that a partition holds about kB keys whatever lambda.  Its slot image,
// about (1 + lambda) kB slots, is staged in shared memory when it fits
// kOwnerCap (lambda <= 4); larger images are written straight to global
// memory, bucket range by bucket range (coalesced for the warp-searched
// buckets such maps consist of).
__host__ __device__ constexpr uint32_t part_log_buckets(uint32_t lambda) {
  return lambda <= 1 ? 10u : lambda == 2 ? 9u : lambda == 4 ? 8u : lambda == 8 ? 7u : 6u;
}
// Level-one buckets of an n-key map with lambda keys per bucket.
__host__ __device__ constexpr uint64_t level1_buckets(uint64_t n, uint32_t lambda) {
  return (n + lambda - 1) / lambda;
}
constexpr int kPartThreads = 512;      // threads of a partition CTA
constexpr uint32_t kThreadSearchMax = 3;  // largest bucket a single thread searches
constexpr uint16_t kOwnerEmpty = 0xFFFF;
constexpr uint16_t kOwnerFill = 0x8000;

// One map of a build pass.  A pass builds a set of maps whose elements are
// numbered 0 .. total-1 in pass order; map j owns pass elements
// [pass_begin, pass_begin + n) which are input elements
// [key_begin, key_begin + n).
struct MapDev {
  uint64_t key_begin;   // first input element (keys / fingerprints / values)
  uint64_t pass_begin;  // first pass element
  uint64_t desc_base;   // descriptor index of the map's bucket 0
  uint64_t slot_base;   // slot index of the map's slot 0
  uint64_t seed;
  uint64_t fpb;         // fingerprint base of this round (string maps)
  HashConsts c1;        // level-one constants of this round
  uint32_t n;           // keys
  uint32_t nb;          // level-one buckets (= descriptors)
  uint32_t round;
  uint32_t slot_cap;    // bound_factor * n
  uint32_t part_begin;  // first partition (pass numbering)
};

// Per-map outcome of a pass, written by the device.
struct MapStatus {
  uint32_t reseed;      // sum s^2 above the bound: next round
  uint32_t dup;         // two equal keys in one bucket
  uint32_t next_round;  // attempts exhausted / equal fingerprints of different strings
  uint32_t timeout;     // a bounded wait ran out
  uint32_t invalid;     // bad string offsets
  uint32_t overflow;    // partitions deferred to the global-memory kernel
  uint32_t max_s;
  uint32_t max_att;
  uint64_t S;           // sum s^2 (valid when reseed == 0)
  uint64_t att_sum;
  uint64_t nonempty;    // buckets with s > 0
};

struct BuildCfg {
  uint32_t attempt_cap;
  uint32_t reject;       // test hook: attempts below this count as failed
  uint32_t spin_limit;   // polls of a look-back wait before giving up
  uint32_t hold_first;   // test hook: partition 0 never publishes (forces a timeout)
  uint32_t thread_max;   // buckets of 2 .. thread_max keys are searched by one thread each
  uint32_t prefetch;     // 1: take the next partition's ticket and stage its keys during the search
};

// Everything a pass's kernels read; passed by value.
struct PassDev {
  const MapDev* maps;
  MapStatus* status;
  const uint64_t* pass_seg;   // [m+1] pass element offsets
  const uint32_t* part_seg;   // [m+1] partition offsets
  uint32_t m;
  uint32_t P;                 // partitions
  uint32_t logB;              // log2 of the buckets per partition
  uint64_t total;             // pass elements
  // inputs
  const uint64_t* hkeys;      // u64 keys, or fingerprints of string keys (input numbering)
  const void* vals;           // int32 / int64 values (input numbering)
  const int64_t* offs;        // string maps: offsets (input numbering), else null
  const uint8_t* ctx;         // string maps: the map set's own context copy
  int vals_i64;
  // scratch
  uint32_t* part_cnt;         // [P]    keys per partition
  uint32_t* part_start;       // [P+1]  exclusive scan of part_cnt
  uint32_t* part_cursor;      // [P]    scatter cursors
  uint64_t* lookback;         // [P]    decoupled look-back words
  uint32_t* ticket;           // partition work queue head
  uint64_t* stage_key;        // [total]
  uint64_t* stage_pay;        // [total * PW]
  uint32_t* ovf_list;         // [P] partitions deferred to the overflow kernel
  uint64_t* ovf_excl;         // [P] their slot prefix
  uint32_t* ovf_count;
  uint64_t* ovf_key;          // [total]      (lazily allocated)
  uint64_t* ovf_pay;          // [total * PW] (lazily allocated)
  // outputs
  uint64_t* desc;             // descriptor array of the set
  uint64_t* slots;            // slot array of the set (2 or 4 words per slot)
  // Inline-singleton records (one-map u64 passes with the option, else null):
  // rec[2b .. 2b+1] = {key, value} of a one-key bucket b, else {a key that
  // does not hash to b, desc[b]}.  That key is 0 except in bucket rec_g0 =
  // g(0), where it is rec_x1 (the least x >= 1 with g(x) != g(0)).
  uint64_t* rec;
  uint64_t rec_x1;
  uint32_t rec_g0;
  BuildCfg cfg;
};

// An NVTX range for the lifetime of the object (host code): the entry points
// and the phases of a build show up by name in a profiler's timeline.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Process-wide count of kernels launched by the library (fks_api.cu).
void note_launches(uint32_t n);

// Launch shapes of a build and of a uint64 lookup: the defaults below, or
// what fks_autotune measured best for a (key kind, keys per bucket) pair
// (fks_tune.cu).  No shape changes a table or a result: every shape runs
// the same steps and keeps the first successful attempt of every bucket.
struct BuildShape {
  uint32_t thread_max;             // buckets of 2 .. thread_max keys are searched by one thread each
  uint32_t part_ctas_per_sm;       // partition-build CTAs per SM (capped by occupancy)
  uint32_t scatter_blocks_per_sm;  // grid of the one-level count / scatter kernels
  uint32_t split_min_log2;         // passes of >= 2^x keys are grouped in two radix levels
  uint32_t prefetch;               // 1: a partition CTA takes its next ticket during the search
};
struct LookupShape {
  uint32_t queries_per_thread;  // 2, 4 or 8 needles in flight per thread
  uint32_t block;               // 128, 256 or 512 threads
  uint32_t blocks_per_sm;       // grid = SMs x this (grid-stride loop)
};
BuildShape default_build_shape(uint32_t lambda);
LookupShape default_lookup_shape();
// The shape a build / lookup uses: a thread's override (set while the
// autotuner measures candidates), else the tuned table, else the default.
BuildShape build_shape_for(int key_kind, uint32_t lambda);
LookupShape lookup_shape_for(uint32_t lambda);

// Optional CUDA events recorded between the phases of a pass:
// ev[0] before counting, ev[1] after counting, ev[2] after the scan,
// ev[3] after the scatter, ev[4] after the partition build.
struct PassEvents {
  cudaEvent_t ev[5];
};

// Two-level grouping of large passes (fks_split.cu).
struct SplitShape {
  uint32_t binsA, binsB, shiftB, tilesA, tilesB_max;
  bool ok;
};
struct SplitDev {
  uint32_t binsA, binsB, shiftB, tilesA, tilesB_max;
  uint32_t* histA;    // [binsA * tilesA] (may alias histB)
  uint32_t* histB;    // [binsB * tilesB_max]
  uint32_t* sums;     // block sums of the device-wide scan
  uint64_t* startA;   // [binsA + 1] level-A bin starts
  uint32_t* tstartB;  // [binsA + 1] first level-B tile of each level-A bin
  uint64_t* keyA;     // level-A output: keys, payloads, partition of each key
  uint64_t* payA;
  uint32_t* gpA;
};
SplitShape split_shape(uint32_t P, uint64_t total);
size_t split_hist_words(const SplitShape& sh);
size_t split_sum_words(const SplitShape& sh);
cudaError_t launch_split(const PassDev& p, const SplitDev& s, bool strings, cudaStream_t stream);

// Device-wide exclusive scan of n elements in place (fks_split.cu); sums
// holds scan_sum_words(n) elements of scratch.  T = uint32_t or uint64_t.
template <class T>
cudaError_t scan_exclusive(T* data, uint64_t n, T* sums, cudaStream_t st);
size_t scan_sum_words(uint64_t n);

// from_array pre-pass (fks_dedup.cu).  launch_dedup_mark fills keep[0 .. u]
// (keep[u] = 0) with the first-occurrence flags; flags[0] = malformed string
// offsets, flags[1] = a probe sequence ran out (not expected).  After an
// in-place exclusive scan of keep (= pos), the pack launchers gather the
// kept elements in input order.
size_t dedup_table_words(uint64_t u);
cudaError_t launch_dedup_mark(const uint64_t* keys, const uint8_t* ctx, const int64_t* offs, const int64_t* d_seg,
                              uint32_t m, uint64_t u, uint64_t* table, size_t table_words, uint32_t* keep,
                              uint32_t* flags, int sms, cudaStream_t st);
cudaError_t launch_dedup_pack_u64(const uint64_t* keys, const void* vals, int vals_i64, uint64_t u,
                                  const uint32_t* pos, uint64_t* okeys, void* ovals, int sms, cudaStream_t st);
cudaError_t launch_dedup_lengths(const int64_t* offs, uint64_t u, const uint32_t* pos, uint64_t* lens, int sms,
                                 cudaStream_t st);
cudaError_t launch_dedup_pack_bytes(const uint8_t* ctx, const int64_t* offs, const void* vals, int vals_i64,
                                    uint64_t u, const uint32_t* pos, const uint64_t* noff, uint8_t* octx,
                                    int64_t* ooffs, void* ovals, int sms, cudaStream_t st);
cudaError_t launch_dedup_segs(const uint32_t* pos, const int64_t* d_seg, uint32_t m, int64_t* oseg, cudaStream_t st);

// Launchers (fks_build.cu).
cudaError_t launch_fingerprints(const uint8_t* ctx, const int64_t* offs, uint64_t n,
                                const MapDev* maps, const uint64_t* pass_seg, uint32_t m,
                                uint64_t total, uint64_t* fps, MapStatus* status,
                                cudaStream_t stream);
cudaError_t launch_pass(const PassDev& p, bool strings, int sms, const BuildShape& shape, cudaStream_t stream,
                        const PassEvents* events);
// The same pass with the keys grouped by launch_split instead of the
// single-level partition scatter.
cudaError_t launch_pass_split(const PassDev& p, const SplitDev& s, bool strings, int sms, const BuildShape& shape,
                              cudaStream_t stream, const PassEvents* events);
cudaError_t launch_overflow(const PassDev& p, bool strings, uint32_t count, cudaStream_t stream);
cudaError_t launch_dupcheck(const uint64_t* hkeys, const int64_t* offs, const uint8_t* ctx,
                            uint64_t n, uint64_t* table, uint32_t* table_idx, uint64_t table_size,
                            uint32_t* flags, uint32_t spin_limit, cudaStream_t stream);

// Lookup side (fks_lookup.cu).
struct LookupMap {
  const uint64_t* desc;
  const uint64_t* slots;   // 2 (u64) or 4 (bytes) words per slot
  const uint8_t* ctx;      // string maps: the map's context
  HashConsts c1;
  uint64_t seed;
  uint64_t fpb;
  uint32_t nb;             // level-one buckets
  uint32_t round;
};
cudaError_t launch_lookup_u64(const LookupMap& M, const uint64_t* q, uint64_t nq, void* out,
                              int out_i64, uint8_t* found, int64_t absent, int sms,
                              const LookupShape& shape, cudaStream_t stream);
// Lookups of a map with inline-singleton records (rec: 2 words per bucket).
cudaError_t launch_lookup_inline(const LookupMap& M, const uint64_t* rec, const uint64_t* q, uint64_t nq, void* out,
                                 int out_i64, uint8_t* found, int64_t absent, int sms, cudaStream_t stream);
cudaError_t launch_lookup_bytes(const LookupMap& M, const uint8_t* qctx, const int64_t* qoffs,
                                uint64_t nq, void* out, int out_i64, uint8_t* found,
                                int64_t absent, int sms, cudaStream_t stream);
cudaError_t launch_lookup_batched(const LookupMap* maps, uint32_t m, int strings,
                                  const uint32_t* ids, const uint64_t* q, const uint8_t* qctx,
                                  const int64_t* qoffs, uint64_t nq, void* out, int out_i64,
                                  uint8_t* found, int64_t absent, int sms, cudaStream_t stream);

// One lookup request of a coalesced serving batch (fks_lookup.cu).
struct LookupReq {
  LookupMap M;
  const uint64_t* q;      // u64 needles
  const uint8_t* qctx;    // string needles
  const int64_t* qoffs;
  void* out;              // nullable
  uint8_t* found;         // nullable
  int64_t absent;
  uint64_t begin;         // first query of this request in the batch
  uint32_t strings;
  uint32_t out_i64;
};
cudaError_t launch_lookup_requests(const LookupReq* reqs, const uint64_t* begins, uint32_t nreq,
                                   uint64_t total, int sms, cudaStream_t stream);

// Host helpers of fks_api.cu used by the serving loop.
bool lookup_view_of(struct ::fks_map* m, LookupMap* out, int* strings, int* out_i64);
int device_sm_count();

// Search-based comparison map (fks_sort.cu).
size_t sort_scratch_bytes(uint64_t n);
cudaError_t launch_sort_pairs(const uint64_t* keys, const uint64_t* vals, uint64_t n, uint64_t* kout,
                              uint64_t* vout, void* scratch, cudaStream_t st);
cudaError_t launch_widen_i32(const int32_t* in, uint64_t n, uint64_t* out, cudaStream_t st);
cudaError_t launch_sorted_search(const uint64_t* keys, const uint64_t* vals, uint64_t n, const uint64_t* q,
                                 uint64_t nq, void* out, int out_i64, uint8_t* found, int64_t absent, int sms,
                                 cudaStream_t st);
// Eytzinger layout of sorted (keys, values): ek, ev hold n + 1 words (slot 0 unused).
cudaError_t launch_eytzinger_layout(const uint64_t* sk, const uint64_t* sv, uint64_t n, uint64_t* ek, uint64_t* ev,
                                    int sms, cudaStream_t st);
cudaError_t launch_eytzinger_search(const uint64_t* ek, const uint64_t* ev, uint64_t n, const uint64_t* q, uint64_t nq,
                                    void* out, int out_i64, uint8_t* found, int64_t absent, int sms, cudaStream_t st);

}  // namespace fks
