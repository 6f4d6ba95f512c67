// fks_tune.cu -- launch shapes of the build and of uint64 lookups, and the
// autotuner that measures them.
//
// A shape fixes how the work is spread over the GPU, never what is computed:
//   build   thread_max         buckets of 2 .. thread_max keys are searched by
//                              one thread each (pairwise compares of the
//                              slot indices); larger buckets by a warp segment of
//                              2^ceil(log2 s) lanes, above 32 keys by the CTA
//                              (threads per bucket, and the small / large
//                              bucket threshold)
//           part_ctas_per_sm   resident partition-build CTAs per SM
//           scatter_blocks_per_sm  grid of the one-level count / scatter
//           split_min_log2     passes of >= 2^x keys group in two radix levels
//   lookup  queries_per_thread needles in flight per thread
//           block              threads per block
//           blocks_per_sm      grid (grid-stride loop)
// Every search keeps the first attempt without a collision, whoever runs it,
// so a table is the same under every shape.
//
// fks_autotune builds a synthetic sample of the requested kind and size,
// measures the candidates one parameter at a time (coordinate descent from
// the current shape; the median of three blocking builds, or of five lookup
// launches timed with CUDA events) and keeps the fastest in a process-wide
// table keyed by (key kind, keys per bucket), which later builds and
// lookups consult.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>

#include "fks.h"
#include "fks_internal.cuh"

namespace fks {

BuildShape default_build_shape(uint32_t lambda) {
  BuildShape s;
  // measured on 2^26-key builds: one-thread searches pay for buckets of up to
  // three keys; with 8 or 16 keys per bucket every bucket goes to a segment
  s.thread_max = lambda <= 4 ? kThreadSearchMax : 1u;
  s.part_ctas_per_sm = 0;  // as many as fit
  s.scatter_blocks_per_sm = 8;
  s.split_min_log2 = 20;
  // staging the next partition during the search pays up to 8 keys per
  // bucket (2^26 keys: 4.01 vs 4.14 ms at lambda 1, 6.01 vs 6.15 ms at 8);
  // with 16, whose partitions need their slot prefix before the search, the
  // longer look-back behind queued partitions costs more (7.29 vs 6.94 ms)
  s.prefetch = lambda <= 8 ? 1u : 0u;
  return s;
}

LookupShape default_lookup_shape() {
  LookupShape s;
  s.queries_per_thread = 4;
  s.block = 256;
  s.blocks_per_sm = 8;
  return s;
}

namespace {

std::mutex g_mu;
std::vector<fks_tuning> g_table;
thread_local const BuildShape* t_build_override = nullptr;  // set while a candidate is measured

const fks_tuning* find_locked(uint32_t kind, uint32_t lambda) {
  for (const fks_tuning& t : g_table)
    if (t.key_kind == kind && t.keys_per_bucket == lambda) return &t;
  return nullptr;
}

BuildShape build_of(const fks_tuning& t) {
  BuildShape s;
  s.thread_max = t.thread_search_max;
  s.part_ctas_per_sm = t.part_ctas_per_sm;
  s.scatter_blocks_per_sm = t.scatter_blocks_per_sm;
  s.split_min_log2 = t.split_min_keys_log2;
  s.prefetch = t.part_prefetch;
  return s;
}

LookupShape lookup_of(const fks_tuning& t) {
  LookupShape s;
  s.queries_per_thread = t.lookup_queries_per_thread;
  s.block = t.lookup_block;
  s.blocks_per_sm = t.lookup_blocks_per_sm;
  return s;
}

void fill(fks_tuning* t, uint32_t kind, uint32_t lambda, const BuildShape& b, const LookupShape& l) {
  memset(t, 0, sizeof(*t));
  t->struct_size = sizeof(fks_tuning);
  t->key_kind = kind;
  t->keys_per_bucket = lambda;
  t->thread_search_max = b.thread_max;
  t->part_ctas_per_sm = b.part_ctas_per_sm;
  t->scatter_blocks_per_sm = b.scatter_blocks_per_sm;
  t->split_min_keys_log2 = b.split_min_log2;
  t->part_prefetch = b.prefetch;
  t->lookup_queries_per_thread = l.queries_per_thread;
  t->lookup_block = l.block;
  t->lookup_blocks_per_sm = l.blocks_per_sm;
}

bool valid_lambda(uint32_t l) { return l == 1 || l == 2 || l == 4 || l == 8 || l == 16; }

bool valid(const fks_tuning& t) {
  return t.struct_size >= sizeof(fks_tuning) && (t.key_kind == FKS_KEY_U64 || t.key_kind == FKS_KEY_BYTES) &&
         valid_lambda(t.keys_per_bucket) && t.thread_search_max >= 1 && t.thread_search_max <= kThreadSearchMax &&
         t.part_ctas_per_sm <= 2 && t.scatter_blocks_per_sm >= 1 && t.scatter_blocks_per_sm <= 64 &&
         t.split_min_keys_log2 >= 10 && t.split_min_keys_log2 <= 40 && t.part_prefetch <= 1 &&
         (t.lookup_queries_per_thread == 2 || t.lookup_queries_per_thread == 4 ||
          t.lookup_queries_per_thread == 8) &&
         (t.lookup_block == 128 || t.lookup_block == 256 || t.lookup_block == 512) && t.lookup_blocks_per_sm >= 1 &&
         t.lookup_blocks_per_sm <= 1024;
}

void store(const fks_tuning& t) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (fks_tuning& e : g_table)
    if (e.key_kind == t.key_kind && e.keys_per_bucket == t.keys_per_bucket) {
      e = t;
      return;
    }
  g_table.push_back(t);
}

// ---------------------------------------------------------------- sample inputs
constexpr uint64_t kQuerySalt = 0xA5A5A5A5A5A5A5A5ull;

// keys[i] = the i-th output of a splitmix64 stream (distinct: mix13 is a
// bijection), vals[i] = i; keys may be NULL
__global__ void k_tune_keys(uint64_t seed, uint64_t n, uint64_t* keys, int64_t* vals) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    if (keys) keys[i] = mix13(seed + (i + 1) * kGamma);
    vals[i] = int64_t(i);
  }
}

// about 90 % members (a key drawn at random) and 10 % random words
__global__ void k_tune_queries(uint64_t seed, const uint64_t* keys, uint64_t n, uint64_t nq, uint64_t* q) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < nq; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t h = mix13((seed ^ kQuerySalt) + (i + 1) * kGamma);
    q[i] = (h & 1023u) < 922u ? keys[((h >> 10) & 0xFFFFFFFFull) * n >> 32] : mix13(h ^ kGamma);
  }
}

// string i: length 8 .. 64; its first seven bytes spell i in base 26 (a-z),
// which keeps the strings distinct, the rest are random a-z
__global__ void k_tune_lengths(uint64_t seed, uint64_t n, uint64_t* lens) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i <= n; i += uint64_t(gridDim.x) * blockDim.x)
    lens[i] = i < n ? 8 + mix13(seed + (i + 1) * kGamma) % 57 : 0;
}

__global__ void k_tune_bytes(uint64_t seed, uint64_t n, const uint64_t* offs, uint8_t* ctx) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t o = offs[i], len = offs[i + 1] - o;
    uint64_t x = i;
    for (uint64_t b = 0; b < len; ++b) {
      uint8_t c;
      if (b < 7) {
        c = uint8_t('a' + x % 26);
        x /= 26;
      } else {
        c = uint8_t('a' + mix13(seed ^ (i * 64 + b)) % 26);
      }
      ctx[o + b] = c;
    }
  }
}

template <class T>
T median(std::vector<T> v) {
  std::sort(v.begin(), v.end());
  return v[v.size() / 2];
}

struct Sample {
  uint64_t* keys = nullptr;
  int64_t* vals = nullptr;
  uint64_t* offs = nullptr;  // strings: n + 1 offsets (int64 values)
  uint8_t* ctx = nullptr;
  uint64_t* sums = nullptr;
  uint64_t* q = nullptr;
  int64_t* out = nullptr;
  uint8_t* found = nullptr;
};

}  // namespace

BuildShape build_shape_for(int key_kind, uint32_t lambda) {
  if (t_build_override) return *t_build_override;
  std::lock_guard<std::mutex> lock(g_mu);
  if (const fks_tuning* t = find_locked(uint32_t(key_kind), lambda)) return build_of(*t);
  return default_build_shape(lambda);
}

LookupShape lookup_shape_for(uint32_t lambda) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (const fks_tuning* t = find_locked(FKS_KEY_U64, lambda)) return lookup_of(*t);
  return default_lookup_shape();
}

}  // namespace fks

using namespace fks;

extern "C" {

fks_status fks_tuning_get(fks_key_kind kind, uint32_t keys_per_bucket, fks_tuning* h_out) {
  if (!h_out || !valid_lambda(keys_per_bucket) || (kind != FKS_KEY_U64 && kind != FKS_KEY_BYTES))
    return FKS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (const fks_tuning* t = find_locked(kind, keys_per_bucket)) {
    *h_out = *t;
    return FKS_OK;
  }
  fill(h_out, kind, keys_per_bucket, default_build_shape(keys_per_bucket), default_lookup_shape());
  return FKS_OK;
}

fks_status fks_tuning_set(const fks_tuning* h_in) {
  if (!h_in || !valid(*h_in)) return FKS_ERR_INVALID_ARG;
  store(*h_in);
  return FKS_OK;
}

void fks_tuning_reset(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
}

// One line per entry: a tag, the version, then the fields in declaration order.
fks_status fks_tuning_save(const char* path) {
  if (!path) return FKS_ERR_INVALID_ARG;
  std::vector<fks_tuning> copy;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    copy = g_table;
  }
  FILE* f = fopen(path, "w");
  if (!f) return FKS_ERR_INVALID_ARG;
  for (const fks_tuning& t : copy)
    fprintf(f, "fks_tuning 2 %u %u %u %u %u %u %u %u %u %u %.6g %.6g %llu %u\n", t.key_kind, t.keys_per_bucket,
            t.thread_search_max, t.part_ctas_per_sm, t.scatter_blocks_per_sm, t.split_min_keys_log2,
            t.lookup_queries_per_thread, t.lookup_block, t.lookup_blocks_per_sm, t.tuned, double(t.build_ms),
            double(t.lookup_ms), static_cast<unsigned long long>(t.sample_keys), t.part_prefetch);
  const bool ok = fflush(f) == 0;
  fclose(f);
  return ok ? FKS_OK : FKS_ERR_INVALID_ARG;
}

fks_status fks_tuning_load(const char* path) {
  if (!path) return FKS_ERR_INVALID_ARG;
  FILE* f = fopen(path, "r");
  if (!f) return FKS_ERR_INVALID_ARG;
  std::vector<fks_tuning> entries;
  char line[512];
  bool bad = false;
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '\n' || line[0] == '#') continue;
    fks_tuning t;
    memset(&t, 0, sizeof(t));
    t.struct_size = sizeof(fks_tuning);
    unsigned version = 0;
    double bms = 0, lms = 0;
    unsigned long long nk = 0;
    const int got = sscanf(line, "fks_tuning %u %u %u %u %u %u %u %u %u %u %u %lg %lg %llu %u", &version, &t.key_kind,
                           &t.keys_per_bucket, &t.thread_search_max, &t.part_ctas_per_sm, &t.scatter_blocks_per_sm,
                           &t.split_min_keys_log2, &t.lookup_queries_per_thread, &t.lookup_block,
                           &t.lookup_blocks_per_sm, &t.tuned, &bms, &lms, &nk, &t.part_prefetch);
    t.build_ms = float(bms);
    t.lookup_ms = float(lms);
    t.sample_keys = nk;
    // version 1 lines have no part_prefetch: the default for their lambda
    if (version == 1 && got == 14) t.part_prefetch = default_build_shape(t.keys_per_bucket).prefetch;
    const bool complete = (version == 1 && got == 14) || (version == 2 && got == 15);
    if (!complete || !valid(t)) {
      bad = true;
      break;
    }
    entries.push_back(t);
  }
  fclose(f);
  if (bad) return FKS_ERR_INVALID_ARG;  // nothing installed from a malformed file
  for (const fks_tuning& t : entries) store(t);
  return FKS_OK;
}

fks_status fks_autotune(fks_key_kind kind, uint32_t keys_per_bucket, uint64_t n, uint64_t nq, uint64_t seed,
                        fks_stream_t stream, fks_tuning* h_out, fks_tune_trial* h_trials, uint32_t max_trials,
                        uint32_t* h_count) {
  NvtxRange range("fks_autotune");
  if (h_count) *h_count = 0;
  if ((kind != FKS_KEY_U64 && kind != FKS_KEY_BYTES) || !valid_lambda(keys_per_bucket)) return FKS_ERR_INVALID_ARG;
  if (n == 0) n = 1ull << 22;
  if (nq == 0) nq = n;
  if (n < 1024 || n >= (1ull << 30) || nq >= (1ull << 32)) return FKS_ERR_INVALID_ARG;
  const bool str = kind == FKS_KEY_BYTES;
  const uint32_t lambda = keys_per_bucket;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  // ---- the sample, in one allocation
  Sample S;
  const uint64_t ctx_cap = str ? n * 64 + 16 : 0;
  const size_t sums_words = str ? scan_sum_words(n + 1) : 0;
  size_t off = 0;
  auto take = [&off](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) & ~size_t(255);
    return at;
  };
  const size_t o_keys = take(str ? 0 : 8 * n), o_vals = take(8 * n), o_offs = take(str ? 8 * (n + 1) : 0),
               o_ctx = take(ctx_cap), o_sums = take(8 * sums_words), o_q = take(str ? 0 : 8 * nq),
               o_out = take(str ? 0 : 8 * nq), o_found = take(str ? 0 : nq);
  uint8_t* block = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&block), off, st) != cudaSuccess) {
    cudaGetLastError();
    return FKS_ERR_OUT_OF_MEMORY;
  }
  S.keys = reinterpret_cast<uint64_t*>(block + o_keys);
  S.vals = reinterpret_cast<int64_t*>(block + o_vals);
  S.offs = reinterpret_cast<uint64_t*>(block + o_offs);
  S.ctx = block + o_ctx;
  S.sums = reinterpret_cast<uint64_t*>(block + o_sums);
  S.q = reinterpret_cast<uint64_t*>(block + o_q);
  S.out = reinterpret_cast<int64_t*>(block + o_out);
  S.found = block + o_found;
  const unsigned grid = unsigned(sms) * 8;
  fks_status result = FKS_OK;
  if (!str) {
    k_tune_keys<<<grid, 256, 0, st>>>(seed, n, S.keys, S.vals);
  } else {
    k_tune_keys<<<grid, 256, 0, st>>>(seed, n, nullptr, S.vals);
    k_tune_lengths<<<grid, 256, 0, st>>>(seed, n, S.offs);
    if (scan_exclusive<uint64_t>(S.offs, n + 1, S.sums, st) != cudaSuccess) result = FKS_ERR_CUDA;
    k_tune_bytes<<<grid, 256, 0, st>>>(seed, n, S.offs, S.ctx);
  }
  note_launches(str ? 3 : 1);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) result = FKS_ERR_CUDA;

  fks_build_opts opts{};
  opts.struct_size = sizeof(opts);
  opts.keys_per_bucket = lambda;
  std::vector<fks_tune_trial> trials;
  auto record = [&](uint32_t param, uint32_t value, float ms) {
    fks_tune_trial t;
    t.param = param;
    t.value = value;
    t.ms = ms;
    trials.push_back(t);
  };
  // one blocking build under `shape`; its wall time in ms, or < 0 on failure
  auto build_once = [&](const BuildShape& shape, fks_map_t* keep) -> float {
    t_build_override = &shape;
    fks_map_t m = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    const fks_status s =
        str ? fks_build_bytes(S.ctx, reinterpret_cast<const int64_t*>(S.offs), S.vals, FKS_VAL_I64, n, seed, &opts,
                              nullptr, stream, &m)
            : fks_build_u64(S.keys, S.vals, FKS_VAL_I64, n, seed, &opts, nullptr, stream, &m);
    const auto t1 = std::chrono::steady_clock::now();
    t_build_override = nullptr;
    if (s != FKS_OK) return -1.0f;
    if (keep) *keep = m;
    else fks_map_destroy(m);
    return float(std::chrono::duration<double, std::milli>(t1 - t0).count());
  };
  auto time_build = [&](const BuildShape& shape) -> float {
    if (build_once(shape, nullptr) < 0) return -1.0f;  // warm-up
    std::vector<float> v;
    for (int r = 0; r < 3; ++r) {
      const float ms = build_once(shape, nullptr);
      if (ms < 0) return -1.0f;
      v.push_back(ms);
    }
    return median(v);
  };

  BuildShape best = build_shape_for(kind, lambda);
  float best_ms = 0;
  if (result == FKS_OK) best_ms = time_build(best);
  if (best_ms < 0) result = FKS_ERR_BUILD_FAILED;
  // try one parameter's candidates from the current best; keep any improvement
  auto sweep = [&](uint32_t param, const std::vector<uint32_t>& values, uint32_t BuildShape::*field) {
    for (uint32_t v : values) {
      if (result != FKS_OK) return;
      BuildShape c = best;
      c.*field = v;
      const float ms = time_build(c);
      if (ms < 0) {
        result = FKS_ERR_BUILD_FAILED;
        return;
      }
      record(param, v, ms);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  };
  sweep(0, {1, 2, 3}, &BuildShape::thread_max);
  sweep(6, {0, 1}, &BuildShape::prefetch);
  sweep(1, {1, 2}, &BuildShape::part_ctas_per_sm);
  {
    // one or two grouping levels at this size: the threshold goes just below
    // or just above log2 n
    uint32_t lg = 0;
    while ((2ull << lg) <= n) ++lg;
    const uint32_t two = std::min(best.split_min_log2, lg), one = std::max(best.split_min_log2, lg + 1);
    sweep(3, {two, one}, &BuildShape::split_min_log2);
  }
  if (n < (1ull << best.split_min_log2)) sweep(2, {4, 8, 16, 32}, &BuildShape::scatter_blocks_per_sm);

  // ---- lookups (uint64 maps)
  LookupShape lbest = lookup_shape_for(lambda);
  float lbest_ms = 0;
  if (result == FKS_OK && !str) {
    fks_map_t m = nullptr;
    if (build_once(best, &m) < 0) result = FKS_ERR_BUILD_FAILED;
    LookupMap L{};
    int strings = 0, i64 = 0;
    if (result == FKS_OK && !lookup_view_of(m, &L, &strings, &i64)) result = FKS_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (result == FKS_OK) {
      k_tune_queries<<<grid, 256, 0, st>>>(seed, S.keys, n, nq, S.q);
      note_launches(1);
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) result = FKS_ERR_CUDA;
    }
    auto time_lookup = [&](const LookupShape& shape) -> float {
      std::vector<float> v;
      for (int r = 0; r < 6; ++r) {
        cudaEventRecord(e0, st);
        if (launch_lookup_u64(L, S.q, nq, S.out, 1, S.found, -1, sms, shape, st) != cudaSuccess) return -1.0f;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r) v.push_back(ms);  // the first launch warms up
      }
      return median(v);
    };
    if (result == FKS_OK) {
      lbest_ms = time_lookup(lbest);
      if (lbest_ms < 0) result = FKS_ERR_CUDA;
    }
    for (uint32_t qpt : {2u, 4u, 8u})
      for (uint32_t blk : {128u, 256u, 512u}) {
        if (result != FKS_OK) break;
        LookupShape c = lbest;
        c.queries_per_thread = qpt;
        c.block = blk;
        const float ms = time_lookup(c);
        if (ms < 0) {
          result = FKS_ERR_CUDA;
          break;
        }
        record(4, qpt << 16 | blk, ms);
        if (ms < lbest_ms) {
          lbest_ms = ms;
          lbest = c;
        }
      }
    for (uint32_t per : {4u, 8u, 32u, 128u, 1024u}) {
      if (result != FKS_OK) break;
      LookupShape c = lbest;
      c.blocks_per_sm = per;
      const float ms = time_lookup(c);
      if (ms < 0) {
        result = FKS_ERR_CUDA;
        break;
      }
      record(5, per, ms);
      if (ms < lbest_ms) {
        lbest_ms = ms;
        lbest = c;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (m) fks_map_destroy(m);
  }
  cudaFreeAsync(block, st);
  cudaStreamSynchronize(st);
  cudaGetLastError();
  if (result != FKS_OK) return result;
  fks_tuning t;
  fill(&t, kind, lambda, best, lbest);
  t.tuned = 1;
  t.build_ms = best_ms;
  t.lookup_ms = str ? 0.0f : lbest_ms;
  t.sample_keys = n;
  store(t);
  if (h_out) *h_out = t;
  if (h_trials)
    for (uint32_t i = 0; i < trials.size() && i < max_trials; ++i) h_trials[i] = trials[i];
  if (h_count) *h_count = uint32_t(trials.size());
  return FKS_OK;
}

}  // extern "C"
