/*
 * fks.h -- C ABI of a B300 (sm_103a) library that builds and queries
 * Fredman-Komlos-Szemeredi two-level, static, collision-free hash maps, the
 * method of Due, Elsman, Henriksen, "Towards Efficient Hash Maps in
 * Functional Array Languages" (arXiv 2508.11443).
 *
 * The interface follows the paper's `map` module type (Sec. 3.2):
 *   from_array_nodup  -> fks_build_u64 / fks_build_bytes (duplicates are
 *                        detected and rejected instead of assumed absent)
 *   lookup -> opt v   -> fks_lookup_u64 / fks_lookup_bytes (value + found)
 *   membership        -> a lookup with out_vals == NULL (Sec. 4)
 * and its key abstraction (Sec. 3.3): fixed-width uint64 keys, or byte-slice
 * keys (offset, length) into a context array.  The map keeps its own copy of
 * the context; the needles of a lookup bring theirs (Sec. 3.1).
 *
 * Conventions for every call below.
 *   Pointers: device pointers unless the parameter name starts with h_.
 *   Streams:  every call is ordered on `stream` (a cudaStream_t; NULL is the
 *             legacy default stream).  Builds block until the device status
 *             of the build is known (one stream synchronisation); lookups do
 *             not block.
 *   Errors:   every call returns an fks_status and never aborts.  Device-side
 *             failures come back through a status word, never a trap.
 *             fks_last_error() gives a one-line description of the last
 *             failure on the calling thread.
 *   Ownership: a map owns copies of its keys, values and context; inputs may
 *             be freed once the build returns.  Handles are freed by
 *             fks_map_destroy / fks_mapset_destroy.
 *   Sizes:    1 <= n < 2^30 keys per map; string length < 2^24 bytes;
 *             context < 2^40 bytes.
 */
#ifndef FKS_H_
#define FKS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* fks_stream_t; /* identical to cudaStream_t */

typedef struct fks_map* fks_map_t;       /* one map                     */
typedef struct fks_sortmap* fks_sortmap_t; /* sorted-array map (comparison point) */
typedef struct fks_mapset* fks_mapset_t; /* maps built by one batched call */

typedef enum {
  FKS_OK = 0,
  FKS_ERR_INVALID_ARG = 1,   /* bad pointer, size, offsets or options          */
  FKS_ERR_DUPLICATE_KEY = 2, /* two equal keys (equal byte strings)            */
  FKS_ERR_OUT_OF_MEMORY = 3, /* the allocator returned NULL                    */
  FKS_ERR_BUILD_FAILED = 4,  /* round_cap level-one rounds failed, no duplicate */
  FKS_ERR_TIMEOUT = 5,       /* a bounded device wait ran out                  */
  FKS_ERR_CUDA = 6,          /* a CUDA runtime call failed                     */
  FKS_ERR_EVICTED = 7        /* serving: the map was evicted                   */
} fks_status;

typedef enum { FKS_VAL_I32 = 0, FKS_VAL_I64 = 1 } fks_val_type;
typedef enum { FKS_KEY_U64 = 0, FKS_KEY_BYTES = 1 } fks_key_kind;

/* Device-memory hook.  alloc returns a device pointer aligned to 256 bytes
 * or NULL; free releases it.  Both are stream-ordered on `stream`.  A NULL
 * hook (or NULL members) selects cudaMallocAsync / cudaFreeAsync. */
typedef struct {
  size_t struct_size; /* sizeof(fks_allocator) */
  void* (*alloc)(size_t bytes, fks_stream_t stream, void* user);
  void (*free)(void* ptr, size_t bytes, fks_stream_t stream, void* user);
  void* user;
} fks_allocator;

/* Build options; a NULL pointer or a 0 field selects the default.
 *
 * keys_per_bucket (lambda) selects the level-one bucket count: the paper
 * draws one bucket per key (g k = Hash const k mod n, Sec. 2.3); lambda in
 * {2, 4, 8, 16} draws nb = ceil(n / lambda) buckets and keeps every other
 * step.  Fewer buckets mean a smaller descriptor array (8 nb bytes), which
 * stays in L2 for large maps, so a lookup costs about one DRAM miss instead
 * of the paper's two (Sec. 5) -- at the price of more slots: E[sum s^2] =
 * n + n (n - 1) / nb, about (1 + lambda) n.  The default bound_factor is
 * 2 (1 + lambda) (4 for lambda = 1), twice that expectation, so each
 * level-one round passes the space bound with probability >= 1/2 as in the
 * paper's analysis.  bound_factor * n must stay below 2^32 (slot offsets
 * are 32-bit descriptor fields); larger builds return FKS_ERR_INVALID_ARG.
 * A struct_size that ends before keys_per_bucket is accepted (lambda 1).
 *
 * inline_singletons = 1 (uint64 keys, lambda 1, fks_build_u64 and its
 * _async / _host forms only; other builds return FKS_ERR_INVALID_ARG) adds a
 * record array of 16 bytes per level-one bucket next to the unchanged
 * tables: a bucket of one key holds {key, value}, any other bucket {x,
 * desc[b]} with x a key that hashes to another bucket (0, or for the one
 * bucket g(0) the least x >= 1 with g(x) != g(0)).  fks_lookup_u64 then reads
 * the record first, and only needles of buckets with two or more keys go on
 * to a slot: about 37 % of a map's keys sit alone in their bucket, whose
 * lookups take one random access instead of the paper's two (Sec. 5).  The
 * map holds 16 more bytes per bucket (fks_map_info: inline_singletons = 1;
 * fks_map_export_records copies the records).
 *
 * dedup = 1 turns a build into the paper's from_array (Sec. 3.2): the input
 * may hold equal keys (equal words, or equal byte strings), and the first
 * occurrence in input order wins -- per map for fks_build_batched.  The map
 * holds the distinct keys (fks_map_info: n).  The paper leaves the winner
 * unspecified; with dedup = 0 (from_array_nodup) equal keys are an error. */
typedef struct {
  size_t struct_size;        /* sizeof(fks_build_opts)                          */
  uint32_t bound_factor;     /* level-one redraw when sum s^2 > bound*n (2 (1 + lambda)) */
  uint32_t attempt_cap;      /* level-two attempts per bucket and round (4095) */
  uint32_t round_cap;        /* level-one rounds (32)                           */
  uint32_t reject_attempts;  /* TEST HOOK: attempts below this count as failed (0) */
  uint32_t spin_limit;       /* bound of every device wait, in polls (1<<20)     */
  uint32_t keys_per_bucket;  /* lambda: 1 (the paper), 2, 4, 8 or 16 (1)        */
  uint32_t dedup;            /* 1: from_array -- duplicate keys allowed (0)     */
  uint32_t inline_singletons; /* 1: inline-singleton records (0)               */
} fks_build_opts;

typedef struct {
  uint64_t n;             /* keys                                     */
  uint64_t seed;          /* build seed                               */
  uint64_t slots;         /* S = sum over buckets of s^2              */
  uint64_t slot_capacity; /* slots reserved (bound_factor * n)        */
  uint64_t bytes;         /* device bytes held by the map             */
  uint64_t attempts_sum;  /* sum of level-two attempt indices         */
  uint64_t context_bytes; /* strings: bytes of the map's context      */
  uint32_t round;         /* level-one round that succeeded           */
  uint32_t max_bucket;    /* largest bucket                           */
  uint32_t max_attempt;   /* largest level-two attempt index          */
  uint32_t key_kind;      /* fks_key_kind                             */
  uint32_t val_type;      /* fks_val_type                             */
  uint32_t overflow_partitions; /* partitions built through global memory */
  uint64_t nonempty_buckets;    /* buckets with s > 0                      */
  uint64_t buckets;             /* level-one buckets nb = descriptors      */
  uint32_t keys_per_bucket;     /* lambda of the build                     */
  uint32_t inline_singletons;   /* 1: the map has inline-singleton records */
} fks_map_info_t;

/* Phase timings of the last build on the calling thread (CUDA events on the
 * build's stream; summed over level-one passes).  Recorded only while
 * fks_profile_enable(1) is in effect on that thread.  Keys are grouped by
 * level-one partition either in one level (count, scan, scatter) or, for
 * large builds, in two radix levels, reported together in group_ms. */
typedef struct {
  float fingerprint_ms; /* string maps: fingerprints of the keys            */
  float count_ms;       /* one level: level-one hash + keys per partition   */
  float scan_ms;        /* one level: scan of the partition counts          */
  float scatter_ms;     /* one level: keys scattered into partition ranges  */
  float part_build_ms;  /* per-partition Hist, Presum, make_2, placement    */
  uint32_t passes;      /* level-one passes run                             */
  uint32_t grouping_levels; /* 1 or 2                                       */
  float group_ms;       /* two levels: the whole grouping                   */
} fks_build_profile;

/* ------------------------------------------------------------------ build
 * fks_build_u64 -- from_array_nodup over uint64 keys (Sec. 2.3 make_1 /
 * make_2 as a data-parallel construction; Sec. 3.2).
 *   keys   uint64[n]          distinct keys (device)
 *   vals   int32[n] or int64[n] per val_type (device)
 *   seed   selects the hash constants; the table is a pure function of
 *          (key set, values, seed): the first successful level-one round and,
 *          per bucket, the first successful level-two attempt are kept.
 *   opts, alloc  may be NULL.   out  receives the handle (NULL on failure).
 * Returns FKS_ERR_DUPLICATE_KEY when two keys are equal. */
fks_status fks_build_u64(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                         uint64_t seed, const fks_build_opts* opts, const fks_allocator* alloc,
                         fks_stream_t stream, fks_map_t* out);

/* fks_build_bytes -- the same over byte-string keys in a context (Sec. 3.1,
 * Sec. 3.3 slices): key i is ctx[offs[i] .. offs[i+1]).
 *   ctx    uint8[offs[n]] (device), copied into the map
 *   offs   int64[n+1] non-decreasing, offs[0] >= 0 (device)
 * Keys are hashed through a 61-bit polynomial fingerprint; equal byte
 * strings are duplicates, equal fingerprints of different strings make the
 * build redraw its constants. */
fks_status fks_build_bytes(const uint8_t* ctx, const int64_t* offs, const void* vals,
                           fks_val_type val_type, uint64_t n, uint64_t seed,
                           const fks_build_opts* opts, const fks_allocator* alloc,
                           fks_stream_t stream, fks_map_t* out);

/* fks_build_u64_async / fks_build_bytes_async -- the same builds, returned
 * at once: the build runs on a host thread of the library (on `stream`, on
 * the calling thread's current device) and the handle reports its outcome.
 * fks_map_info waits for the build and returns its status (FKS_OK, or the
 * error the blocking call would have returned); lookups, export and destroy
 * wait for it as well.  A handle whose build failed holds no tables (every
 * call on it returns the build's error) and must still be destroyed.  The
 * inputs must stay valid until the build is known to be done. */
fks_status fks_build_u64_async(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                               uint64_t seed, const fks_build_opts* opts, const fks_allocator* alloc,
                               fks_stream_t stream, fks_map_t* out);
fks_status fks_build_bytes_async(const uint8_t* ctx, const int64_t* offs, const void* vals,
                                 fks_val_type val_type, uint64_t n, uint64_t seed,
                                 const fks_build_opts* opts, const fks_allocator* alloc,
                                 fks_stream_t stream, fks_map_t* out);

/* ------------------------------------------------------------------ lookup
 * fks_lookup_u64 -- lookup -> opt v (Sec. 3.2) with the membership test of
 * Sec. 2.2: level-one descriptor, then one level-two slot, then a compare.
 *   q          uint64[nq] needles (device)
 *   out_vals   int32[nq] / int64[nq] per the map's val_type, or NULL
 *   out_found  uint8[nq] (1 = present), or NULL
 *   absent     written to out_vals for needles that are not in the map
 *              (must fit int32 for int32 maps)
 * nq == 0 is a no-op.  Does not block. */
fks_status fks_lookup_u64(fks_map_t map, const uint64_t* q, uint64_t nq, void* out_vals,
                          uint8_t* out_found, int64_t absent, fks_stream_t stream);

/* fks_lookup_bytes -- needles ctx qctx[qoffs[i] .. qoffs[i+1]) (device),
 * a context of their own (Sec. 3.1); a hit needs equal fingerprint, length
 * and bytes. */
fks_status fks_lookup_bytes(fks_map_t map, const uint8_t* qctx, const int64_t* qoffs, uint64_t nq,
                            void* out_vals, uint8_t* out_found, int64_t absent,
                            fks_stream_t stream);

/* ------------------------------------------------------------------ batched
 * fks_build_batched -- m independent maps over one concatenated input, the
 * same construction per segment with map-local buckets, so map j's tables
 * equal those of a per-call build of segment j with seed h_seeds[j].
 *   keys      uint64[total] for FKS_KEY_U64 (else NULL)
 *   ctx,offs  for FKS_KEY_BYTES: one context, offs int64[total+1] (else NULL)
 *   h_seg     int64[m+1] segment offsets in host or device memory (device
 *             offsets are copied to the host first), h_seg[0] = 0, every segment
 *             non-empty
 *   h_seeds   uint64[m] HOST build seeds
 *   vals      int32/int64[total] (device)
 * The status of each map is returned in h_status[m] (may be NULL); the call
 * returns FKS_OK only if every map was built. */
fks_status fks_build_batched(fks_key_kind kind, const uint64_t* keys, const uint8_t* ctx,
                             const int64_t* offs, const int64_t* h_seg, const uint64_t* h_seeds,
                             uint32_t m, const void* vals, fks_val_type val_type,
                             const fks_build_opts* opts, const fks_allocator* alloc,
                             fks_stream_t stream, fks_mapset_t* out, fks_status* h_status);

/* fks_lookup_batched -- (map_id, key) needles against a map set in one
 * launch.  map_ids uint32[nq] (device); an id >= m is reported absent.
 * Key kind FKS_KEY_U64 uses q; FKS_KEY_BYTES uses qctx/qoffs. */
fks_status fks_lookup_batched(fks_mapset_t set, const uint32_t* map_ids, const uint64_t* q,
                              const uint8_t* qctx, const int64_t* qoffs, uint64_t nq,
                              void* out_vals, uint8_t* out_found, int64_t absent,
                              fks_stream_t stream);

/* Number of maps of a set, and a borrowed handle of map j (valid until the
 * set is destroyed; do not destroy it). */
uint32_t fks_mapset_size(fks_mapset_t set);
fks_map_t fks_mapset_get(fks_mapset_t set, uint32_t j);

/* ------------------------------------------------------------------ recorded batched builds
 * A batched build recorded once as a CUDA graph and replayed: for a caller
 * that rebuilds the same set of maps again and again from refreshed data
 * (same buffers, same segment sizes), so that each rebuild costs one graph
 * launch instead of a dozen kernel launches and table uploads.  The paper
 * builds each map once; this is the launch-sequence form of its batched
 * construction (one data-parallel pass over all maps' keys, Sec. 2.5).
 *
 * fks_build_graph_create -- arguments as for fks_build_batched, without the
 * seeds: the input buffers (keys, or ctx/offs; vals) are bound to the graph
 * and must stay valid until it is destroyed; their contents may change
 * between runs, but not their sizes (for string keys offs[total], the
 * context size, must stay the same).  Allocates the set's tables and the
 * build's scratch once, and records the first pass (every map at level-one
 * round 0: table upload, fingerprints, grouping, partition build, status
 * download) as a graph on a stream of the library's own.  dedup = 1 is
 * rejected (it changes the sizes).  Synchronises `stream`.
 *
 * fks_build_graph_run -- rebuild every map from the buffers' current
 * contents with seeds h_seeds[m] (host): one launch of the recorded pass on
 * `stream`, one synchronisation, then the maps that must redraw (a space
 * bound or level-two failure, probability well below 1/2 per map) run
 * through the ordinary pass loop.  The tables equal those of
 * fks_build_batched with the same inputs and seeds.  h_status[m] (nullable)
 * receives each map's status; returns FKS_OK only if every map was built.
 * Runs of one graph are serialised; a run blocks until it is done.
 *
 * fks_build_graph_mapset -- the maps of the last run, for fks_lookup_batched,
 * fks_mapset_get, export and info.  Owned by the graph: valid until
 * fks_build_graph_destroy (fks_mapset_destroy on it does nothing); each run
 * rewrites its tables in place, so lookups must not overlap a run.
 *
 * fks_build_graph_kernels -- kernels one replay of the recorded pass runs. */
typedef struct fks_build_graph* fks_build_graph_t;
fks_status fks_build_graph_create(fks_key_kind kind, const uint64_t* keys, const uint8_t* ctx,
                                  const int64_t* offs, const int64_t* h_seg, uint32_t m, const void* vals,
                                  fks_val_type val_type, const fks_build_opts* opts, const fks_allocator* alloc,
                                  fks_stream_t stream, fks_build_graph_t* out);
fks_status fks_build_graph_run(fks_build_graph_t g, const uint64_t* h_seeds, fks_stream_t stream,
                               fks_status* h_status);
fks_mapset_t fks_build_graph_mapset(fks_build_graph_t g);
uint32_t fks_build_graph_kernels(fks_build_graph_t g);
void fks_build_graph_destroy(fks_build_graph_t g);

/* ------------------------------------------------------------------ launch shapes and the autotuner
 * How a build and a uint64 lookup spread their work over the GPU.  No shape
 * changes a table or a result: every level-two search keeps the first
 * attempt without a collision, whichever threads run it.  The paper leaves
 * this mapping to its compiler; here it is measured.
 *
 *   thread_search_max      buckets of 2 .. T keys are searched by one thread
 *                          each (pairwise compares of their slot indices); larger
 *                          ones by a warp segment of 2^ceil(log2 s) lanes,
 *                          above 32 keys by the whole CTA: the threads per
 *                          bucket and the small / large bucket threshold (1..3)
 *   part_ctas_per_sm       resident partition-build CTAs per SM (0 = as many
 *                          as fit, else 1 or 2)
 *   scatter_blocks_per_sm  blocks per SM of the one-level count / scatter (1..64)
 *   split_min_keys_log2    passes of >= 2^x keys are grouped in two radix
 *                          levels instead of one (10..40)
 *   part_prefetch          1: a partition CTA takes its next partition and
 *                          stages its keys while it searches the current one;
 *                          0: only once it is free (shorter look-back waits
 *                          for partitions that write their slots directly)
 *   lookup_queries_per_thread, lookup_block, lookup_blocks_per_sm
 *                          needles in flight per thread (2, 4, 8), threads
 *                          per block (128, 256, 512) and the grid cap in
 *                          blocks per SM (1..1024; a grid-stride loop covers
 *                          what the cap leaves) of fks_lookup_u64
 * A process-wide table holds one entry per (key_kind, keys_per_bucket);
 * builds and uint64 lookups of maps with that lambda use it, else the
 * defaults (thread_search_max 3, or 1 for lambda >= 8; 0; 8; 20;
 * part_prefetch 1, or 0 for lambda 16; 4; 256; 8). */
typedef struct {
  size_t struct_size;           /* sizeof(fks_tuning)                            */
  uint32_t key_kind;            /* fks_key_kind of the entry                     */
  uint32_t keys_per_bucket;     /* lambda of the entry                           */
  uint32_t thread_search_max;
  uint32_t part_ctas_per_sm;
  uint32_t scatter_blocks_per_sm;
  uint32_t split_min_keys_log2;
  uint32_t lookup_queries_per_thread; /* lookup fields: FKS_KEY_U64 entries only */
  uint32_t lookup_block;
  uint32_t lookup_blocks_per_sm;
  uint32_t tuned;               /* 1: measured by fks_autotune                   */
  float build_ms;               /* the sample build at the chosen shape          */
  float lookup_ms;              /* the sample lookup at the chosen shape         */
  uint64_t sample_keys;         /* keys of the sample it was measured on         */
  uint32_t part_prefetch;
  uint32_t reserved;
} fks_tuning;

/* One measured candidate: param 0 thread_search_max, 1 part_ctas_per_sm,
 * 2 scatter_blocks_per_sm, 3 split_min_keys_log2, 4 lookup_queries_per_thread
 * << 16 | lookup_block, 5 lookup_blocks_per_sm, 6 part_prefetch; ms is the
 * median time. */
typedef struct {
  uint32_t param;
  uint32_t value;
  float ms;
} fks_tune_trial;

/* fks_autotune -- measure the shapes on a synthetic sample and keep the
 * fastest in the table.  The sample: n keys (0: 2^22; 1024 <= n < 2^30) from
 * a splitmix64 stream for FKS_KEY_U64, or distinct a-z strings of 8..64
 * bytes for FKS_KEY_BYTES; uint64 lookups of nq needles (0: n) at about 90 %
 * hits.  Coordinate descent from the current entry: each build candidate is
 * the median of three blocking builds, each lookup candidate the median of
 * five launches (CUDA events).  h_out (nullable) receives the entry,
 * h_trials[max_trials] (nullable) the candidates measured and *h_count their
 * number.  Allocates the sample with cudaMallocAsync on `stream`; blocks. */
fks_status fks_autotune(fks_key_kind kind, uint32_t keys_per_bucket, uint64_t n, uint64_t nq, uint64_t seed,
                        fks_stream_t stream, fks_tuning* h_out, fks_tune_trial* h_trials, uint32_t max_trials,
                        uint32_t* h_count);
/* the entry in effect for (kind, keys_per_bucket): tuned, or the defaults */
fks_status fks_tuning_get(fks_key_kind kind, uint32_t keys_per_bucket, fks_tuning* h_out);
/* install an entry (e.g. one saved from an earlier process); every field is
 * checked against the ranges above (FKS_ERR_INVALID_ARG otherwise) */
fks_status fks_tuning_set(const fks_tuning* h_in);
/* forget every entry: back to the defaults */
void fks_tuning_reset(void);
/* the table to / from a text file (one line per entry), so that a service
 * tunes once per GPU type and later processes start from the result.  A
 * malformed or out-of-range line makes fks_tuning_load return
 * FKS_ERR_INVALID_ARG and install nothing; loaded entries replace the
 * table's entries for the same (key_kind, keys_per_bucket). */
fks_status fks_tuning_save(const char* path);
fks_status fks_tuning_load(const char* path);

/* ------------------------------------------------------------------ no allocation
 * fks_build_u64_noalloc -- the same build as fks_build_u64, for callers that
 * must not allocate device memory: a service whose device memory is all
 * pre-reserved in its own pool or budget (a library allocation would bypass
 * it, or fail), or a latency-critical path that cannot afford cudaMalloc /
 * cudaFree, which may synchronise the device.  The paper has no counterpart;
 * this is an engineering entry point of this library.
 *
 * Nothing is allocated: the caller passes the inputs and the output tables,
 * and the build's scratch is one fixed device array compiled into the
 * library (about 8.4 MB, held on every GPU that loads the library until the
 * process exits).  Hence n <= FKS_NOALLOC_MAX_KEYS; larger n returns
 * FKS_ERR_INVALID_ARG.
 *   keys, vals, val_type, n, seed, opts   as for fks_build_u64, with one
 *                  level-one bucket per key (keys_per_bucket other than 0
 *                  or 1 returns FKS_ERR_INVALID_ARG; bound_factor <= 4) and
 *                  distinct keys (dedup = 1 returns FKS_ERR_INVALID_ARG)
 *   desc_out       uint64[n] (device): the bucket descriptors
 *   slots_out      slot_capacity slots of 16 bytes (device), slot_capacity >=
 *                  bound_factor * n; the first info.slots slots are the table
 *   h_info         (host, nullable) sizes and statistics of the result
 * The tables written are byte-for-byte those fks_build_u64 would build for
 * the same (keys, values, seed), as fks_map_export returns them.
 * The first call on a device looks up the scratch array's device address
 * (once per device); make that first call before any stream capture.
 * All calls share the scratch array: calls whose work overlaps on the GPU
 * (two host threads, or two streams) race and must be serialised by the
 * caller.  Blocks until the result is known, like fks_build_u64.  Returns a
 * status only (fks_last_error is not updated). */
#define FKS_NOALLOC_MAX_KEYS 262144u
fks_status fks_build_u64_noalloc(const uint64_t* keys, const void* vals, fks_val_type val_type,
                                 uint64_t n, uint64_t seed, const fks_build_opts* opts,
                                 uint64_t* desc_out, void* slots_out, uint64_t slot_capacity,
                                 fks_map_info_t* h_info, fks_stream_t stream);

/* ------------------------------------------------------------------ search-based map
 * The comparison point of the paper's evaluation (mk_arraymap, Sec. 3.4;
 * Table 1 "binary search"): the pairs sorted by key (here an LSD radix
 * sort, stable, 8 passes of 8 bits) and lookups by binary search.
 * fks_sortmap_build does not block; keys are assumed distinct (a lookup of
 * a repeated key returns the value of its first sorted occurrence). */
fks_status fks_sortmap_build(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                             const fks_allocator* alloc, fks_stream_t stream, fks_sortmap_t* out);
fks_status fks_sortmap_lookup(fks_sortmap_t map, const uint64_t* q, uint64_t nq, void* out_vals,
                              uint8_t* out_found, int64_t absent, fks_stream_t stream);
/* fks_eytzmap_build -- the paper's locality variant of the same map (Sec. 3.4;
 * the third row of its Table 1): the sorted pairs stored in Eytzinger order,
 * the implicit binary search tree level by level (node k, 1-based, has
 * children 2k and 2k + 1), so the top levels a search visits first are
 * contiguous and stay cached.  The result is an fks_sortmap_t: lookups go
 * through fks_sortmap_lookup, which descends the tree. */
fks_status fks_eytzmap_build(const uint64_t* keys, const void* vals, fks_val_type val_type, uint64_t n,
                             const fks_allocator* alloc, fks_stream_t stream, fks_sortmap_t* out);
/* keys and their values (int64) to host memory in storage order: sorted, or
 * Eytzinger order (nodes 1..n) for maps from fks_eytzmap_build; synchronises */
fks_status fks_sortmap_export(fks_sortmap_t map, uint64_t* h_keys, int64_t* h_vals, fks_stream_t stream);
void fks_sortmap_destroy(fks_sortmap_t map);

/* ------------------------------------------------------------------ serving
 * A request loop over resident maps: build and lookup requests are
 * submitted as they arrive (from any thread) and complete asynchronously.
 *   - Builds are admitted in arrival order against a device-memory budget:
 *     least-recently-used resident maps are evicted until the new map fits
 *     (accounted size 72 B/key for uint64 maps, 136 B/key + context bytes
 *     for string maps).  An evicted map that still has lookups in flight is
 *     freed when they finish.  Builds run on worker threads with their own
 *     streams.
 *   - FKS_SERVE_BATCHED (continuous batching): every lookup whose map is
 *     ready joins the next coalesced launch; lookups that arrive while a
 *     batch runs go into the following one.  A lookup of a map still being
 *     built waits for that build.
 *   - FKS_SERVE_PER_CALL: one request at a time in arrival order, each as
 *     its own launch followed by a synchronisation (the comparison point).
 * Latency of a request = submission to the moment the server observed its
 * completion on the host.  All device pointers of a request must stay valid
 * until it completes; results are written to the request's own buffers. */
typedef struct fks_server* fks_server_t;
typedef enum { FKS_SERVE_BATCHED = 0, FKS_SERVE_PER_CALL = 1 } fks_serve_mode;
typedef enum { FKS_REQ_BUILD = 0, FKS_REQ_LOOKUP = 1 } fks_request_type;

typedef struct {
  size_t struct_size;        /* sizeof(fks_server_opts)                     */
  uint64_t memory_budget;    /* bytes of resident maps (accounted sizes)    */
  uint32_t max_maps;         /* map ids are 0 .. max_maps-1                 */
  uint32_t mode;             /* fks_serve_mode                              */
  uint32_t build_workers;    /* threads running builds (default 2)          */
  uint32_t max_batch_requests; /* lookups per coalesced launch (default 4096) */
  uint32_t max_inflight_batches; /* coalesced launches in flight (default 2) */
} fks_server_opts;

typedef struct {
  size_t struct_size;        /* sizeof(fks_request)                          */
  uint32_t type;             /* fks_request_type                            */
  uint32_t map_id;           /* build: id the new map takes; lookup: target */
  uint32_t key_kind;         /* fks_key_kind                                */
  uint32_t val_type;         /* fks_val_type (build)                        */
  /* build: uint64 keys, or ctx/offs (ctx_bytes = offs[n]); device memory  */
  const uint64_t* keys;
  const uint8_t* ctx;
  const int64_t* offs;
  uint64_t ctx_bytes;
  const void* vals;
  uint64_t n;
  uint64_t seed;
  /* lookup: q (uint64) or qctx/qoffs (strings), outputs; device memory     */
  const uint64_t* q;
  const uint8_t* qctx;
  const int64_t* qoffs;
  uint64_t nq;
  void* out_vals;            /* nullable; int32/int64 per the map           */
  uint8_t* out_found;        /* nullable                                    */
  int64_t absent;
} fks_request;

typedef struct {
  uint64_t submitted, completed, builds, lookups, queries;
  uint64_t batches;          /* lookup launches                             */
  uint64_t evictions, rejected;
  uint64_t resident_bytes, peak_resident_bytes;
  double span_s;             /* first submission to last completion         */
  double p50_us, p99_us, p999_us;              /* all requests              */
  double lookup_p50_us, lookup_p99_us, build_p50_us, build_p99_us;
} fks_server_stats_t;

fks_status fks_server_create(const fks_server_opts* opts, fks_server_t* out);
/* non-blocking; h_ticket identifies the request for fks_server_wait */
fks_status fks_server_submit(fks_server_t srv, const fks_request* req, uint64_t* h_ticket);
/* load generator: submits reqs[i] at h_arrival_us[i] microseconds after the
 * call (spinning on the host clock); returns once all are submitted */
fks_status fks_server_replay(fks_server_t srv, const fks_request* reqs, const double* h_arrival_us,
                             uint64_t count, uint64_t* h_tickets);
/* blocks until the request completed; its status and latency (us) */
fks_status fks_server_wait(fks_server_t srv, uint64_t ticket, fks_status* h_result, double* h_latency_us);
/* blocks until every submitted request completed */
fks_status fks_server_drain(fks_server_t srv);
fks_status fks_server_stats(fks_server_t srv, fks_server_stats_t* h_out);
/* a borrowed handle of a resident map (NULL if not resident); waits for
 * every submitted request first -- call it while no client submits */
fks_map_t fks_server_map(fks_server_t srv, uint32_t map_id);
void fks_server_destroy(fks_server_t srv);

/* ------------------------------------------------------------------ host buffers
 * The end-to-end path of a caller whose data lives in host memory; not in
 * the paper (whose arrays live on the device).  Pinned buffers give
 * asynchronous copies that overlap; pageable buffers work at the speed of
 * the driver's staged copies.
 *
 * fks_build_u64_host -- fks_build_u64 over host keys and values: they are
 * uploaded to device memory (stream-ordered pool), the map is built from the
 * copies, which are freed afterwards.  Arguments as for fks_build_u64.
 *
 * fks_lookup_u64_host -- fks_lookup_u64 over host needles and results:
 *   h_q       uint64[nq] needles (host)
 *   h_out     int32[nq] / int64[nq] per the map's val_type (host), or NULL
 *   h_found   uint8[nq] (host), or NULL
 * The needles go through the device in chunks of 2^23: the upload of one
 * chunk, the lookup of the previous one (on `stream`) and the download of
 * the results before it overlap (three device buffers of the stream-ordered
 * pool, two streams of the calling thread's own).  Blocks until the results
 * are in host memory.  uint64 maps only (FKS_ERR_INVALID_ARG otherwise). */
fks_status fks_build_u64_host(const uint64_t* h_keys, const void* h_vals, fks_val_type val_type, uint64_t n,
                              uint64_t seed, const fks_build_opts* opts, const fks_allocator* alloc,
                              fks_stream_t stream, fks_map_t* out);
fks_status fks_lookup_u64_host(fks_map_t map, const uint64_t* h_q, uint64_t nq, void* h_out, uint8_t* h_found,
                               int64_t absent, fks_stream_t stream);

/* ------------------------------------------------------------------ tables
 * fks_map_info -- sizes and build statistics (host struct). */
fks_status fks_map_info(fks_map_t map, fks_map_info_t* h_out);

/* fks_map_export -- copy the tables to host memory (synchronises `stream`):
 *   h_desc   uint64[buckets] bucket descriptors (info.buckets of them): slot offset (bits 0..31) | s
 *            (bits 32..51) | level-two attempt (bits 52..63)
 *   h_slots  S slots: uint64 maps {key, value} (16 B); string maps {fp,
 *            offset | length << 40, value, 0} (32 B); empty slots hold the
 *            bucket's lowest occupied slot with value -1
 *   h_ctx    string maps: the map's context (context_bytes); else ignored
 * Any pointer may be NULL. */
fks_status fks_map_export(fks_map_t map, uint64_t* h_desc, void* h_slots, uint8_t* h_ctx,
                          fks_stream_t stream);

/* fks_map_export_records -- copy a map's inline-singleton records to host
 * memory (synchronises `stream`): h_rec uint64[2 * buckets], bucket b at
 * h_rec[2b], h_rec[2b + 1] as described at fks_build_opts.  A map built
 * without the option: FKS_ERR_INVALID_ARG. */
fks_status fks_map_export_records(fks_map_t map, uint64_t* h_rec, fks_stream_t stream);

/* fks_map_import -- a map from tables that fks_map_export wrote (checkpoint /
 * resume: export, store the buffers and the info anywhere, import in another
 * process or on another GPU).  Not in the paper, whose maps live only as long
 * as the program that built them.
 *   h_info   what fks_map_info returned for the exported map: n, seed, round,
 *            slots, slot_capacity, buckets, keys_per_bucket, key_kind,
 *            val_type, context_bytes and the statistics are taken from it
 *   h_desc   uint64[buckets], h_slots (slots of 16 or 32 bytes), h_ctx
 *            uint8[context_bytes] for string maps: host memory, as exported
 * The descriptors are checked against the metadata before anything is
 * uploaded (every non-empty bucket's s^2 slots in order inside the slot
 * array, sum s = n, sum s^2 = slots); a mismatch returns FKS_ERR_INVALID_ARG.
 * The map answers lookups exactly as the exported one (the level-one and
 * fingerprint constants are re-derived from seed and round).  Inline-singleton
 * records are not part of a checkpoint: a map exported with them is imported
 * without (info.inline_singletons = 0) and answers through its descriptors
 * and slots, with the same results.  Blocks until the upload is done; the
 * handle is freed by fks_map_destroy. */
fks_status fks_map_import(const fks_map_info_t* h_info, const uint64_t* h_desc, const void* h_slots,
                          const uint8_t* h_ctx, const fks_allocator* alloc, fks_stream_t stream, fks_map_t* out);

void fks_map_destroy(fks_map_t map);
void fks_mapset_destroy(fks_mapset_t set);

const char* fks_status_str(fks_status status);
const char* fks_last_error(void);

/* ------------------------------------------------------------------ metrics */
void fks_profile_enable(int on);                       /* per calling thread */
fks_status fks_last_build_profile(fks_build_profile* h_out);
uint64_t fks_kernel_launches(void); /* kernels launched by this library so far */

#ifdef __cplusplus
}
#endif
#endif /* FKS_H_ */
