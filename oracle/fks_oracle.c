/*
 * fks_oracle.c -- plain, slow, single-threaded CPU oracle for the FKS
 * two-level static hash map (Due, Elsman, Henriksen, "Towards Efficient Hash
 * Maps in Functional Array Languages", arXiv 2508.11443).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant table with
 * the CUDA library; every function below is written out independently from
 * the paper's definitions (and, where the paper is silent, from the readings
 * listed at the top of each function).
 *
 * What it computes, in the paper's order:
 *   - the hash-set construction (const, consts) and the function
 *       h k = offsets[g k] + (Hash consts[g k] k  mod  shape[g k]),
 *       g k = Hash const k mod n,  shape = (s^2 of Hist n (g K)),
 *       offsets = Presum shape                          (Sec. 2.2)
 *   - make_1: one random const, hashes mod n, Hist, Groupby, make_2 per
 *     group                                             (Sec. 2.3, level one)
 *   - make_2: draw constants until no slot of the m^2 range is hit twice
 *                                                      (Sec. 2.3, level two)
 *   - placement of every key at h k, the remaining slots filled with a key of
 *     K, values in an accompanying array, and the membership test
 *     arr[h a] = a                                      (Sec. 2.2)
 *   - keys that are byte slices of a context array      (Sec. 3.1, 3.3)
 *
 * Readings of points the paper leaves open (each also stated in the design
 * notes of the repository):
 *   R1  Random/Hash (Sec. 2.1 asks only for a universal family): constants
 *       are outputs of the splitmix64 generator (Steele, Lea, Flood 2014) at a
 *       counter built from (round, tag, attempt, index); Hash is the vector
 *       multiply-shift of Thorup ("High speed hashing for integers and
 *       strings", 2015), strongly universal into 32 bits:
 *         H(m0,m1,add; k) = (m0*lo32(k) + m1*hi32(k) + add  mod 2^64) >> 32
 *   R2  "mod m" is replaced by the multiply-high range reduction
 *       (H * m) >> 32, which is < m for every m <= 2^32 (Lemire 2019).
 *   R3  Presum is exclusive (needed for h k in [0, S), Sec. 2.2 property 1).
 *   R4  Space bound: if S = sum s^2 > bound_factor * n the level-one
 *       constant is redrawn (next round).  The paper only states E[S] = O(n).
 *   R5  make_2 retries forever in the paper; here: attempts 0..attempt_cap-1,
 *       at attempt 64 an exact test for equal keys in the bucket
 *       (duplicates -> DUPLICATE; equal fingerprints of different strings ->
 *       next round), after attempt_cap failures -> next round.  After
 *       round_cap rounds an exact global duplicate test decides between
 *       DUPLICATE and BUILD_FAILED.
 *   R6  An empty bucket (s = 0) means "absent" with no second probe.
 *   R7  The filler key of an empty slot is the key at the lowest occupied
 *       slot of the same bucket; its value is all ones (-1).
 *   R8  Byte-string keys hash through a 61-bit polynomial fingerprint
 *       (Carter-Wegman polynomial hashing mod the Mersenne prime 2^61-1) of
 *       [length, little-endian 32-bit words...]; the base is drawn per round.
 *
 * Table layout produced (the device library writes the same bytes):
 *   desc[b]  = slot_off (bits 0..31) | s (bits 32..51) | attempt (bits 52..63)
 *   u64 slot = { key, value }                       2 x uint64
 *   str slot = { fp, off | len << 40, value, 0 }    4 x uint64
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- status */
enum {
  OR_OK = 0,
  OR_INVALID_ARG = 1,
  OR_DUPLICATE_KEY = 2,
  OR_OUT_OF_MEMORY = 3,
  OR_BUILD_FAILED = 4
};

/* ------------------------------------------------- R1: splitmix64 stream */
/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014): state advances by the odd
 * constant gamma = 2^64 / golden ratio; each output is the "mix13" finaliser
 * of the state.  The i-th output (i = 0, 1, ...) for a seed is therefore
 * mix(seed + (i + 1) * gamma). */
static uint64_t or_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t seed, uint64_t i) {
  return or_mix(seed + (i + 1u) * 0x9E3779B97F4A7C15ULL);
}

#define OR_TAG_L1 0xFFFFFFFFull /* level-one constant        */
#define OR_TAG_FP 0xFFFFFFFEull /* string fingerprint base   */

/* counter = round (bits 48..63) | tag (bits 14..45) | attempt (bits 2..13)
 *           | constant index (bits 0..1) */
static uint64_t or_counter(uint32_t round, uint64_t tag, uint32_t attempt, uint32_t j) {
  return ((uint64_t)round << 48) | (tag << 14) | ((uint64_t)attempt << 2) | (uint64_t)j;
}

/* Random : () -> [3]Int, made deterministic by its coordinates. */
void or_derive(uint64_t seed, uint32_t round, uint64_t tag, uint32_t attempt, uint64_t out[3]) {
  for (uint32_t j = 0; j < 3; ++j) out[j] = or_splitmix64(seed, or_counter(round, tag, attempt, j));
}

/* Hash : [3]Int -> u64 -> 32-bit value (R1). */
uint32_t or_hash(const uint64_t c[3], uint64_t k) {
  uint64_t lo = k & 0xFFFFFFFFull, hi = k >> 32;
  uint64_t acc = c[0] * lo + c[1] * hi + c[2]; /* wraps mod 2^64 */
  return (uint32_t)(acc >> 32);
}

/* range reduction onto [0, m), m <= 2^32 (R2). */
uint64_t or_reduce(uint32_t h, uint64_t m) {
  return ((uint64_t)h * m) >> 32;
}

/* --------------------------------------- R8: fingerprint of a byte string */
#define OR_P61 ((1ull << 61) - 1)

static uint64_t or_mulmod61(uint64_t a, uint64_t b) {
  unsigned __int128 p = (unsigned __int128)a * b;
  return (uint64_t)(p % OR_P61);
}

uint64_t or_fp_base(uint64_t seed, uint32_t round) {
  uint64_t c[3];
  or_derive(seed, round, OR_TAG_FP, 0, c);
  return c[0] % (OR_P61 - 1) + 1; /* in [1, p-1] */
}

/* Horner over the sequence [len, w_0, ..., w_{m-1}], w_t the little-endian
 * 32-bit word of bytes 4t..4t+3 (zero padded past the end). */
uint64_t or_fingerprint(const uint8_t* bytes, uint64_t len, uint64_t base) {
  uint64_t h = len % OR_P61;
  for (uint64_t t = 0; t < len; t += 4) {
    uint64_t w = 0;
    for (uint64_t q = 0; q < 4 && t + q < len; ++q) w |= (uint64_t)bytes[t + q] << (8 * q);
    h = (or_mulmod61(h, base) + w) % OR_P61;
  }
  return h;
}

/* ------------------------------------------------------------ map model */
typedef struct {
  uint64_t n;          /* keys                                  */
  uint64_t seed;
  uint32_t round;      /* level-one round that succeeded        */
  uint32_t max_s;      /* largest bucket                        */
  uint64_t S;          /* slots = sum s^2                       */
  uint64_t c1[3];      /* level-one constants                   */
  uint64_t attempts_sum;   /* sum over non-empty buckets of attempt */
  uint64_t nonempty;
  uint32_t rounds_used;    /* rounds tried (round + 1 on success)   */
  uint32_t max_attempt;
  uint64_t nb;             /* level-one buckets = descriptors       */
} or_info;

typedef struct {
  uint32_t bound_factor;   /* default 2 * (1 + keys_per_bucket), i.e. 4 */
  uint32_t round_cap;      /* default 32   */
  uint32_t attempt_cap;    /* default 4095 */
  uint32_t reject_attempts;/* test hook: attempts below this count as failures */
  uint32_t keys_per_bucket;/* lambda: nb = ceil(n / lambda) level-one buckets (default 1) */
} or_opts;

/* Level-one bucket count.  The paper takes one bucket per key (g k = Hash
 * const k mod n, Sec. 2.3).  The bucket-count variant takes nb = ceil(n /
 * lambda) buckets; the FKS argument is unchanged: E[sum s^2] = n + n (n - 1)
 * / nb < (1 + lambda) n, so a bound of 2 (1 + lambda) n holds with
 * probability at least 1/2 per round (Markov), as 4n does for lambda = 1. */
static uint64_t or_buckets(uint64_t n, uint32_t lambda) { return (n + lambda - 1) / lambda; }

#define OR_DUP_CHECK_AT 64u

/* Key access: the hashed key (u64 key or fingerprint) and an exact equality
 * of two members (u64: equal keys; strings: equal byte sequences). */
typedef struct {
  const uint64_t* hkey;     /* hashed key per member          */
  const uint8_t* ctx;       /* strings: context, else NULL    */
  const int64_t* offs;      /* strings: offsets[n+1]          */
} or_keys;

static int or_same_member(const or_keys* K, uint64_t i, uint64_t j) {
  if (!K->ctx) return K->hkey[i] == K->hkey[j];
  int64_t li = K->offs[i + 1] - K->offs[i], lj = K->offs[j + 1] - K->offs[j];
  if (li != lj) return 0;
  return memcmp(K->ctx + K->offs[i], K->ctx + K->offs[j], (size_t)li) == 0;
}

static int or_cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : x > y;
}

/* collision (Sec. 2.3): Or (Map (> 1) (Hist m^2 hs)).  Written literally with
 * a histogram when m^2 is small, else as "two equal values after sorting",
 * which is the same predicate. */
static int or_collision(const uint64_t* hs, uint64_t m, uint64_t range) {
  int hit = 0;
  if (range <= (1u << 22)) {
    uint32_t* hist = (uint32_t*)calloc(range, sizeof(uint32_t));
    for (uint64_t i = 0; i < m; ++i) hist[hs[i]] += 1;
    for (uint64_t x = 0; x < range; ++x) hit |= hist[x] > 1;
    free(hist);
  } else {
    uint64_t* c = (uint64_t*)malloc(m * sizeof(uint64_t));
    memcpy(c, hs, m * sizeof(uint64_t));
    qsort(c, m, sizeof(uint64_t), or_cmp_u64);
    for (uint64_t i = 1; i < m; ++i) hit |= c[i] == c[i - 1];
    free(c);
  }
  return hit;
}

enum { L2_OK = 0, L2_DUP = 1, L2_NEXT_ROUND = 2 };

/* make_2 (Sec. 2.3, level two) for bucket b whose members are idx[0..m).
 * Returns the first attempt whose constants give no collision. */
static int or_make2(const or_keys* K, const uint64_t* idx, uint64_t m, uint64_t seed,
                    uint32_t round, uint64_t b, const or_opts* o, uint32_t* attempt_out) {
  uint64_t range = m * m;
  uint64_t* hs = (uint64_t*)malloc(m * sizeof(uint64_t));
  int res = L2_NEXT_ROUND;
  for (uint32_t a = 0; a < o->attempt_cap; ++a) {
    if (a == OR_DUP_CHECK_AT) {
      int equal_hkey = 0, dup = 0;
      for (uint64_t x = 0; x < m; ++x)
        for (uint64_t y = x + 1; y < m; ++y)
          if (K->hkey[idx[x]] == K->hkey[idx[y]]) {
            equal_hkey = 1;
            dup |= or_same_member(K, idx[x], idx[y]);
          }
      if (dup) { res = L2_DUP; break; }
      if (equal_hkey) { res = L2_NEXT_ROUND; break; }
    }
    uint64_t cs[3];
    or_derive(seed, round, b, a, cs);
    for (uint64_t x = 0; x < m; ++x) hs[x] = or_reduce(or_hash(cs, K->hkey[idx[x]]), range);
    if (a < o->reject_attempts) continue;
    if (!or_collision(hs, m, range)) { *attempt_out = a; res = L2_OK; break; }
  }
  free(hs);
  return res;
}

/* exact global duplicate test after round_cap failed rounds (R5). */
static const or_keys* g_sort_keys; /* qsort has no context argument in C99 */
static int or_cmp_idx(const void* a, const void* b) {
  uint64_t i = *(const uint64_t*)a, j = *(const uint64_t*)b;
  const or_keys* K = g_sort_keys;
  if (!K->ctx) return K->hkey[i] < K->hkey[j] ? -1 : K->hkey[i] > K->hkey[j];
  int64_t li = K->offs[i + 1] - K->offs[i], lj = K->offs[j + 1] - K->offs[j];
  if (li != lj) return li < lj ? -1 : 1;
  return memcmp(K->ctx + K->offs[i], K->ctx + K->offs[j], (size_t)li);
}

static int or_has_duplicates(const or_keys* K, uint64_t n) {
  uint64_t* idx = (uint64_t*)malloc(n * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  g_sort_keys = K;
  qsort(idx, n, sizeof(uint64_t), or_cmp_idx);
  int dup = 0;
  for (uint64_t i = 1; i < n && !dup; ++i) dup = or_same_member(K, idx[i - 1], idx[i]);
  free(idx);
  return dup;
}

/* make_1 (Sec. 2.3, level one) followed by placement (Sec. 2.2).
 *   slot_words = 2 (u64 keys) or 4 (strings); slots[] holds slot_cap slots.
 *   payload(i, slot) writes the member's words into its slot. */
static int or_build_common(const or_keys* K, const int64_t* vals, uint64_t n, uint64_t seed,
                           const or_opts* o, uint64_t* desc, uint64_t* slots, uint64_t slot_cap,
                           uint32_t slot_words, or_info* info, uint64_t* hkey_buf,
                           const uint8_t* ctx, const int64_t* offs) {
  const uint64_t nb = or_buckets(n, o->keys_per_bucket);
  uint64_t* hashes = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* shape = (uint64_t*)malloc(nb * sizeof(uint64_t));
  uint64_t* gstart = (uint64_t*)malloc((nb + 1) * sizeof(uint64_t));
  uint64_t* grouped = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* cursor = (uint64_t*)malloc(nb * sizeof(uint64_t));
  uint32_t* attempt = (uint32_t*)malloc(nb * sizeof(uint32_t));
  int status = OR_BUILD_FAILED;
  (void)slot_cap; /* checked by the callers against bound_factor * n */
  memset(info, 0, sizeof(*info));
  info->n = n;
  info->seed = seed;
  info->nb = nb;

  for (uint32_t r = 0; r < o->round_cap; ++r) {
    info->rounds_used = r + 1;
    if (ctx) { /* R8: the fingerprint base is redrawn every round */
      uint64_t base = or_fp_base(seed, r);
      for (uint64_t i = 0; i < n; ++i)
        hkey_buf[i] = or_fingerprint(ctx + offs[i], (uint64_t)(offs[i + 1] - offs[i]), base);
    }
    /* const = Random (); hashes = Map ((mod nb) . Hash const) keys */
    uint64_t c1[3];
    or_derive(seed, r, OR_TAG_L1, 0, c1);
    for (uint64_t i = 0; i < n; ++i) hashes[i] = or_reduce(or_hash(c1, K->hkey[i]), nb);
    /* shape = Hist nb hashes (Rep n 1) */
    memset(shape, 0, nb * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i) shape[hashes[i]] += 1;
    /* R4: the space bound (bound_factor * n, n = keys) */
    uint64_t S = 0;
    for (uint64_t b = 0; b < nb; ++b) S += shape[b] * shape[b];
    if (S > (uint64_t)o->bound_factor * n) continue;
    /* Groupby nb hashes keys (stable counting sort; order is irrelevant) */
    gstart[0] = 0;
    for (uint64_t b = 0; b < nb; ++b) gstart[b + 1] = gstart[b] + shape[b];
    for (uint64_t b = 0; b < nb; ++b) cursor[b] = gstart[b];
    for (uint64_t i = 0; i < n; ++i) grouped[cursor[hashes[i]]++] = i;
    /* consts = Map make_2 (groups) */
    int any_dup = 0, any_next = 0;
    uint64_t att_sum = 0, nonempty = 0;
    uint32_t max_att = 0, max_s = 0;
    for (uint64_t b = 0; b < nb; ++b) {
      attempt[b] = 0;
      if (shape[b] == 0) continue;
      nonempty += 1;
      if (shape[b] > max_s) max_s = (uint32_t)shape[b];
      if (shape[b] == 1) continue; /* one key never collides: attempt 0 */
      uint32_t a = 0;
      int res = or_make2(K, grouped + gstart[b], shape[b], seed, r, b, o, &a);
      if (res == L2_DUP) any_dup = 1;
      else if (res == L2_NEXT_ROUND) any_next = 1;
      else {
        attempt[b] = a;
        att_sum += a;
        if (a > max_att) max_att = a;
      }
    }
    if (any_dup) { status = OR_DUPLICATE_KEY; goto done; }
    if (any_next) continue;

    /* offsets = Presum shape^2 (exclusive, R3); descriptors */
    uint64_t off = 0;
    for (uint64_t b = 0; b < nb; ++b) {
      desc[b] = off | (shape[b] << 32) | ((uint64_t)attempt[b] << 52);
      off += shape[b] * shape[b];
    }
    /* place every key at h k */
    uint8_t* used = (uint8_t*)calloc(S ? S : 1, 1);
    for (uint64_t i = 0; i < n; ++i) {
      uint64_t b = hashes[i], s = shape[b];
      uint64_t cs[3];
      or_derive(seed, r, b, attempt[b], cs);
      uint64_t j = (desc[b] & 0xFFFFFFFFull) + or_reduce(or_hash(cs, K->hkey[i]), s * s);
      uint64_t* sl = slots + j * slot_words;
      used[j] = 1;
      if (slot_words == 2) {
        sl[0] = K->hkey[i];
        sl[1] = (uint64_t)vals[i];
      } else {
        sl[0] = K->hkey[i];
        sl[1] = (uint64_t)offs[i] | ((uint64_t)(offs[i + 1] - offs[i]) << 40);
        sl[2] = (uint64_t)vals[i];
        sl[3] = 0;
      }
    }
    /* R7: fill the rest of each bucket's range with its lowest occupied slot */
    for (uint64_t b = 0; b < nb; ++b) {
      uint64_t s = shape[b];
      if (s < 2) continue;
      uint64_t lo = desc[b] & 0xFFFFFFFFull, hi = lo + s * s, first = hi;
      for (uint64_t j = lo; j < hi; ++j)
        if (used[j]) { first = j; break; }
      for (uint64_t j = lo; j < hi; ++j) {
        if (used[j]) continue;
        uint64_t* sl = slots + j * slot_words;
        const uint64_t* src = slots + first * slot_words;
        if (slot_words == 2) {
          sl[0] = src[0];
          sl[1] = ~0ull;
        } else {
          sl[0] = src[0];
          sl[1] = src[1];
          sl[2] = ~0ull;
          sl[3] = 0;
        }
      }
    }
    free(used);
    info->round = r;
    info->S = S;
    info->max_s = max_s;
    memcpy(info->c1, c1, sizeof(c1));
    info->attempts_sum = att_sum;
    info->nonempty = nonempty;
    info->max_attempt = max_att;
    status = OR_OK;
    goto done;
  }
  /* R5: every round failed; decide between duplicates and plain failure */
  status = or_has_duplicates(K, n) ? OR_DUPLICATE_KEY : OR_BUILD_FAILED;
done:
  free(hashes); free(shape); free(gstart); free(grouped); free(cursor); free(attempt);
  return status;
}

static void or_default_opts(or_opts* o, const or_opts* in) {
  o->keys_per_bucket = (in && in->keys_per_bucket) ? in->keys_per_bucket : 1;
  o->bound_factor = 2 * (1 + o->keys_per_bucket);
  o->round_cap = 32;
  o->attempt_cap = 4095;
  o->reject_attempts = 0;
  if (in) {
    if (in->bound_factor) o->bound_factor = in->bound_factor;
    if (in->round_cap) o->round_cap = in->round_cap;
    if (in->attempt_cap) o->attempt_cap = in->attempt_cap;
    o->reject_attempts = in->reject_attempts;
  }
}

/* Sizes every build accepts: n keys below 2^30, lambda in 1 .. 16, and a
 * slot range whose offsets fit the descriptor's 32-bit field. */
static int or_sizes_ok(const or_opts* o, uint64_t n, uint64_t slot_cap) {
  if (n == 0 || n >= (1ull << 30)) return 0;
  if (o->keys_per_bucket < 1 || o->keys_per_bucket > 16) return 0;
  if ((uint64_t)o->bound_factor * n > 0xFFFFFFFFull) return 0;
  return slot_cap >= (uint64_t)o->bound_factor * n;
}

/* Build over uint64 keys.  desc[nb], slots[2 * slot_cap] (uint64 words),
 * nb = ceil(n / keys_per_bucket). */
int or_build_u64(const uint64_t* keys, const int64_t* vals, uint64_t n, uint64_t seed,
                 const or_opts* opts, uint64_t* desc, uint64_t* slots, uint64_t slot_cap,
                 or_info* info) {
  or_opts o;
  or_default_opts(&o, opts);
  if (!or_sizes_ok(&o, n, slot_cap)) return OR_INVALID_ARG;
  or_keys K = {keys, NULL, NULL};
  return or_build_common(&K, vals, n, seed, &o, desc, slots, slot_cap, 2, info, NULL, NULL, NULL);
}

/* Build over byte-string keys: key i is ctx[offs[i] .. offs[i+1]).
 * desc[nb], slots[4 * slot_cap] (uint64 words). */
int or_build_bytes(const uint8_t* ctx, const int64_t* offs, const int64_t* vals, uint64_t n,
                   uint64_t seed, const or_opts* opts, uint64_t* desc, uint64_t* slots,
                   uint64_t slot_cap, or_info* info) {
  or_opts o;
  or_default_opts(&o, opts);
  if (!or_sizes_ok(&o, n, slot_cap)) return OR_INVALID_ARG;
  for (uint64_t i = 0; i < n; ++i) {
    int64_t len = offs[i + 1] - offs[i];
    if (offs[i] < 0 || len < 0 || len >= (1ll << 24) || offs[i + 1] >= (1ll << 40))
      return OR_INVALID_ARG;
  }
  uint64_t* fps = (uint64_t*)malloc(n * sizeof(uint64_t));
  or_keys K = {fps, ctx, offs};
  int st = or_build_common(&K, vals, n, seed, &o, desc, slots, slot_cap, 4, info, fps, ctx, offs);
  free(fps);
  return st;
}

/* from_array (Sec. 3.2): the constructor that accepts duplicate keys.  The
 * paper leaves the surviving pair unspecified; reading: the first occurrence
 * in input order wins.  keep[e] = 1 iff no earlier element of the same
 * segment has an equal key (u64: equal words; strings: equal bytes).  seg
 * holds m + 1 segment offsets (NULL: one segment).  Written as its
 * definition: sort the indices by (segment, key, index) and keep the first
 * index of every run of equal (segment, key). */
static const uint64_t* g_dd_keys;
static const uint8_t* g_dd_ctx;
static const int64_t* g_dd_offs;
static const uint32_t* g_dd_segid;
static int or_cmp_dedup(const void* a, const void* b) {
  uint64_t i = *(const uint64_t*)a, j = *(const uint64_t*)b;
  if (g_dd_segid[i] != g_dd_segid[j]) return g_dd_segid[i] < g_dd_segid[j] ? -1 : 1;
  int c = 0;
  if (g_dd_keys) {
    c = g_dd_keys[i] < g_dd_keys[j] ? -1 : g_dd_keys[i] > g_dd_keys[j];
  } else {
    int64_t li = g_dd_offs[i + 1] - g_dd_offs[i], lj = g_dd_offs[j + 1] - g_dd_offs[j];
    if (li != lj) c = li < lj ? -1 : 1;
    else c = memcmp(g_dd_ctx + g_dd_offs[i], g_dd_ctx + g_dd_offs[j], (size_t)li);
  }
  if (c) return c;
  return i < j ? -1 : i > j;
}

static int or_same_key(uint64_t i, uint64_t j) {
  if (g_dd_segid[i] != g_dd_segid[j]) return 0;
  if (g_dd_keys) return g_dd_keys[i] == g_dd_keys[j];
  int64_t li = g_dd_offs[i + 1] - g_dd_offs[i], lj = g_dd_offs[j + 1] - g_dd_offs[j];
  return li == lj && memcmp(g_dd_ctx + g_dd_offs[i], g_dd_ctx + g_dd_offs[j], (size_t)li) == 0;
}

/* keys (u64) or ctx/offs (strings); returns the number of kept elements. */
uint64_t or_dedup(const uint64_t* keys, const uint8_t* ctx, const int64_t* offs, uint64_t u,
                  const int64_t* seg, uint32_t m, uint8_t* keep) {
  uint64_t* idx = (uint64_t*)malloc((u ? u : 1) * sizeof(uint64_t));
  uint32_t* segid = (uint32_t*)malloc((u ? u : 1) * sizeof(uint32_t));
  for (uint64_t e = 0; e < u; ++e) idx[e] = e;
  if (seg) {
    for (uint32_t j = 0; j < m; ++j)
      for (int64_t e = seg[j]; e < seg[j + 1]; ++e) segid[e] = j;
  } else {
    for (uint64_t e = 0; e < u; ++e) segid[e] = 0;
  }
  g_dd_keys = keys;
  g_dd_ctx = ctx;
  g_dd_offs = offs;
  g_dd_segid = segid;
  qsort(idx, u, sizeof(uint64_t), or_cmp_dedup);
  uint64_t kept = 0;
  for (uint64_t r = 0; r < u; ++r) {
    int first = r == 0 || !or_same_key(idx[r - 1], idx[r]);
    keep[idx[r]] = (uint8_t)first;
    kept += (uint64_t)first;
  }
  free(idx);
  free(segid);
  return kept;
}

/* Lookup (Sec. 2.2 membership test; Sec. 3.2 lookup -> opt v).
 * nb = the map's level-one buckets (n for the paper's construction).
 * found[i] = 1 and out[i] = value for members, found[i] = 0 and
 * out[i] = absent otherwise. */
void or_lookup_u64(const uint64_t* desc, const uint64_t* slots, uint64_t nb, uint64_t seed,
                   uint32_t round, const uint64_t* q, uint64_t nq, int64_t absent,
                   int64_t* out, uint8_t* found) {
  uint64_t c1[3];
  or_derive(seed, round, OR_TAG_L1, 0, c1);
  for (uint64_t i = 0; i < nq; ++i) {
    uint64_t b = or_reduce(or_hash(c1, q[i]), nb);
    uint64_t d = desc[b], s = (d >> 32) & 0xFFFFF;
    int hit = 0;
    int64_t v = absent;
    if (s > 0) { /* R6 */
      uint64_t cs[3];
      or_derive(seed, round, b, (uint32_t)(d >> 52), cs);
      uint64_t j = (d & 0xFFFFFFFFull) + or_reduce(or_hash(cs, q[i]), s * s);
      if (slots[2 * j] == q[i]) { hit = 1; v = (int64_t)slots[2 * j + 1]; }
    }
    if (out) out[i] = v;
    if (found) found[i] = (uint8_t)hit;
  }
}

/* Lookup of byte-string needles: needle i is qctx[qoffs[i] .. qoffs[i+1]);
 * the map's own context is mctx (the needle context may differ, Sec. 3.1). */
void or_lookup_bytes(const uint64_t* desc, const uint64_t* slots, const uint8_t* mctx, uint64_t nb,
                     uint64_t seed, uint32_t round, const uint8_t* qctx, const int64_t* qoffs,
                     uint64_t nq, int64_t absent, int64_t* out, uint8_t* found) {
  uint64_t c1[3];
  or_derive(seed, round, OR_TAG_L1, 0, c1);
  uint64_t base = or_fp_base(seed, round);
  for (uint64_t i = 0; i < nq; ++i) {
    uint64_t len = (uint64_t)(qoffs[i + 1] - qoffs[i]);
    uint64_t fp = or_fingerprint(qctx + qoffs[i], len, base);
    uint64_t b = or_reduce(or_hash(c1, fp), nb);
    uint64_t d = desc[b], s = (d >> 32) & 0xFFFFF;
    int hit = 0;
    int64_t v = absent;
    if (s > 0) {
      uint64_t cs[3];
      or_derive(seed, round, b, (uint32_t)(d >> 52), cs);
      uint64_t j = (d & 0xFFFFFFFFull) + or_reduce(or_hash(cs, fp), s * s);
      const uint64_t* sl = slots + 4 * j;
      uint64_t off = sl[1] & ((1ull << 40) - 1), slen = sl[1] >> 40;
      if (sl[0] == fp && slen == len && memcmp(mctx + off, qctx + qoffs[i], len) == 0) {
        hit = 1;
        v = (int64_t)sl[2];
      }
    }
    if (out) out[i] = v;
    if (found) found[i] = (uint8_t)hit;
  }
}

/* Level-one histogram of one round over nb buckets (for kernel-level
 * parity checks). */
void or_l1_counts(const uint64_t* hkeys, uint64_t n, uint64_t nb, uint64_t seed, uint32_t round,
                  uint32_t* cnt) {
  uint64_t c1[3];
  or_derive(seed, round, OR_TAG_L1, 0, c1);
  memset(cnt, 0, nb * sizeof(uint32_t));
  for (uint64_t i = 0; i < n; ++i) cnt[or_reduce(or_hash(c1, hkeys[i]), nb)] += 1;
}

/* Fingerprints of n strings for one round (for kernel-level parity checks). */
void or_fingerprints(const uint8_t* ctx, const int64_t* offs, uint64_t n, uint64_t seed,
                     uint32_t round, uint64_t* out) {
  uint64_t base = or_fp_base(seed, round);
  for (uint64_t i = 0; i < n; ++i)
    out[i] = or_fingerprint(ctx + offs[i], (uint64_t)(offs[i + 1] - offs[i]), base);
}

/* Eytzinger layout (Sec. 3.4, the locality variant of the sorted-array map):
 * the implicit binary search tree of the sorted keys stored level by level.
 * e[1..n] (1-based; e[0] unused): node k has children 2k and 2k+1, and an
 * in-order walk of the tree visits the keys in sorted order.  Filled here
 * by that definition: an in-order traversal that assigns sorted[0], [1], ...
 * to the nodes it visits. */
static void or_eyt_fill(const uint64_t* sk, const int64_t* sv, uint64_t n, uint64_t k, uint64_t* next,
                        uint64_t* ek, int64_t* ev) {
  if (k > n) return;
  or_eyt_fill(sk, sv, n, 2 * k, next, ek, ev);
  ek[k] = sk[*next];
  ev[k] = sv[*next];
  *next += 1;
  or_eyt_fill(sk, sv, n, 2 * k + 1, next, ek, ev);
}

void or_eytzinger_layout(const uint64_t* sorted_keys, const int64_t* sorted_vals, uint64_t n, uint64_t* ek,
                         int64_t* ev) {
  uint64_t next = 0;
  ek[0] = 0;
  ev[0] = 0;
  or_eyt_fill(sorted_keys, sorted_vals, n, 1, &next, ek, ev);
}

/* Search of the Eytzinger array: descend k -> 2k + (e[k] < q) until k > n;
 * the last node where the walk went left holds the smallest key >= q.
 * Returns that node if its key equals q, else 0. */
uint64_t or_eytzinger_search(const uint64_t* ek, uint64_t n, uint64_t q) {
  uint64_t k = 1, cand = 0;
  while (k <= n) {
    if (ek[k] < q) {
      k = 2 * k + 1;
    } else {
      cand = k;
      k = 2 * k;
    }
  }
  return (cand && ek[cand] == q) ? cand : 0;
}

/* Sorted-array map (Sec. 3.4, mk_arraymap): binary search returning the
 * index or -1; used as the search-based comparison point. */
int64_t or_binary_search(const uint64_t* sorted, uint64_t n, uint64_t q) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (sorted[mid] < q) lo = mid + 1; else hi = mid;
  }
  return (lo < n && sorted[lo] == q) ? (int64_t)lo : -1;
}
