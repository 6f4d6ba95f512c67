// fks_lookup.cu -- lookups against FKS two-level hash maps.
//
// The membership test of Sec. 2.2 (arr[h a] = a) and lookup -> opt v of
// Sec. 3.2: one dependent read of the bucket descriptor desc[g q], one
// dependent read of the slot offsets[g q] + Hash consts[g q] q mod s^2, one
// compare.  An empty bucket answers "absent" without the second read.
//
// The two reads are random 8 B / 16 B accesses into tables far larger than
// L2, so the kernel is bound by DRAM sector throughput: each thread keeps
// kQ queries in flight (all descriptor reads issued before any slot read),
// queries are read and results written with vector accesses, and the random
// reads bypass L1 allocation.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fks_internal.cuh"
#include "fks_strings.cuh"

namespace fks {
namespace {

constexpr int kLookupThreads = 256;

// L2 policies: descriptors are kept (evict_last) so the L2 holds as many of
// them as fits; slots are read once (evict_first).
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_stream() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t ld_na_u64(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ ulonglong2 ld_na_u128(const uint64_t* p, uint64_t pol) {
  ulonglong2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(v.x), "=l"(v.y)
               : "l"(p), "l"(pol));
  return v;
}

// One 32-byte load (a single request, like a 16-byte one): a whole string
// slot {fingerprint, offset | length << 40, value, 0}.  p is 32-byte aligned.
__device__ __forceinline__ ulonglong4_32a ld_na_u256(const uint64_t* p, uint64_t pol) {
  ulonglong4_32a v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
               : "=l"(v.x), "=l"(v.y), "=l"(v.z), "=l"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

// Lookups through inline-singleton records: one 16-byte probe of rec[b]
// answers every needle whose bucket holds no key or one key (hit or miss);
// only the others go on to their slot, as in k_lookup_u64.  A record {x, y}
// is a one-key bucket's {key, value} exactly when x hashes to b; otherwise y
// is desc[b] (and x, hashing elsewhere, equals no needle of bucket b).
template <bool kI64>
__global__ void __launch_bounds__(512) k_lookup_inline(LookupMap M, const uint64_t* __restrict__ rec,
                                                       const uint64_t* __restrict__ q, uint64_t nq,
                                                       void* __restrict__ out, uint8_t* __restrict__ found,
                                                       int64_t absent, int vec) {
  constexpr int kQ = 4;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kQ;
  const uint64_t keep = policy_keep(), strm = policy_stream();
  for (uint64_t base = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kQ; base < nq; base += stride) {
    const bool full = vec && base + kQ <= nq;
    uint64_t k[kQ];
    if (full) {
#pragma unroll
      for (int i = 0; i < kQ; i += 2) {
        const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(q + base + i));
        k[i] = v.x;
        k[i + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) k[i] = base + i < nq ? __ldcs(q + base + i) : 0;
    }
    uint32_t b[kQ];
    ulonglong2 r[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      b[i] = reduce32(hash32(M.c1, k[i]), M.nb);
      r[i] = ld_na_u128(rec + 2ull * b[i], keep);
    }
    ulonglong2 sl[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      sl[i] = make_ulonglong2(~k[i], 0);
      if (r[i].x == k[i]) {
        sl[i] = r[i];  // the bucket's one key
      } else if (reduce32(hash32(M.c1, r[i].x), M.nb) != b[i]) {
        const uint64_t d = r[i].y;  // a descriptor record
        const uint32_t s = desc_s(d);
        if (s) {
          const HashConsts c = derive(M.seed, M.round, b[i], desc_attempt(d));
          const uint32_t jj = desc_off(d) + reduce32(hash32(c, k[i]), s * s);
          sl[i] = ld_na_u128(M.slots + 2ull * jj, strm);
        }
      }
    }
    int64_t v[kQ];
    uint32_t f = 0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const bool hit = sl[i].x == k[i];
      v[i] = hit ? int64_t(sl[i].y) : absent;
      f |= uint32_t(hit) << (8 * i);
    }
    if (full) {
      if (out) {
        if (kI64) {
          __stcs(reinterpret_cast<longlong2*>(static_cast<int64_t*>(out) + base), make_longlong2(v[0], v[1]));
          __stcs(reinterpret_cast<longlong2*>(static_cast<int64_t*>(out) + base + 2), make_longlong2(v[2], v[3]));
        } else {
          __stcs(reinterpret_cast<int4*>(static_cast<int32_t*>(out) + base),
                 make_int4(int(v[0]), int(v[1]), int(v[2]), int(v[3])));
        }
      }
      if (found) __stcs(reinterpret_cast<unsigned int*>(found + base), f);
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        if (base + i >= nq) break;
        if (out) {
          if (kI64) static_cast<int64_t*>(out)[base + i] = v[i];
          else static_cast<int32_t*>(out)[base + i] = int32_t(v[i]);
        }
        if (found) found[base + i] = uint8_t((f >> (8 * i)) & 1u);
      }
    }
  }
}

template <int kQ, bool kI64, int NT>
__global__ void __launch_bounds__(NT) k_lookup_u64(LookupMap M, const uint64_t* __restrict__ q, uint64_t nq,
                                                   void* __restrict__ out, uint8_t* __restrict__ found,
                                                   int64_t absent, int vec) {
  static_assert(kQ == 2 || kQ == 4 || kQ == 8, "2, 4 or 8 needles per thread");
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kQ;
  const uint64_t keep = policy_keep(), strm = policy_stream();
  for (uint64_t base = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kQ; base < nq;
       base += stride) {
    const bool full = vec && base + kQ <= nq;
    uint64_t k[kQ];
    if (full) {
#pragma unroll
      for (int i = 0; i < kQ; i += 2) {
        const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(q + base + i));
        k[i] = v.x;
        k[i + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) k[i] = base + i < nq ? __ldcs(q + base + i) : 0;
    }
    uint32_t b[kQ];
    uint64_t d[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      b[i] = reduce32(hash32(M.c1, k[i]), M.nb);
      d[i] = ld_na_u64(M.desc + b[i], keep);
    }
    ulonglong2 sl[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const uint32_t s = desc_s(d[i]);
      sl[i] = make_ulonglong2(~k[i], 0);
      if (s) {
        const HashConsts c = derive(M.seed, M.round, b[i], desc_attempt(d[i]));
        const uint32_t jj = desc_off(d[i]) + reduce32(hash32(c, k[i]), s * s);
        sl[i] = ld_na_u128(M.slots + 2ull * jj, strm);
      }
    }
    int64_t v[kQ];
    uint64_t f = 0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const bool hit = sl[i].x == k[i];
      v[i] = hit ? int64_t(sl[i].y) : absent;
      f |= uint64_t(hit) << (8 * i);
    }
    if (full) {
      if (out) {
        if (kI64) {
#pragma unroll
          for (int i = 0; i < kQ; i += 2)
            __stcs(reinterpret_cast<longlong2*>(static_cast<int64_t*>(out) + base + i),
                   make_longlong2(v[i], v[i + 1]));
        } else if (kQ == 2) {
          __stcs(reinterpret_cast<int2*>(static_cast<int32_t*>(out) + base), make_int2(int(v[0]), int(v[1])));
        } else {
#pragma unroll
          for (int i = 0; i < kQ; i += 4)
            __stcs(reinterpret_cast<int4*>(static_cast<int32_t*>(out) + base + i),
                   make_int4(int(v[i]), int(v[i + 1]), int(v[i + 2 < kQ ? i + 2 : 0]), int(v[i + 3 < kQ ? i + 3 : 0])));
        }
      }
      if (found) {
        if (kQ == 2) __stcs(reinterpret_cast<unsigned short*>(found + base), static_cast<unsigned short>(f));
        else if (kQ == 4) __stcs(reinterpret_cast<unsigned int*>(found + base), static_cast<unsigned int>(f));
        else __stcs(reinterpret_cast<unsigned long long*>(found + base), static_cast<unsigned long long>(f));
      }
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        if (base + i >= nq) break;
        if (out) {
          if (kI64) static_cast<int64_t*>(out)[base + i] = v[i];
          else static_cast<int32_t*>(out)[base + i] = int32_t(v[i]);
        }
        if (found) found[base + i] = uint8_t(f >> (8 * i));
      }
    }
  }
}

// One needle of a string map; returns whether it is present.
__device__ __forceinline__ bool lookup_one_bytes(const LookupMap& M, const uint8_t* s,
                                                 uint32_t len, int64_t* val) {
  const uint64_t keep = policy_keep(), strm = policy_stream();
  const uint64_t h = fingerprint(s, len, M.fpb);
  const uint32_t b = reduce32(hash32(M.c1, h), M.nb);
  const uint64_t d = ld_na_u64(M.desc + b, keep);
  const uint32_t sz = desc_s(d);
  if (!sz) return false;
  const HashConsts c = derive(M.seed, M.round, b, desc_attempt(d));
  const uint32_t jj = desc_off(d) + reduce32(hash32(c, h), sz * sz);
  const ulonglong4_32a w = ld_na_u256(M.slots + 4ull * jj, strm);  // the whole slot, value included
  if (w.x != h || offlen_len(w.y) != len) return false;
  if (!bytes_equal(M.ctx + offlen_off(w.y), s, len)) return false;
  *val = int64_t(w.z);
  return true;
}

// String needles against one map, one needle per lane.  A needle longer
// than kLongString bytes is fingerprinted and compared by the whole warp
// (lanes take its words), so that one long string does not hold up the
// other 31 lanes for its whole length; shorter needles go through each
// lane's own loop, which costs less than passing 32 needles one by one
// through the warp's reductions (measured: 2^24 needles of 4-64 bytes,
// 1.21 ms per lane against 4.83 ms with every needle shared).
template <bool kI64>
__global__ void __launch_bounds__(kLookupThreads, 8) k_lookup_bytes(LookupMap M, const uint8_t* __restrict__ qctx,
                                                                 const int64_t* __restrict__ qoffs, uint64_t nq,
                                                                 void* __restrict__ out,
                                                                 uint8_t* __restrict__ found, int64_t absent) {
  __shared__ uint64_t pw[33];
  if (threadIdx.x < 33) pw[threadIdx.x] = pow61(M.fpb, threadIdx.x);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t keep = policy_keep(), strm = policy_stream();
  const uint64_t nwarps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t base = (uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < nq;
       base += nwarps * 32) {
    const uint64_t i = base + lane;
    int64_t o0 = 0, o1 = 0;
    if (i < nq) {
      o0 = __ldg(reinterpret_cast<const long long*>(qoffs) + i);
      o1 = __ldg(reinterpret_cast<const long long*>(qoffs) + i + 1);
    }
    const bool ok = i < nq && o0 >= 0 && o1 >= o0 && o1 - o0 < (int64_t(1) << 24);
    const uint32_t len = ok ? uint32_t(o1 - o0) : 0u;
    const bool lng = len > kLongString;
    uint64_t fp = 0;
    if (ok && !lng) fp = fingerprint(qctx + o0, len, M.fpb);
    for (uint32_t todo = __ballot_sync(0xFFFFFFFFu, lng); todo; todo &= todo - 1) {
      const int j = __ffs(todo) - 1;
      const int64_t oj = __shfl_sync(0xFFFFFFFFu, o0, j);
      const uint32_t lj = __shfl_sync(0xFFFFFFFFu, len, j);
      const uint64_t h = warp_fingerprint(qctx + oj, lj, pw);
      if (int(lane) == j) fp = h;
    }
    bool cand = false;
    uint64_t coff = 0, cval = 0;
    if (ok) {
      const uint32_t b = reduce32(hash32(M.c1, fp), M.nb);
      const uint64_t d = ld_na_u64(M.desc + b, keep);
      const uint32_t sz = desc_s(d);
      if (sz) {
        const HashConsts c = derive(M.seed, M.round, b, desc_attempt(d));
        const uint32_t jj = desc_off(d) + reduce32(hash32(c, fp), sz * sz);
        const ulonglong4_32a w = ld_na_u256(M.slots + 4ull * jj, strm);  // the whole slot, value included
        cand = w.x == fp && offlen_len(w.y) == len;
        coff = offlen_off(w.y);
        cval = w.z;
      }
    }
    bool hit = cand && !lng && bytes_equal(qctx + o0, M.ctx + coff, len);
    for (uint32_t todo = __ballot_sync(0xFFFFFFFFu, cand && lng); todo; todo &= todo - 1) {
      const int j = __ffs(todo) - 1;
      const int64_t oj = __shfl_sync(0xFFFFFFFFu, o0, j);
      const uint32_t lj = __shfl_sync(0xFFFFFFFFu, len, j);
      const uint64_t cj = __shfl_sync(0xFFFFFFFFu, coff, j);
      const bool eq = warp_bytes_equal(qctx + oj, M.ctx + cj, lj);
      if (int(lane) == j) hit = eq;
    }
    if (i < nq) {
      const int64_t v = hit ? int64_t(cval) : absent;
      if (out) {
        if (kI64) static_cast<int64_t*>(out)[i] = v;
        else static_cast<int32_t*>(out)[i] = int32_t(v);
      }
      if (found) found[i] = uint8_t(hit);
    }
  }
}

// (map_id, needle) pairs against a set of maps; the small table of maps stays
// in L1/L2.
template <bool kI64, bool kStr>
__global__ void __launch_bounds__(kLookupThreads) k_lookup_batched(
    const LookupMap* __restrict__ maps, uint32_t m, const uint32_t* __restrict__ ids,
    const uint64_t* __restrict__ q, const uint8_t* __restrict__ qctx,
    const int64_t* __restrict__ qoffs, uint64_t nq, void* __restrict__ out,
    uint8_t* __restrict__ found, int64_t absent) {
  // uint64 needles: four descriptor loads in flight per thread before any
  // slot load; string needles are each a chain of dependent loads
  constexpr int kQ = kStr ? 2 : 4;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kQ;
  const uint64_t keep = policy_keep(), strm = policy_stream();
  for (uint64_t base = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kQ; base < nq;
       base += stride) {
    int64_t v[kQ];
    bool hit[kQ];
    if (!kStr) {
      uint64_t k[kQ], d[kQ];
      uint32_t b[kQ], id[kQ];
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const bool ok = base + i < nq;
        id[i] = ok ? __ldg(ids + base + i) : m;
        k[i] = ok ? __ldcs(q + base + i) : 0;
        d[i] = 0;
        b[i] = 0;
        if (id[i] < m) {
          b[i] = reduce32(hash32(maps[id[i]].c1, k[i]), maps[id[i]].nb);
          d[i] = ld_na_u64(maps[id[i]].desc + b[i], keep);
        }
      }
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const uint32_t s = desc_s(d[i]);
        hit[i] = false;
        v[i] = absent;
        if (s) {
          const LookupMap& M = maps[id[i]];
          const HashConsts c = derive(M.seed, M.round, b[i], desc_attempt(d[i]));
          const uint32_t jj = desc_off(d[i]) + reduce32(hash32(c, k[i]), s * s);
          const ulonglong2 sl = ld_na_u128(M.slots + 2ull * jj, strm);
          hit[i] = sl.x == k[i];
          if (hit[i]) v[i] = int64_t(sl.y);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        hit[i] = false;
        v[i] = absent;
        if (base + i >= nq) continue;
        const uint32_t id = __ldg(ids + base + i);
        const int64_t o0 = __ldg(reinterpret_cast<const long long*>(qoffs) + base + i);
        const int64_t o1 = __ldg(reinterpret_cast<const long long*>(qoffs) + base + i + 1);
        if (id < m && o0 >= 0 && o1 >= o0 && o1 - o0 < (int64_t(1) << 24))
          hit[i] = lookup_one_bytes(maps[id], qctx + o0, uint32_t(o1 - o0), &v[i]);
        if (!hit[i]) v[i] = absent;
      }
    }
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      if (base + i >= nq) break;
      if (out) {
        if (kI64) static_cast<int64_t*>(out)[base + i] = v[i];
        else static_cast<int32_t*>(out)[base + i] = int32_t(v[i]);
      }
      if (found) found[base + i] = uint8_t(hit[i]);
    }
  }
}

// All queries of many lookup requests (different maps, key kinds, output
// buffers) in one launch: query i belongs to the request whose
// [begin, begin + nq) holds it.
__global__ void __launch_bounds__(kLookupThreads) k_lookup_requests(const LookupReq* __restrict__ reqs,
                                                                    const uint64_t* __restrict__ begins,
                                                                    uint32_t nreq, uint64_t total) {
  __shared__ uint64_t sb[1025];
  const bool cached = nreq <= 1024;
  if (cached) {
    for (uint32_t i = threadIdx.x; i <= nreq; i += blockDim.x) sb[i] = begins[i];
    __syncthreads();
  }
  const uint64_t* b = cached ? sb : begins;
  const uint64_t keep = policy_keep(), strm = policy_stream();
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride) {
    uint32_t lo = 0, hi = nreq;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (b[mid] <= i) lo = mid; else hi = mid;
    }
    const LookupReq& R = reqs[lo];
    const uint64_t local = i - b[lo];
    int64_t v = R.absent;
    bool hit = false;
    if (!R.strings) {
      const uint64_t k = __ldcs(R.q + local);
      const uint32_t bk = reduce32(hash32(R.M.c1, k), R.M.nb);
      const uint64_t d = ld_na_u64(R.M.desc + bk, keep);
      const uint32_t s = desc_s(d);
      if (s) {
        const HashConsts c = derive(R.M.seed, R.M.round, bk, desc_attempt(d));
        const ulonglong2 sl = ld_na_u128(R.M.slots + 2ull * (desc_off(d) + reduce32(hash32(c, k), s * s)), strm);
        hit = sl.x == k;
        if (hit) v = int64_t(sl.y);
      }
    } else {
      const int64_t o0 = __ldg(reinterpret_cast<const long long*>(R.qoffs) + local);
      const int64_t o1 = __ldg(reinterpret_cast<const long long*>(R.qoffs) + local + 1);
      if (o0 >= 0 && o1 >= o0 && o1 - o0 < (int64_t(1) << 24))
        hit = lookup_one_bytes(R.M, R.qctx + o0, uint32_t(o1 - o0), &v);
      if (!hit) v = R.absent;
    }
    if (R.out) {
      if (R.out_i64) static_cast<int64_t*>(R.out)[local] = v;
      else static_cast<int32_t*>(R.out)[local] = int32_t(v);
    }
    if (R.found) R.found[local] = uint8_t(hit);
  }
}

unsigned grid_for(uint64_t work, int sms, int per_sm) {
  uint64_t blocks = (work + kLookupThreads - 1) / kLookupThreads;
  const uint64_t cap = uint64_t(sms) * per_sm;
  return unsigned(blocks < cap ? (blocks ? blocks : 1) : cap);
}

}  // namespace

template <int kQ, int NT>
static void lookup_u64_at(const LookupMap& M, const uint64_t* q, uint64_t nq, void* out, int out_i64, uint8_t* found,
                          int64_t absent, int vec, unsigned grid, cudaStream_t stream) {
  if (out_i64) k_lookup_u64<kQ, true, NT><<<grid, NT, 0, stream>>>(M, q, nq, out, found, absent, vec);
  else k_lookup_u64<kQ, false, NT><<<grid, NT, 0, stream>>>(M, q, nq, out, found, absent, vec);
}

template <int kQ>
static void lookup_u64_q(const LookupMap& M, const uint64_t* q, uint64_t nq, void* out, int out_i64, uint8_t* found,
                         int64_t absent, int vec, uint32_t block, unsigned grid, cudaStream_t stream) {
  if (block == 128) lookup_u64_at<kQ, 128>(M, q, nq, out, out_i64, found, absent, vec, grid, stream);
  else if (block == 512) lookup_u64_at<kQ, 512>(M, q, nq, out, out_i64, found, absent, vec, grid, stream);
  else lookup_u64_at<kQ, 256>(M, q, nq, out, out_i64, found, absent, vec, grid, stream);
}

cudaError_t launch_lookup_inline(const LookupMap& M, const uint64_t* rec, const uint64_t* q, uint64_t nq, void* out,
                                 int out_i64, uint8_t* found, int64_t absent, int sms, cudaStream_t stream) {
  if (nq == 0) return cudaSuccess;
  const int vec = ((reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(out) |
                    reinterpret_cast<uintptr_t>(found)) & 15u) == 0;
  uint64_t blocks = (nq + 4 * 512 - 1) / (4 * 512);
  const uint64_t cap = uint64_t(sms) * 1024;
  if (blocks > cap) blocks = cap;
  if (out_i64) k_lookup_inline<true><<<unsigned(blocks), 512, 0, stream>>>(M, rec, q, nq, out, found, absent, vec);
  else k_lookup_inline<false><<<unsigned(blocks), 512, 0, stream>>>(M, rec, q, nq, out, found, absent, vec);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_lookup_u64(const LookupMap& M, const uint64_t* q, uint64_t nq, void* out,
                              int out_i64, uint8_t* found, int64_t absent, int sms,
                              const LookupShape& shape, cudaStream_t stream) {
  if (nq == 0) return cudaSuccess;
  const uint32_t kq = shape.queries_per_thread == 2 || shape.queries_per_thread == 8 ? shape.queries_per_thread : 4u;
  const uint32_t block = shape.block == 128 || shape.block == 512 ? shape.block : 256u;
  const uint32_t per_sm = shape.blocks_per_sm ? shape.blocks_per_sm : 8u;
  // vector loads and stores need 16-byte aligned needles, values and flags
  const int vec = ((reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(out) |
                    reinterpret_cast<uintptr_t>(found)) & 15u) == 0;
  const uint64_t threads = (nq + kq - 1) / kq;
  uint64_t blocks = (threads + block - 1) / block;
  const uint64_t cap = uint64_t(sms) * per_sm;
  if (blocks > cap) blocks = cap;
  const unsigned grid = unsigned(blocks ? blocks : 1);
  if (kq == 2) lookup_u64_q<2>(M, q, nq, out, out_i64, found, absent, vec, block, grid, stream);
  else if (kq == 8) lookup_u64_q<8>(M, q, nq, out, out_i64, found, absent, vec, block, grid, stream);
  else lookup_u64_q<4>(M, q, nq, out, out_i64, found, absent, vec, block, grid, stream);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_lookup_bytes(const LookupMap& M, const uint8_t* qctx, const int64_t* qoffs,
                                uint64_t nq, void* out, int out_i64, uint8_t* found,
                                int64_t absent, int sms, cudaStream_t stream) {
  if (nq == 0) return cudaSuccess;
  const unsigned grid = grid_for(nq, sms, 8);
  if (out_i64)
    k_lookup_bytes<true><<<grid, kLookupThreads, 0, stream>>>(M, qctx, qoffs, nq, out, found, absent);
  else
    k_lookup_bytes<false><<<grid, kLookupThreads, 0, stream>>>(M, qctx, qoffs, nq, out, found, absent);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_lookup_requests(const LookupReq* reqs, const uint64_t* begins, uint32_t nreq,
                                   uint64_t total, int sms, cudaStream_t stream) {
  if (total == 0 || nreq == 0) return cudaSuccess;
  k_lookup_requests<<<grid_for(total, sms, 8), kLookupThreads, 0, stream>>>(reqs, begins, nreq, total);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_lookup_batched(const LookupMap* maps, uint32_t m, int strings,
                                  const uint32_t* ids, const uint64_t* q, const uint8_t* qctx,
                                  const int64_t* qoffs, uint64_t nq, void* out, int out_i64,
                                  uint8_t* found, int64_t absent, int sms, cudaStream_t stream) {
  if (nq == 0) return cudaSuccess;
  // uint64 needles: one pass of the grid over all of them (as the tuned
  // single-map lookup); strings: up to 8 blocks per SM
  const unsigned grid = strings ? grid_for((nq + 1) / 2, sms, 8) : grid_for((nq + 3) / 4, sms, 1024);
#define FKS_LB(I64, STR)                                                                      \
  k_lookup_batched<I64, STR><<<grid, kLookupThreads, 0, stream>>>(maps, m, ids, q, qctx, qoffs, \
                                                                  nq, out, found, absent)
  if (out_i64) {
    if (strings) FKS_LB(true, true); else FKS_LB(true, false);
  } else {
    if (strings) FKS_LB(false, true); else FKS_LB(false, false);
  }
#undef FKS_LB
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fks
