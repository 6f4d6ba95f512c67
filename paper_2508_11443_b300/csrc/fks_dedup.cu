// fks_dedup.cu -- from_array (Sec. 3.2): the constructor that accepts
// duplicate keys.  The paper leaves the surviving pair unspecified; here the
// first occurrence in input order wins (per map for batched builds).  This
// is a pre-pass in front of the build (from_array_nodup on the kept pairs):
//
//   k_dedup_insert  every element claims or joins the entry of its key in
//                   an open-addressing table of 64-bit words (hash tag << 32
//                   | index + 1); equal keys keep the smallest index with
//                   one atomicMin (the tags of equal keys are equal)
//   k_dedup_keep    keep[e] = 1 iff e is the index stored for its key
//   scan            exclusive scan of keep, in place -> output positions
//                   (keep[e] = pos[e + 1] - pos[e])
//   k_dedup_pack_*  kept keys / values (and, for strings, bytes and new
//                   offsets) gathered in input order
//
// Equality is exact: equal 64-bit words, or equal length and bytes for
// strings, and the same segment; the tag only filters.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fks_internal.cuh"
#include "fks_strings.cuh"

namespace fks {
namespace {

constexpr uint64_t kDedupFpBase = 0x1F3D5B79A2C4E6F1ull % (kP61 - 1) + 1;  // fixed fingerprint base

__device__ __forceinline__ uint32_t seg_of(const int64_t* seg, uint32_t m, uint64_t e) {
  uint32_t lo = 0, hi = m;  // largest j with seg[j] <= e
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (uint64_t(__ldg(reinterpret_cast<const long long*>(seg) + mid)) <= e) lo = mid; else hi = mid;
  }
  return lo;
}

struct DedupArgs {
  const uint64_t* keys;  // u64 keys, or null for strings
  const uint8_t* ctx;
  const int64_t* offs;
  const int64_t* seg;    // device [m + 1] or null (one segment)
  uint32_t m;
  uint64_t u;
  uint64_t* table;
  uint64_t mask;         // table size - 1
  uint32_t* keep;        // [u + 1]
  uint32_t* flags;       // [0]: invalid offsets, [1]: probe limit reached
};

// Offsets of string element e, or false when they are malformed.
__device__ __forceinline__ bool str_span(const DedupArgs& a, uint64_t e, int64_t* o0, uint32_t* len) {
  const int64_t x = __ldg(reinterpret_cast<const long long*>(a.offs) + e);
  const int64_t y = __ldg(reinterpret_cast<const long long*>(a.offs) + e + 1);
  if (x < 0 || y < x || y - x >= (int64_t(1) << 24) || y >= (int64_t(1) << 40)) return false;
  *o0 = x;
  *len = uint32_t(y - x);
  return true;
}

__device__ __forceinline__ bool same_key(const DedupArgs& a, uint64_t o, uint64_t e, uint32_t seg_e) {
  if (a.m > 1 && seg_of(a.seg, a.m, o) != seg_e) return false;
  if (a.keys) return __ldg(reinterpret_cast<const unsigned long long*>(a.keys) + o) ==
                     __ldg(reinterpret_cast<const unsigned long long*>(a.keys) + e);
  int64_t xo, xe;
  uint32_t lo, le;
  if (!str_span(a, o, &xo, &lo) || !str_span(a, e, &xe, &le) || lo != le) return false;
  return bytes_equal(a.ctx + xo, a.ctx + xe, le);
}

// 64-bit tag of element e (false for malformed string offsets).
__device__ __forceinline__ bool tag_of(const DedupArgs& a, uint64_t e, uint32_t seg_e, uint64_t* tag) {
  uint64_t h;
  if (a.keys) {
    h = __ldg(reinterpret_cast<const unsigned long long*>(a.keys) + e);
  } else {
    int64_t o0;
    uint32_t len;
    if (!str_span(a, e, &o0, &len)) return false;
    h = fingerprint(a.ctx + o0, len, kDedupFpBase);
  }
  *tag = mix13(h ^ (uint64_t(seg_e) * kGamma));
  return true;
}

__global__ void __launch_bounds__(256) k_dedup_insert(DedupArgs a) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < a.u; e += stride) {
    const uint32_t sg = a.m > 1 ? seg_of(a.seg, a.m, e) : 0u;
    uint64_t tag;
    if (!tag_of(a, e, sg, &tag)) {
      atomicExch(a.flags, 1u);
      continue;
    }
    const uint64_t hi = tag >> 32, mine = (hi << 32) | (e + 1);
    uint64_t h = tag & a.mask;
    bool placed = false;
    for (uint64_t probe = 0; probe <= a.mask; ++probe, h = (h + 1) & a.mask) {
      unsigned long long* slot = reinterpret_cast<unsigned long long*>(a.table + h);
      uint64_t cur = *reinterpret_cast<volatile unsigned long long*>(slot);
      if (cur == 0) {
        cur = atomicCAS(slot, 0ull, (unsigned long long)mine);
        if (cur == 0) {
          placed = true;
          break;
        }
      }
      if ((cur >> 32) != hi) continue;
      if (same_key(a, (cur & 0xFFFFFFFFull) - 1, e, sg)) {
        atomicMin(slot, (unsigned long long)mine);  // equal tag bits: the smaller index wins
        placed = true;
        break;
      }
    }
    if (!placed) atomicExch(a.flags + 1, 1u);
  }
}

__global__ void __launch_bounds__(256) k_dedup_keep(DedupArgs a) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < a.u; e += stride) {
    const uint32_t sg = a.m > 1 ? seg_of(a.seg, a.m, e) : 0u;
    uint64_t tag;
    uint32_t keep = 1;  // malformed elements pass through (the call fails on the flag)
    if (tag_of(a, e, sg, &tag)) {
      const uint64_t hi = tag >> 32;
      uint64_t h = tag & a.mask;
      for (uint64_t probe = 0; probe <= a.mask; ++probe, h = (h + 1) & a.mask) {
        const uint64_t cur = a.table[h];
        if (cur == 0) break;  // not reached: every element was placed
        if ((cur >> 32) != hi) continue;
        const uint64_t o = (cur & 0xFFFFFFFFull) - 1;
        if (o == e) break;
        if (same_key(a, o, e, sg)) {
          keep = 0;
          break;
        }
      }
    }
    a.keep[e] = keep;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.keep[a.u] = 0;
}

__global__ void __launch_bounds__(256) k_dedup_pack_u64(const uint64_t* __restrict__ keys, const void* vals,
                                                        int vals_i64, uint64_t u, const uint32_t* __restrict__ pos,
                                                        uint64_t* __restrict__ okeys, void* ovals) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < u; e += stride) {
    const uint32_t p = pos[e];
    if (pos[e + 1] == p) continue;
    okeys[p] = keys[e];
    if (vals_i64) static_cast<int64_t*>(ovals)[p] = static_cast<const int64_t*>(vals)[e];
    else static_cast<int32_t*>(ovals)[p] = static_cast<const int32_t*>(vals)[e];
  }
}

// Byte length of each kept string (0 for dropped or malformed ones).
__global__ void __launch_bounds__(256) k_dedup_lengths(const int64_t* __restrict__ offs, uint64_t u,
                                                       const uint32_t* __restrict__ pos, uint64_t* __restrict__ lens) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < u; e += stride) {
    const int64_t x = offs[e], y = offs[e + 1];
    const bool ok = pos[e + 1] != pos[e] && x >= 0 && y >= x && y - x < (int64_t(1) << 24);
    lens[e] = ok ? uint64_t(y - x) : 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) lens[u] = 0;
}

// Kept strings: bytes to their new offsets (one warp copies 32 strings, one
// after the other, lanes over the bytes), new offsets and values.
__global__ void __launch_bounds__(256) k_dedup_pack_bytes(const uint8_t* __restrict__ ctx, const int64_t* __restrict__ offs,
                                                          const void* vals, int vals_i64, uint64_t u,
                                                          const uint32_t* __restrict__ pos,
                                                          const uint64_t* __restrict__ noff,
                                                          uint8_t* __restrict__ octx, int64_t* __restrict__ ooffs,
                                                          void* ovals) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t w0 = (uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; w0 < u; w0 += warps * 32) {
    const uint64_t e = w0 + lane;
    uint64_t src = 0, dst = 0, len = 0;
    if (e < u && pos[e + 1] != pos[e]) {
      const uint32_t p = pos[e];
      dst = noff[e];
      len = noff[e + 1] - dst;  // 0 for malformed spans
      src = len ? uint64_t(offs[e]) : 0ull;
      ooffs[p] = int64_t(dst);
      if (vals_i64) static_cast<int64_t*>(ovals)[p] = static_cast<const int64_t*>(vals)[e];
      else static_cast<int32_t*>(ovals)[p] = static_cast<const int32_t*>(vals)[e];
    }
    for (uint32_t j = 0; j < 32; ++j) {
      const uint64_t s_ = __shfl_sync(0xFFFFFFFFu, src, j), d_ = __shfl_sync(0xFFFFFFFFu, dst, j),
                     l_ = __shfl_sync(0xFFFFFFFFu, len, j);
      for (uint64_t b = lane; b < l_; b += 32) octx[d_ + b] = ctx[s_ + b];
    }
  }
}

__global__ void k_dedup_tail(const uint32_t* __restrict__ pos, const uint64_t* __restrict__ noff, uint64_t u,
                             int64_t* __restrict__ ooffs) {
  ooffs[pos[u]] = int64_t(noff[u]);
}

// New segment offsets: position of each old segment start.
__global__ void k_dedup_segs(const uint32_t* __restrict__ pos, const int64_t* __restrict__ seg, uint32_t m,
                             int64_t* __restrict__ oseg) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= m; j += gridDim.x * blockDim.x)
    oseg[j] = int64_t(pos[seg[j]]);
}

unsigned grid_for(uint64_t n, int sms) {
  const uint64_t b = (n + 255) / 256, cap = uint64_t(sms) * 16;
  return unsigned(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

size_t dedup_table_words(uint64_t u) {
  uint64_t size = 1;
  while (size < 2 * u) size <<= 1;
  return size_t(size);
}

cudaError_t launch_dedup_mark(const uint64_t* keys, const uint8_t* ctx, const int64_t* offs, const int64_t* d_seg,
                              uint32_t m, uint64_t u, uint64_t* table, size_t table_words, uint32_t* keep,
                              uint32_t* flags, int sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(table, 0, sizeof(uint64_t) * table_words, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * 2, st);
  if (e != cudaSuccess) return e;
  DedupArgs a{keys, ctx, offs, d_seg, m, u, table, uint64_t(table_words) - 1, keep, flags};
  k_dedup_insert<<<grid_for(u, sms), 256, 0, st>>>(a);
  k_dedup_keep<<<grid_for(u, sms), 256, 0, st>>>(a);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_dedup_pack_u64(const uint64_t* keys, const void* vals, int vals_i64, uint64_t u,
                                  const uint32_t* pos, uint64_t* okeys, void* ovals, int sms, cudaStream_t st) {
  k_dedup_pack_u64<<<grid_for(u, sms), 256, 0, st>>>(keys, vals, vals_i64, u, pos, okeys, ovals);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dedup_lengths(const int64_t* offs, uint64_t u, const uint32_t* pos, uint64_t* lens, int sms,
                                 cudaStream_t st) {
  k_dedup_lengths<<<grid_for(u, sms), 256, 0, st>>>(offs, u, pos, lens);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dedup_pack_bytes(const uint8_t* ctx, const int64_t* offs, const void* vals, int vals_i64,
                                    uint64_t u, const uint32_t* pos, const uint64_t* noff, uint8_t* octx,
                                    int64_t* ooffs, void* ovals, int sms, cudaStream_t st) {
  k_dedup_pack_bytes<<<grid_for((u + 31) / 32 * 32, sms), 256, 0, st>>>(ctx, offs, vals, vals_i64, u, pos, noff,
                                                                          octx, ooffs, ovals);
  k_dedup_tail<<<1, 1, 0, st>>>(pos, noff, u, ooffs);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_dedup_segs(const uint32_t* pos, const int64_t* d_seg, uint32_t m, int64_t* oseg, cudaStream_t st) {
  k_dedup_segs<<<(m + 256) / 256, 256, 0, st>>>(pos, d_seg, m, oseg);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fks
