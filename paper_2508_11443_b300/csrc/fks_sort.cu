// fks_sort.cu -- the search-based map the paper compares against
// (mk_arraymap, Sec. 3.4): keys sorted together with their values, lookups
// by binary search returning the index or "absent".  The paper sorts with a
// comparison merge sort because its key abstraction offers no digits; uint64
// keys do, so this uses a least-significant-digit radix sort, 8 passes of 8
// bits, each pass stable:
//   count   per tile of kSortTile keys, a shared histogram of the digit
//   scan    exclusive scan of the digit-major histogram (device wide)
//   scatter per tile, warp-stable ranks (__match_any_sync within a warp,
//           warps in order), then each key to its digit's next position
#include <cuda_runtime.h>
#include <stdint.h>

#include "fks_internal.cuh"

namespace fks {
namespace {

constexpr uint32_t kSortTile = 2048;
constexpr int kSortThreads = 256;  // 8 warps x 256 keys each, 32 per round
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint32_t kPerWarp = kSortTile / kSortWarps;
constexpr uint32_t kRounds = kPerWarp / 32;

__device__ __forceinline__ uint32_t lane() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_count(const uint64_t* __restrict__ keys, uint64_t n,
                                                             uint32_t shift, uint32_t tiles,
                                                             uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t t0 = uint64_t(blockIdx.x) * kSortTile;
  for (uint32_t i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    if (t0 + i < n) atomicAdd(h + uint32_t((__ldcs(keys + t0 + i) >> shift) & 255u), 1u);
  }
  __syncthreads();
  hist[uint64_t(threadIdx.x) * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t* __restrict__ kin,
                                                               const uint64_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout,
                                                               uint64_t* __restrict__ vout, uint64_t n,
                                                               uint32_t shift, uint32_t tiles,
                                                               const uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kSortWarps][256];
  const uint32_t w = threadIdx.x >> 5;
  for (uint32_t d = lane(); d < 256; d += 32) cnt[w][d] = 0;
  __syncwarp();
  const uint64_t base = uint64_t(blockIdx.x) * kSortTile + uint64_t(w) * kPerWarp;
  uint64_t k[kRounds], v[kRounds];
  uint32_t dg[kRounds], rk[kRounds];
#pragma unroll
  for (uint32_t r = 0; r < kRounds; ++r) {
    const uint64_t e = base + r * 32 + lane();
    const bool ok = e < n;
    k[r] = ok ? __ldcs(kin + e) : 0;
    v[r] = ok ? __ldcs(vin + e) : 0;
    dg[r] = ok ? uint32_t((k[r] >> shift) & 255u) : 256u;
  }
#pragma unroll
  for (uint32_t r = 0; r < kRounds; ++r) {
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dg[r]);
    const uint32_t leader = __ffs(peers) - 1;
    const uint32_t before = dg[r] < 256u ? cnt[w][dg[r]] : 0u;
    rk[r] = before + __popc(peers & lanemask_lt());
    __syncwarp();
    if (lane() == leader && dg[r] < 256u) cnt[w][dg[r]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit, the keys of earlier warps of this tile come first
  if (threadIdx.x < 256) {
    uint32_t run = hist[uint64_t(threadIdx.x) * tiles + blockIdx.x];
    for (int ww = 0; ww < kSortWarps; ++ww) {
      const uint32_t c = cnt[ww][threadIdx.x];
      cnt[ww][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (uint32_t r = 0; r < kRounds; ++r) {
    if (dg[r] < 256u) {
      const uint32_t dst = cnt[w][dg[r]] + rk[r];
      kout[dst] = k[r];
      vout[dst] = v[r];
    }
  }
}

// Binary search (lower bound) of each needle; index or absent (Sec. 3.4:
// binary_search returns -1 for a needle that is not there).
template <bool kI64>
__global__ void __launch_bounds__(256) k_search(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                                                uint64_t n, const uint64_t* __restrict__ q, uint64_t nq,
                                                void* __restrict__ out, uint8_t* __restrict__ found,
                                                int64_t absent) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nq; i += stride) {
    const uint64_t x = __ldcs(q + i);
    uint64_t lo = 0, len = n;
    while (len > 0) {
      const uint64_t half = len >> 1;
      if (__ldg(keys + lo + half) < x) {
        lo += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    const bool hit = lo < n && __ldg(keys + lo) == x;
    const int64_t v = hit ? int64_t(__ldg(vals + lo)) : absent;
    if (out) {
      if (kI64) static_cast<int64_t*>(out)[i] = v;
      else static_cast<int32_t*>(out)[i] = int32_t(v);
    }
    if (found) found[i] = uint8_t(hit);
  }
}

// ---------------------------------------------------------------- Eytzinger
// The locality variant of the sorted-array map (Sec. 3.4): the implicit
// search tree of the sorted keys stored level by level, 1-based (node k has
// children 2k and 2k + 1; slot 0 unused).  Nodes 1..n form a complete
// binary tree, so subtree sizes have a closed form and every node finds its
// in-order rank -- the sorted position of its key -- in O(log n).
__device__ __forceinline__ uint32_t ilog2(uint64_t v) { return 63u - uint32_t(__clzll(static_cast<long long>(v))); }

// Nodes in the subtree of v (complete tree of n nodes, last level at depth H).
__device__ __forceinline__ uint64_t subtree_size(uint64_t v, uint64_t n, uint32_t H) {
  if (v > n) return 0;
  const uint32_t t = H - ilog2(v);                // levels below v down to the last
  const uint64_t first = v << t, span = 1ull << t;  // v's nodes on the last level
  const uint64_t last = first > n ? 0 : (n - first + 1 < span ? n - first + 1 : span);
  return span - 1 + last;
}

__device__ __forceinline__ uint64_t inorder_rank(uint64_t k, uint64_t n, uint32_t H) {
  uint64_t r = subtree_size(2 * k, n, H);
  for (uint64_t c = k; c > 1; c >>= 1)
    if (c & 1) r += subtree_size(c - 1, n, H) + 1;  // a right child: the left sibling's subtree and the parent
  return r;
}

__global__ void __launch_bounds__(256) k_eytz_gather(const uint64_t* __restrict__ sk, const uint64_t* __restrict__ sv,
                                                     uint64_t n, uint64_t* __restrict__ ek, uint64_t* __restrict__ ev) {
  const uint32_t H = ilog2(n);
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t k = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; k <= n; k += stride) {
    if (k == 0) {
      ek[0] = 0;
      ev[0] = 0;
      continue;
    }
    const uint64_t r = inorder_rank(k, n, H);
    ek[k] = __ldg(sk + r);
    ev[k] = __ldg(sv + r);
  }
}

// Descend k -> 2k + (e[k] < q), kQ needles per thread in step (all their
// loads of one level in flight together); the answer is the last node where
// the walk went left, if its key equals the needle.
template <int kQ, bool kI64>
__global__ void __launch_bounds__(256) k_eytz_search(const uint64_t* __restrict__ ek, const uint64_t* __restrict__ ev,
                                                     uint64_t n, const uint64_t* __restrict__ q, uint64_t nq,
                                                     void* __restrict__ out, uint8_t* __restrict__ found,
                                                     int64_t absent) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kQ;
  for (uint64_t base = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kQ; base < nq; base += stride) {
    uint64_t x[kQ], k[kQ], cand[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      x[i] = base + i < nq ? __ldcs(q + base + i) : 0ull;
      k[i] = 1;
      cand[i] = 0;
    }
    bool more = n >= 1;
    while (more) {
      uint64_t key[kQ];
#pragma unroll
      for (int i = 0; i < kQ; ++i) key[i] = k[i] <= n ? __ldg(ek + k[i]) : 0ull;
      more = false;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        if (k[i] <= n) {
          const bool right = key[i] < x[i];
          if (!right) cand[i] = k[i];
          k[i] = 2 * k[i] + (right ? 1 : 0);
          more |= k[i] <= n;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      if (base + i >= nq) break;
      const bool hit = cand[i] != 0 && __ldg(ek + cand[i]) == x[i];
      const int64_t v = hit ? int64_t(__ldg(ev + cand[i])) : absent;
      if (out) {
        if (kI64) static_cast<int64_t*>(out)[base + i] = v;
        else static_cast<int32_t*>(out)[base + i] = int32_t(v);
      }
      if (found) found[base + i] = uint8_t(hit);
    }
  }
}

__global__ void k_widen_i32(const int32_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ out) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = uint64_t(int64_t(in[i]));
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n) {
  const uint64_t tiles = (n + kSortTile - 1) / kSortTile;
  const uint64_t hist = 256 * tiles;
  const size_t bytes = 2 * 8 * n + 4 * hist + 4 * scan_sum_words(hist) + 1024;
  return (bytes + 255) & ~size_t(255);  // buffers placed after the scratch stay aligned
}

// Sort (keys, vals) ascending by key into (kout, vout); vals are 64-bit
// words.  scratch holds sort_scratch_bytes(n).
cudaError_t launch_sort_pairs(const uint64_t* keys, const uint64_t* vals, uint64_t n, uint64_t* kout,
                              uint64_t* vout, void* scratch, cudaStream_t st) {
  const uint32_t tiles = uint32_t((n + kSortTile - 1) / kSortTile);
  uint64_t* tk = static_cast<uint64_t*>(scratch);
  uint64_t* tv = tk + n;
  uint32_t* hist = reinterpret_cast<uint32_t*>(tv + n);
  uint32_t* sums = hist + 256ull * tiles;
  const uint64_t* ik = keys;
  const uint64_t* iv = vals;
  // 8 passes; even passes write (tk, tv), odd passes (kout, vout): the last
  // pass lands in kout/vout
  for (uint32_t pass = 0; pass < 8; ++pass) {
    uint64_t* ok = (pass & 1) ? kout : tk;
    uint64_t* ov = (pass & 1) ? vout : tv;
    const uint32_t shift = 8 * pass;
    k_sort_count<<<tiles, kSortThreads, 0, st>>>(ik, n, shift, tiles, hist);
    cudaError_t e = scan_exclusive<uint32_t>(hist, 256ull * tiles, sums, st);
    if (e != cudaSuccess) return e;
    k_sort_scatter<<<tiles, kSortThreads, 0, st>>>(ik, iv, ok, ov, n, shift, tiles, hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ik = ok;
    iv = ov;
  }
  note_launches(8 * 2);  // the scans count their own
  return cudaSuccess;
}

cudaError_t launch_widen_i32(const int32_t* in, uint64_t n, uint64_t* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const uint64_t blocks = (n + 255) / 256, cap = uint64_t(device_sm_count()) * 8;
  k_widen_i32<<<unsigned(blocks < cap ? blocks : cap), 256, 0, st>>>(in, n, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sorted_search(const uint64_t* keys, const uint64_t* vals, uint64_t n, const uint64_t* q,
                                 uint64_t nq, void* out, int out_i64, uint8_t* found, int64_t absent, int sms,
                                 cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  uint64_t blocks = (nq + 255) / 256;
  const uint64_t cap = uint64_t(sms) * 8;
  if (blocks > cap) blocks = cap;
  if (out_i64) k_search<true><<<unsigned(blocks), 256, 0, st>>>(keys, vals, n, q, nq, out, found, absent);
  else k_search<false><<<unsigned(blocks), 256, 0, st>>>(keys, vals, n, q, nq, out, found, absent);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fks

namespace fks {

cudaError_t launch_eytzinger_layout(const uint64_t* sk, const uint64_t* sv, uint64_t n, uint64_t* ek, uint64_t* ev,
                                    int sms, cudaStream_t st) {
  uint64_t blocks = (n + 1 + 255) / 256;
  const uint64_t cap = uint64_t(sms) * 16;
  if (blocks > cap) blocks = cap;
  k_eytz_gather<<<unsigned(blocks), 256, 0, st>>>(sk, sv, n, ek, ev);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_eytzinger_search(const uint64_t* ek, const uint64_t* ev, uint64_t n, const uint64_t* q, uint64_t nq,
                                    void* out, int out_i64, uint8_t* found, int64_t absent, int sms, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  constexpr int kQ = 4;
  uint64_t blocks = (nq + 256 * kQ - 1) / (256 * kQ);
  const uint64_t cap = uint64_t(sms) * 8;
  if (blocks > cap) blocks = cap;
  if (out_i64) k_eytz_search<kQ, true><<<unsigned(blocks), 256, 0, st>>>(ek, ev, n, q, nq, out, found, absent);
  else k_eytz_search<kQ, false><<<unsigned(blocks), 256, 0, st>>>(ek, ev, n, q, nq, out, found, absent);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fks
