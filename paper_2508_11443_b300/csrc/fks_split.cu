// fks_split.cu -- grouping of a build pass's keys by level-one partition in
// two radix levels (most significant digit first), for large passes.
//
// The paper groups keys by their level-one bucket with Hist + Groupby (Sec.
// 2.3-2.5).  Here keys are first brought into contiguous partition ranges
// (a partition = up to 1024 consecutive buckets), each then handled by one CTA in
// k_part_build.  A single scatter with one atomic per key into ~n/1024
// partitions is bound by the L2 atomic rate; two levels of at most a few
// hundred bins each make every write part of a contiguous run and use no
// global atomics:
//
//   level A: digit = partition >> sB   (bins over the whole pass)
//   level B: digit = partition & (2^sB - 1), inside each level-A bin
//
// and each level is count (per tile of kTile keys, a shared histogram) ->
// exclusive scan of the bin-major histogram -> scatter (a shared counting
// sort of the tile, then coalesced writes).  Level A also stores each key's
// partition so level B does not hash again.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fks_internal.cuh"

namespace fks {
namespace {

constexpr uint32_t kTile = 4096;     // keys per tile
constexpr int kSplitThreads = 512;
constexpr uint32_t kMaxBins = 1024;  // bins of one level (larger shapes use the one-level path)
constexpr uint32_t kScanItems = 8192;  // elements per block of the device-wide scan
constexpr int kScanThreads = 512;

__device__ __forceinline__ uint32_t lane() { return threadIdx.x & 31u; }

// The j in [lo, hi) with seg[j] <= e < seg[j + 1] (seg[lo] <= e < seg[hi]).
template <class T>
__device__ __forceinline__ uint32_t seg_in(const T* seg, uint32_t lo, uint32_t hi, uint64_t e) {
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (uint64_t(seg[mid]) <= e) lo = mid; else hi = mid;
  }
  return lo;
}
template <class T>
__device__ __forceinline__ uint32_t seg_of(const T* seg, uint32_t m, uint64_t e) {
  return seg_in(seg, 0u, m, e);
}

// The maps a tile [e0, e1) of a pass spans: [tj[0], tj[1]), found by one
// thread in `seg` (which must be complete: a barrier before the call when it
// is the shared copy) and published by a barrier after it, so that each
// element's search covers those maps only -- most tiles lie inside one map.
__device__ __forceinline__ void tile_maps(const PassDev& p, const uint64_t* seg, uint64_t e0, uint64_t e1,
                                          uint32_t* tj) {
  if (threadIdx.x == 0) {
    tj[0] = p.m == 1 ? 0u : seg_of(seg, p.m, e0);
    tj[1] = p.m == 1 ? 1u : seg_of(seg, p.m, e1 > e0 ? e1 - 1 : e0) + 1;
  }
}

// ------------------------------------------------------------ element access
// Partition and payload of pass element e, read from the pass inputs.
template <bool kStr>
struct Elem {
  uint64_t key, p0, p1;
  uint32_t gp;
};

// Two halves so that a thread issues the loads of all its elements before
// it uses any of them: load_elem reads (the partition field holds the map),
// finish_elem hashes and packs.
template <bool kStr>
__device__ __forceinline__ Elem<kStr> load_elem(const PassDev& p, const uint64_t* seg, const uint32_t* tj,
                                                uint64_t e) {
  const uint32_t j = p.m == 1 ? 0u : seg_in(seg, tj[0], tj[1], e);
  const MapDev& M = p.maps[j];
  const uint64_t in = M.key_begin + (e - M.pass_begin);
  Elem<kStr> x;
  x.key = __ldcs(reinterpret_cast<const unsigned long long*>(p.hkeys) + in);
  const int64_t v = p.vals_i64 ? __ldcs(static_cast<const long long*>(p.vals) + in)
                               : int64_t(__ldcs(static_cast<const int*>(p.vals) + in));
  x.gp = j;
  if (!kStr) {
    x.p0 = uint64_t(v);
    x.p1 = 0;
  } else {
    const int64_t o0 = __ldg(reinterpret_cast<const long long*>(p.offs) + in);
    const int64_t o1 = __ldg(reinterpret_cast<const long long*>(p.offs) + in + 1);
    const bool valid = o0 >= 0 && o1 >= o0 && o1 - o0 < (int64_t(1) << 24) && o1 < (int64_t(1) << 40);
    x.p0 = valid ? offlen_pack(uint64_t(o0), uint64_t(o1 - o0)) : 0ull;  // invalid: empty slice
    x.p1 = uint64_t(v);
  }
  return x;
}

template <bool kStr>
__device__ __forceinline__ void finish_elem(const PassDev& p, Elem<kStr>& x) {
  const MapDev& M = p.maps[x.gp];
  x.gp = M.part_begin + (reduce32(hash32(M.c1, x.key), M.nb) >> p.logB);
}

__device__ __forceinline__ uint64_t key_only(const PassDev& p, const uint64_t* seg, const uint32_t* tj, uint64_t e,
                                             uint32_t* j) {
  *j = p.m == 1 ? 0u : seg_in(seg, tj[0], tj[1], e);
  const MapDev& M = p.maps[*j];
  return __ldcs(reinterpret_cast<const unsigned long long*>(p.hkeys) + M.key_begin + (e - M.pass_begin));
}
__device__ __forceinline__ uint32_t gp_of(const PassDev& p, uint32_t j, uint64_t k) {
  const MapDev& M = p.maps[j];
  return M.part_begin + (reduce32(hash32(M.c1, k), M.nb) >> p.logB);
}

// Level-B tile t -> (level-A bin, first element, end element).
__device__ __forceinline__ bool tile_b(const SplitDev& s, const uint32_t* tstart, uint32_t t,
                                       uint32_t* bin, uint64_t* e0, uint64_t* e1) {
  if (t >= tstart[s.binsA]) return false;
  const uint32_t a = seg_of(tstart, s.binsA, t);
  const uint64_t s0 = s.startA[a], s1 = s.startA[a + 1];
  *bin = a;
  *e0 = s0 + uint64_t(t - tstart[a]) * kTile;
  *e1 = min(s1, *e0 + kTile);
  return true;
}

__device__ __forceinline__ uint64_t histB_index(const SplitDev& s, const uint32_t* tstart, uint32_t a,
                                                uint32_t d, uint32_t t) {
  const uint32_t nt = tstart[a + 1] - tstart[a];
  return uint64_t(tstart[a]) * s.binsB + uint64_t(d) * nt + (t - tstart[a]);
}

// ------------------------------------------------------------ level A
__global__ void __launch_bounds__(kSplitThreads) k_countA(PassDev p, SplitDev s) {
  __shared__ uint32_t hist[kMaxBins];
  __shared__ uint64_t sh_seg[2049];
  const uint64_t* seg = p.pass_seg;
  if (p.m > 1 && p.m <= 2048) {
    for (uint32_t i = threadIdx.x; i <= p.m; i += blockDim.x) sh_seg[i] = p.pass_seg[i];
    seg = sh_seg;
  }
  for (uint32_t i = threadIdx.x; i < s.binsA; i += blockDim.x) hist[i] = 0;
  const uint32_t tile = blockIdx.x;
  const uint64_t e0 = uint64_t(tile) * kTile, e1 = min(p.total, e0 + kTile);
  __shared__ uint32_t tj[2];
  __syncthreads();  // sh_seg is complete before thread 0 searches it
  tile_maps(p, seg, e0, e1, tj);
  __syncthreads();
  constexpr uint32_t kPer = kTile / kSplitThreads;
  uint64_t k[kPer];
  uint32_t jm[kPer];
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {  // all loads first
    const uint64_t e = e0 + threadIdx.x + u * kSplitThreads;
    k[u] = e < e1 ? key_only(p, seg, tj, e, &jm[u]) : 0ull;
  }
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {
    const uint64_t e = e0 + threadIdx.x + u * kSplitThreads;
    if (e < e1) atomicAdd(hist + (gp_of(p, jm[u], k[u]) >> s.shiftB), 1u);
  }
  __syncthreads();
  for (uint32_t a = threadIdx.x; a < s.binsA; a += blockDim.x) s.histA[uint64_t(a) * s.tilesA + tile] = hist[a];
}

template <bool kStr>
__global__ void __launch_bounds__(kSplitThreads, 2) k_scatterA(PassDev p, SplitDev s) {
  constexpr int PW = kStr ? 2 : 1;
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem);
  uint64_t* spay = skey + kTile;
  uint32_t* sgp = reinterpret_cast<uint32_t*>(spay + PW * kTile);
  __shared__ uint32_t cur[kMaxBins], lstart[kMaxBins], dbase[kMaxBins], wsum[kSplitThreads / 32];
  __shared__ uint64_t sh_seg[2049];
  const uint64_t* seg = p.pass_seg;
  if (p.m > 1 && p.m <= 2048) {
    for (uint32_t i = threadIdx.x; i <= p.m; i += blockDim.x) sh_seg[i] = p.pass_seg[i];
    seg = sh_seg;
  }
  const uint32_t tile = blockIdx.x;
  for (uint32_t i = threadIdx.x; i < s.binsA; i += blockDim.x) {
    cur[i] = 0;
    dbase[i] = s.histA[uint64_t(i) * s.tilesA + tile];  // this tile's output start per bin
  }
  const uint64_t e0 = uint64_t(tile) * kTile, e1 = min(p.total, e0 + kTile);
  __shared__ uint32_t tj[2];
  __syncthreads();  // sh_seg is complete before thread 0 searches it
  tile_maps(p, seg, e0, e1, tj);
  __syncthreads();
  const uint32_t cnt = uint32_t(e1 - e0);
  constexpr uint32_t kPer = kTile / kSplitThreads;
  Elem<kStr> x[kPer];
  uint32_t rank[kPer];
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {  // all loads first
    const uint32_t i = threadIdx.x + u * kSplitThreads;
    if (i < cnt) x[u] = load_elem<kStr>(p, seg, tj, e0 + i);
  }
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {
    const uint32_t i = threadIdx.x + u * kSplitThreads;
    if (i < cnt) {
      finish_elem<kStr>(p, x[u]);
      rank[u] = atomicAdd(cur + (x[u].gp >> s.shiftB), 1u);
    }
  }
  __syncthreads();
  // exclusive scan of the tile histogram (binsA <= kMaxBins)
  {
    constexpr uint32_t kPerBin = kMaxBins / kSplitThreads;
    uint32_t c[kPerBin], sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPerBin; ++q) {
      const uint32_t b = threadIdx.x * kPerBin + q;
      c[q] = b < s.binsA ? cur[b] : 0u;
      sum += c[q];
    }
    uint32_t inc = sum;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
      if (lane() >= uint32_t(d)) inc += y;
    }
    if (lane() == 31) wsum[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t base = 0;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) base += wsum[w];
    uint32_t run = base + inc - sum;
#pragma unroll
    for (uint32_t q = 0; q < kPerBin; ++q) {
      const uint32_t b = threadIdx.x * kPerBin + q;
      if (b < s.binsA) lstart[b] = run;
      run += c[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {
    const uint32_t i = threadIdx.x + u * kSplitThreads;
    if (i < cnt) {
      const uint32_t pos = lstart[x[u].gp >> s.shiftB] + rank[u];
      skey[pos] = x[u].key;
      spay[PW * pos] = x[u].p0;
      if (kStr) spay[PW * pos + 1] = x[u].p1;
      sgp[pos] = x[u].gp;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const uint32_t gp = sgp[i], a = gp >> s.shiftB;
    const uint64_t dst = uint64_t(dbase[a]) + (i - lstart[a]);
    s.keyA[dst] = skey[i];
    s.payA[PW * dst] = spay[PW * i];
    if (kStr) s.payA[PW * dst + 1] = spay[PW * i + 1];
    s.gpA[dst] = gp;
  }
}

// level-A bin starts, level-B tiles per bin (one CTA)
__global__ void __launch_bounds__(1024) k_binsA(PassDev p, SplitDev s) {
  __shared__ uint32_t wsum[32];
  const uint32_t t = threadIdx.x;
  // startA[a] = histA scanned at (a, tile 0); startA[binsA] = total
  for (uint32_t a = t; a < s.binsA; a += blockDim.x) s.startA[a] = s.histA[uint64_t(a) * s.tilesA];
  if (t == 0) s.startA[s.binsA] = p.total;
  __syncthreads();
  // tiles of level B per bin, exclusive scan (binsA <= kMaxBins, 2 per thread)
  uint32_t c[2], sum = 0;
  for (int q = 0; q < 2; ++q) {
    const uint32_t a = t * 2 + q;
    c[q] = a < s.binsA ? uint32_t((s.startA[a + 1] - s.startA[a] + kTile - 1) / kTile) : 0u;
    sum += c[q];
  }
  uint32_t inc = sum;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane() >= uint32_t(d)) inc += y;
  }
  if (lane() == 31) wsum[t >> 5] = inc;
  __syncthreads();
  uint32_t base = 0;
  for (uint32_t w = 0; w < (t >> 5); ++w) base += wsum[w];
  uint32_t run = base + inc - sum;
  for (int q = 0; q < 2; ++q) {
    const uint32_t a = t * 2 + q;
    if (a < s.binsA) s.tstartB[a] = run;
    if (a == s.binsA - 1) s.tstartB[s.binsA] = run + c[q];
    run += c[q];
  }
}

// ------------------------------------------------------------ level B
__global__ void __launch_bounds__(kSplitThreads) k_countB(PassDev p, SplitDev s) {
  __shared__ uint32_t hist[kMaxBins];
  const uint32_t t = blockIdx.x;
  uint32_t a;
  uint64_t e0, e1;
  if (!tile_b(s, s.tstartB, t, &a, &e0, &e1)) return;
  for (uint32_t i = threadIdx.x; i < s.binsB; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint32_t mask = s.binsB - 1;
  constexpr uint32_t kPer = kTile / kSplitThreads;
  uint32_t g[kPer];
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {  // all loads first
    const uint64_t e = e0 + threadIdx.x + u * kSplitThreads;
    g[u] = e < e1 ? __ldcs(s.gpA + e) : 0u;
  }
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u)
    if (e0 + threadIdx.x + u * kSplitThreads < e1) atomicAdd(hist + (g[u] & mask), 1u);
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < s.binsB; d += blockDim.x) s.histB[histB_index(s, s.tstartB, a, d, t)] = hist[d];
  (void)p;
}

template <bool kStr>
__global__ void __launch_bounds__(kSplitThreads, 2) k_scatterB(PassDev p, SplitDev s) {
  constexpr int PW = kStr ? 2 : 1;
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem);
  uint64_t* spay = skey + kTile;
  uint16_t* sdig = reinterpret_cast<uint16_t*>(spay + PW * kTile);
  __shared__ uint32_t cur[kMaxBins], lstart[kMaxBins], dbase[kMaxBins], wsum[kSplitThreads / 32];
  const uint32_t t = blockIdx.x;
  uint32_t a;
  uint64_t e0, e1;
  if (!tile_b(s, s.tstartB, t, &a, &e0, &e1)) return;
  for (uint32_t i = threadIdx.x; i < s.binsB; i += blockDim.x) {
    cur[i] = 0;
    dbase[i] = s.histB[histB_index(s, s.tstartB, a, i, t)];  // this tile's output start per bin
  }
  __syncthreads();
  const uint32_t cnt = uint32_t(e1 - e0), mask = s.binsB - 1;
  constexpr uint32_t kPer = kTile / kSplitThreads;
  uint64_t k[kPer], q0[kPer], q1[kPer];
  uint32_t d[kPer], rank[kPer];
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {  // all loads first
    const uint32_t i = threadIdx.x + u * kSplitThreads;
    if (i < cnt) {
      const uint64_t e = e0 + i;
      k[u] = __ldcs(reinterpret_cast<const unsigned long long*>(s.keyA) + e);
      q0[u] = __ldcs(reinterpret_cast<const unsigned long long*>(s.payA) + PW * e);
      q1[u] = kStr ? __ldcs(reinterpret_cast<const unsigned long long*>(s.payA) + PW * e + 1) : 0ull;
      d[u] = __ldcs(s.gpA + e) & mask;
    }
  }
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u)
    if (threadIdx.x + u * kSplitThreads < cnt) rank[u] = atomicAdd(cur + d[u], 1u);
  __syncthreads();
  {
    constexpr uint32_t kPerBin = kMaxBins / kSplitThreads;
    uint32_t c[kPerBin], sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPerBin; ++q) {
      const uint32_t b = threadIdx.x * kPerBin + q;
      c[q] = b < s.binsB ? cur[b] : 0u;
      sum += c[q];
    }
    uint32_t inc = sum;
    for (int dd = 1; dd < 32; dd <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, dd);
      if (lane() >= uint32_t(dd)) inc += y;
    }
    if (lane() == 31) wsum[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t base = 0;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) base += wsum[w];
    uint32_t run = base + inc - sum;
#pragma unroll
    for (uint32_t q = 0; q < kPerBin; ++q) {
      const uint32_t b = threadIdx.x * kPerBin + q;
      if (b < s.binsB) lstart[b] = run;
      run += c[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (uint32_t u = 0; u < kPer; ++u) {
    const uint32_t i = threadIdx.x + u * kSplitThreads;
    if (i < cnt) {
      const uint32_t pos = lstart[d[u]] + rank[u];
      skey[pos] = k[u];
      spay[PW * pos] = q0[u];
      if (kStr) spay[PW * pos + 1] = q1[u];
      sdig[pos] = uint16_t(d[u]);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const uint32_t dg = sdig[i];
    const uint64_t dst = uint64_t(dbase[dg]) + (i - lstart[dg]);
    p.stage_key[dst] = skey[i];
    p.stage_pay[PW * dst] = spay[PW * i];
    if (kStr) p.stage_pay[PW * dst + 1] = spay[PW * i + 1];
  }
}

// partition starts from the scanned level-B histogram; clears the state the
// partition kernel expects zero
__global__ void __launch_bounds__(256) k_part_starts(PassDev p, SplitDev s) {
  const uint32_t gstride = gridDim.x * blockDim.x;
  for (uint32_t gp = blockIdx.x * blockDim.x + threadIdx.x; gp < p.P; gp += gstride) {
    const uint32_t a = gp >> s.shiftB, d = gp & (s.binsB - 1);
    const uint32_t nt = s.tstartB[a + 1] - s.tstartB[a];
    p.part_start[gp] = nt ? s.histB[histB_index(s, s.tstartB, a, d, s.tstartB[a])] : uint32_t(s.startA[a]);
    p.lookback[gp] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.part_start[p.P] = uint32_t(p.total);
    *p.ticket = 0;
    *p.ovf_count = 0;
  }
}

// ------------------------------------------------------------ device-wide exclusive scan
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T* in, uint64_t n, T* sums) {
  __shared__ T ws[kScanThreads / 32];
  const uint64_t b0 = uint64_t(blockIdx.x) * kScanItems;
  T v = 0;
  for (uint64_t i = b0 + threadIdx.x; i < min(n, b0 + kScanItems); i += kScanThreads) v += in[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
  if (lane() == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) tot += ws[w];
    sums[blockIdx.x] = tot;
  }
}

template <class T>
__global__ void __launch_bounds__(1024) k_scan_sums(T* sums, uint32_t nb) {
  __shared__ T ws[32];
  __shared__ T carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < nb; c0 += 1024) {
    const uint32_t i = c0 + threadIdx.x;
    const T v = i < nb ? sums[i] : T(0);
    T inc = v;
    for (int d = 1; d < 32; d <<= 1) {
      const T y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
      if (lane() >= uint32_t(d)) inc += y;
    }
    if (lane() == 31) ws[threadIdx.x >> 5] = inc;
    __syncthreads();
    T base = carry;
    for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) base += ws[w];
    if (i < nb) sums[i] = base + inc - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = base + inc;
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(T* data, uint64_t n, const T* sums) {
  __shared__ T ws[kScanThreads / 32];
  constexpr uint32_t kPer = kScanItems / kScanThreads;  // 16 consecutive per thread
  const uint64_t b0 = uint64_t(blockIdx.x) * kScanItems + uint64_t(threadIdx.x) * kPer;
  T v[kPer], sum = 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    v[q] = b0 + q < n ? data[b0 + q] : T(0);
    sum += v[q];
  }
  T inc = sum;
  for (int d = 1; d < 32; d <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane() >= uint32_t(d)) inc += y;
  }
  if (lane() == 31) ws[threadIdx.x >> 5] = inc;
  __syncthreads();
  T run = sums[blockIdx.x];
  for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) run += ws[w];
  run += inc - sum;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    if (b0 + q < n) data[b0 + q] = run;
    run += v[q];
  }
}

}  // namespace

template <class T>
cudaError_t scan_exclusive(T* data, uint64_t n, T* sums, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const uint32_t nb = uint32_t((n + kScanItems - 1) / kScanItems);
  k_scan_reduce<T><<<nb, kScanThreads, 0, st>>>(data, n, sums);
  k_scan_sums<T><<<1, 1024, 0, st>>>(sums, nb);
  k_scan_down<T><<<nb, kScanThreads, 0, st>>>(data, n, sums);
  note_launches(3);
  return cudaGetLastError();
}
template cudaError_t scan_exclusive<uint32_t>(uint32_t*, uint64_t, uint32_t*, cudaStream_t);
template cudaError_t scan_exclusive<uint64_t>(uint64_t*, uint64_t, uint64_t*, cudaStream_t);

size_t scan_sum_words(uint64_t n) { return size_t((n + kScanItems - 1) / kScanItems) + 2; }

SplitShape split_shape(uint32_t P, uint64_t total) {
  SplitShape sh{};
  uint32_t L = 0;
  while ((1ull << L) < P) ++L;
  sh.shiftB = L / 2;
  sh.binsB = 1u << sh.shiftB;
  sh.binsA = (P + sh.binsB - 1) >> sh.shiftB;
  if (sh.binsA == 0) sh.binsA = 1;
  sh.tilesA = uint32_t((total + kTile - 1) / kTile);
  sh.tilesB_max = sh.tilesA + sh.binsA;
  sh.ok = sh.binsA <= kMaxBins && sh.binsB <= kMaxBins;
  return sh;
}

size_t split_hist_words(const SplitShape& sh) {
  const uint64_t a = uint64_t(sh.binsA) * sh.tilesA, b = uint64_t(sh.binsB) * sh.tilesB_max;
  return size_t(a > b ? a : b);
}

size_t split_sum_words(const SplitShape& sh) {
  return split_hist_words(sh) / kScanItems + 2;
}

cudaError_t launch_split(const PassDev& p, const SplitDev& s, bool strings, cudaStream_t st) {
  cudaError_t e;
  const int PW = strings ? 2 : 1;
  const size_t smemA = size_t(kTile) * 8 * (1 + PW) + size_t(kTile) * 4;
  const size_t smemB = size_t(kTile) * 8 * (1 + PW) + size_t(kTile) * 2;
  // the scatters' shared-memory attribute, set once per process (thread-safe
  // static initialisation; concurrent first builds wait for it)
  static const cudaError_t attr = [] {
    cudaError_t r = cudaSuccess;
    const int a = int(kTile * 8 * 3 + kTile * 4), b = int(kTile * 8 * 3 + kTile * 2);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_scatterA<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, a);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_scatterA<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, a);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_scatterB<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(k_scatterB<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return r;
  }();
  if (attr != cudaSuccess) return attr;
  k_countA<<<s.tilesA, kSplitThreads, 0, st>>>(p, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = scan_exclusive<uint32_t>(s.histA, uint64_t(s.binsA) * s.tilesA, s.sums, st)) != cudaSuccess) return e;
  if (strings) k_scatterA<true><<<s.tilesA, kSplitThreads, smemA, st>>>(p, s);
  else k_scatterA<false><<<s.tilesA, kSplitThreads, smemA, st>>>(p, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_binsA<<<1, 1024, 0, st>>>(p, s);
  k_countB<<<s.tilesB_max, kSplitThreads, 0, st>>>(p, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // entries past the last real level-B tile are never written or read; they
  // only trail the real ones in the scan
  if ((e = scan_exclusive<uint32_t>(s.histB, uint64_t(s.binsB) * s.tilesB_max, s.sums, st)) != cudaSuccess) return e;
  if (strings) k_scatterB<true><<<s.tilesB_max, kSplitThreads, smemB, st>>>(p, s);
  else k_scatterB<false><<<s.tilesB_max, kSplitThreads, smemB, st>>>(p, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t blocks = (p.P + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_part_starts<<<blocks, 256, 0, st>>>(p, s);
  note_launches(6);  // the two scans count their own three
  return cudaGetLastError();
}

}  // namespace fks
