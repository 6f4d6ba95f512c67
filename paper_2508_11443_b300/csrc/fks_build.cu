// fks_build.cu -- device construction of FKS two-level hash maps.
//
// The paper's data-parallel construction (Sec. 2.3-2.5) groups keys by their
// level-one hash with Hist + Groupby (the sortless form tags every key with
// its bucket and re-runs only the buckets that collided).  On sm_103a the
// same steps are arranged around the memory hierarchy:
//
//   pass 1  k_partition<count>   g k for every key; keys per partition of
//                                2^logB consecutive buckets (1024 with one
//                                bucket per key; about 1024 keys in any
//                                case), L2 atomics on a small counter array,
//                                warp-aggregated
//   pass 2  k_scan_parts         exclusive scan of the partition counts
//   pass 3  k_partition<scatter> keys (+ payload) scattered into contiguous
//                                partition ranges
//   pass 4  k_part_build         one CTA per partition, a persistent work
//                                queue: Hist of the partition's buckets in
//                                shared memory, exclusive Presum of s and s^2,
//                                a decoupled look-back across partitions for
//                                the map-level slot offsets (Presum shape),
//                                Groupby into shared memory, level-two search
//                                per bucket (make_2: the first attempt with no
//                                collision inside s^2 slots), descriptors and
//                                slot image written out coalesced.
//
// The level-one space bound (sum s^2 <= bound * n) is checked on the running
// slot prefix; a map that exceeds it is redrawn by the host (next round).
// Partitions with more keys than shared memory holds are deferred to
// k_part_overflow, which runs the same steps on global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fks_internal.cuh"
#include "fks_strings.cuh"

namespace fks {
namespace {

constexpr int kUnroll = 4;
constexpr uint64_t kLbFlagA = 1ull << 62;
constexpr uint64_t kLbFlagP = 2ull << 62;
constexpr uint64_t kLbVal = (1ull << 62) - 1;
constexpr uint64_t kSat = 1ull << 61;

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t sat(uint64_t x) { return x < kSat ? x : kSat; }

template <class T>
__device__ __forceinline__ uint32_t upper_seg(const T* seg, uint32_t m, uint64_t e) {
  // largest j in [0, m) with seg[j] <= e  (seg[0] = 0 <= e < seg[m])
  uint32_t lo = 0, hi = m;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (uint64_t(seg[mid]) <= e) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t load_val(const void* vals, int i64, uint64_t i) {
  return i64 ? __ldg(static_cast<const long long*>(vals) + i)
             : int64_t(__ldg(static_cast<const int*>(vals) + i));
}

// -------------------------------------------------------------- fingerprints
__global__ void __launch_bounds__(256) k_fingerprints(const uint8_t* __restrict__ ctx,
                                                      const int64_t* __restrict__ offs,
                                                      const MapDev* __restrict__ maps,
                                                      const uint64_t* __restrict__ pass_seg,
                                                      uint32_t m, uint64_t total,
                                                      uint64_t* __restrict__ fps,
                                                      MapStatus* status) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const uint32_t j = m == 1 ? 0u : upper_seg(pass_seg, m, e);
    const MapDev& M = maps[j];
    const uint64_t in = M.key_begin + (e - M.pass_begin);
    const int64_t o0 = __ldg(reinterpret_cast<const long long*>(offs) + in);
    const int64_t o1 = __ldg(reinterpret_cast<const long long*>(offs) + in + 1);
    const int64_t len = o1 - o0;
    if (o0 < 0 || len < 0 || len >= (int64_t(1) << 24) || o1 >= (int64_t(1) << 40)) {
      atomicExch(&status[j].invalid, 1u);
      fps[in] = 0;
      continue;
    }
    fps[in] = fingerprint(ctx + o0, uint32_t(len), M.fpb);
  }
}

// The same for a one-map pass: a string longer than kLongString bytes is
// fingerprinted by the whole warp (lanes take its words), so that it does
// not hold up the other lanes for its whole length; shorter ones by their
// own lane.
__global__ void __launch_bounds__(256, 8) k_fingerprints_map(const uint8_t* __restrict__ ctx,
                                                           const int64_t* __restrict__ offs,
                                                           const MapDev* __restrict__ maps, uint64_t total,
                                                           uint64_t* __restrict__ fps, MapStatus* status) {
  __shared__ uint64_t pw[33];
  const uint64_t key_begin = maps[0].key_begin, pass_begin = maps[0].pass_begin;
  if (threadIdx.x < 33) pw[threadIdx.x] = pow61(maps[0].fpb, threadIdx.x);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nwarps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t base = (uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < total;
       base += nwarps * 32) {
    const uint64_t e = base + lane;
    const uint64_t in = key_begin + (e - pass_begin);
    int64_t o0 = 0, o1 = 0;
    if (e < total) {
      o0 = __ldg(reinterpret_cast<const long long*>(offs) + in);
      o1 = __ldg(reinterpret_cast<const long long*>(offs) + in + 1);
    }
    const int64_t len = o1 - o0;
    const bool bad = e < total && (o0 < 0 || len < 0 || len >= (int64_t(1) << 24) || o1 >= (int64_t(1) << 40));
    if (bad) atomicExch(&status[0].invalid, 1u);
    const bool ok = e < total && !bad;
    const bool lng = ok && uint64_t(len) > kLongString;
    uint64_t fp = 0;
    if (ok && !lng) fp = fingerprint(ctx + o0, uint32_t(len), pw[1]);
    for (uint32_t todo = __ballot_sync(0xFFFFFFFFu, lng); todo; todo &= todo - 1) {
      const int j = __ffs(todo) - 1;
      const int64_t oj = __shfl_sync(0xFFFFFFFFu, o0, j);
      const uint32_t lj = uint32_t(__shfl_sync(0xFFFFFFFFu, len, j));
      const uint64_t h = warp_fingerprint(ctx + oj, lj, pw);
      if (int(lane) == j) fp = h;
    }
    if (e < total) fps[in] = fp;  // 0 for invalid offsets
  }
}

// -------------------------------------------------------------- partitioning
// Warp-aggregated claim of `count` consecutive cells of ctr[idx]: lanes with
// the same idx share one atomic (the paper's Hist, Sec. 2.1, with atomics).
template <bool kNeedPos>
__device__ __forceinline__ uint32_t claim(uint32_t* ctr, uint32_t idx, bool valid, bool agg) {
  if (!agg) {
    if (!valid) return 0;
    if (kNeedPos) return atomicAdd(ctr + idx, 1u);
    atomicAdd(ctr + idx, 1u);
    return 0;
  }
  const uint32_t key = valid ? idx : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
  const uint32_t leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (valid && lane_id() == leader) {
    if (kNeedPos) base = atomicAdd(ctr + idx, uint32_t(__popc(peers)));
    else atomicAdd(ctr + idx, uint32_t(__popc(peers)));
  }
  if (!kNeedPos) return 0;
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & lanemask_lt());
}

template <bool kScatter, bool kStr>
__global__ void __launch_bounds__(256) k_partition(PassDev p, int agg) {
  extern __shared__ uint64_t sh_seg[];
  const uint64_t* seg = p.pass_seg;
  if (p.m > 1 && p.m <= 2048) {
    for (uint32_t i = threadIdx.x; i <= p.m; i += blockDim.x) sh_seg[i] = p.pass_seg[i];
    __syncthreads();
    seg = sh_seg;
  }
  const uint32_t lane = lane_id();
  const uint64_t warp0 = (uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u)) * kUnroll;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kUnroll;
  const MapDev* maps = p.maps;
  // the one-map case keeps its parameters in registers
  const uint64_t kb0 = maps[0].key_begin, pb0 = maps[0].pass_begin;
  const HashConsts c10 = maps[0].c1;
  const uint32_t n0 = maps[0].nb, part0 = maps[0].part_begin;
  const uint32_t logB = p.logB;
  const uint64_t* __restrict__ hkeys = p.hkeys;
  for (uint64_t base = warp0; base < p.total; base += stride) {
    uint64_t k[kUnroll], in[kUnroll], pv[kUnroll], po[kUnroll];
    uint32_t gp[kUnroll];
    bool ok[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t e = base + uint64_t(u) * 32 + lane;
      ok[u] = e < p.total;
      pv[u] = po[u] = 0;
      if (p.m == 1) {
        in[u] = kb0 + (e - pb0);
        k[u] = ok[u] ? __ldcs(reinterpret_cast<const unsigned long long*>(hkeys) + in[u]) : 0;
        gp[u] = part0 + (reduce32(hash32(c10, k[u]), n0) >> logB);
      } else {
        const uint32_t j = ok[u] ? upper_seg(seg, p.m, e) : 0u;
        in[u] = maps[j].key_begin + (e - maps[j].pass_begin);
        k[u] = ok[u] ? __ldcs(reinterpret_cast<const unsigned long long*>(hkeys) + in[u]) : 0;
        const HashConsts c1 = maps[j].c1;
        gp[u] = maps[j].part_begin + (reduce32(hash32(c1, k[u]), maps[j].nb) >> logB);
      }
      if (kScatter && ok[u]) {  // payload loads issued before the claims
        pv[u] = uint64_t(load_val(p.vals, p.vals_i64, in[u]));
        if (kStr) {
          const int64_t o0 = __ldg(reinterpret_cast<const long long*>(p.offs) + in[u]);
          const int64_t o1 = __ldg(reinterpret_cast<const long long*>(p.offs) + in[u] + 1);
          const bool valid = o0 >= 0 && o1 >= o0 && o1 - o0 < (int64_t(1) << 24) && o1 < (int64_t(1) << 40);
          // invalid offsets (the map fails with INVALID_ARG) become an empty slice
          po[u] = valid ? offlen_pack(uint64_t(o0), uint64_t(o1 - o0)) : 0ull;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (!kScatter) {
        claim<false>(p.part_cnt, gp[u], ok[u], agg);
      } else {
        const uint32_t pos = claim<true>(p.part_cursor, gp[u], ok[u], agg);
        if (ok[u]) {
          p.stage_key[pos] = k[u];
          if (!kStr) p.stage_pay[pos] = pv[u];
          else reinterpret_cast<ulonglong2*>(p.stage_pay)[pos] = make_ulonglong2(po[u], pv[u]);
        }
      }
    }
  }
}

// One CTA: exclusive scan of the partition counts; clears the look-back words,
// the work-queue head and the overflow counter for the build kernel.
__global__ void __launch_bounds__(1024) k_scan_parts(PassDev p) {
  __shared__ uint32_t wsum[32];
  const uint32_t T = blockDim.x, t = threadIdx.x;
  const uint32_t per = (p.P + T - 1) / T;
  const uint32_t lo = min(p.P, t * per), hi = min(p.P, lo + per);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; ++i) {
    sum += p.part_cnt[i];
    p.lookback[i] = 0;
  }
  uint32_t incl = sum;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane_id() >= uint32_t(d)) incl += x;
  }
  if (lane_id() == 31) wsum[t >> 5] = incl;
  __syncthreads();
  if (t < 32) {
    uint32_t w = t < (T >> 5) ? wsum[t] : 0u, wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, wi, d);
      if (t >= uint32_t(d)) wi += x;
    }
    wsum[t] = wi - w;
  }
  __syncthreads();
  uint32_t run = wsum[t >> 5] + incl - sum;
  for (uint32_t i = lo; i < hi; ++i) {
    p.part_start[i] = run;
    p.part_cursor[i] = run;
    run += p.part_cnt[i];
  }
  if (t == T - 1) p.part_start[p.P] = run;
  if (t == 0) {
    *p.ticket = 0;
    *p.ovf_count = 0;
  }
}

// -------------------------------------------------------------- partition CTA
// Search classes of a bucket of s >= 2 keys: 0 = one thread (s <= thr), 1..5 =
// a segment of 2^cls lanes (s <= 32), 6 = the whole CTA.
constexpr uint32_t kClasses = 7;
// With at most kCap keys a class of buckets of >= s_min keys has at most
// kCap / s_min entries (s_min = 2, 2, 3, 5, 9, 17, 33 for classes 0..6; class
// 1 holds buckets of 2 keys only when one-thread searches stop at a single
// key): fixed list regions in the work array, a select chain over
// compile-time constants (the index is a runtime value in the kernel).
constexpr uint32_t kRegion1 = kCap / 2, kRegion2 = kRegion1 + kCap / 2, kRegion3 = kRegion2 + kCap / 3,
                   kRegion4 = kRegion3 + kCap / 5, kRegion5 = kRegion4 + kCap / 9,
                   kRegion6 = kRegion5 + kCap / 17, kWorkEntries = kRegion6 + kCap / 33;
__host__ __device__ __forceinline__ constexpr uint32_t class_region(uint32_t c) {
  return c == 0 ? 0u
         : c == 1 ? kRegion1
         : c == 2 ? kRegion2
         : c == 3 ? kRegion3
         : c == 4 ? kRegion4
         : c == 5 ? kRegion5
         : kRegion6;
}
static_assert(kCap != 2048 || kWorkEntries == 3548, "class regions of a 2048-key partition");

__host__ __device__ constexpr uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Shared memory of a partition CTA.  raw*: the partition's staged keys and
// payloads as delivered by the bulk-copy engine (the key range may start one
// element early to keep the copy 16-byte aligned); g*: the same entries
// grouped by bucket; owner: the partition's slot image as member indices.
template <int PW>
struct Smem {
  static constexpr uint32_t kRawN = kCap + 2;
  static constexpr uint32_t kRawKey = 0;
  static constexpr uint32_t kRawPay = align16(kRawKey + kRawN * 8);
  static constexpr uint32_t kGkey = align16(kRawPay + kRawN * 8 * PW);
  static constexpr uint32_t kGpay = kGkey + kCap * 8;
  static constexpr uint32_t kOwner = kGpay + kCap * 8 * PW;
  static constexpr uint32_t kCnt = kOwner + kOwnerCap * 2;
  static constexpr uint32_t kGst = kCnt + kB * 4;
  static constexpr uint32_t kSoff = kGst + (kB + 4) * 4;
  static constexpr uint32_t kAtt = kSoff + kB * 4;
  static constexpr uint32_t kWork = align16(kAtt + kB * 2);  // class lists of the buckets to search
  static constexpr uint32_t kBytes = align16(kWork + kWorkEntries * 2);
};

struct PartCtl {
  uint32_t gp, skip, nbig, maxs, maxatt, flag_a, flag_b, nonempty;
  uint32_t failed;  // a bucket found no constants: this pass of the map is discarded
  uint32_t nwork;
  uint32_t ccnt[8], cbase[8], ccur[8];  // search classes: list sizes, starts, cursors
  uint32_t next_gp, next_issued, abort;
  uint64_t next_e0, next_e1;  // staged range of partition next_gp
  uint64_t excl, Spart, attsum;
  unsigned long long fillmin;  // (slot << 32) | member of a CTA-searched bucket
  uint32_t wsum[kPartThreads / 32];
  uint64_t wsum2[kPartThreads / 32];
};

struct MapRegs {
  HashConsts c1;
  uint64_t seed, desc_base, slot_base;
  uint32_t nb, round, slot_cap, part_begin, part_end;  // nb: level-one buckets
};

__device__ __forceinline__ MapRegs load_map(const PassDev& p, uint32_t j) {
  const MapDev& M = p.maps[j];
  MapRegs r;
  r.c1 = M.c1;
  r.seed = M.seed;
  r.desc_base = M.desc_base;
  r.slot_base = M.slot_base;
  r.nb = M.nb;
  r.round = M.round;
  r.slot_cap = M.slot_cap;
  r.part_begin = M.part_begin;
  r.part_end = p.part_seg[j + 1];
  return r;
}

// ---- bulk copies into shared memory, completion on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One thread: start the copy of partition gp's staged range into raw* and
// record the range in *r0, *r1.  Returns 1 if a copy was issued (the caller
// waits on the mbarrier).
template <int PW>
__device__ uint32_t issue_stage(const PassDev& p, uint32_t gp, uint64_t* raw_key, uint64_t* raw_pay,
                                uint64_t* bar, uint64_t* r0, uint64_t* r1) {
  if (gp >= p.P) return 0;
  const uint64_t e0 = p.part_start[gp], e1 = p.part_start[gp + 1];
  *r0 = e0;
  *r1 = e1;
  if (e1 == e0 || e1 - e0 > kCap) return 0;
  const uint64_t a0 = e0 & ~1ull;                 // 16-byte aligned start of the key copy
  const uint32_t nk = uint32_t((e1 - a0 + 1) & ~1ull);  // even element count
  const uint32_t bk = nk * 8u;
  const uint32_t bp = PW == 1 ? bk : uint32_t(e1 - e0) * 16u;
  const uint64_t* sp = PW == 1 ? p.stage_pay + a0 : p.stage_pay + 2 * e0;
  fence_proxy_async_smem();
  mbar_expect_tx(bar, bk + bp);
  bulk_g2s(raw_key, p.stage_key + a0, bk, bar);
  bulk_g2s(raw_pay, sp, bp, bar);
  return 1;
}

// Exclusive Presum of s and s^2 over the partition's nb <= kB buckets
// (cnt[] holds s).  Leaves gst[] the group starts (gst[nb] = keys), soff[]
// the partition-local slot offsets, ctl.Spart = sum s^2, ctl.maxs,
// ctl.nonempty.
__device__ void scan_buckets(const uint32_t* cnt, uint32_t* gst, uint32_t* soff, PartCtl& ctl, uint32_t nb) {
  const uint32_t t = threadIdx.x;
  constexpr uint32_t kPer = kB / kPartThreads;
  uint32_t c[kPer], ls = 0, mx = 0, ne = 0;
  uint64_t ls2 = 0;
#pragma unroll
  for (uint32_t i = 0; i < kPer; ++i) {
    c[i] = t * kPer + i < nb ? cnt[t * kPer + i] : 0u;
    ls += c[i];
    ls2 += uint64_t(c[i]) * c[i];
    mx = max(mx, c[i]);
    ne += c[i] != 0;
  }
  uint32_t inc = ls;
  uint64_t inc2 = ls2;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    const uint64_t x2 = __shfl_up_sync(0xFFFFFFFFu, inc2, d);
    if (lane_id() >= uint32_t(d)) {
      inc += x;
      inc2 += x2;
    }
  }
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  ne = __reduce_add_sync(0xFFFFFFFFu, ne);
  if (lane_id() == 31) {
    ctl.wsum[t >> 5] = inc;
    ctl.wsum2[t >> 5] = inc2;
  }
  if (lane_id() == 0) {
    atomicMax(&ctl.maxs, mx);
    atomicAdd(&ctl.nonempty, ne);
  }
  __syncthreads();
  uint32_t we = 0;
  uint64_t we2 = 0;
  for (uint32_t w = 0; w < (t >> 5); ++w) {
    we += ctl.wsum[w];
    we2 += ctl.wsum2[w];
  }
  uint32_t run = we + inc - ls;
  uint64_t run2 = we2 + inc2 - ls2;
#pragma unroll
  for (uint32_t i = 0; i < kPer; ++i) {
    if (t * kPer + i < nb) {
      gst[t * kPer + i] = run;
      soff[t * kPer + i] = uint32_t(run2 < 0xFFFFFFFFull ? run2 : 0xFFFFFFFFull);
    }
    run += c[i];
    run2 += uint64_t(c[i]) * c[i];
  }
  if (t == kPartThreads - 1) {  // past every bucket: run = keys, run2 = sum s^2
    gst[nb] = run;
    ctl.Spart = run2;
  }
  __syncthreads();
}

// Hist of a partition's buckets straight from global memory (overflow path).
__device__ __noinline__ void count_global(const PassDev& p, const MapRegs& M, uint32_t b0, uint64_t e0,
                                          uint64_t e1, uint32_t* cnt) {
  for (uint64_t e = e0 + threadIdx.x; e < e1; e += kPartThreads) {
    const uint64_t k = p.stage_key[e];
    atomicAdd(cnt + (reduce32(hash32(M.c1, k), M.nb) - b0), 1u);
  }
}

// Decoupled look-back, in two halves so that the wait can be deferred.
// publish_aggregate (one thread): make this partition's slot count visible
// (the first partition of a map publishes its inclusive prefix at once).
__device__ __forceinline__ void publish_aggregate(const PassDev& p, uint32_t gp, uint32_t first,
                                                  uint64_t agg) {
  if (p.cfg.hold_first && gp == 0) return;
  st_relaxed(p.lookback + gp, (gp == first ? kLbFlagP : kLbFlagA) | sat(agg));
}

// resolve_prefix (one warp): exclusive slot prefix of partition gp within
// its map, 32 predecessors per step, then publish the inclusive prefix.
// Every wait is bounded by cfg.spin_limit polls.
__device__ uint64_t resolve_prefix(const PassDev& p, uint32_t gp, uint32_t first, uint64_t agg,
                                   bool* timed_out) {
  const uint32_t lane = lane_id();
  const bool hold = p.cfg.hold_first && gp == 0;
  *timed_out = false;
  if (gp == first) return 0;
  uint64_t excl = 0;
  int64_t hi = int64_t(gp) - 1;
  uint32_t polls = 0, ns = 32;
  for (;;) {
    const int64_t q = hi - int64_t(lane);
    const bool real = q >= int64_t(first);
    uint64_t w = real ? ld_relaxed(p.lookback + q) : kLbFlagP;
    bool to = false;
    while (__any_sync(0xFFFFFFFFu, w == 0)) {
      if (++polls > p.cfg.spin_limit) {
        to = true;
        break;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
      if (w == 0) w = ld_relaxed(p.lookback + q);
    }
    if (to) {
      *timed_out = true;
      excl = kSat;
      break;
    }
    const uint32_t pm = __ballot_sync(0xFFFFFFFFu, (w >> 62) == 2);
    const uint32_t upto = pm ? uint32_t(__ffs(pm) - 1) : 31u;
    uint64_t v = lane <= upto ? (w & kLbVal) : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
    excl = sat(excl + v);
    if (pm) break;
    hi -= 32;
  }
  if (lane == 0 && !hold) st_relaxed(p.lookback + gp, kLbFlagP | sat(excl + agg));
  return excl;
}

// One warp: resolve the prefix and record the partition's outcome in ctl
// and in the map's status.
__device__ void finish_prefix(const PassDev& p, const MapRegs& M, uint32_t gp, uint32_t j, uint64_t Sp,
                              PartCtl& ctl) {
  bool to = false;
  const uint64_t excl = resolve_prefix(p, gp, M.part_begin, Sp, &to);
  if (lane_id() == 0) {
    const uint64_t incl = excl + Sp;
    ctl.excl = excl;
    ctl.skip = (to || incl > M.slot_cap) ? 1u : 0u;
    if (to) atomicExch(&p.status[j].timeout, 1u);
    if (incl > M.slot_cap) atomicExch(&p.status[j].reseed, 1u);
    if (gp + 1 == M.part_end) p.status[j].S = incl;
    atomicMax(&p.status[j].max_s, ctl.maxs);
    atomicAdd(reinterpret_cast<unsigned long long*>(&p.status[j].nonempty), (unsigned long long)ctl.nonempty);
  }
}

// Equal keys of two members: u64 maps compare keys; string maps compare bytes.
template <int PW>
__device__ __forceinline__ bool same_member(const PassDev& p, const uint64_t* gpay, uint32_t x,
                                            uint32_t y) {
  if (PW == 1) return true;  // called only for equal keys
  const uint64_t ox = gpay[2 * x], oy = gpay[2 * y];
  const uint32_t lx = offlen_len(ox), ly = offlen_len(oy);
  if (lx != ly) return false;
  return bytes_equal(p.ctx + offlen_off(ox), p.ctx + offlen_off(oy), lx);
}

enum { kSearchDup = -1, kSearchNext = -2 };

template <int PW>
__device__ __forceinline__ void write_slot(const PassDev& p, uint64_t idx, uint64_t key,
                                           const uint64_t* pay, bool fill) {
  if (PW == 1) {
    reinterpret_cast<ulonglong2*>(p.slots)[idx] = make_ulonglong2(key, fill ? ~0ull : pay[0]);
  } else {
    ulonglong2* d = reinterpret_cast<ulonglong2*>(p.slots) + 2 * idx;
    d[0] = make_ulonglong2(key, pay[0]);
    d[1] = make_ulonglong2(fill ? ~0ull : pay[1], 0ull);
  }
}

// make_2 + placement for a bucket of 2 or 3 keys by one thread: the first
// attempt whose slot indices in the s^2 <= 9 slots are pairwise distinct,
// then every slot of the range written once (member, or the filler: the
// lowest occupied slot's key with value -1).  Returns the attempt, or
// kSearchDup / kSearchNext.
template <int PW>
__device__ int search_place_small(const PassDev& p, const uint64_t* gkey, const uint64_t* gpay, uint32_t g0,
                                  uint32_t s, uint64_t seed, uint32_t round, uint32_t b, uint16_t* owner,
                                  uint32_t so, uint64_t slot0, bool owner_mode) {
  const uint32_t m = s * s;
  const bool three = s == 3;
  const uint64_t k0 = gkey[g0], k1 = gkey[g0 + 1], k2 = three ? gkey[g0 + 2] : 0ull;
  uint32_t j0 = 0, j1 = 0, j2 = 0;
  int found = kSearchNext;
  for (uint32_t a = 0; a < p.cfg.attempt_cap; ++a) {
    if (a == kDupCheckAttempt) {
      const bool e01 = k0 == k1, e02 = three && k0 == k2, e12 = three && k1 == k2;
      if (e01 || e02 || e12) {  // every equal pair
        bool dup = e01 && same_member<PW>(p, gpay, g0, g0 + 1);
        dup |= e02 && same_member<PW>(p, gpay, g0, g0 + 2);
        dup |= e12 && same_member<PW>(p, gpay, g0 + 1, g0 + 2);
        return dup ? kSearchDup : kSearchNext;
      }
    }
    const HashConsts c = derive(seed, round, b, a);
    j0 = reduce32(hash32(c, k0), m);
    j1 = reduce32(hash32(c, k1), m);
    j2 = three ? reduce32(hash32(c, k2), m) : 0xFFFFu;
    const bool col = j0 == j1 || (three && (j0 == j2 || j1 == j2));
    if (a < p.cfg.reject) continue;
    if (!col) {
      found = int(a);
      break;
    }
  }
  if (found < 0) return found;
  const uint32_t jmin = min(j0, min(j1, j2));
  const uint32_t xmin = jmin == j0 ? 0u : (jmin == j1 ? 1u : 2u);
  for (uint32_t t = 0; t < m; ++t) {
    const uint32_t x = t == j0 ? 0u : (t == j1 ? 1u : (t == j2 ? 2u : 3u));
    const bool fill = x == 3u;
    const uint32_t src = g0 + (fill ? xmin : x);
    if (owner_mode) owner[so + t] = uint16_t(fill ? (kOwnerFill | src) : src);
    else write_slot<PW>(p, slot0 + t, gkey[src], gpay + PW * src, fill);
  }
  return found;
}

// make_2 + placement for up to 32 / G buckets of 2 <= s <= G keys by one warp
// (G = 2^cls lanes per bucket, 2 <= G <= 32).  Lane x of segment q holds key
// x of bucket list[q]; every segment tries attempts 0, 1, 2, ... in step and
// keeps its first attempt without a collision (two of its lanes on one slot,
// found with one __match_any_sync over (segment, slot) tags for the whole
// warp), as the sequential make_2.  Statistics go to *amax / *asum (lane 0
// of each segment).
template <int PW>
__device__ void search_place_seg(const PassDev& p, const uint64_t* gkey, const uint64_t* gpay,
                                 const uint32_t* gst, const uint32_t* soff, const uint16_t* list,
                                 uint32_t cnt, uint32_t cls, uint64_t seed, uint32_t round, uint32_t b0,
                                 uint16_t* owner, uint64_t slot_part, bool owner_mode, uint32_t j,
                                 PartCtl& ctl, uint16_t* att, uint32_t* amax, uint64_t* asum) {
  const uint32_t lane = lane_id(), G = 1u << cls;
  const uint32_t q = lane >> cls, x = lane & (G - 1u);
  const uint32_t segmask = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u) << (q * G);
  const bool segv = q < cnt;
  uint32_t lb = 0, g0 = 0, s = 0;
  if (segv) {
    lb = list[q];
    g0 = gst[lb];
    s = gst[lb + 1] - g0;
  }
  const bool mine = segv && x < s;
  const uint64_t key = mine ? gkey[g0 + x] : 0ull;
  const uint32_t m = s * s;
  bool done = !segv;
  int result = kSearchNext;
  uint32_t myj = 0;
  for (uint32_t a = 0; a < p.cfg.attempt_cap; ++a) {
    if (__all_sync(0xFFFFFFFFu, done)) break;
    if (a == kDupCheckAttempt) {
      const uint32_t members = __ballot_sync(0xFFFFFFFFu, mine && !done);
      const uint32_t same = __match_any_sync(0xFFFFFFFFu, key) & members & segmask;
      bool eq = false, dup = false;
      if (mine && !done && __popc(same) > 1) {
        eq = true;
        for (uint32_t lower = same & lanemask_lt(); lower; lower &= lower - 1)  // every equal pair
          dup |= same_member<PW>(p, gpay, g0 + (uint32_t(__ffs(lower) - 1) - q * G), g0 + x);
      }
      const uint32_t eqm = __ballot_sync(0xFFFFFFFFu, eq), dupm = __ballot_sync(0xFFFFFFFFu, dup);
      if (!done && (eqm & segmask)) {
        result = (dupm & segmask) ? kSearchDup : kSearchNext;
        done = true;
      }
    }
    const bool live = mine && !done;
    uint32_t jj = 0;
    if (live) jj = reduce32(hash32(derive(seed, round, b0 + lb, a), key), m);
    // (segment, slot) tag; idle lanes carry distinct values above every tag
    const uint32_t tag = live ? ((q << 16) | jj) : 0xFFFFFFFFu - lane;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, tag);
    const uint32_t colm = __ballot_sync(0xFFFFFFFFu, live && __popc(peers) > 1);
    if (!done && a >= p.cfg.reject && !(colm & segmask)) {
      done = true;
      result = int(a);
      myj = jj;
    }
  }
  // placement: members, then the filler (lowest occupied slot, value -1)
  const bool ok = segv && result >= 0;
  uint32_t v = (mine && ok) ? ((myj << 5) | x) : 0xFFFFFFFFu;
  for (uint32_t d = G >> 1; d > 0; d >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, d));
  const uint32_t xmin = v & 31u;
  const uint32_t so = segv ? soff[lb] : 0u;
  if (owner_mode) {
    if (mine && ok) owner[so + myj] = uint16_t(g0 + x);
    __syncwarp();
    if (ok)
      for (uint32_t t = x; t < m; t += G)
        if (owner[so + t] == kOwnerEmpty) owner[so + t] = uint16_t(kOwnerFill | (g0 + xmin));
  } else {
    if (ok)
      for (uint32_t t = x; t < m; t += G)
        write_slot<PW>(p, slot_part + so + t, gkey[g0 + xmin], gpay + PW * (g0 + xmin), true);
    __syncwarp();
    if (mine && ok) write_slot<PW>(p, slot_part + so + myj, key, gpay + PW * (g0 + x), false);
  }
  if (segv && x == 0) {
    if (result >= 0) {
      att[lb] = uint16_t(result);
      *amax = max(*amax, uint32_t(result));
      *asum += uint64_t(result);
    } else {
      atomicExch(result == kSearchDup ? &p.status[j].dup : &p.status[j].next_round, 1u);
      ctl.failed = 1;
    }
  }
}

// make_2 + placement for a bucket of more than 32 keys, by the CTA.
template <int PW>
__device__ __noinline__ void search_place_cta(const PassDev& p, const uint64_t* k, const uint64_t* gpay,
                                              uint32_t g0, uint32_t s, uint64_t seed, uint32_t round,
                                              uint32_t b, uint16_t* owner, uint32_t so, uint64_t slot0,
                                              bool owner_mode, uint32_t j, PartCtl& ctl,
                                              uint16_t* att_out) {
  const uint32_t t = threadIdx.x, m = s * s;
  int found = kSearchNext;
  for (uint32_t a = 0; a < p.cfg.attempt_cap; ++a) {
    if (a == kDupCheckAttempt) {
      if (t == 0) ctl.flag_a = ctl.flag_b = 0;
      __syncthreads();
      for (uint32_t x = t; x < s; x += kPartThreads)
        for (uint32_t y = x + 1; y < s; ++y)
          if (k[x] == k[y]) {
            ctl.flag_a = 1;
            if (same_member<PW>(p, gpay, g0 + x, g0 + y)) ctl.flag_b = 1;
          }
      __syncthreads();
      const uint32_t eq = ctl.flag_a, dup = ctl.flag_b;
      __syncthreads();
      if (dup) { found = kSearchDup; break; }
      if (eq) { found = kSearchNext; break; }
    }
    const HashConsts c = derive(seed, round, b, a);
    if (t == 0) ctl.flag_a = 0;
    __syncthreads();
    for (uint32_t x = t; x < s; x += kPartThreads) {
      const uint32_t jx = reduce32(hash32(c, k[x]), m);
      for (uint32_t y = 0; y < s; ++y)
        if (y != x && reduce32(hash32(c, k[y]), m) == jx) {
          ctl.flag_a = 1;
          break;
        }
    }
    __syncthreads();
    const uint32_t col = ctl.flag_a;
    __syncthreads();
    if (a >= p.cfg.reject && !col) { found = int(a); break; }
  }
  if (found < 0) {
    if (t == 0) {
      if (found == kSearchDup) atomicExch(&p.status[j].dup, 1u);
      else atomicExch(&p.status[j].next_round, 1u);
      *att_out = 0;
      ctl.failed = 1;
    }
    __syncthreads();
    return;
  }
  const HashConsts c = derive(seed, round, b, uint32_t(found));
  if (t == 0) {
    *att_out = uint16_t(found);
    ctl.fillmin = ~0ull;
    atomicMax(&ctl.maxatt, uint32_t(found));
    ctl.attsum += uint64_t(found);
  }
  __syncthreads();
  for (uint32_t x = t; x < s; x += kPartThreads) {
    const uint32_t jx = reduce32(hash32(c, k[x]), m);
    atomicMin(&ctl.fillmin, (static_cast<unsigned long long>(jx) << 32) | x);
  }
  __syncthreads();
  const uint32_t xmin = uint32_t(ctl.fillmin & 0xFFFFFFFFull);
  if (owner_mode) {
    for (uint32_t x = t; x < s; x += kPartThreads) owner[so + reduce32(hash32(c, k[x]), m)] = uint16_t(g0 + x);
    __syncthreads();
    for (uint32_t q = t; q < m; q += kPartThreads)
      if (owner[so + q] == kOwnerEmpty) owner[so + q] = uint16_t(kOwnerFill | (g0 + xmin));
  } else {
    for (uint32_t q = t; q < m; q += kPartThreads)
      write_slot<PW>(p, slot0 + q, k[xmin], gpay + PW * (g0 + xmin), true);
    __syncthreads();
    for (uint32_t x = t; x < s; x += kPartThreads)
      write_slot<PW>(p, slot0 + reduce32(hash32(c, k[x]), m), k[x], gpay + PW * (g0 + x), false);
  }
  __syncthreads();
}

// Search classes of a bucket of s >= 2 keys: 0 = one thread (s <= thr), 1..5 =
// a segment of 2^cls lanes (s <= 32), 6 = the whole CTA.
__device__ __forceinline__ uint32_t search_class(uint32_t s, uint32_t thr) {
  if (s <= thr) return 0;
  if (s > 32) return 6;
  return 32u - uint32_t(__clz(int(s - 1)));  // ceil(log2 s)
}

// Level-two search (make_2) of every bucket of a grouped partition, then the
// placement of its keys: slot image in shared memory (owner mode) or direct
// writes.  Empty and single-key buckets need no search (attempt 0); the
// others are listed by class, one shared atomic per warp and class -- into
// fixed regions in one pass when the partition holds at most kCap keys
// (kFixed), else counted first and placed in a second pass.  Small buckets
// are searched by single threads from the low warps, mid-size ones in
// packed warp segments from the high warps (no barrier between the two),
// buckets above 32 keys by the whole CTA.
//
// resolve: the slot prefix of partition gp (size Sp) is resolved here, by
// the first warp without single-thread searches, while the others search.
template <int PW, bool kFixed>
__device__ void search_partition(const PassDev& p, const MapRegs& M, uint32_t j, uint32_t b0,
                                 uint32_t nb, uint64_t slot_part, bool owner_mode,
                                 const uint64_t* gkey, const uint64_t* gpay, uint16_t* owner,
                                 const uint32_t* gst, const uint32_t* soff, uint16_t* att,
                                 uint16_t* work, PartCtl& ctl, bool resolve, uint32_t gp, uint64_t Sp) {
  const uint32_t thr = p.cfg.thread_max;
  const uint32_t lane = lane_id();
  if (kFixed && threadIdx.x < kClasses) ctl.cbase[threadIdx.x] = class_region(threadIdx.x);
  // pass 1: singletons placed, classes counted (kFixed: listed)
  for (uint32_t lb0 = threadIdx.x & ~31u; lb0 < nb; lb0 += kPartThreads) {
    const uint32_t lb = lb0 + lane;
    uint32_t g0 = 0, s = 0;
    if (lb < nb) {
      g0 = gst[lb];
      s = gst[lb + 1] - g0;
      att[lb] = 0;
      if (s == 1) {
        if (owner_mode) owner[soff[lb]] = uint16_t(g0);
        else write_slot<PW>(p, slot_part + soff[lb], gkey[g0], gpay + PW * g0, false);
      }
    }
    const uint32_t c = (lb < nb && s > 1) ? search_class(s, thr) : kClasses;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, c);
    const uint32_t leader = uint32_t(__ffs(peers) - 1);
    if (kFixed) {
      uint32_t base = 0;
      if (c < kClasses && lane == leader) base = atomicAdd(&ctl.ccnt[c], uint32_t(__popc(peers)));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (c < kClasses) work[class_region(c) + base + __popc(peers & lanemask_lt())] = uint16_t(lb);
    } else if (c < kClasses && lane == leader) {
      atomicAdd(&ctl.ccnt[c], uint32_t(__popc(peers)));
    }
  }
  __syncthreads();
  if (!kFixed && threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t c = 0; c < kClasses; ++c) {
      ctl.cbase[c] = run;
      ctl.ccur[c] = run;
      run += ctl.ccnt[c];
    }
  }
  if (!kFixed) __syncthreads();
  // pass 2: the class lists
  for (uint32_t lb0 = threadIdx.x & ~31u; !kFixed && lb0 < nb; lb0 += kPartThreads) {
    const uint32_t lb = lb0 + lane;
    uint32_t s = 0;
    if (lb < nb) s = gst[lb + 1] - gst[lb];
    const uint32_t c = (lb < nb && s > 1) ? search_class(s, thr) : kClasses;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, c);
    const uint32_t leader = uint32_t(__ffs(peers) - 1);
    uint32_t base = 0;
    if (c < kClasses && lane == leader) base = atomicAdd(&ctl.ccur[c], uint32_t(__popc(peers)));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (c < kClasses) work[base + __popc(peers & lanemask_lt())] = uint16_t(lb);
  }
  if (!kFixed) __syncthreads();
  uint32_t my_max = 0;
  uint64_t my_sum = 0;
  // single-thread searches, from thread 0 up
  const uint32_t n0 = ctl.ccnt[0];
  if (resolve && (threadIdx.x >> 5) == min(kPartThreads / 32 - 1, (n0 + 31) / 32))
    finish_prefix(p, M, gp, j, Sp, ctl);
  for (uint32_t w = threadIdx.x; w < n0; w += kPartThreads) {
    const uint32_t lb = work[ctl.cbase[0] + w];
    const uint32_t g0 = gst[lb], s = gst[lb + 1] - g0;
    const int a = search_place_small<PW>(p, gkey, gpay, g0, s, M.seed, M.round, b0 + lb, owner, soff[lb],
                                         slot_part + soff[lb], owner_mode);
    if (a >= 0) {
      att[lb] = uint16_t(a);
      my_max = max(my_max, uint32_t(a));
      my_sum += uint64_t(a);
    } else {
      atomicExch(a == kSearchDup ? &p.status[j].dup : &p.status[j].next_round, 1u);
      ctl.failed = 1;
    }
  }
  // warp segments, from the last warp down: chunk k of class c holds 32 / 2^c buckets
  {
    uint32_t chunks[6], total = 0;
#pragma unroll
    for (uint32_t c = 1; c <= 5; ++c) {
      const uint32_t per = 32u >> c;
      chunks[c] = (ctl.ccnt[c] + per - 1) / per;
      total += chunks[c];
    }
    constexpr uint32_t kWarps = kPartThreads / 32;
    for (uint32_t k = kWarps - 1 - (threadIdx.x >> 5); k < total; k += kWarps) {
      uint32_t c = 1, r = k;
      while (r >= chunks[c]) r -= chunks[c++];
      const uint32_t per = 32u >> c;
      const uint32_t first = r * per;
      const uint32_t cnt = min(per, ctl.ccnt[c] - first);
      search_place_seg<PW>(p, gkey, gpay, gst, soff, work + ctl.cbase[c] + first, cnt, c, M.seed, M.round, b0,
                           owner, slot_part, owner_mode, j, ctl, att, &my_max, &my_sum);
    }
  }
  // statistics: one shared atomic per warp
  my_max = __reduce_max_sync(0xFFFFFFFFu, my_max);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) my_sum += __shfl_xor_sync(0xFFFFFFFFu, my_sum, d);
  if (lane == 0) {
    if (my_max) atomicMax(&ctl.maxatt, my_max);
    if (my_sum) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl.attsum), my_sum);
  }
  __syncthreads();
  // s > 32 (adversarial inputs, or many keys per bucket): the whole CTA, one bucket at a time
  const uint32_t n6 = ctl.ccnt[6];
  if (n6) {
    for (uint32_t i = 0; i < n6; ++i) {
      const uint32_t lb = work[ctl.cbase[6] + i];
      const uint32_t g0 = gst[lb], s = gst[lb + 1] - g0;
      search_place_cta<PW>(p, gkey + g0, gpay, g0, s, M.seed, M.round, b0 + lb, owner, soff[lb],
                           slot_part + soff[lb], owner_mode, j, ctl, att + lb);
    }
    __syncthreads();
  }
}

// Descriptors of the partition's buckets and, in owner mode, its slot image
// (both coalesced).
template <int PW>
__device__ void write_partition(const PassDev& p, const MapRegs& M, uint32_t b0, uint32_t nb,
                                uint64_t excl, bool owner_mode, const uint64_t* gkey,
                                const uint64_t* gpay, const uint16_t* owner, const uint32_t* gst,
                                const uint32_t* soff, const uint16_t* att, uint64_t Sp) {
  const uint32_t t = threadIdx.x;
  for (uint32_t lb = t; lb < nb; lb += kPartThreads) {
    const uint32_t s = gst[lb + 1] - gst[lb];
    const uint64_t d = desc_pack(uint32_t(excl + soff[lb]), s, att[lb]);
    p.desc[M.desc_base + b0 + lb] = d;
    if (PW == 1 && p.rec) {  // inline-singleton record of the bucket
      const uint32_t b = b0 + lb;
      ulonglong2 r;
      r.x = s == 1 ? gkey[gst[lb]] : (b == p.rec_g0 ? p.rec_x1 : 0ull);
      r.y = s == 1 ? gpay[gst[lb]] : d;
      reinterpret_cast<ulonglong2*>(p.rec)[M.desc_base + b] = r;
    }
  }
  if (owner_mode) {
    const uint64_t slot_part = M.slot_base + excl;
    for (uint32_t q = t; q < uint32_t(Sp); q += kPartThreads) {
      const uint16_t o = owner[q];
      if (o == kOwnerEmpty) continue;  // only when a bucket failed (never written then)
      const uint32_t idx = o & 0x7FFFu;
      write_slot<PW>(p, slot_part + q, gkey[idx], gpay + PW * idx, (o & kOwnerFill) != 0);
    }
  }
}

__device__ __forceinline__ void flush_stats(const PassDev& p, uint32_t j, const PartCtl& ctl) {
  if (ctl.maxatt) atomicMax(&p.status[j].max_att, ctl.maxatt);
  if (ctl.attsum)
    atomicAdd(reinterpret_cast<unsigned long long*>(&p.status[j].att_sum), (unsigned long long)ctl.attsum);
}

// The partition CTA: a persistent loop over a ticketed queue of partitions.
// While partition i is searched and written, the bulk-copy engine already
// stages partition i+1 into shared memory.
template <int PW>
__global__ void __launch_bounds__(kPartThreads, PW == 1 ? 2 : 1) k_part_build(PassDev p) {
  extern __shared__ __align__(128) uint8_t smem[];
  using L = Smem<PW>;
  uint64_t* raw_key = reinterpret_cast<uint64_t*>(smem + L::kRawKey);
  uint64_t* raw_pay = reinterpret_cast<uint64_t*>(smem + L::kRawPay);
  uint64_t* gkey = reinterpret_cast<uint64_t*>(smem + L::kGkey);
  uint64_t* gpay = reinterpret_cast<uint64_t*>(smem + L::kGpay);
  uint16_t* owner = reinterpret_cast<uint16_t*>(smem + L::kOwner);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + L::kCnt);
  uint32_t* gst = reinterpret_cast<uint32_t*>(smem + L::kGst);
  uint32_t* soff = reinterpret_cast<uint32_t*>(smem + L::kSoff);
  uint16_t* att = reinterpret_cast<uint16_t*>(smem + L::kAtt);
  uint16_t* work = reinterpret_cast<uint16_t*>(smem + L::kWork);
  __shared__ PartCtl ctl;
  // the current partition's map, out of registers; two copies so that the
  // next partition's can be written while the previous write-out still reads
  __shared__ MapRegs sM[2];
  uint32_t iter = 0;
  __shared__ __align__(8) uint64_t bar;
  const uint32_t t = threadIdx.x;
  constexpr uint32_t kPerThread = kCap / kPartThreads;
  uint32_t parity = 0;
  if (t == 0) {
    mbar_init(&bar, 1);
    ctl.abort = 0;
    ctl.next_gp = atomicAdd(p.ticket, 1u);
    ctl.next_issued = issue_stage<PW>(p, ctl.next_gp, raw_key, raw_pay, &bar, &ctl.next_e0, &ctl.next_e1);
  }
  __syncthreads();
  uint32_t last_j = 0xFFFFFFFFu;  // thread 32: the map held in sM[(iter & 1) ^ 1]
  for (;;) {
    if (!p.cfg.prefetch && iter > 0) {
      // Without prefetch the next ticket is taken only when the CTA is free:
      // a partition is then never queued behind another partition's search,
      // so the predecessors whose aggregates its look-back needs are already
      // running (what partitions that write their slots directly wait for).
      if (t == 0 && !ctl.abort) {
        ctl.next_gp = atomicAdd(p.ticket, 1u);
        ctl.next_issued = issue_stage<PW>(p, ctl.next_gp, raw_key, raw_pay, &bar, &ctl.next_e0, &ctl.next_e1);
      }
      __syncthreads();
    }
    const uint32_t gp = ctl.next_gp;
    const uint32_t issued = ctl.next_issued;
    if (gp >= p.P || ctl.abort) break;
    const uint32_t j = p.m == 1 ? 0u : upper_seg(p.part_seg, p.m, gp);
    if (t == 32) {  // visible after the barrier below; global reads only when the map changes
      sM[iter & 1] = j == last_j ? sM[(iter & 1) ^ 1] : load_map(p, j);
      last_j = j;
    }
    const MapRegs& M = sM[iter & 1];
    ++iter;
    const uint64_t e0 = ctl.next_e0, e1 = ctl.next_e1;
    const uint32_t ne = uint32_t(e1 - e0 < 0xFFFFFFFFull ? e1 - e0 : 0xFFFFFFFFull);
    for (uint32_t i = t; i < (1u << p.logB); i += kPartThreads) cnt[i] = 0;
    if (issued) {  // bounded wait for the staged copy
      uint32_t polls = 0;
      while (!mbar_try_wait(&bar, parity)) {
        if (++polls > p.cfg.spin_limit) {
          ctl.abort = 1;
          break;
        }
      }
      parity ^= 1u;
    }
    __syncthreads();
    if (ctl.abort) {
      if (t == 0) atomicExch(&p.status[j].timeout, 1u);
      break;
    }
    if (t == 0) {  // every reader of last iteration's values passed the barrier above
      ctl.maxs = ctl.maxatt = ctl.nonempty = ctl.nbig = ctl.failed = ctl.nwork = 0;
      ctl.attsum = 0;
      for (uint32_t c = 0; c < 8; ++c) ctl.ccnt[c] = 0;
    }
    // M (written by thread 32 above) is visible past the barrier
    const uint32_t b0 = (gp - M.part_begin) << p.logB;
    const uint32_t nb = min(1u << p.logB, M.nb - b0);  // buckets of this partition
    const bool overflow = ne > kCap;
    const uint32_t shift = uint32_t(e0 & 1ull);  // raw key index of element e0
    uint16_t lbr[kPerThread], rk[kPerThread];
    if (!overflow) {
      // Hist of the partition's buckets from shared memory; the atomic's
      // return value is the key's rank within its bucket.
#pragma unroll
      for (uint32_t u = 0; u < kPerThread; ++u) {
        const uint32_t i = t + u * kPartThreads;
        if (i < ne) {
          const uint64_t k = raw_key[shift + i];
          const uint32_t lb = reduce32(hash32(M.c1, k), M.nb) - b0;
          lbr[u] = uint16_t(lb);
          rk[u] = uint16_t(atomicAdd(cnt + lb, 1u));
        }
      }
    } else {
      count_global(p, M, b0, e0, e1, cnt);
    }
    __syncthreads();
    scan_buckets(cnt, gst, soff, ctl, nb);
    const uint64_t Sp = ctl.Spart;
    const bool owner_mode = Sp <= kOwnerCap;
    // The slot prefix of this partition (look-back across partitions) is
    // needed only by the write-out: publish the aggregate now and resolve
    // the prefix after the search, unless the partition writes its slots
    // directly (oversized slot image) or is deferred to the overflow kernel.
    const bool early = overflow || !owner_mode;
    if (t < 32) {
      if (t == 0) publish_aggregate(p, gp, M.part_begin, Sp);
      if (early) finish_prefix(p, M, gp, j, Sp, ctl);
    }
    if (!overflow) {
#pragma unroll
      for (uint32_t u = 0; u < kPerThread; ++u) {
        const uint32_t i = t + u * kPartThreads;
        if (i < ne) {
          const uint32_t pos = gst[lbr[u]] + rk[u];
          gkey[pos] = raw_key[shift + i];
#pragma unroll
          for (int w = 0; w < PW; ++w) gpay[PW * pos + w] = raw_pay[PW * ((PW == 1 ? shift : 0) + i) + w];
        }
      }
      if (owner_mode)
        for (uint32_t q = t; q < uint32_t(Sp); q += kPartThreads) owner[q] = kOwnerEmpty;
    }
    __syncthreads();
    // raw* is free again: stage the next partition while this one is searched
    // (by the last warp, which rarely has search work: the worklist fills
    // the low warps first)
    if (p.cfg.prefetch && t == kPartThreads - 32) {
      ctl.next_gp = atomicAdd(p.ticket, 1u);
      ctl.next_issued = issue_stage<PW>(p, ctl.next_gp, raw_key, raw_pay, &bar, &ctl.next_e0, &ctl.next_e1);
    }
    if (early && ctl.skip) {
      __syncthreads();
      continue;
    }
    if (overflow) {
      if (t == 0) {
        const uint32_t slot = atomicAdd(p.ovf_count, 1u);
        p.ovf_list[slot] = gp;
        p.ovf_excl[slot] = ctl.excl;
        atomicAdd(&p.status[j].overflow, 1u);
      }
      __syncthreads();
      continue;
    }
    // the slot prefix is needed only by the write-out: resolved during the search
    search_partition<PW, true>(p, M, j, b0, nb, M.slot_base + ctl.excl, owner_mode, gkey, gpay, owner, gst,
                               soff, att, work, ctl, !early, gp, Sp);
    if (!ctl.failed && !ctl.skip)
      write_partition<PW>(p, M, b0, nb, ctl.excl, owner_mode, gkey, gpay, owner, gst, soff, att, Sp);
    if (t == 0) flush_stats(p, j, ctl);
  }
  // never leave with a bulk copy in flight
  if (t == 0 && ctl.next_issued && ctl.abort) {
    uint32_t polls = 0;
    while (!mbar_try_wait(&bar, parity) && ++polls < p.cfg.spin_limit) {
    }
  }
}

// Partitions deferred because they hold more than kCap keys: grouped through
// global memory (the rare, adversarial case).  Group indices are
// partition-local; the grouped buffer starts at the partition's first element.
template <int PW>
__global__ void __launch_bounds__(kPartThreads, 1) k_part_overflow(PassDev p) {
  extern __shared__ __align__(128) uint8_t smem[];
  using L = Smem<PW>;
  uint16_t* owner = reinterpret_cast<uint16_t*>(smem + L::kOwner);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + L::kCnt);
  uint32_t* gst = reinterpret_cast<uint32_t*>(smem + L::kGst);
  uint32_t* soff = reinterpret_cast<uint32_t*>(smem + L::kSoff);
  uint16_t* att = reinterpret_cast<uint16_t*>(smem + L::kAtt);
  uint16_t* work = reinterpret_cast<uint16_t*>(smem + L::kWork);
  __shared__ PartCtl ctl;
  const uint32_t t = threadIdx.x;
  const uint32_t gp = p.ovf_list[blockIdx.x];
  const uint32_t j = p.m == 1 ? 0u : upper_seg(p.part_seg, p.m, gp);
  const MapRegs M = load_map(p, j);
  const uint32_t b0 = (gp - M.part_begin) << p.logB;
  const uint32_t nb = min(1u << p.logB, M.nb - b0);
  const uint64_t e0 = p.part_start[gp], e1 = p.part_start[gp + 1];
  const uint64_t excl = p.ovf_excl[blockIdx.x];
  uint64_t* gkey = p.ovf_key + e0;
  uint64_t* gpay = p.ovf_pay + PW * e0;
  for (uint32_t i = t; i < nb; i += kPartThreads) cnt[i] = 0;
  if (t == 0) {
    ctl.maxs = ctl.maxatt = ctl.nonempty = ctl.nbig = ctl.failed = ctl.nwork = 0;
    ctl.attsum = 0;
    for (uint32_t c = 0; c < 8; ++c) ctl.ccnt[c] = 0;
  }
  __syncthreads();
  count_global(p, M, b0, e0, e1, cnt);
  __syncthreads();
  scan_buckets(cnt, gst, soff, ctl, nb);
  const uint64_t Sp = ctl.Spart;
  const bool owner_mode = Sp <= kOwnerCap;
  for (uint32_t i = t; i < nb; i += kPartThreads) cnt[i] = gst[i];
  if (owner_mode)
    for (uint32_t q = t; q < uint32_t(Sp); q += kPartThreads) owner[q] = kOwnerEmpty;
  __syncthreads();
  for (uint64_t e = e0 + t; e < e1; e += kPartThreads) {
    const uint64_t k = p.stage_key[e];
    const uint32_t lb = reduce32(hash32(M.c1, k), M.nb) - b0;
    const uint32_t pos = atomicAdd(cnt + lb, 1u);
    gkey[pos] = k;
#pragma unroll
    for (int w = 0; w < PW; ++w) gpay[PW * pos + w] = p.stage_pay[PW * e + w];
  }
  __syncthreads();
  search_partition<PW, false>(p, M, j, b0, nb, M.slot_base + excl, owner_mode, gkey, gpay, owner, gst, soff,
                              att, work, ctl, false, gp, Sp);
  if (!ctl.failed)
    write_partition<PW>(p, M, b0, nb, excl, owner_mode, gkey, gpay, owner, gst, soff, att, Sp);
  if (t == 0) flush_stats(p, j, ctl);
}

// -------------------------------------------------------------- duplicate test
// Exact global duplicate test after every level-one round failed: insertion
// into an open-addressing set; flags[0] = duplicate found, flags[1] = keys
// equal to the empty marker (u64 maps), flags[2] = a wait ran out.
__global__ void __launch_bounds__(256) k_dupcheck(const uint64_t* __restrict__ hkeys,
                                                  const int64_t* __restrict__ offs,
                                                  const uint8_t* __restrict__ ctx, uint64_t n,
                                                  uint64_t* table, uint32_t* tidx,
                                                  uint64_t size, uint32_t* flags,
                                                  uint32_t spin_limit) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t mask = size - 1;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t k = hkeys[i];
    if (!offs && k == ~0ull) {
      if (atomicAdd(flags + 1, 1u) >= 1u) atomicExch(flags, 1u);
      continue;
    }
    uint64_t h = mix13(k) & mask;
    for (uint64_t probe = 0; probe < size; ++probe, h = (h + 1) & mask) {
      const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(table + h), ~0ull, k);
      if (old == ~0ull) {
        if (offs) atomicExch(tidx + h, uint32_t(i + 1));
        break;
      }
      if (old != k) continue;
      if (!offs) {
        atomicExch(flags, 1u);
        break;
      }
      uint32_t other = 0, polls = 0;
      while ((other = atomicAdd(tidx + h, 0u)) == 0u) {
        if (++polls > spin_limit) break;
        __nanosleep(64);
      }
      if (other == 0u) {
        atomicExch(flags + 2, 1u);
        break;
      }
      const uint64_t oi = other - 1;
      const int64_t li = offs[i + 1] - offs[i], lo = offs[oi + 1] - offs[oi];
      if (li == lo && bytes_equal(ctx + offs[i], ctx + offs[oi], uint32_t(li))) {
        atomicExch(flags, 1u);
        break;
      }
    }
  }
}

}  // namespace

// ================================================================ launchers
cudaError_t launch_fingerprints(const uint8_t* ctx, const int64_t* offs, uint64_t n,
                                const MapDev* maps, const uint64_t* pass_seg, uint32_t m,
                                uint64_t total, uint64_t* fps, MapStatus* status,
                                cudaStream_t stream) {
  (void)n;
  if (total == 0) return cudaSuccess;
  const uint64_t blocks = (total + 255) / 256;
  if (m == 1)  // grid-stride over at most 8 blocks per SM: each block derives its powers of R once
    k_fingerprints_map<<<unsigned(blocks < uint64_t(device_sm_count()) * 8 ? blocks : uint64_t(device_sm_count()) * 8),
                         256, 0, stream>>>(ctx, offs, maps, total, fps, status);
  else
    k_fingerprints<<<unsigned(blocks < 65535ull * 16 ? blocks : 65535ull * 16), 256, 0, stream>>>(
        ctx, offs, maps, pass_seg, m, total, fps, status);
  note_launches(1);
  return cudaGetLastError();
}

// The partition kernels' shared-memory attribute and the partition kernel's
// resident CTAs per SM, set up once per process (thread-safe static
// initialisation; concurrent first builds wait for it).
template <int PW>
struct BuildKernelSetup {
  cudaError_t err = cudaSuccess;
  int occ = 1;
  BuildKernelSetup() {
    const int smem = int(Smem<PW>::kBytes);
    err = cudaFuncSetAttribute(k_part_build<PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_part_overflow<PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int o = 0;
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_part_build<PW>, kPartThreads, smem);
    occ = o > 0 ? o : 1;
  }
};

template <int PW>
static cudaError_t launch_build_kernel(const PassDev& p, int sms, const BuildShape& shape, cudaStream_t stream) {
  static const BuildKernelSetup<PW> setup;
  if (setup.err != cudaSuccess) return setup.err;
  const int occ = setup.occ;
  const int smem = int(Smem<PW>::kBytes);
  const uint64_t per_sm = shape.part_ctas_per_sm && int(shape.part_ctas_per_sm) < occ ? shape.part_ctas_per_sm : occ;
  const uint64_t want = uint64_t(sms) * per_sm;
  const unsigned grid = unsigned(p.P < want ? p.P : want);
  k_part_build<PW><<<grid, kPartThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pass(const PassDev& p, bool strings, int sms, const BuildShape& shape, cudaStream_t stream,
                        const PassEvents* ev) {
  if (p.total == 0 || p.P == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(p.part_cnt, 0, sizeof(uint32_t) * p.P, stream);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev->ev[0], stream);
  // Warp aggregation pays off when a warp's keys share partitions (small maps).
  const int agg = (p.total / p.P) < 64 || p.P < 64 ? 1 : 0;
  const size_t seg_smem = (p.m > 1 && p.m <= 2048) ? sizeof(uint64_t) * (p.m + 1) : 0;
  uint64_t blocks = (p.total + 256 * kUnroll - 1) / (256 * kUnroll);
  const uint64_t maxb = uint64_t(sms) * (shape.scatter_blocks_per_sm ? shape.scatter_blocks_per_sm : 8u);
  if (blocks > maxb) blocks = maxb;
  if (strings) k_partition<false, true><<<unsigned(blocks), 256, seg_smem, stream>>>(p, agg);
  else k_partition<false, false><<<unsigned(blocks), 256, seg_smem, stream>>>(p, agg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev->ev[1], stream);
  k_scan_parts<<<1, 1024, 0, stream>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev->ev[2], stream);
  if (strings) k_partition<true, true><<<unsigned(blocks), 256, seg_smem, stream>>>(p, agg);
  else k_partition<true, false><<<unsigned(blocks), 256, seg_smem, stream>>>(p, agg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev->ev[3], stream);
  e = strings ? launch_build_kernel<2>(p, sms, shape, stream) : launch_build_kernel<1>(p, sms, shape, stream);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev->ev[4], stream);
  note_launches(4);
  return cudaSuccess;
}

cudaError_t launch_pass_split(const PassDev& p, const SplitDev& s, bool strings, int sms, const BuildShape& shape,
                              cudaStream_t stream, const PassEvents* ev) {
  if (p.total == 0 || p.P == 0) return cudaSuccess;
  if (ev) cudaEventRecord(ev->ev[0], stream);
  cudaError_t e = launch_split(p, s, strings, stream);
  if (e != cudaSuccess) return e;
  if (ev) {
    cudaEventRecord(ev->ev[1], stream);
    cudaEventRecord(ev->ev[2], stream);
    cudaEventRecord(ev->ev[3], stream);
  }
  e = strings ? launch_build_kernel<2>(p, sms, shape, stream) : launch_build_kernel<1>(p, sms, shape, stream);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev->ev[4], stream);
  note_launches(1);
  return cudaSuccess;
}

cudaError_t launch_overflow(const PassDev& p, bool strings, uint32_t count, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  if (strings) {
    k_part_overflow<2><<<count, kPartThreads, Smem<2>::kBytes, stream>>>(p);
  } else {
    k_part_overflow<1><<<count, kPartThreads, Smem<1>::kBytes, stream>>>(p);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dupcheck(const uint64_t* hkeys, const int64_t* offs, const uint8_t* ctx,
                            uint64_t n, uint64_t* table, uint32_t* table_idx, uint64_t table_size,
                            uint32_t* flags, uint32_t spin_limit, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(table, 0xFF, sizeof(uint64_t) * table_size, stream);
  if (e != cudaSuccess) return e;
  if (table_idx && (e = cudaMemsetAsync(table_idx, 0, sizeof(uint32_t) * table_size, stream)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * 4, stream)) != cudaSuccess) return e;
  uint64_t blocks = (n + 255) / 256;
  const uint64_t maxb = uint64_t(device_sm_count()) * 16;
  if (blocks > maxb) blocks = maxb;
  k_dupcheck<<<unsigned(blocks), 256, 0, stream>>>(hkeys, offs, ctx, n, table, table_idx,
                                                  table_size, flags, spin_limit);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fks
