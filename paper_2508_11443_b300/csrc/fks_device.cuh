// fks_device.cuh -- arithmetic of the FKS two-level hash map on sm_103a.
//
// The construction (Sec. 2.2 of Due, Elsman, Henriksen, arXiv 2508.11443):
//   g k = Hash const k mod n                      level one, n buckets
//   h k = offsets[g k] + Hash consts[g k] k mod shape[g k]
//   shape[b] = s_b^2, offsets = exclusive Presum shape
// with Random drawing the constants of a universal family (Sec. 2.1).
//
// Choices made where the paper leaves the family open:
//   * Random is the splitmix64 generator (Steele, Lea, Flood, OOPSLA 2014)
//     evaluated at a counter (round, tag, attempt, index); tag is the bucket
//     for level two, or a reserved value for level one / the fingerprint base.
//   * Hash is Thorup's vector multiply-shift over the two 32-bit halves of a
//     key, strongly universal into 32 bits.
//   * "mod m" is the multiply-high reduction (h * m) >> 32 (Lemire), exact on
//     [0, m) for m < 2^32 and free of division.
//   * Byte strings are hashed through a polynomial fingerprint modulo the
//     Mersenne prime 2^61 - 1 of [length, little-endian 32-bit words].
// These functions are __host__ __device__ so the host side of the library
// derives level-one constants with the same code the kernels run.
#pragma once
#include <stdint.h>

#ifndef FKS_HD
#define FKS_HD __host__ __device__ __forceinline__
#endif

namespace fks {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;  // splitmix64 state increment
constexpr uint64_t kTagLevel1 = 0xFFFFFFFFull;      // level-one constants
constexpr uint64_t kTagFingerprint = 0xFFFFFFFEull;  // fingerprint base
constexpr uint64_t kP61 = (1ull << 61) - 1;
constexpr uint32_t kDupCheckAttempt = 64;  // attempt at which a bucket is tested for equal keys

// splitmix64 output finaliser (Stafford's "mix13").
FKS_HD uint64_t mix13(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct HashConsts {
  uint64_t m0, m1, add;
};

// Constants for (round, tag, attempt): splitmix64 outputs number
// ctr, ctr + 1, ctr + 2 with ctr = round<<48 | tag<<14 | attempt<<2.
FKS_HD HashConsts derive(uint64_t seed, uint32_t round, uint64_t tag, uint32_t attempt) {
  const uint64_t ctr = (uint64_t(round) << 48) | (tag << 14) | (uint64_t(attempt) << 2);
  const uint64_t s0 = seed + (ctr + 1) * kGamma;
  HashConsts c;
  c.m0 = mix13(s0);
  c.m1 = mix13(s0 + kGamma);
  c.add = mix13(s0 + 2 * kGamma);
  return c;
}

// Vector multiply-shift: (m0 * lo32(k) + m1 * hi32(k) + add) >> 32.
FKS_HD uint32_t hash32(const HashConsts& c, uint64_t k) {
  const uint64_t acc = c.m0 * (k & 0xFFFFFFFFull) + c.m1 * (k >> 32) + c.add;
  return uint32_t(acc >> 32);
}

// floor(h * m / 2^32): the reduction onto [0, m).  m < 2^32 always holds
// (m = n < 2^30 at level one, m = s^2 <= 4n at level two).
FKS_HD uint32_t reduce32(uint32_t h, uint32_t m) {
#ifdef __CUDA_ARCH__
  return __umulhi(h, m);
#else
  return uint32_t((uint64_t(h) * m) >> 32);
#endif
}

// ---------------------------------------------------------------- 2^61 - 1
FKS_HD uint64_t mulmod61(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  const uint64_t lo = a * b, hi = __umul64hi(a, b);
#else
  const unsigned __int128 p = (unsigned __int128)a * b;
  const uint64_t lo = uint64_t(p), hi = uint64_t(p >> 64);
#endif
  // a, b < 2^61: p < 2^122; p = hi*2^64 + lo = (hi << 3 | lo >> 61) * 2^61 + (lo & P)
  uint64_t x = (lo & kP61) + ((lo >> 61) | (hi << 3));
  x = (x & kP61) + (x >> 61);
  return x >= kP61 ? x - kP61 : x;
}

FKS_HD uint64_t addmod61(uint64_t a, uint64_t w) {  // a < p, w < 2^32
  uint64_t x = a + w;
  return x >= kP61 ? x - kP61 : x;
}

FKS_HD uint64_t fp_base(uint64_t seed, uint32_t round) {
  return derive(seed, round, kTagFingerprint, 0).m0 % (kP61 - 1) + 1;
}

// ---------------------------------------------------------------- layouts
// Bucket descriptor: slot offset (32) | s (20) | attempt (12).
FKS_HD uint64_t desc_pack(uint32_t off, uint32_t s, uint32_t attempt) {
  return uint64_t(off) | (uint64_t(s) << 32) | (uint64_t(attempt) << 52);
}
FKS_HD uint32_t desc_off(uint64_t d) { return uint32_t(d); }
FKS_HD uint32_t desc_s(uint64_t d) { return uint32_t(d >> 32) & 0xFFFFFu; }
FKS_HD uint32_t desc_attempt(uint64_t d) { return uint32_t(d >> 52); }

// String slot word 1: offset into the map's context (40) | length (24).
FKS_HD uint64_t offlen_pack(uint64_t off, uint64_t len) { return off | (len << 40); }
FKS_HD uint64_t offlen_off(uint64_t w) { return w & ((1ull << 40) - 1); }
FKS_HD uint32_t offlen_len(uint64_t w) { return uint32_t(w >> 40); }

}  // namespace fks
