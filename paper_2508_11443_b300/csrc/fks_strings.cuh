// fks_strings.cuh -- device helpers for byte-string keys (Sec. 3.1: a key is
// an (offset, length) slice of a context): word reads, the polynomial
// fingerprint of R8 and exact byte equality.
#pragma once
#include <stdint.h>

#include "fks_device.cuh"

namespace fks {

// t-th little-endian 32-bit word of the byte string s[0 .. len), zero padded.
// Reads only aligned words that hold at least one byte of the string.
__device__ __forceinline__ uint32_t str_word(const uint8_t* s, uint32_t len, uint32_t t) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(s) + 4u * t;
  const uint32_t r = len - 4u * t;  // bytes left, >= 1
  const uint32_t take = r < 4u ? r : 4u;
  const uint32_t sh = uint32_t(a & 3u);
  const uint32_t* A = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t lo = __ldg(A);
  const uint32_t hi = (sh + take > 4u) ? __ldg(A + 1) : 0u;
  uint32_t w = __funnelshift_r(lo, hi, sh * 8u);
  if (take < 4u) w &= (1u << (8u * take)) - 1u;
  return w;
}

// Horner over [len, word 0, word 1, ...] modulo 2^61 - 1 at base `base`.
__device__ __forceinline__ uint64_t fingerprint(const uint8_t* s, uint32_t len, uint64_t base) {
  uint64_t h = len;
  const uint32_t words = (len + 3u) >> 2;
  for (uint32_t t = 0; t < words; ++t) h = addmod61(mulmod61(h, base), str_word(s, len, t));
  return h;
}

__device__ __forceinline__ bool bytes_equal(const uint8_t* a, const uint8_t* b, uint32_t len) {
  const uint32_t words = (len + 3u) >> 2;
  for (uint32_t t = 0; t < words; ++t)
    if (str_word(a, len, t) != str_word(b, len, t)) return false;
  return true;
}

}  // namespace fks
