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

// ---------------------------------------------------------------- warp-cooperative forms
// Strings longer than this many bytes are fingerprinted and compared by the
// whole warp; shorter ones by their own lane.
constexpr uint32_t kLongString = 128;

// a + b mod 2^61 - 1 for a, b < 2^61 - 1
__device__ __forceinline__ uint64_t addp61(uint64_t a, uint64_t b) {
  const uint64_t x = a + b;
  return x >= kP61 ? x - kP61 : x;
}

// base^e mod 2^61 - 1 by squaring
__device__ __forceinline__ uint64_t pow61(uint64_t base, uint32_t e) {
  uint64_t r = 1;
  while (e) {
    if (e & 1u) r = mulmod61(r, base);
    base = mulmod61(base, base);
    e >>= 1;
  }
  return r;
}

// The fingerprint of s[0 .. len) by the whole warp (every lane passes the
// same s, len; pw[t] = base^t for t <= 32).  Horner's value
//   len * R^m + sum_t w_t * R^(m - 1 - t)   (m words, mod 2^61 - 1)
// evaluated 32 words at a time: lane x multiplies word c + x by its power,
// the warp sums the products, and the running value moves up by R^k.
// Exact modular arithmetic: the same value as fingerprint().
__device__ __forceinline__ uint64_t warp_fingerprint(const uint8_t* s, uint32_t len, const uint64_t* pw) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t words = (len + 3u) >> 2;
  uint64_t h = len;
  for (uint32_t c = 0; c < words; c += 32) {
    const uint32_t k = words - c < 32u ? words - c : 32u;
    uint64_t term = lane < k ? mulmod61(str_word(s, len, c + lane), pw[k - 1 - lane]) : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) term = addp61(term, __shfl_xor_sync(0xFFFFFFFFu, term, d));
    h = addp61(mulmod61(h, pw[k]), term);
  }
  return h;
}

// a[0 .. len) == b[0 .. len) by the whole warp, 32 words per step.
__device__ __forceinline__ bool warp_bytes_equal(const uint8_t* a, const uint8_t* b, uint32_t len) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t words = (len + 3u) >> 2;
  for (uint32_t c = 0; c < words; c += 32) {
    const bool differ = c + lane < words && str_word(a, len, c + lane) != str_word(b, len, c + lane);
    if (__any_sync(0xFFFFFFFFu, differ)) return false;
  }
  return true;
}

}  // namespace fks
