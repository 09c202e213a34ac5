// modarith.cuh -- modular arithmetic of the counting residue planes (device):
// 61-bit primes 2^61 - c in 8-byte residues and 31-bit primes 2^31 - c in
// 4-byte ones, c < 2^10, reduced after Crandall's pseudo-Mersenne method.
#pragma once
#include <stdint.h>

namespace tn {

static constexpr uint64_t M61 = (1ull << 61) - 1;

// a * b mod p for p = 2^61 - c, a, b < p, c < 2^10.  The 122-bit product is
// folded twice with 2^61 = c (mod p) (pseudo-Mersenne reduction, Crandall 1992).
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t lo = a * b;
  uint64_t hi = __umul64hi(a, b);
  uint64_t x1 = (hi << 3) | (lo >> 61);   // product >> 61, < 2^61
  uint64_t x0 = lo & M61;
  uint64_t t_lo = x1 * c;
  uint64_t t_hi = __umul64hi(x1, c);
  uint64_t y_lo = t_lo + x0;
  uint64_t y_hi = t_hi + (y_lo < t_lo ? 1ull : 0ull);
  uint64_t y1 = (y_hi << 3) | (y_lo >> 61);  // < 2^11
  uint64_t z = y1 * c + (y_lo & M61);        // < 2^61 + 2^21 < 2p
  uint64_t p = M61 + 1 - c;
  return z >= p ? z - p : z;
}

__device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t p = M61 + 1 - c;
  uint64_t s = a + b;
  return s >= p ? s - p : s;
}

// The same for p = 2^31 - c (c < 2^10) on 4-byte residues: the 62-bit product
// is folded twice with 2^31 = c (mod p).
static constexpr uint64_t M31 = (1ull << 31) - 1;
__device__ __forceinline__ uint32_t mulmod31(uint32_t a, uint32_t b, uint64_t c) {
  const uint64_t x = (uint64_t)a * b;                  // < 2^62
  const uint64_t y = (x >> 31) * c + (x & M31);        // < 2^41
  const uint64_t z = (y >> 31) * c + (y & M31);        // < 2^31 + 2^20 < 2p
  const uint64_t p = M31 + 1 - c;
  return (uint32_t)(z >= p ? z - p : z);
}
__device__ __forceinline__ uint32_t addmod31(uint32_t a, uint32_t b, uint64_t c) {
  const uint32_t p = (uint32_t)(M31 + 1 - c);
  const uint32_t s = a + b;                            // < 2p < 2^32
  return s >= p ? s - p : s;
}
// residue arithmetic by plane width
__device__ __forceinline__ uint64_t mulmodR(uint64_t a, uint64_t b, uint64_t c) {
  return mulmod61(a, b, c);
}
__device__ __forceinline__ uint32_t mulmodR(uint32_t a, uint32_t b, uint64_t c) {
  return mulmod31(a, b, c);
}
__device__ __forceinline__ uint64_t addmodR(uint64_t a, uint64_t b, uint64_t c) {
  return addmod61(a, b, c);
}
__device__ __forceinline__ uint32_t addmodR(uint32_t a, uint32_t b, uint64_t c) {
  return addmod31(a, b, c);
}

}  // namespace tn
