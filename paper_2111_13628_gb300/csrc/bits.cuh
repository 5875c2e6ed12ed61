// Bit-sliced helpers shared by the multi-spin-coded kernels (32 replicas per 32-bit word).
#pragma once
#include <stdint.h>

namespace nmc {

__device__ __forceinline__ uint32_t maj3b(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (a & c) | (b & c);
}

// Transposes the 8x8 bit matrix held as 8 bytes (byte j = row j) so that byte i holds
// column i: with row j = bit plane j of 8 replicas, byte i becomes replica i's value.
__device__ __forceinline__ unsigned long long transpose8(unsigned long long x) {
  unsigned long long t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return x;
}

// Gathers byte q of each of the 8 planes p[0..7] into one 64-bit word (byte j from plane j).
__device__ __forceinline__ unsigned long long gather_bytes(const uint32_t *p, int q) {
  const uint32_t sel = (uint32_t)q | ((uint32_t)(4 + q) << 4);
  const uint32_t t01 = __byte_perm(p[0], p[1], sel), t23 = __byte_perm(p[2], p[3], sel);
  const uint32_t t45 = __byte_perm(p[4], p[5], sel), t67 = __byte_perm(p[6], p[7], sel);
  return (unsigned long long)__byte_perm(t01, t23, 0x5410) |
         ((unsigned long long)__byte_perm(t45, t67, 0x5410) << 32);
}

}  // namespace nmc
