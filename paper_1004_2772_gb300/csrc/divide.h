// Division by a run-time invariant divisor with one multiply-high, for tables
// whose line count is not a power of two (Section 3.1 allows any table size
// through division by a constant; the method is the unsigned case of
// Granlund and Montgomery, "Division by Invariant Integers using
// Multiplication", PLDI 1994, Fig. 4.1, also in Warren, "Hacker's Delight",
// ch. 10).
//
// For a divisor 1 <= d <= 2^32 and l = ceil(log2 d):
//   m   = floor(2^64 * (2^l - d) / d) + 1          (fits in 64 bits)
//   sh1 = min(l, 1),  sh2 = max(l - 1, 0)
//   t   = mulhi64(m, n)
//   n / d = (t + ((n - t) >> sh1)) >> sh2          for every 64-bit n.
#pragma once

#include <stdint.h>

namespace vss {

struct DivU64 {
  uint64_t m;    // magic multiplier
  uint32_t d;    // divisor
  uint32_t sh;   // sh1 | sh2 << 8
};

#if defined(__CUDACC__)
#define VSS_HD __host__ __device__ __forceinline__
#else
#define VSS_HD inline
#endif

VSS_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

VSS_HD uint64_t div_q(const DivU64& v, uint64_t n) {
  const uint64_t t = mulhi64(v.m, n);
  return (t + ((n - t) >> (v.sh & 0xFFu))) >> (v.sh >> 8);
}

VSS_HD uint32_t div_r(const DivU64& v, uint64_t n) {  // n mod d (d <= 2^32 - 1)
  return (uint32_t)(n - div_q(v, n) * v.d);
}

// Host: the constants for divisor d (1 <= d < 2^32).
inline DivU64 make_div(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < (uint64_t)d) ++l;
  const unsigned __int128 num = ((unsigned __int128)1 << 64) * ((1ull << l) - d);
  DivU64 v;
  v.m = (uint64_t)(num / d) + 1;
  v.d = d;
  const uint32_t sh1 = l < 1 ? l : 1, sh2 = l > 1 ? l - 1 : 0;
  v.sh = sh1 | (sh2 << 8);
  return v;
}

#undef VSS_HD

}  // namespace vss
