// fastdiv.h -- unsigned 32-bit division by a divisor fixed at set-up, as a multiply-high, an
// add and two shifts (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, the round-up method for N = 32 bits, which is exact for every
// 32-bit numerator).  Site coordinates come from the linear site index this way in every
// lattice kernel.  Plain C++ so that host code and tests can use it as well.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define LBMD_HD __host__ __device__ __forceinline__
#else
#define LBMD_HD inline
#endif

namespace lbmd {

struct FastDiv {
  uint32_t d;    // divisor, >= 1
  uint32_t m;    // multiplier: floor(2^32 (2^l - d) / d) + 1 with l = ceil(log2 d)
  uint32_t s1;   // min(l, 1)
  uint32_t s2;   // max(l - 1, 0)
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;  // l = ceil(log2 d)
  f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

LBMD_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// n / f.d for every 32-bit n
LBMD_HD uint32_t fast_div(uint32_t n, const FastDiv &f) {
  const uint32_t t = mulhi32(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

}  // namespace lbmd
