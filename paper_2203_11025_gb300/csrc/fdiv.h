// Division by a divisor fixed at launch, as a multiply-high and a shift: for 0 <= n < 2^31,
// n / d = (umulhi(n, m) + n) >> s with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1
// (the round-up multiplier of Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994).  The convolution kernels divide item indices by tile counts with
// it; the host builds the multiplier once per launch.  Host and device code share this file
// (the host form of umulhi is the high word of the 64-bit product).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define HELM_FDIV_HD __host__ __device__
#else
#define HELM_FDIV_HD
#endif

namespace helm {

struct FDiv { uint32_t d, m, s; };

inline FDiv make_fdiv(uint32_t d) {
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  const uint64_t m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;   // < 2^32 for d >= 1
  return {d, (uint32_t)m, s};
}

HELM_FDIV_HD inline int fdiv(const FDiv& f, int n) {
#ifdef __CUDA_ARCH__
  const uint32_t hi = __umulhi((uint32_t)n, f.m);
#else
  const uint32_t hi = (uint32_t)(((uint64_t)(uint32_t)n * f.m) >> 32);
#endif
  return (int)((hi + (uint32_t)n) >> f.s);
}

}  // namespace helm
