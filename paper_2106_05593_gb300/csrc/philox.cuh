// Counter-based Philox4x32-10 generator (J. K. Salmon, M. A. Moraes, R. O. Dror,
// D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds
// of two 32x32 -> 64-bit products of counter words 0 and 2, mixed with the round
// key, which is advanced by the two Weyl increments between rounds.
#pragma once

#include <cuda_runtime.h>

namespace mmc {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    // one 32 x 32 -> 64-bit product per multiplier (both halves at once)
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const unsigned lo0 = (unsigned)p0, hi0 = (unsigned)(p0 >> 32);
    const unsigned lo1 = (unsigned)p1, hi1 = (unsigned)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// The same generator with the ten round keys given (rk[2 r], rk[2 r + 1] = the
// key after r bumps): a launch computes them once on the host, so that the
// rounds read them from the kernel's parameter space.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const unsigned *rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const unsigned lo0 = (unsigned)p0, hi0 = (unsigned)(p0 >> 32);
    const unsigned lo1 = (unsigned)p1, hi1 = (unsigned)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// uniform in (0, 1): ((r >> 9) + 1/2) * 2^-23, exact in FP32.  Built from the
// bits: 1 + (r >> 9) 2^-23 is a float in [1, 2) whose mantissa is r >> 9, and
// subtracting 1 - 2^-24 is exact (Sterbenz: the operands are within a factor 2).
__device__ __forceinline__ float uniform01(unsigned r) {
  return __uint_as_float(0x3F800000u | (r >> 9)) - 0.99999994039535522461f;
}

}  // namespace mmc
