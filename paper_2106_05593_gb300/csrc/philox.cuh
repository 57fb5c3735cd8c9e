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
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// uniform in (0, 1): ((r >> 9) + 1/2) * 2^-23, exact in FP32
__device__ __forceinline__ float uniform01(unsigned r) {
  return ((float)(r >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

}  // namespace mmc
