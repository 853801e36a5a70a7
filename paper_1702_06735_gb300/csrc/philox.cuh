// Philox4x32-10 counter-based random numbers (J. K. Salmon, M. A. Moraes,
// R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): a 128-bit counter and a 64-bit key give 128 random bits through
// ten rounds of two 32x32 -> 64-bit multiplications, with the key bumped by
// the Weyl constants between rounds.  Any (key, counter) pair is drawn
// independently, so every thread draws its own stream without state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tdmix {

struct Philox4 {
  uint32_t v[4];
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(Philox4 c, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;  // round multipliers
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;  // key increments
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = uint64_t(M0) * c.v[0];
    const uint64_t p1 = uint64_t(M1) * c.v[2];
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    c = Philox4{{hi1 ^ c.v[1] ^ k0, lo1, hi0 ^ c.v[3] ^ k1, lo0}};
  }
  return c;
}

// A double in [0, 1) from 53 random bits (the top 32 of a, top 21 of b).
__host__ __device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
  return double((uint64_t(a) << 21) | (b >> 11)) * (1.0 / 9007199254740992.0);
}

}  // namespace tdmix
