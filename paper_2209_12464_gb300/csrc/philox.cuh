// Counter-based Gaussian test matrix for RU-QLP's sketch (Section III-A
// step 1: Omega with iid N(0,1) entries), generated on the device.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): 10 rounds of
//   (hi0, lo0) = 0xD2511F53 * c0,  (hi1, lo1) = 0xCD9E8D57 * c2,
//   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key bumped by (0x9E3779B9, 0xBB67AE85) after each round.
// Entry (i, j) of Omega uses counter (j, i mod 2^32, i / 2^32, 0) and key
// (seed mod 2^32, seed / 2^32); its first two output words give
// u1 = (x0 + 1/2) 2^-32, u2 = (x1 + 1/2) 2^-32 in (0, 1) and
//   Omega_ij = sqrt(-2 ln u1) cos(2 pi u2)      (Box-Muller, first variate),
// evaluated in FP64.
#pragma once
#include <stdint.h>

namespace ruqlp {

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ double omega_entry(uint64_t seed, int64_t i, int j) {
  uint32_t c[4] = {(uint32_t)j, (uint32_t)((uint64_t)i & 0xFFFFFFFFu),
                   (uint32_t)((uint64_t)i >> 32), 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  const double u1 = ((double)c[0] + 0.5) * 2.3283064365386963e-10;  // 2^-32
  const double u2 = ((double)c[1] + 0.5) * 2.3283064365386963e-10;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

}  // namespace ruqlp
