// Counter-based Gaussian draws shared by the slice engines: Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC'11) and the Box-Muller transform (Box &
// Muller, 1958).  A 4x32-bit counter and 2x32-bit key go through ten rounds;
// each round multiplies words 0 and 2 by fixed odd constants and mixes the
// product halves with words 1, 3 and the round key, the key words advancing
// by Weyl increments between rounds.  Two uniforms u = (w + 1/2)/2^32 give
// r = sqrt(-2 ln u1) and (r cos 2 pi u2, r sin 2 pi u2).
#pragma once

#include <stdint.h>

namespace trrng {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi_a = __umulhi(0xD2511F53u, c[0]), lo_a = 0xD2511F53u * c[0];
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c[2]), lo_b = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi_b ^ c[1] ^ k0, n2 = hi_a ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo_b;
    c[2] = n2;
    c[3] = lo_a;
  }
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1) {
  const float u1 = ((float)a + 0.5f) * 2.3283064365386963e-10f;   // (a + 1/2) / 2^32
  const float u2 = ((float)b + 0.5f) * 2.3283064365386963e-10f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double &z0, double &z1) {
  const double u1 = ((double)a + 0.5) * 2.3283064365386963e-10;
  const double u2 = ((double)b + 0.5) * 2.3283064365386963e-10;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}


}  // namespace trrng
