// Counter-based normal numbers of Alg. 1's start block, shared by every
// kernel that draws it: Philox4x32-10 (Salmon et al., "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011) and the Box-Muller transform.
#pragma once

#include <cstdint>

namespace isvd {

// Philox4x32-10: ten rounds on the counter (c0..c3) with key (k0, k1).
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
}

// Normals j = 4q .. 4q+3 of row i: counter (q, i mod 2^32, i / 2^32, 0),
// words (0,1) and (2,3) through Box-Muller with u = (word + 1/2) 2^-32.
__device__ __forceinline__ void gaussian_quad(uint32_t k0, uint32_t k1, int64_t i, int32_t q, float z[4]) {
  uint32_t c0 = (uint32_t)q, c1 = (uint32_t)i, c2 = (uint32_t)((uint64_t)i >> 32), c3 = 0u;
  philox4x32_10(c0, c1, c2, c3, k0, k1);
  const uint32_t w[4] = {c0, c1, c2, c3};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    // u = (w + 1/2) 2^-32.  Near u = 1 the float form of u loses the
    // distance 1 - u = (~w + 1/2) 2^-32, so ln u is taken as log1p of that
    // distance and 2u as the equivalent angle 2u - 2 (period 2 of sincospi).
    const uint32_t wa = w[2 * h], wb = w[2 * h + 1];
    const float lnu = (wa < 0x80000000u) ? logf(fmaf((float)wa, 2.3283064365386963e-10f, 1.1641532182693481e-10f))
                                         : log1pf(-fmaf((float)(~wa), 2.3283064365386963e-10f,
                                                        1.1641532182693481e-10f));
    const float t = (wb < 0x80000000u) ? fmaf((float)wb, 4.6566128730773926e-10f, 2.3283064365386963e-10f)
                                       : -fmaf((float)(~wb), 4.6566128730773926e-10f, 2.3283064365386963e-10f);
    const float rho = sqrtf(-2.0f * lnu);
    float sn, cs;
    sincospif(t, &sn, &cs);
    z[2 * h] = rho * cs;
    z[2 * h + 1] = rho * sn;
  }
}

}  // namespace isvd
