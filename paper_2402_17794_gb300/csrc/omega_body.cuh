// Philox4x32-10 and Box-Muller device functions shared by the single-problem
// and grouped Gaussian kernels (see omega.cu for the layout of Omega).
#pragma once

#include "internal.h"

namespace rsvd {
namespace omega {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                             uint32_t& c3, uint32_t k0, uint32_t k1) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
  uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
  uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0;
  c1 = lo1;
  c2 = n2;
  c3 = lo0;
}

__device__ __forceinline__ double uniform52(uint32_t wa, uint32_t wb) {
  uint64_t x = ((uint64_t)(wa >> 6) << 26) | (uint64_t)(wb >> 6);
  return ((double)x + 0.5) * 0x1p-52;
}

__device__ __forceinline__ void philox10(uint64_t t, uint32_t stream, uint32_t k0, uint32_t k1,
                                         uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3) {
  c0 = (uint32_t)t;
  c1 = (uint32_t)(t >> 32);
  c2 = stream;
  c3 = 0;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c0, c1, c2, c3, k0, k1);
  }
}

__device__ __forceinline__ double gaussian_at(uint64_t t, uint32_t stream, uint32_t k0,
                                              uint32_t k1) {
  uint32_t c0, c1, c2, c3;
  philox10(t, stream, k0, k1, c0, c1, c2, c3);
  double u1 = uniform52(c0, c1);
  double u2 = uniform52(c2, c3);
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// FP32 Box-Muller on u = (w >> 8 + 1/2) 2^-24 from words 0 and 2.
__device__ __forceinline__ float gaussian_at_f32(uint64_t t, uint32_t stream, uint32_t k0,
                                                 uint32_t k1) {
  uint32_t c0, c1, c2, c3;
  philox10(t, stream, k0, k1, c0, c1, c2, c3);
  const float u1 = ((float)(c0 >> 8) + 0.5f) * 0x1p-24f;
  const float u2 = ((float)(c2 >> 8) + 0.5f) * 0x1p-24f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}


// FP64 Gaussian for linear index t of Omega and a 64-bit seed.
__device__ __forceinline__ double gaussian_value_f64(uint64_t t, uint32_t stream, uint64_t seed) {
  return gaussian_at(t, stream, (uint32_t)seed, (uint32_t)(seed >> 32));
}

}  // namespace omega
}  // namespace rsvd
