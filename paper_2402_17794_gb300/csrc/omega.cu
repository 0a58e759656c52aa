// Step 1 of Algorithm 4 (Section 3.3): the n x l Gaussian test matrix Omega.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) gives four 32-bit words
// per counter; two words make a 52-bit uniform u = (x + 1/2) 2^-52 (exact in
// FP64, strictly inside (0, 1)); Box-Muller (1958) turns (u1, u2) into
// z = sqrt(-2 ln u1) cos(2 pi u2).  Element (i, j) of the column-major
// Omega uses counter (lo32(t), hi32(t), stream, 0), t = j*n + i, and key
// (lo32(seed), hi32(seed)).  The work is O(n l) (Section 3.1.1's sampling
// cost), negligible beside one pass over A, so the kernel is a plain
// grid-stride loop with coalesced column-major stores.
#include <cuda_bf16.h>

#include "internal.h"

namespace rsvd {
namespace {

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

__global__ void gaussian_f32_fast_kernel(int64_t n, int l, uint32_t k0, uint32_t k1,
                                         uint32_t stream, float* __restrict__ out, int64_t ldo) {
  const uint64_t total = (uint64_t)n * (uint64_t)l;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t j = t / (uint64_t)n, i = t - j * (uint64_t)n;
    out[i + j * (uint64_t)ldo] = gaussian_at_f32(t, stream, k0, k1);
  }
}

template <typename T>
__device__ __forceinline__ T to_out(double z);
template <>
__device__ __forceinline__ double to_out<double>(double z) { return z; }
template <>
__device__ __forceinline__ float to_out<float>(double z) { return (float)z; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(double z) {
  return __double2bfloat16(z);
}

template <typename T>
__global__ void gaussian_kernel(int64_t n, int l, uint32_t k0, uint32_t k1, uint32_t stream,
                                T* __restrict__ out, int64_t ldo) {
  const uint64_t total = (uint64_t)n * (uint64_t)l;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t j = t / (uint64_t)n, i = t - j * (uint64_t)n;
    out[i + j * (uint64_t)ldo] = to_out<T>(gaussian_at(t, stream, k0, k1));
  }
}

}  // namespace

cudaError_t launch_gaussian(int64_t n, int l, uint64_t seed, uint32_t stream_id, int out_dtype,
                            void* out, int64_t ldo, cudaStream_t st) {
  const uint64_t total = (uint64_t)n * (uint64_t)l;
  int threads = 256;
  uint64_t want = (total + threads - 1) / threads;
  int blocks = (int)(want < 152 * 16 ? (want ? want : 1) : 152 * 16);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (out_dtype == RSVD_F64) {
    gaussian_kernel<double><<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id, (double*)out, ldo);
    note_launch();
  } else if (out_dtype == kOutF32Fast) {
    gaussian_f32_fast_kernel<<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id, (float*)out,
                                                         ldo);
    note_launch();
  } else if (out_dtype == RSVD_F32) {
    gaussian_kernel<float><<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id, (float*)out, ldo);
    note_launch();
  } else if (out_dtype == RSVD_BF16) {
    gaussian_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id,
                                                               (__nv_bfloat16*)out, ldo);
    note_launch();
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rsvd
