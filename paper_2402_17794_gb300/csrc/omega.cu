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

#include "omega_body.cuh"

namespace rsvd {
namespace {

using namespace omega;

__global__ void gaussian_f32_fast_kernel(int64_t n, int l, uint32_t k0, uint32_t k1,
                                         uint32_t stream, float* __restrict__ out, int64_t ldo,
                                         uint64_t t0) {
  const uint64_t total = (uint64_t)n * (uint64_t)l;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t j = t / (uint64_t)n, i = t - j * (uint64_t)n;
    out[i + j * (uint64_t)ldo] = gaussian_at_f32(t0 + t, stream, k0, k1);
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
                                T* __restrict__ out, int64_t ldo, uint64_t t0) {
  const uint64_t total = (uint64_t)n * (uint64_t)l;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t j = t / (uint64_t)n, i = t - j * (uint64_t)n;
    out[i + j * (uint64_t)ldo] = to_out<T>(gaussian_at(t0 + t, stream, k0, k1));
  }
}

}  // namespace

cudaError_t launch_gaussian(int64_t n, int l, uint64_t seed, uint32_t stream_id, int out_dtype,
                            void* out, int64_t ldo, cudaStream_t st, int64_t col0) {
  const uint64_t t0 = (uint64_t)col0 * (uint64_t)n;   // first column drawn is column col0
  const uint64_t total = (uint64_t)n * (uint64_t)l;
  int threads = 256;
  uint64_t want = (total + threads - 1) / threads;
  int blocks = (int)(want < 152 * 16 ? (want ? want : 1) : 152 * 16);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (out_dtype == RSVD_F64) {
    gaussian_kernel<double><<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id, (double*)out,
                                                        ldo, t0);
    note_launch();
  } else if (out_dtype == kOutF32Fast) {
    gaussian_f32_fast_kernel<<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id, (float*)out,
                                                         ldo, t0);
    note_launch();
  } else if (out_dtype == RSVD_F32) {
    gaussian_kernel<float><<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id, (float*)out,
                                                       ldo, t0);
    note_launch();
  } else if (out_dtype == RSVD_BF16) {
    gaussian_kernel<__nv_bfloat16><<<blocks, threads, 0, st>>>(n, l, k0, k1, stream_id,
                                                               (__nv_bfloat16*)out, ldo, t0);
    note_launch();
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rsvd
