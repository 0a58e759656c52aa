// Gram products G = Y^T Y of CholeskyQR2 (the orth(.) of Algorithm 4,
// Section 3.3) on the CUDA cores, FP64 or FP32.
//
// Y is tall and skinny (up to 65536 rows, l <= 272 columns in FP32, 160 in
// FP64) and G is l x l
// and symmetric, so only the upper triangle is formed:
//
//  * every CTA takes a contiguous range of rows and forms its rows' whole
//    contribution to the upper triangle;
//  * thread t owns one B x B block (bi <= bj) of G in registers, so each
//    value of Y read from shared memory feeds B multiply-adds;
//  * rows are staged KB at a time by cp.async into a row-major shared tile
//    (double buffered), so a block row's B values are contiguous;
//  * the per-CTA partials are summed in CTA order by a second kernel, so
//    the result does not depend on scheduling.
#include <algorithm>

#include "internal.h"

namespace rsvd {
namespace {

constexpr int KB = 32;   // rows of Y per shared-memory stage

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(T) : 0;   // 0 source bytes: zero fill
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared tile row stride: the blocks' width plus 4 elements, so a warp that
// stores 8 rows x 4 columns (FP32) hits 32 distinct banks, and rows stay
// 16-byte aligned.
__host__ __device__ inline int gram_ldt(int l, int B) { return (l + B - 1) / B * B + 4; }

// Stages rows [r, r + KB) of Y into tile (row-major, stride ldt).  Threads
// go down columns in groups of G rows (one 32-byte sector), consecutive
// groups take consecutive columns.
template <typename T>
__device__ __forceinline__ void stage_rows(const T* __restrict__ Y, int64_t ldy, int64_t r,
                                           int64_t r_end, int l, T* tile, int ldt) {
  constexpr int G = 32 / sizeof(T);
  const int total = KB * l;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int g = e / G, rr = e - g * G;
    const int c = g % l;
    const int row = (g / l) * G + rr;
    const int64_t gr = r + row;
    const bool ok = gr < r_end;
    cp_async_elem(tile + row * ldt + c, Y + (ok ? gr : r) + (int64_t)c * ldy, ok);
  }
}

// Loads n = B values from 16-byte aligned shared memory as 16-byte vectors.
template <int B>
__device__ __forceinline__ void ld_frag(const float* p, float (&v)[B]) {
#pragma unroll
  for (int q = 0; q < B / 4; ++q) {
    const float4 x = *reinterpret_cast<const float4*>(p + 4 * q);
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
}
template <int B>
__device__ __forceinline__ void ld_frag(const double* p, double (&v)[B]) {
#pragma unroll
  for (int q = 0; q < B / 2; ++q) {
    const double2 x = *reinterpret_cast<const double2*>(p + 2 * q);
    v[2 * q] = x.x;
    v[2 * q + 1] = x.y;
  }
}

// Threads per CTA the kernel is compiled for (the upper-triangle blocks of
// the largest l that the block edge serves, rounded up to warps).
template <typename T, int B>
constexpr int gram_max_threads() {
  return (sizeof(T) == 4 && B == 8) ? 608 : (sizeof(T) == 8 ? 832 : 544);
}

template <typename T, int B>
__global__ void __launch_bounds__(gram_max_threads<T, B>())
gram_kernel(const T* __restrict__ Y, int64_t ldy, int64_t rows, int l, int64_t chunk,
            T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char gram_smem[];
  T* tiles = reinterpret_cast<T*>(gram_smem);
  const int nb = (l + B - 1) / B;
  const int ldt = gram_ldt(l, B);
  const int tid = threadIdx.x;

  // this thread's block (bi, bj), bi <= bj, enumerated row by row
  int bi = -1, bj = -1;
  {
    int u = tid;
    for (int a = 0; a < nb; ++a) {
      const int len = nb - a;
      if (u < len) {
        bi = a;
        bj = a + u;
        break;
      }
      u -= len;
    }
  }
  // padded columns (l .. nb*B) stay zero in both stages
  for (int e = tid; e < 2 * KB * (ldt - l); e += blockDim.x) {
    const int w = ldt - l;
    const int s = e / (KB * w), rem = e - s * KB * w;
    tiles[s * KB * ldt + (rem / w) * ldt + l + rem % w] = T(0);
  }

  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = (r0 + chunk < rows) ? r0 + chunk : rows;
  T acc[B][B];
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int b = 0; b < B; ++b) acc[a][b] = T(0);

  const int nstage = (int)((r1 - r0 + KB - 1) / KB);
  if (nstage > 0) stage_rows(Y, ldy, r0, r1, l, tiles, ldt);
  cp_async_commit();
  for (int s = 0; s < nstage; ++s) {
    T* cur = tiles + (s & 1) * KB * ldt;
    if (s + 1 < nstage)
      stage_rows(Y, ldy, r0 + (int64_t)(s + 1) * KB, r1, l, tiles + ((s + 1) & 1) * KB * ldt, ldt);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if (bi >= 0) {
      const T* pa = cur + bi * B;
      const T* pb = cur + bj * B;
#pragma unroll 2
      for (int r = 0; r < KB; ++r) {
        T va[B], vb[B];
        ld_frag<B>(pa + r * ldt, va);
        ld_frag<B>(pb + r * ldt, vb);
#pragma unroll
        for (int a = 0; a < B; ++a)
#pragma unroll
          for (int b = 0; b < B; ++b) acc[a][b] = fma(va[a], vb[b], acc[a][b]);
      }
    }
    __syncthreads();
  }
  if (bi < 0) return;
  T* out = part + (size_t)blockIdx.x * l * l;
#pragma unroll
  for (int a = 0; a < B; ++a) {
    const int i = bi * B + a;
    if (i >= l) break;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int c = bj * B + b;
      if (c < l) out[i + (size_t)c * l] = acc[a][b];
    }
  }
}

// G (ldg) = sum of the partials, in CTA order; both triangles written.
template <typename T>
__global__ void gram_reduce_kernel(const T* __restrict__ part, int parts, int l, T* __restrict__ G,
                                   int64_t ldg) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * l) return;
  const int i = e % l, c = e / l;
  if (i > c) return;
  T s = T(0);
  for (int p = 0; p < parts; ++p) s += part[(size_t)p * l * l + e];
  G[i + (int64_t)c * ldg] = s;
  G[c + (int64_t)i * ldg] = s;
}

template <typename T, int B>
cudaError_t launch_b(const T* Y, int64_t ldy, int64_t rows, int l, T* G, int64_t ldg, T* part,
                     int grid, int64_t chunk, cudaStream_t st) {
  const int nb = (l + B - 1) / B;
  const int threads = std::max(64, (nb * (nb + 1) / 2 + 31) / 32 * 32);
  const size_t smem = (size_t)2 * KB * gram_ldt(l, B) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(gram_kernel<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set = true;
  }
  gram_kernel<T, B><<<grid, threads, smem, st>>>(Y, ldy, rows, l, chunk, part);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_reduce_kernel<T><<<(l * l + 255) / 256, 256, 0, st>>>(part, grid, l, G, ldg);
  note_launch();
  return cudaGetLastError();
}

// Micro-block edge for (T, l); 0 when the kernel does not cover l.
template <typename T>
int block_edge(int l) {
  if (sizeof(T) == 4) return l <= 64 ? 4 : (l <= 272 ? 8 : 0);
  return l <= 160 ? 4 : 0;   // 40 x 41 / 2 = 820 blocks of 4 x 4 at l = 160
}

}  // namespace

template <typename T>
bool gram_supported(int l) {
  return block_edge<T>(l) > 0;
}

template <typename T>
cudaError_t launch_gram(const T* Y, int64_t ldy, int64_t rows, int l, T* G, int64_t ldg, T* part,
                        size_t part_elems, int num_sms, cudaStream_t st) {
  if (rows <= 0 || l <= 0) return cudaSuccess;
  int grid = (int)std::min<int64_t>(num_sms, (rows + KB - 1) / KB);
  grid = (int)std::min<int64_t>(grid, (int64_t)(part_elems / ((size_t)l * l)));
  if (grid < 1) return cudaErrorInvalidValue;
  int64_t chunk = (rows + grid - 1) / grid;
  chunk = (chunk + KB - 1) / KB * KB;
  grid = (int)((rows + chunk - 1) / chunk);
  const int b = block_edge<T>(l);
  if (b == 4) return launch_b<T, 4>(Y, ldy, rows, l, G, ldg, part, grid, chunk, st);
  if constexpr (sizeof(T) == 4) {
    if (b == 8) return launch_b<T, 8>(Y, ldy, rows, l, G, ldg, part, grid, chunk, st);
  }
  return cudaErrorInvalidValue;
}

template bool gram_supported<double>(int);
template bool gram_supported<float>(int);
template cudaError_t launch_gram<double>(const double*, int64_t, int64_t, int, double*, int64_t,
                                         double*, size_t, int, cudaStream_t);
template cudaError_t launch_gram<float>(const float*, int64_t, int64_t, int, float*, int64_t,
                                        float*, size_t, int, cudaStream_t);

}  // namespace rsvd
