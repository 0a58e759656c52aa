// Shared body of the tall-skinny SIMT products (single-problem and grouped
// launches): constants and the 64 x (16*TN) tile device function.
#pragma once

#include "internal.h"

namespace rsvd {
namespace simt {

constexpr int BM = 64;
constexpr int BK = 16;
constexpr int THREADS = 256;
constexpr int AS_LD = BM + 1;  // padded row

// One 64 x (16*TN) output tile over the contraction range [kb, ke):
// Cout (ld ldc) = op(A)[r0:r0+64, kb:ke] X[kb:ke, c0:c0+16*TN], where op(A) = A
// (M x K, lda) or A^T (A stored K x M).  Rows >= M and columns >= N are
// neither read nor written.
template <typename T, int TN, bool TRANS>
__device__ __forceinline__ void gemm_tile(const T* __restrict__ A, int64_t lda,
                                          const T* __restrict__ X, int64_t ldx,
                                          T* __restrict__ Cout, int64_t ldc, int64_t M, int N,
                                          int64_t r0, int c0, int64_t kb, int64_t ke) {
  constexpr int BN = 16 * TN;
  constexpr int XS_LD = BN + 1;
  __shared__ T As[2][BK * AS_LD];
  __shared__ T Xs[2][BK * XS_LD];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  constexpr int A_PER = BM * BK / THREADS;             // 4
  constexpr int X_PER = (BN * BK + THREADS - 1) / THREADS;
  T ra[A_PER], rx[X_PER];

  auto load_tiles = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      int idx = tid + e * THREADS;
      int r, kk;
      if (!TRANS) { r = idx % BM; kk = idx / BM; }
      else { kk = idx % BK; r = idx / BK; }
      int64_t gr = r0 + r, gk = k0 + kk;
      T v = T(0);
      if (gr < M && gk < ke) v = TRANS ? A[gk + gr * lda] : A[gr + gk * lda];
      ra[e] = v;
    }
#pragma unroll
    for (int e = 0; e < X_PER; ++e) {
      int idx = tid + e * THREADS;
      int kk = idx % BK, c = idx / BK;
      int64_t gk = k0 + kk;
      T v = T(0);
      if (idx < BN * BK && c0 + c < N && gk < ke) v = X[gk + (int64_t)(c0 + c) * ldx];
      rx[e] = v;
    }
  };
  auto store_tiles = [&](int buf) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      int idx = tid + e * THREADS;
      int r, kk;
      if (!TRANS) { r = idx % BM; kk = idx / BM; }
      else { kk = idx % BK; r = idx / BK; }
      As[buf][kk * AS_LD + r] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < X_PER; ++e) {
      int idx = tid + e * THREADS;
      if (idx < BN * BK) {
        int kk = idx % BK, c = idx / BK;
        Xs[buf][kk * XS_LD + c] = rx[e];
      }
    }
  };

  T acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  int buf = 0;
  if (kb < ke) {
    load_tiles(kb);
    store_tiles(0);
  }
  __syncthreads();
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) load_tiles(k0 + BK);
    const T* as = As[buf];
    const T* xs = Xs[buf];
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], x[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = as[kk * AS_LD + tx + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) x[j] = xs[kk * XS_LD + ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    if (more) store_tiles(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gr = r0 + tx + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gc = c0 + ty + 16 * j;
      if (gc < N) Cout[gr + (int64_t)gc * ldc] = acc[i][j];
    }
  }
}

}  // namespace simt
}  // namespace rsvd
