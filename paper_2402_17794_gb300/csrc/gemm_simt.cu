// Tall-skinny products on the CUDA cores, FP64 or FP32: the passes over A
// of the plain path (Algorithm 4, steps 2, 5 and 6, Section 3.3) and the
// O(m l^2) products of CholeskyQR2 (Gram Y^T Y, Y R^-1) and of the lift
// U = Q U~ (step 8) in both paths.
//
// On GB300 FP64 runs at 2 DFMA per clock per SM (about 1.2 TFLOP/s for the
// GPU) while HBM streams ~6.8 TB/s, so an FP64 pass over A at l = 80
// (20 flop per byte of A) is bound by the FP64 pipe by two orders of
// magnitude, not by memory.  The kernel is therefore shaped to keep the
// DFMA pipe busy: 64 x BN output tiles (BN = 16*TN matched to l so no
// column of work is padded away), 4 x TN accumulators per thread, both
// operands staged in padded shared memory (conflict-free 8-byte accesses)
// with a register double buffer, and split-K so that every SM holds several
// CTAs.  Split-K partials are summed by a second kernel in a fixed order,
// so results do not depend on scheduling.
#include <algorithm>

#include "gemm_body.cuh"

namespace rsvd {
namespace {

using simt::BK;
using simt::BM;
using simt::THREADS;

template <typename T, int TN, bool TRANS>
__global__ void __launch_bounds__(THREADS)
gemm_simt_kernel(const T* __restrict__ A, int64_t lda, const T* __restrict__ X,
                 int64_t ldx, T* __restrict__ C, int64_t ldc, int64_t M, int64_t K, int N,
                 int64_t k_per_split, int64_t part_stride, int x_upper) {
  const int64_t kb = (int64_t)blockIdx.z * k_per_split;
  int64_t ke = (kb + k_per_split < K) ? kb + k_per_split : K;
  if (x_upper) {  // X upper triangular: this column tile needs k < its last column + 1
    const int64_t kc = (int64_t)(blockIdx.y + 1) * 16 * TN;
    if (kc < ke) ke = kc;
  }
  simt::gemm_tile<T, TN, TRANS>(A, lda, X, ldx, C + (int64_t)blockIdx.z * part_stride, ldc, M, N,
                                (int64_t)blockIdx.x * BM, blockIdx.y * 16 * TN, kb, ke);
}

template <typename T>
__global__ void splitk_reduce_kernel(const T* __restrict__ part, int splits,
                                     int64_t part_stride, int64_t M, int N, T* __restrict__ C,
                                     int64_t ldc) {
  const int64_t total = M * (int64_t)N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = t / M, r = t - c * M;
    T s = T(0);
    for (int z = 0; z < splits; ++z) s += part[z * part_stride + t];
    C[r + c * ldc] = s;
  }
}

template <typename T, int TN>
void launch_tn(const GemmArgs<T>& g, dim3 grid, T* out, int64_t ldo, int64_t kps,
               int64_t pstride, cudaStream_t st) {
  if (g.trans)
    gemm_simt_kernel<T, TN, true><<<grid, THREADS, 0, st>>>(g.A, g.lda, g.X, g.ldx, out, ldo, g.M,
                                                            g.K, g.N, kps, pstride, 0);
  else
    gemm_simt_kernel<T, TN, false><<<grid, THREADS, 0, st>>>(g.A, g.lda, g.X, g.ldx, out, ldo,
                                                             g.M, g.K, g.N, kps, pstride,
                                                             g.x_upper ? 1 : 0);
  note_launch();
}

}  // namespace

template <typename T>
cudaError_t launch_gemm(const GemmArgs<T>& g, T* part, size_t part_elems, int num_sms,
                        cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  // Column tiles of at most 96 columns, each a multiple of 16 wide.
  int col_tiles = (g.N + 95) / 96;
  int per = (g.N + col_tiles - 1) / col_tiles;
  int tn = (per + 15) / 16;
  int bn = 16 * tn;
  col_tiles = (g.N + bn - 1) / bn;
  int64_t row_tiles = (g.M + BM - 1) / BM;
  // Split K so the grid covers every SM several times, keeping >= 256 of K
  // per split, and never more slices than the partial buffer holds.
  int64_t tiles = row_tiles * col_tiles;
  int64_t target = (int64_t)num_sms * 6;
  int64_t splits = (target + tiles - 1) / tiles;
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, g.K / 256));
  splits = std::min<int64_t>(splits, kMaxSplits);
  int64_t pstride = g.M * (int64_t)g.N;
  if (splits > 1 && (part == nullptr || (size_t)(splits * pstride) > part_elems))
    splits = part ? std::max<int64_t>(1, (int64_t)(part_elems / (size_t)pstride)) : 1;
  if (splits < 1) splits = 1;
  int64_t kps = (g.K + splits - 1) / splits;
  kps = (kps + BK - 1) / BK * BK;
  splits = (g.K + kps - 1) / kps;
  if (splits < 1) splits = 1;
  dim3 grid((unsigned)row_tiles, (unsigned)col_tiles, (unsigned)splits);
  T* out = splits > 1 ? part : g.C;
  int64_t ldo = splits > 1 ? g.M : g.ldc;
  switch (tn) {
    case 1: launch_tn<T, 1>(g, grid, out, ldo, kps, pstride, st); break;
    case 2: launch_tn<T, 2>(g, grid, out, ldo, kps, pstride, st); break;
    case 3: launch_tn<T, 3>(g, grid, out, ldo, kps, pstride, st); break;
    case 4: launch_tn<T, 4>(g, grid, out, ldo, kps, pstride, st); break;
    case 5: launch_tn<T, 5>(g, grid, out, ldo, kps, pstride, st); break;
    case 6: launch_tn<T, 6>(g, grid, out, ldo, kps, pstride, st); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  int64_t total = pstride;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 8);
  splitk_reduce_kernel<T><<<blocks, 256, 0, st>>>(part, (int)splits, pstride, g.M, g.N, g.C, g.ldc);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmArgs<double>&, double*, size_t, int,
                                         cudaStream_t);
template cudaError_t launch_gemm<float>(const GemmArgs<float>&, float*, size_t, int, cudaStream_t);

}  // namespace rsvd
