// Second kernel of a stream-K pass over A (tcgen05 passes): sums the per-CTA
// partials of every output tile whose k-range was split between CTAs.
#include "umma.h"

namespace rsvd {
namespace {

// Sums the per-CTA partials of every tile whose k-range was split, in CTA
// order.  Grid: (tile, group of kFixCols output columns); one thread per
// output row of the tile.  Tiles written whole by one CTA are skipped.  The
// (at most a few) CTAs sharing the tile are resolved once per block.
__global__ void apass_fixup_kernel(const float* __restrict__ part, int grid, int64_t total, int kt,
                                   int bmt, int l, int64_t rows_out, float* __restrict__ out,
                                   int64_t ldo, int accumulate) {
  constexpr int kMaxShare = 32;
  __shared__ int s_src[kMaxShare];
  __shared__ int s_n;
  const int64_t t = blockIdx.x;
  if (threadIdx.x == 0) {
    auto begin = [&](int c) { return (int64_t)((__int128)total * c / grid); };
    auto cta_of = [&](int64_t g) {
      int c = (int)((__int128)g * grid / total);
      while (c + 1 < grid && begin(c + 1) <= g) ++c;
      while (c > 0 && begin(c) > g) --c;
      return c;
    };
    const int cf = cta_of(t * kt), cl = cta_of((t + 1) * kt - 1);
    int n = 0;
    if (cf != cl) {
      for (int cc = cf; cc <= cl && n < kMaxShare; ++cc) {
        const int64_t b = begin(cc);
        if (b >= begin(cc + 1)) continue;
        s_src[n++] = cc * 2 + ((b / kt == t) ? 0 : 1);   // partial slot of CTA cc
      }
    }
    s_n = n;
  }
  __syncthreads();
  const int n = s_n;
  if (n == 0) return;  // written directly by one CTA
  const int64_t per_tile = (int64_t)bmt * l;
  const int c0 = blockIdx.y * kFixCols;
  for (int r = threadIdx.x; r < bmt; r += blockDim.x) {
    const int64_t row = t * bmt + r;
    if (row >= rows_out) continue;
#pragma unroll
    for (int cc = 0; cc < kFixCols; ++cc) {
      const int c = c0 + cc;
      if (c >= l) break;
      float s = 0.f;
      for (int j = 0; j < n; ++j) s += part[(size_t)s_src[j] * per_tile + (size_t)c * bmt + r];
      float* d = out + row + (int64_t)c * ldo;
      *d = accumulate ? *d + s : s;
    }
  }
}

}  // namespace

int launch_apass_fixup(const float* part, int grid, int64_t total, int kt, int bmt, int l,
                       int64_t rows_out, int64_t tiles, float* out, int64_t ldo, int accumulate,
                       cudaStream_t st) {
  const dim3 fgrid((unsigned)tiles, (unsigned)((l + kFixCols - 1) / kFixCols));
  apass_fixup_kernel<<<fgrid, 256, 0, st>>>(part, grid, total, kt, bmt, l, rows_out, out, ldo,
                                            accumulate);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

}  // namespace rsvd
