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

__global__ void apass_fixup_list_kernel(const float* __restrict__ part, int bmt, int l,
                                        int64_t rows_out, float* __restrict__ out, int64_t ldo,
                                        int accumulate, const __grid_constant__ FixList fl) {
  const int i = blockIdx.x;
  const int64_t t = fl.tile[i];
  const int s0 = fl.off[i], s1 = fl.off[i + 1];
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
      for (int j = s0; j < s1; ++j) s += part[(size_t)fl.src[j] * per_tile + (size_t)c * bmt + r];
      float* d = out + row + (int64_t)c * ldo;
      *d = accumulate ? *d + s : s;
    }
  }
}

}  // namespace

// Host mirror of the pass kernel's stream-K ranges: CTA c of `grid` takes
// iterations [total c / grid, total (c+1) / grid).
int64_t host_begin(int64_t total, int c, int grid) {
  return (int64_t)((__int128)total * c / grid);
}

int host_cta_of(int64_t g, int64_t total, int grid) {
  int c = (int)((__int128)g * grid / total);
  while (c + 1 < grid && host_begin(total, c + 1, grid) <= g) ++c;
  while (c > 0 && host_begin(total, c, grid) > g) --c;
  return c;
}

// Fills fl with the split tiles in the same order and with the same slots as
// the device-side search; false when it does not fit.
bool build_fix_list(int grid, int64_t total, int kt, int64_t tiles, FixList& fl) {
  fl.n = 0;
  int ns = 0;
  for (int c = 0; c < grid; ++c) {
    // only tiles that hold a CTA boundary can be split
    const int64_t b = host_begin(total, c, grid);
    if (b % kt == 0) continue;
    const int64_t t = b / kt;
    if (fl.n > 0 && fl.tile[fl.n - 1] == t) continue;
    const int cf = host_cta_of(t * kt, total, grid), cl = host_cta_of((t + 1) * kt - 1, total, grid);
    if (cf == cl) continue;
    if (fl.n >= kFixMaxTiles) return false;
    fl.tile[fl.n] = (int)t;
    fl.off[fl.n] = ns;
    for (int cc = cf; cc <= cl; ++cc) {
      const int64_t bc = host_begin(total, cc, grid);
      if (bc >= host_begin(total, cc + 1, grid)) continue;
      if (ns >= kFixMaxSrc) return false;
      fl.src[ns++] = cc * 2 + ((bc / kt == t) ? 0 : 1);
    }
    ++fl.n;
  }
  fl.off[fl.n] = ns;
  (void)tiles;
  return true;
}

int launch_apass_fixup(const float* part, int grid, int64_t total, int kt, int bmt, int l,
                       int64_t rows_out, int64_t tiles, float* out, int64_t ldo, int accumulate,
                       cudaStream_t st) {
  static thread_local FixList fl;
  if (build_fix_list(grid, total, kt, tiles, fl)) {
    if (fl.n == 0) return RSVD_OK;   // every tile written whole by one CTA
    const dim3 fgrid((unsigned)fl.n, (unsigned)((l + kFixCols - 1) / kFixCols));
    apass_fixup_list_kernel<<<fgrid, 256, 0, st>>>(part, bmt, l, rows_out, out, ldo, accumulate,
                                                   fl);
  } else {
    const dim3 fgrid((unsigned)tiles, (unsigned)((l + kFixCols - 1) / kFixCols));
    apass_fixup_kernel<<<fgrid, 256, 0, st>>>(part, grid, total, kt, bmt, l, rows_out, out, ldo,
                                              accumulate);
  }
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

}  // namespace rsvd
