// tcgen05 BF16 passes over A (mixed path): host interface.
#pragma once

#include "internal.h"

namespace rsvd {

struct ApassCall {
  bool ax;              // true: Y = A X (contracts n); false: Z = A^T X (contracts m)
  const void* A;        // BF16 (or FP8, see fp8) m x n, column-major, lda % 8 == 0,
                        // 16-byte aligned
  int64_t m, n, lda;
  const void* X;        // BF16 operand: (n for ax, m otherwise) x x_cols, ldx % 8 == 0
  int64_t ldx;
  int x_cols;           // columns present in X (the rest of the last part reads as zero)
  int l;                // output columns
  int slices;           // operand slices summed into the output (1..3)
  int slice_stride;     // column offset between slices (>= l rounded up to 16)
  float* out;           // FP32 (m or n) x l, column-major
  int64_t ldo;
  float* part;          // partial slots
  size_t part_floats;
  bool accumulate = false;  // out += A X instead of out = A X
  // FP8 A: E4M3 codes (lda % 16 == 0) with FP32 power-of-two scales, one per
  // 128 x 128 tile, tile (I, J) at scales[I + J * lds]
  bool fp8 = false;
  const float* scales = nullptr;
  int64_t lds = 0;
  long long wait_cycles = 0;  // bound of each pipeline wait in clock64 cycles; 0: ~1 s
};

// Floats of partial-slot workspace a pass with `l` output columns needs.
size_t apass_partial_floats(int num_sms, int l);

// Enqueues the pass (main kernel + split-tile fixup).  Returns RSVD_OK or a
// positive RSVD_ERR_* code (unsupported alignment/shape -- including operand
// slices too wide for two shared-memory stages --, workspace, CUDA).
int launch_apass_bf16(const ApassCall& c, int num_sms, int* status, cudaStream_t st);

// Fixup of a stream-K pass: `grid` CTAs shared `total` (tile, k-block)
// iterations, `kt` k-blocks per tile of `bmt` rows; CTA c wrote the partials of
// its first and last (split) tiles to part slots 2c and 2c+1 (bmt x l floats
// each, column-major).  Writes (or adds to, `accumulate`) out for those tiles.
constexpr int kFixCols = 8;   // output columns per fixup block
int launch_apass_fixup(const float* part, int grid, int64_t total, int kt, int bmt, int l,
                       int64_t rows_out, int64_t tiles, float* out, int64_t ldo, int accumulate,
                       cudaStream_t st);

}  // namespace rsvd
