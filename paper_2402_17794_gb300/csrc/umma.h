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

// The split tiles of a stream-K pass and their partial slots, listed on the
// host (a kernel parameter): grid CTAs share `total` (tile, k-block)
// iterations with kt k-blocks per tile; CTA c takes [total c / grid,
// total (c+1) / grid) and writes the partials of its first and last (split)
// tiles to slots 2c and 2c+1.
constexpr int kFixMaxTiles = 192;
constexpr int kFixMaxSrc = 512;
struct FixList {
  int n;                          // split tiles
  int tile[kFixMaxTiles];
  int off[kFixMaxTiles + 1];      // sources of tile i: src[off[i] .. off[i+1])
  int src[kFixMaxSrc];            // partial slot (CTA * 2 + 0 first / 1 last tile)
};
int64_t host_begin(int64_t total, int c, int grid);
int host_cta_of(int64_t g, int64_t total, int grid);
// false when the list does not fit FixList.
bool build_fix_list(int grid, int64_t total, int kt, int64_t tiles, FixList& fl);

// FP64-accurate passes over A on the tensor cores (exact products of BF16
// digit slices).  Preparation of A, once per A: its row exponents and six
// digit slices (slices: 6 x ncol columns of ldsl rows, ncol = n rounded up to
// 128; rmax: m ints).
int f64tc_prepare_a(const double* A, int64_t m, int64_t n, int64_t lda, void* slices,
                    int64_t ldsl, int64_t ncol, int* rmax, int* status, int num_sms,
                    cudaStream_t st);
struct F64tcCall {
  bool ax;                 // true: out = A X (X n x l); false: out = A^T X (X m x l)
  const void* slices;      // from f64tc_prepare_a
  int64_t m, n, ldsl, ncol;
  const int* rmax;
  const double* X;
  int64_t ldx;
  int l;                   // output columns (any; blocks of <= 80 per pass)
  double* out;
  int64_t ldo;
  // workspace
  void* xslices;           // 6 * 80 rows of ldxs BF16 (ldxs >= rows of X, multiple of 8)
  int64_t ldxs;
  int* fexp;               // 80 ints
  int64_t* raw_t;          // (m or n) x 80 int64
  float* raw_r;            // (m or n) x 80 float
  int64_t* part_t;         // partial slots: num_sms * 2 * 128 * 80
  float* part_r;
  long long wait_cycles = 0;
};
constexpr int kF64tcMaxL = 80;   // output columns per pass (six TMEM regions of <= 80)
int launch_apass_f64tc(const F64tcCall& c, int num_sms, int* status, cudaStream_t st);

// FP8 passes with block-scaled MMA (kind::mxf8f6f4).  The operand: the FP32
// X (rows x l <= 256, ld ldx) split by launch_split_e4m3 into `slices` E4M3
// slices of its column-normalised values (slice j column c at
// out[(j * l16 + c) * ldo + r], l16 = l rounded up to 16, ldo >= rows,
// ldo % 16 == 0), one exponent per 64-row chunk (mx8_xexp_count(rows) ints)
// and the power-of-two column scales (l16 floats) the pass multiplies its
// output columns by; colbits: l unsigned of scratch.
// The chunk (64 or 128 rows, the stage depth the pass will use) comes from
// mx8_chunk_rows; 0 means the shape is not supported.
int64_t mx8_xexp_count(int64_t rows);   // chunk exponents for 64-row chunks (an upper bound)
int mx8_chunk_rows(bool ax, int64_t m, int64_t n, int l, int slices);
int launch_split_e4m3(const float* X, int64_t rows, int l, int64_t ldx, int slices, int chunk,
                      uint8_t* out, int64_t ldo, int* xexp, float* colscale, unsigned* colbits,
                      cudaStream_t st);
struct Mx8Call {
  bool ax;                 // true: Y = A X (contracts n); false: Z = A^T X (contracts m)
  const void* A;           // E4M3 m x n, column-major, lda % 16 == 0, 16-byte aligned
  int64_t m, n, lda;
  const float* scales;     // power-of-two scale of each 128 x 128 tile, (I, J) at I + J * lds
  int64_t lds;
  const void* X;           // E4M3 slices from launch_split_e4m3 (n rows for ax, m otherwise)
  int64_t ldx;
  const int* xexp;
  const float* colscale;
  int chunk;               // rows per exponent: mx8_chunk_rows of this call
  int slices;              // 2, 4 or 6
  int l;                   // output columns (<= 256)
  float* out;              // FP32 (m or n) x l, column-major
  int64_t ldo;
  float* part;             // partial slots, as for the BF16 passes
  size_t part_floats;
  bool accumulate = false;
  long long wait_cycles = 0;
};
int launch_apass_mx8(const Mx8Call& c, int num_sms, int* status, cudaStream_t st);

}  // namespace rsvd
