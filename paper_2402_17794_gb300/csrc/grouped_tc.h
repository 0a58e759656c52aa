// Grouped FP32 products on the tcgen05 tensor cores: many uneven tall-skinny
// GEMMs of a batch (Algorithm 4 applied per problem, Section 3.3) in one
// persistent launch.  Host interface.
#pragma once

#include <vector>

#include "internal.h"

namespace rsvd {

// One product of a grouped launch, FP32 in and out:
//   C (M x N, ldc) = op(A) X,  op(A) = A (M x K, lda) in the AX form or
//   A^T (A stored K x M, lda) in the ATX form;  X K x N (ldx).
// M == 0 marks a product that is skipped (a problem outside this step).
// X enters the MMAs as three BF16 slices (x = x1 + x2 + x3, exact for
// |x| >= 2^-110), written
// by the split kernel to `xs` as the shared-memory images the MMAs read: for
// column tile ct (columns ct t .. ct t + t - 1) and contraction block kb,
// image (ct * kpad / 64 + kb) holds 3t rows of 128 bytes -- row j is slice
// j / t, column ct t + j % t, entries kb 64 .. kb 64 + 63 -- with the 16-byte
// chunk c of row j stored at chunk c ^ (j % 8) (the 128-byte swizzle), zero
// past K and past N.  One bulk copy moves an image into a pipeline stage.
struct GtcGemm {
  const float* A;
  const float* X;
  float* C;
  uint16_t* xs;
  int64_t lda, ldx, ldc;
  int M, K, N;
  int x_upper;    // X is upper triangular: entries below its diagonal read as zero
  int kpad;       // K rounded up to 64
  int ncols;      // N rounded up to the column tile
  int t;          // the product's column tile (gtc_tile)
  int pad_;
};

// Work unit: output rows [row0, row0 + 128) and columns [col0, col0 + t) of
// product `prob`, contraction blocks [kb0, kb1) of 64.  slot < 0: the unit
// owns its whole contraction and writes C; otherwise it writes a 128 x t
// partial to partial slot `slot`, and a fix entry sums the slots of the tile.
// t (the product's column tile) depends only on the product's N.
struct GtcUnit {
  int prob, row0, col0, kb0, kb1, slot, t, pad_;
};
struct GtcFix {
  int prob, row0, col0, slot0, nslot, t;
};

constexpr int kGtcMaxTile = 80;   // column tile limit: three slices side by side in one MMA (N <= 256)
constexpr int kGtcBlockK = 64;    // contraction per stage

// Host-side schedule of one grouped launch: units in CTA order, CTA c takes
// units [cta_off[c], cta_off[c + 1]).  Units are dealt longest first to the
// least loaded CTA (LPT), so a launch's time follows the total work, not the
// largest problem.  A product whose contraction exceeds `chunk_kb` blocks is
// split into chunks of at most that many blocks (partial slots + fix
// entries); the split depends only on the product's own K, so a product's
// result is the same in any batch.
struct GtcSchedule {
  std::vector<GtcUnit> units;
  std::vector<int> cta_off;
  std::vector<GtcFix> fix;
  int grid = 0;
  int slots = 0;
  int tmax = 16;   // largest column tile (sets the stage and accumulator sizes)
};
struct GtcShape {
  int M, K, N;
};
// Buckets of the tuning table: K or N in (64 * 2^(b-1), 64 * 2^b].
__host__ __device__ inline int gtc_bucket(int v) {
  int b = 0;
  while (b < 31 && (64 << b) < v) ++b;
  return b;
}
// Column tile of a product with N columns under tile limit cap (0: 80): N
// split into ceil(N / cap) tiles of equal width rounded up to 16.
__host__ __device__ inline int gtc_tile_rule(int N, int cap) {
  if (cap <= 0) cap = kGtcMaxTile;
  const int tiles = (N + cap - 1) / cap;
  const int w = (N + tiles - 1) / tiles;
  return (w + 15) / 16 * 16;
}
struct GtcCaps {
  int cap[32];   // tile limit per N bucket (0: default)
};
void gtc_caps(GtcCaps& c);   // the process-wide tuned limits

// force_chunk > 0 splits every product into chunks of that many blocks (the
// tuner's candidates); otherwise each product's chunk comes from
// gtc_chunk(ax, K).  caps: tile limits to use instead of the tuned ones.
void gtc_schedule(const GtcShape* shapes, int count, bool ax, int num_sms, GtcSchedule& out,
                  int force_chunk = 0, const GtcCaps* caps = nullptr);

// Device pointers of one launch (schedule already on the device).
struct GtcLaunch {
  bool ax;
  const GtcGemm* gemm;
  int count;
  int tmax;              // the schedule's largest column tile
  const GtcUnit* units;
  const int* cta_off;
  int grid;
  const GtcFix* fix;
  int nfix;
  float* part;           // slots * 128 * tmax floats
  int* status;           // RSVD_ERR_TIMEOUT bit on an expired wait
  long long wait_cycles;
};

// Enqueues the grouped pass (and the fix-up of split tiles).  The X slices
// must be current (gtc_split).  Returns RSVD_OK or RSVD_ERR_*.
int launch_gtc(const GtcLaunch& L, cudaStream_t st);

// Writes the BF16 slices of every product's X (table already on the device).
int launch_gtc_split(const GtcGemm* gemm, int count, int max_kpad, int max_ncols,
                     cudaStream_t st);

// Stages of a pass whose largest column tile is t.
int gtc_stages(int t);

// A product's column tile: N split into ceil(N / cap) tiles of equal width
// rounded up to 16, cap = the tuned tile limit for N's bucket (default 80).
int gtc_tile(int N);
// Contraction blocks per unit for a product of this form, K and M: the tuned
// value for (form, K's bucket, M <= 128 or not), else kGtcDefaultChunk.
int gtc_chunk(bool ax, int K, int M);
// Process-wide tuning table: the first value set for a bucket stays, so a
// product's schedule (and its result) is the same in every batch of the
// process.
bool gtc_chunk_tuned(bool ax, int K, int M);
void gtc_set_chunk(bool ax, int K, int M, int chunk_kb);
bool gtc_tile_tuned(int N);
void gtc_set_tile_cap(int N, int cap);
int gtc_generation();   // counts the changes of the table (schedules built before are stale)
constexpr int kGtcDefaultChunk = 64;

}  // namespace rsvd
