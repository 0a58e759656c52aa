// Grouped (batched) randomized SVD: host interface.
#pragma once

#include "internal.h"

namespace rsvd {

// Workspace carve-up of a batch plan (byte offsets): per-problem slices of
// the n x l, m x l and (m+n) x l pools are laid end to end, then one block of
// l x l matrices and a status word per problem, then the context table.
struct BatchLayout {
  size_t om, z, qb, y, qm, tmp, small, ctx, total;
  // tensor engine (FP32 plans): the product table of a grouped step, the BF16
  // slices of each problem's operand X, the work schedules of the ten product
  // shapes of a solve, partial slots of split tiles and a timeout word
  size_t gtab, xs, sched, part, gflags;
  size_t sched_bytes, part_floats;
  int xs_ncols;   // column capacity of a problem's slice slab
};

// rsvd_batch_set_engine values
constexpr int kBatchSimt = 0;
constexpr int kBatchTensor = 1;

BatchLayout make_batch_layout(int max_count, int64_t rows_total, int64_t cols_total, int l,
                              int dtype);
size_t batch_ctx_bytes(int max_count);
int solve_batched(rsvd_plan_t plan, int count, const rsvd_problem_t* problems);
int batch_status(rsvd_plan_t plan, int count, int* codes);
// Times the split-K chunk (and, for N > 80, the column tile limit) candidates
// of the tensor engine on this batch's products and records the fastest per
// shape bucket in the process-wide table.
int batch_autotune(rsvd_plan_t plan, int count, const rsvd_problem_t* problems);
void batch_tc_free(rsvd_plan_t plan);
// rsvd_grouped_gemm_f32 (arguments already checked)
int grouped_gemm_f32(rsvd_plan_t plan, int count, const rsvd_gemm_t* gemms, int trans);

}  // namespace rsvd
