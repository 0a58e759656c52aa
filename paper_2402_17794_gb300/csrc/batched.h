// Grouped (batched) randomized SVD: host interface.
#pragma once

#include "internal.h"

namespace rsvd {

// Workspace carve-up of a batch plan (byte offsets): per-problem slices of
// the n x l, m x l and (m+n) x l pools are laid end to end, then one block of
// l x l matrices and a status word per problem, then the context table.
struct BatchLayout {
  size_t om, z, qb, y, qm, tmp, small, ctx, total;
};

BatchLayout make_batch_layout(int max_count, int64_t rows_total, int64_t cols_total, int l,
                              int dtype);
size_t batch_ctx_bytes(int max_count);
int solve_batched(rsvd_plan_t plan, int count, const rsvd_problem_t* problems);
int batch_status(rsvd_plan_t plan, int count, int* codes);

}  // namespace rsvd
