// Mixed-precision path (BF16 A on tcgen05 tensor cores): internal interface.
#pragma once

#include "internal.h"

namespace rsvd {

struct MixedLayout {
  size_t bytes;
};

struct MixedArgs {
  const void* A;
  int64_t m, n, lda;
  int k, p, q;
  uint64_t seed;
  void* U;
  int64_t ldu;
  double* S;
  void* VT;
  int64_t ldvt;
};

MixedLayout mixed_layout(int64_t m, int64_t n, int l);
int solve_mixed(rsvd_plan_t plan, const MixedArgs& a);
int mixed_apply(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, const void* X,
                int64_t ldx, int l, void* Y, int64_t ldy, bool trans);

}  // namespace rsvd
