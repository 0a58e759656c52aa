// Mixed-precision path: not built yet in this library version.
#include "mixed.h"

namespace rsvd {

MixedLayout mixed_layout(int64_t, int64_t, int) { return MixedLayout{0}; }

int solve_mixed(rsvd_plan_t, const MixedArgs&) { return RSVD_ERR_UNSUPPORTED; }

int mixed_apply(rsvd_plan_t, const void*, int64_t, int64_t, int64_t, const void*, int64_t, int,
                void*, int64_t, bool) {
  return RSVD_ERR_UNSUPPORTED;
}

}  // namespace rsvd
