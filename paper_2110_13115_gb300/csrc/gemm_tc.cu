// First-stage reconstruction on tcgen05 tensor cores (placeholder until the kernel lands).
#include "common.cuh"
#include "internal.h"

namespace rb {
int stage1_tc(const rb_filter_desc&, const rb_basis&, const Geometry&, const Workspace&, rb_candidate*,
              cudaStream_t) {
  set_detail("tensor-core first stage not built");
  return RB_ERR_UNSUPPORTED;
}
}  // namespace rb
