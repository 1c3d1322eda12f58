// One-pass qdot with deferred selection (placeholder until the kernel lands).
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
bool one_pass_supported(int64_t, const qdot_params*, bool) { return false; }
OnePassPlan plan_one_pass(int64_t, const qdot_params*) { return OnePassPlan(); }
cudaError_t launch_one_pass(const double*, const double*, int64_t, const qdot_params*, const OnePassPlan&, void*,
                            qdot_result*, qdot_selection*, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace qd
