// Semi-implicit step (placeholder until the scheme's kernels land).
#include "glasma_internal.cuh"

namespace glasma {

int launch_step_implicit(glasma_ctx* c, bool hop, int* iters) {
  (void)c;
  (void)hop;
  *iters = 0;
  return set_error(GLASMA_ERR_INVALID_ARG, "implicit scheme not available in this build");
}

}  // namespace glasma
