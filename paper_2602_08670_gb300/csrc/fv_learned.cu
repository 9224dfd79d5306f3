// fv_learned.cu — learned-stencil step (placeholder until the CNN kernels land).
#include "fv_internal.h"

namespace fvs {
cudaError_t enqueue_learned_step(fv_state*, const fv_net*) { return cudaErrorNotSupported; }
void learned_workspace_free(fv_state*) {}
}  // namespace fvs
