// Mixed-precision dynamical-core step (FP32 horizontal stencils, FP64 column).
#include "icon_internal.h"

namespace icon {
void enqueue_step_mixed(icon_state*, double, int, cudaStream_t) {}
}  // namespace icon
