// stencil_heat3.cu -- instantiations of the fused and plain propagator
// kernels for one right-hand side (kept apart so the builds run in parallel).
#include "stencil_impl.cuh"

namespace rnp {
RNP_STENCIL_DEFINE(KP_HEAT3, heat3)
}  // namespace rnp
