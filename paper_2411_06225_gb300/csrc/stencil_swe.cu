// stencil_swe.cu -- instantiations of the fused and plain propagator
// kernels for one right-hand side (kept apart so the builds run in parallel).
#include "stencil_impl.cuh"

namespace rnp {
RNP_STENCIL_DEFINE_SPLIT(KP_SWE, swe)
}  // namespace rnp
