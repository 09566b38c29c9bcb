// stencil_swe_wall.cu -- the shallow-water instantiations of the mixed
// kernel with reflecting walls (kept apart so the builds run in parallel).
#include "stencil_impl.cuh"

namespace rnp {
RNP_STENCIL_DEFINE_WALL(KP_SWE, swe)
}  // namespace rnp
