// stencil_wide.cu -- instantiations of the wide mixed-precision stencil
// kernel (128 to 800 threads per CTA at 72 registers, state in tensor
// memory) for the reaction-diffusion operators, kept apart so the build runs
// in parallel with the other operators.
#include "stencil_impl.cuh"

namespace rnp {

FusedFn mixed_wide_fn(int kp, int PX, int RS, bool XS, bool WALL, bool RK, bool iso) {
  if (XS || WALL || !iso) return nullptr;
  switch (kp) {
    case KP_DIFFREACT: return RK ? mixed_wide_for<KP_DIFFREACT, true>(PX, RS)
                                 : mixed_wide_for<KP_DIFFREACT, false>(PX, RS);
    case KP_BRUSS2: return RK ? mixed_wide_for<KP_BRUSS2, true>(PX, RS)
                              : mixed_wide_for<KP_BRUSS2, false>(PX, RS);
    case KP_BRUSS3: return RK ? mixed_wide_for<KP_BRUSS3, true>(PX, RS)
                              : mixed_wide_for<KP_BRUSS3, false>(PX, RS);
  }
  return nullptr;
}

}  // namespace rnp
