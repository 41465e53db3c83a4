// Instantiations of the step kernels with the paper-literal options
// (Eq. 35 forward gradient, Eq. 37 extrapolated outlet) compiled in; a
// translation unit of its own so that it builds in parallel with
// lbms_launch.cu, which holds the default instantiations.
#include "lbms_step_launch.cuh"

namespace lbms {

cudaError_t launch_step_variant_literal(const Launch& L, int variant, cudaStream_t st) {
    using launch_detail::step_t;
    LBMS_STEP_DISPATCH(true);
}

}  // namespace lbms
