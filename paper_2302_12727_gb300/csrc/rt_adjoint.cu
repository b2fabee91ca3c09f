// Reverse-mode derivative of the sub-cycled transport step (placeholder until the
// adjoint kernels land).
#include "rt_internal.cuh"

namespace rt {
rt_status run_adjoint(rt_ctx* c, int, int, bool, bool, const void*, const void*, void*, double*) {
    return fail(c, RT_ERR_INVALID, "adjoint not available in this build");
}
}  // namespace rt
