// Explicit instantiation and dispatch of the treecode kernels for one
// arithmetic type (included by treecode_f32.cu / treecode_f64.cu).
#include "treecode.cuh"

namespace pgb {

template <typename real, int P>
static void launch_p(int stage, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel, void* mom,
                     cudaStream_t s) {
    using v4 = typename V4<real>::t;
    if (stage == PGB_STAGE_UPWARD && up.n_leaves > 0)
        k_upward<real, P><<<(unsigned)up.n_leaves, 128, 0, s>>>(up, (const v4*)src, (real*)mom);
    if (stage == PGB_STAGE_EVAL && ev.n_groups > 0)
        k_eval<real, P><<<(unsigned)((ev.n_groups + 3) / 4), 128, 0, s>>>(ev, (const v4*)src, (const v4*)xrel,
                                                                         (const real*)mom);
}

}  // namespace pgb
