// Explicit instantiation and dispatch of the treecode kernels for one
// arithmetic type (included by treecode_f32.cu / treecode_f64.cu).
#include <algorithm>

#include "treecode.cuh"

namespace pgb {

template <typename real, int P>
static void launch_p(int stage, const UpArgs& up, const std::vector<int64_t>& up_levels, const EvalArgs& ev,
                     const void* src, const void* xrel, void* mom, void* far, cudaStream_t s) {
    using v4 = typename V4<real>::t;
    (void)up_levels;
    if (stage == PGB_STAGE_UPWARD) launch_upward<real, P>(up, src, mom, s);
    // M2P: 8 warps per block in FP32, 4 in FP64 (its registers would
    // otherwise fill an SM), fewer at the highest orders (shared memory)
    constexpr int NW = m2p_warps<real, P>();
    const bool persist = ev.p2p_work != nullptr;
    // P2P: 8 warps per block in both precisions (with 4, a persistent FP64
    // block per SM could not keep the FP64 pipe busy)
    constexpr int NWP = 8;
    if (stage == PGB_STAGE_P2P && ev.n_pitems > 0)
        k_p2p<real, NWP><<<(unsigned)(persist ? ev.persist_blocks : ev.n_pitems), NWP * 32, 0, s>>>(
            ev, (const v4*)src, (const v4*)xrel);
    if (stage == PGB_STAGE_M2P && ev.n_fitems > 0)
        k_m2p<real, P, NW><<<(unsigned)(persist ? ev.persist_blocks : ev.n_fitems), NW * 32, 0, s>>>(
            ev, (const v4*)xrel, (const real*)far);
}

}  // namespace pgb
