// Explicit instantiation and dispatch of the treecode kernels for one
// arithmetic type (included by treecode_f32.cu / treecode_f64.cu).
#include <algorithm>

#include "treecode.cuh"

namespace pgb {

template <typename real, int P>
static void launch_p(int stage, const UpArgs& up, const std::vector<int64_t>& up_levels, const EvalArgs& ev,
                     const void* src, const void* xrel, void* mom, void* far, cudaStream_t s) {
    using v4 = typename V4<real>::t;
    if (stage == PGB_STAGE_UPWARD && up.n_leaves > 0) {
        const int64_t grid = up.p2m_grid > 0 ? std::min<int64_t>(up.n_leaves, up.p2m_grid) : up.n_leaves;
        k_p2m_leaves<real, P><<<(unsigned)grid, 128, 0, s>>>(up, (const v4*)src, (real*)mom);
        // inner nodes level by level, deepest first
        for (int l = (int)up_levels.size() - 3; l >= 0; --l) {  // the deepest level holds only leaves
            UpArgs u = up;
            u.lvl_begin = up_levels[l];
            u.lvl_end = up_levels[l + 1];
            if (u.lvl_end > u.lvl_begin)
                k_m2m_level<real, P><<<(unsigned)(u.lvl_end - u.lvl_begin), 256, 0, s>>>(u, (real*)mom);
        }
        // moments -> far-field coefficients of every node
        if (up.n_nodes > 0) {
            const int64_t g = up.p2m_grid > 0 ? std::min<int64_t>(up.n_nodes, up.p2m_grid) : up.n_nodes;
            k_far_coef<real, P><<<(unsigned)g, 128, 0, s>>>(up, (const real*)mom);
        }
    }
    // FP64 M2P: 4 warps per block (its registers would otherwise fill an SM)
    constexpr int NW = sizeof(real) == 8 ? 4 : 8;
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
