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
        // P2M, moment shifts and far-field coefficients in one launch
        const int64_t grid = up.p2m_grid > 0 ? std::min<int64_t>(up.n_leaves, up.p2m_grid) : up.n_leaves;
        k_upward<real, P><<<(unsigned)grid, 128, 0, s>>>(up, (const v4*)src, (real*)mom);
        (void)up_levels;
        if constexpr (sizeof(real) == sizeof(float)) {
            // FP32: a block per (node, table), a thread per output
            if (up.n_nodes > 0)
                k_far_f32<P><<<dim3((unsigned)up.n_nodes, 2), far_tr(P), 0, s>>>(up, (const float*)mom);
            return;
        }
        // FP64: a few blocks per SM, each with the packed table in shared
        // memory, taking the nodes in turn
        constexpr size_t smem = far_coef_smem<real, P>();
        static bool attr_set = false;  // per instantiation
        if (!attr_set) {
            PGB_CUDA(cudaFuncSetAttribute(k_far_coef<real, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            attr_set = true;
        }
        int dev = 0, n_sm = 0;
        PGB_CUDA(cudaGetDevice(&dev));
        PGB_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        int64_t gf = std::min<int64_t>(up.n_nodes, 4 * (int64_t)n_sm);
        if (up.p2m_grid > 0) gf = std::min<int64_t>(gf, up.p2m_grid);
        k_far_coef<real, P><<<(unsigned)std::max<int64_t>(gf, 1), 128, smem, s>>>(up, (const real*)mom);
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
