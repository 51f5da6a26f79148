// Launches of the double-single kernels for one order P (included by
// treecode_ds.cu for P 0..8 and treecode_ds_hi.cu for P 10, 12, 15, so that
// the two halves compile in parallel).
#pragma once
#include <algorithm>

#include "treecode.cuh"

namespace pgb {

template <int P>
inline void launch_ds(int stage, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel, void* mom,
                      const void* far, cudaStream_t s) {
    constexpr int NW = m2p_warps<ds, P>();  // M2P warps per block (registers, as the FP64 kernel)
    constexpr int NWP = 8;                   // P2P warps per block
    const bool persist = ev.p2p_work != nullptr;
    // P2M and the moment shifts, then the far-field coefficients, all in
    // double-single on the FP32 pipe
    if (stage == PGB_STAGE_UPWARD) launch_upward<ds, P>(up, src, mom, s);
    if (stage == PGB_STAGE_P2P && ev.n_pitems > 0)
        k_p2p<ds, NWP><<<(unsigned)(persist ? ev.persist_blocks : ev.n_pitems), NWP * 32, 0, s>>>(
            ev, (const ds4*)src, (const dbl4*)xrel);
    if (stage == PGB_STAGE_M2P && ev.n_fitems > 0)
        k_m2p<ds, P, NW><<<(unsigned)(persist ? ev.persist_blocks : ev.n_fitems), NW * 32, 0, s>>>(
            ev, (const dbl4*)xrel, (const ds*)far);
}

}  // namespace pgb
