// Double-single kernels of the FP64-class product (upward pass, far-field
// coefficients, P2P, M2P): they read the FP64 source terms split into
// double-single once per product and the FP64 target offsets, and compute
// in double-single on the FP32 pipe.
#include <algorithm>

#include "treecode.cuh"

namespace pgb {

template <int P>
static void launch_ds(int stage, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel, void* mom,
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

// FP64 source terms split into double-single once per product, so that the
// P2P tiles stage them without conversion.
__global__ void k_src_to_ds(const dbl4* __restrict__ in, ds4* __restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = cvt4<ds>(in[i]);
}

// src_ds (2 n_src entries of 32 bytes) = the FP64 source terms src64 split
// into double-single.
void convert_src_ds(const void* src64, void* src_ds, int64_t n, cudaStream_t s) {
    if (n > 0) k_src_to_ds<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const dbl4*)src64, (ds4*)src_ds, n);
}

void treecode_launch_ds(int stage, int P, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel,
                        void* mom, const void* far, cudaStream_t s) {
    switch (P) {
        case 0: launch_ds<0>(stage, up, ev, src, xrel, mom, far, s); break;
        case 1: launch_ds<1>(stage, up, ev, src, xrel, mom, far, s); break;
        case 2: launch_ds<2>(stage, up, ev, src, xrel, mom, far, s); break;
        case 3: launch_ds<3>(stage, up, ev, src, xrel, mom, far, s); break;
        case 4: launch_ds<4>(stage, up, ev, src, xrel, mom, far, s); break;
        case 5: launch_ds<5>(stage, up, ev, src, xrel, mom, far, s); break;
        case 6: launch_ds<6>(stage, up, ev, src, xrel, mom, far, s); break;
        case 7: launch_ds<7>(stage, up, ev, src, xrel, mom, far, s); break;
        case 8: launch_ds<8>(stage, up, ev, src, xrel, mom, far, s); break;
        case 10: launch_ds<10>(stage, up, ev, src, xrel, mom, far, s); break;
        case 12: launch_ds<12>(stage, up, ev, src, xrel, mom, far, s); break;
        case 15: launch_ds<15>(stage, up, ev, src, xrel, mom, far, s); break;
        default: fail(PGB_EINVAL, "P out of range");
    }
}

}  // namespace pgb
