// Double-single kernels of the FP64-class product (upward pass, far-field
// coefficients, P2P, M2P): they read the FP64 source terms split into
// double-single once per product and the FP64 target offsets, and compute
// in double-single on the FP32 pipe.
#include "treecode_ds_inst.cuh"

namespace pgb {

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

void treecode_launch_ds_hi(int stage, int P, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel,
                           void* mom, const void* far, cudaStream_t s);

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
        case 10:
        case 12:
        case 15: treecode_launch_ds_hi(stage, P, up, ev, src, xrel, mom, far, s); break;
        default: fail(PGB_EINVAL, "P out of range");
    }
}

}  // namespace pgb
