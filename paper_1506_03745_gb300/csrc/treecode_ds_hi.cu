// Double-single kernels of the orders above 8 (see treecode_ds.cu).
#include "treecode_ds_inst.cuh"

namespace pgb {

void treecode_launch_ds_hi(int stage, int P, const UpArgs& up, const EvalArgs& ev, const void* src, const void* xrel,
                           void* mom, const void* far, cudaStream_t s) {
    switch (P) {
        case 10: launch_ds<10>(stage, up, ev, src, xrel, mom, far, s); break;
        case 12: launch_ds<12>(stage, up, ev, src, xrel, mom, far, s); break;
        case 15: launch_ds<15>(stage, up, ev, src, xrel, mom, far, s); break;
        default: fail(PGB_EINVAL, "P out of range");
    }
}

}  // namespace pgb
