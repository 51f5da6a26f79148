// FP32 treecode kernels (P2M/M2M upward pass, fused P2P + M2P evaluation).
#include "treecode_inst.cuh"

namespace pgb {
void treecode_launch_f32(int stage, int P, const UpArgs& up, const std::vector<int64_t>& lv, const EvalArgs& ev,
                         const void* src, const void* xrel, void* mom, void* far, cudaStream_t s) {
    switch (P) {
        case 0: launch_p<float, 0>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 1: launch_p<float, 1>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 2: launch_p<float, 2>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 3: launch_p<float, 3>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 4: launch_p<float, 4>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 5: launch_p<float, 5>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 6: launch_p<float, 6>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 7: launch_p<float, 7>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 8: launch_p<float, 8>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 10: launch_p<float, 10>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 12: launch_p<float, 12>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        case 15: launch_p<float, 15>(stage, up, lv, ev, src, xrel, mom, far, s); break;
        default: fail(PGB_EINVAL, "P out of range");
    }
}
}  // namespace pgb
