// One-to-many attention (FP32 form, SIMT) for C = 64: the instantiations of k_attend_impl.cuh.
#include "k_attend_impl.cuh"

namespace quark {

cudaError_t attend_fp32_c64(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st) {
    return launch_c<float, 64>(a, heads, tr, last, st);
}

}  // namespace quark
