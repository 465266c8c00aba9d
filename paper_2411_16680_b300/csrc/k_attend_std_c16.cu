// Standard multi-head cross attention (both forms, SIMT) for C = 16: the instantiations of
// k_attend_impl.cuh.
#include "k_attend_impl.cuh"

namespace quark {

cudaError_t attend_std_c16(const AttendArgs& a, int heads, Transition tr, bool last, bool bf16, cudaStream_t st) {
    return bf16 ? launch_std_c<__nv_bfloat16, 16>(a, heads, tr, last, st) : launch_std_c<float, 16>(a, heads, tr, last, st);
}

}  // namespace quark
