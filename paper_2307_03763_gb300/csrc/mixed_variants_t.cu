// mixed_variants_t.cu -- the persistent likelihood kernel with the T channel,
// with and without the phase output.
#include "mixed_common.cuh"

namespace gb {

const void* mixed_kernel_fn_t(int part, bool im) {
    if (im) return part == 0 ? (const void*)loglik_mixed_kernel<32, true, true> : (const void*)loglik_mixed_kernel<8, true, true>;
    return part == 0 ? (const void*)loglik_mixed_kernel<32, false, true> : (const void*)loglik_mixed_kernel<8, false, true>;
}

}  // namespace gb
