// mixed_variants.cu -- the persistent likelihood kernel with the phase output
// (dh_im); the instantiations with the T channel are in mixed_variants_t.cu.
// Compiled apart from the plain kernel so that the instantiations build in
// parallel.
#include "mixed_common.cuh"

namespace gb {

const void* mixed_kernel_fn_variant(int part, bool im, bool t3) {
    if (t3) return mixed_kernel_fn_t(part, im);
    return part == 0 ? (const void*)loglik_mixed_kernel<32, true, false> : (const void*)loglik_mixed_kernel<8, true, false>;
}

}  // namespace gb
