// mixed_grad_t.cu -- the mixed-precision adjoint gradient kernel with the T
// channel, compiled apart so that the instantiations build in parallel.
#include "mixed_grad.cuh"

namespace gb {

const void* grad_mixed_kernel_fn_t(int part) {
    return part == 0 ? (const void*)grad_mixed_kernel<32, true> : (const void*)grad_mixed_kernel<8, true>;
}

}  // namespace gb
