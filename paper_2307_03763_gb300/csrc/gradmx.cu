// gradmx.cu -- gradient of the window log-likelihood, mixed precision.
#include "gb_internal.cuh"

namespace gb {

int launch_grad_mixed(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                      const double* wE, const double* theta, double* logL, double* grad, cudaStream_t s) {
    (void)plan; (void)dA; (void)dE; (void)wA; (void)wE; (void)theta; (void)logL; (void)grad; (void)s;
    return set_error(ctx, GB_EINVAL, "gb_loglik_grad: GB_MIXED is not available in this build");
}

}  // namespace gb
