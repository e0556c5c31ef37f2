// mixed_grad.cu -- the mixed-precision adjoint gradient (A and E) and its
// launcher; the instantiation with the T channel is in mixed_grad_t.cu.
#include "mixed_grad.cuh"

namespace gb {

int launch_grad_mixed(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                      const double* wE, const double* theta, double* logL, double* grad, const double* dT,
                      const double* wT, cudaStream_t s) {
    if (plan.n_tiles == 0) return GB_OK;
    const bool t3 = dT != nullptr;
    prep_mixed_kernel<<<plan.n_win, 256, 0, s>>>(plan.d_win, plan.d_meta, plan.d_prep, (const double2*)dA,
                                                 (const double2*)dE, wA, wE, (const double2*)dT, wT, plan.n_prep,
                                                 ctx->obs.T_obs, transfer_frequency(ctx), plan.d_head);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "prep_mixed launch");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int n_small = plan.n_tiles - plan.n_large;
    for (int part = 0; part < 2; ++part) {
        const int n_items = part == 0 ? plan.n_large : n_small;
        if (n_items == 0) continue;
        const int nmax = part == 0 ? 1024 : (plan.n_max < 256 ? plan.n_max : 256);
        const size_t smem = (sizeof(CandGx) + sizeof(EpiG)) * kWarpsMx * 32 +
                            sizeof(float2) * kWarpsMx * (t3 ? 3 : 2) * (size_t)nmax;
        const void* kfn = t3 ? grad_mixed_kernel_fn_t(part)
                             : (part == 0 ? (const void*)grad_mixed_kernel<32, false>
                                          : (const void*)grad_mixed_kernel<8, false>);
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(ctx, e, "grad_mixed: smem attribute");
        int grid = sms * resident_blocks(kfn, kWarpsMx * 32, smem);
        const int need = (n_items + kWarpsMx - 1) / kWarpsMx;
        if (grid > need) grid = need;
        const Tile* items = plan.d_tiles + (part == 0 ? 0 : plan.n_large);
        int* head = plan.d_head + (part == 0 ? 1 : 0);
        TabSet32 tabs = tabset32(ctx);
        const float2* tw = (const float2*)ctx->d_tw32;
        double Tobs = ctx->obs.T_obs, fstar = transfer_frequency(ctx);
        int* status = ctx->d_status;
        unsigned long long budget = ctx->budget_ns;
        long long n_prep = plan.n_prep;
        int n_it = n_items, n_mx = nmax;
        void* args[] = {(void*)&plan.d_win, (void*)&plan.d_meta, (void*)&plan.d_prep, (void*)&items, &n_it, &head,
                        &tabs, &tw, &Tobs, &fstar, (void*)&theta, &logL, &grad, &status, &n_mx, &budget, &n_prep};
        e = cudaLaunchKernel(kfn, dim3(grid), dim3(kWarpsMx * 32), args, smem, s);
        ++ctx->launches;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(ctx, e, "grad_mixed launch");
    }
    return GB_OK;
}

}  // namespace gb
