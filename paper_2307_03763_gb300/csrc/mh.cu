// mh.cu -- independence Metropolis-Hastings chains from precomputed values
// (Sec. III.G, Alg. 4, Eq. 13).
//
// The proposal does not depend on the chain state, so all log-likelihoods are
// computed first and each chain is one scan over its proposals.  The scan is
// sequential only through the current state c: while c stays the same, the
// acceptance tests of the following proposals are independent of each other.
// One warp per chain therefore tests the next 32 proposals against the same c
// in parallel, finds the first acceptance with a ballot, records the
// rejections before it, moves c there and continues after it.  Every test is
// the same IEEE expression as in a one-at-a-time scan, so the chain is
// identical to the sequential one bit for bit.
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

__device__ __forceinline__ bool accept_test(double li, double gi, double ui, double lc, double gc, double T,
                                            int literal) {
    const double dl = __dadd_rn(li, -lc);
    const double dg = __dadd_rn(gc, -gi);
    double delta;
    if (T == 1.0)   // x / 1 == x exactly: skip the division
        delta = __dadd_rn(dl, dg);
    else
        delta = literal ? __ddiv_rn(__dadd_rn(dl, dg), T) : __dadd_rn(__ddiv_rn(dl, T), dg);
    return !isnan(delta) && (ui < fmin(0.0, delta));
}

__global__ void mh_kernel(int n_chains, int n, const double* __restrict__ logL,
                          const double* __restrict__ log_g, const double* __restrict__ log_u,
                          const double* __restrict__ temperature, int literal,
                          int32_t* __restrict__ chain, int32_t* __restrict__ n_accept) {
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n_chains) return;   // uniform per warp
    const size_t base = (size_t)r * (size_t)n;
    const double* L = logL + base;
    const double* G = log_g + base;
    const double* U = log_u + base;
    int32_t* out = chain + base;
    const double T = temperature[r];
    int c = 0;
    double lc = L[0], gc = G[0];
    int acc = 0;
    if (lane == 0) out[0] = 0;
    int p = 1;
    while (p < n) {
        const int i = p + lane;
        double li = 0.0, gi = 0.0;
        bool ok = false;
        if (i < n) {
            li = L[i];
            gi = G[i];
            ok = accept_test(li, gi, U[i], lc, gc, T, literal);
        }
        const unsigned ball = __ballot_sync(0xffffffffu, ok);
        const int first = ball ? __ffs(ball) - 1 : 32;
        if (lane < first && i < n) out[i] = c;
        if (first < 32) {
            const int inew = p + first;
            if (lane == first) out[inew] = inew;
            lc = __shfl_sync(0xffffffffu, li, first);
            gc = __shfl_sync(0xffffffffu, gi, first);
            c = inew;
            ++acc;
            p = inew + 1;
        } else {
            p += 32;
        }
    }
    if (n_accept && lane == 0) n_accept[r] = acc;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int gb_mh_independence(gb_ctx_t* ctx, int32_t n_chains, int32_t n, const double* logL,
                                  const double* log_g, const double* log_u, const double* temperature,
                                  int32_t literal, int32_t* chain_idx, int32_t* n_accept, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_chains < 0 || n < 0) return set_error(ctx, GB_EINVAL, "gb_mh_independence: negative size");
    if (n_chains == 0 || n == 0) return GB_OK;
    if (!logL || !log_g || !log_u || !temperature || !chain_idx)
        return set_error(ctx, GB_EINVAL, "gb_mh_independence: null pointer");
    if (literal != 0 && literal != 1) return set_error(ctx, GB_EINVAL, "gb_mh_independence: literal must be 0 or 1");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_independence: cudaSetDevice");
    const int threads = 128;   // four chains per block, one warp each
    const int blocks = (int)(((int64_t)n_chains * 32 + threads - 1) / threads);
    mh_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(
        n_chains, n, logL, log_g, log_u, temperature, literal, chain_idx, n_accept);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_independence launch");
    return GB_OK;
}
