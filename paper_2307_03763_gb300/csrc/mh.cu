// mh.cu -- independence Metropolis-Hastings chains from precomputed values
// (Sec. III.G, Alg. 4, Eq. 13).
//
// The proposal does not depend on the chain state, so all log-likelihoods are
// computed first and each chain is one scan over its proposals.  One CTA runs
// one chain: all its threads turn a chunk of proposals into weights
//   w_i = logL_i/T - log g_i   (default reading),  v_i = logL_i - log g_i (literal)
// in shared memory, then one warp scans the chunk.  The scan is sequential
// only through the current state c: while c stays the same, the acceptance
// tests of the following proposals are independent, so the warp tests 32 at a
// time against c, finds the first acceptance with a ballot, records the
// rejections before it and moves c there.
//
// Each test is decided first in float with a rigorous error margin and falls
// back to the IEEE double expression only when the margin cannot decide: on
// GB300 a double instruction occupies the FP64 pipe of a sub-partition for
// tens of cycles, and a scan is a chain of dependent tests.  The decision is
// always the one the double expression takes, so the chains are identical bit
// for bit to a one-at-a-time double-precision scan.
#include <cfloat>
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kMhThreads = 256;
constexpr int kMhChunk = 8192;   // proposals staged in shared memory at a time

// one weight per proposal; x / 1 == x exactly, so T = 1 skips the division
__device__ __forceinline__ double weight(double l, double g, double T, int literal) {
    return (literal || T == 1.0) ? __dadd_rn(l, -g) : __dadd_rn(__ddiv_rn(l, T), -g);
}

// Eq. 13 in double: Delta = w_i - w_c (default) or (v_i - v_c)/T (literal);
// accept iff log u < min(0, Delta); a NaN Delta rejects.
__device__ __forceinline__ bool accept_exact(double wi, double ui, double wc, double T, int literal) {
    double delta = __dadd_rn(wi, -wc);
    if (literal && T != 1.0) delta = __ddiv_rn(delta, T);
    return !isnan(delta) && (ui < fmin(0.0, delta));
}

// The same decision from float copies W = fl(w), U = fl(u) when Delta = w_i - w_c:
// 1 accept, 0 reject, -1 undecided.  With rounding to nearest,
//   |fl(W_i - W_c) - fl64(w_i - w_c)| < 2^-23 (|W_i| + |W_c| + |D|) and
//   |U - u| < 2^-23 |U|,
// so a gap between U and D above M = 2^-22 (|W_i| + |W_c| + |D| + |U|) decides
// u < Delta exactly; U < 0 implies u < 0.  Non-finite values are undecided.
__device__ __forceinline__ int accept_fast(float Wi, float Ui, float Wc) {
    if (!(fabsf(Wi) <= FLT_MAX) || !(fabsf(Wc) <= FLT_MAX) || !(Ui < 0.0f)) return -1;
    const float D = Wi - Wc;
    if (!(fabsf(D) <= FLT_MAX)) return -1;
    const float M = 2.384185791015625e-07f * (fabsf(Wi) + fabsf(Wc) + fabsf(D) + fabsf(Ui)) + 1e-37f;
    if (Ui - D > M) return 0;
    if (D - Ui > M) return 1;
    return -1;
}

__global__ void __launch_bounds__(kMhThreads) mh_kernel(int n, int chunk, const double* __restrict__ logL,
                                                        const double* __restrict__ log_g,
                                                        const double* __restrict__ log_u,
                                                        const double* __restrict__ temperature, int literal,
                                                        int32_t* __restrict__ chain, int32_t* __restrict__ n_accept) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* ws = (double*)smem_raw;   // chunk
    float* Wf = (float*)(ws + chunk); // chunk
    float* Uf = Wf + chunk;           // chunk
    const int r = blockIdx.x;
    const size_t base = (size_t)r * (size_t)n;
    const double* L = logL + base;
    const double* G = log_g + base;
    const double* U = log_u + base;
    int32_t* out = chain + base;
    const double T = temperature[r];
    const bool fast = !literal || T == 1.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int c = 0;
    double wc = weight(L[0], G[0], T, literal);
    float Wc = (float)wc;
    int acc = 0;
    if (threadIdx.x == 0) out[0] = 0;
    for (int p0 = 1; p0 < n; p0 += chunk) {
        const int len = min(chunk, n - p0);
        __syncthreads();   // the previous chunk is scanned
        for (int j = threadIdx.x; j < len; j += blockDim.x) {
            const double w = weight(L[p0 + j], G[p0 + j], T, literal);
            ws[j] = w;
            Wf[j] = (float)w;
            Uf[j] = (float)U[p0 + j];
        }
        __syncthreads();
        if (warp != 0) continue;
        int lo = 0;
        while (lo < len) {
            int a = len;
            for (int b = lo; b < len; b += 32) {
                const int j = b + lane;
                bool ok = false;
                if (j < len) {
                    const double wj = ws[j];
                    // w = -inf (a proposal outside the prior) is never accepted
                    if (__double_as_longlong(wj) != (long long)0xFFF0000000000000ULL) {
                        int d = fast ? accept_fast(Wf[j], Uf[j], Wc) : -1;
                        if (d < 0) d = accept_exact(wj, U[p0 + j], wc, T, literal) ? 1 : 0;
                        ok = d == 1;
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, ok);
                const int stop = ball ? b + __ffs(ball) - 1 : min(len, b + 32);
                if (j < stop) out[p0 + j] = c;   // rejections up to the acceptance
                if (ball) {
                    a = stop;
                    break;
                }
            }
            if (a < len) {
                c = p0 + a;
                wc = ws[a];
                Wc = Wf[a];
                if (lane == 0) out[c] = c;
                ++acc;
            }
            lo = a + 1;
        }
    }
    if (threadIdx.x == 0 && n_accept) n_accept[r] = acc;
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
    const int chunk = n - 1 < kMhChunk ? (n - 1 > 0 ? n - 1 : 1) : kMhChunk;
    const size_t smem = (sizeof(double) + 2 * sizeof(float)) * (size_t)chunk;
    e = cudaFuncSetAttribute(mh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_independence: smem attribute");
    mh_kernel<<<n_chains, kMhThreads, smem, (cudaStream_t)stream>>>(n, chunk, logL, log_g, log_u, temperature,
                                                                     literal, chain_idx, n_accept);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_independence launch");
    return GB_OK;
}
