// noise.cu -- noise estimate within a frequency segment (Sec. III.C).
//
// Each window's noise is the median of its periodogram, 2 |d_k|^2 / T over
// the window's W bins (the data are continuous-Fourier-transform samples, so
// this is the paper's 2 |DFT|^2 / (N f_sample)), taken as a constant for the
// whole segment; loud signals in a few bins barely move a median.  For
// Gaussian noise the median of the exponentially distributed |d|^2 is ln 2
// times the mean, so an unbiased estimate divides by ln 2 (optional).
// One CTA per (window, channel): the W values are sorted in shared memory
// (bitonic, padded to a power of two) and the middle value (the mean of the
// middle pair for even W) is taken.
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kNoiseThreads = 256;
constexpr int kNoiseMaxW = 4096;
constexpr double kLn2 = 0.69314718055994531;

__global__ void __launch_bounds__(kNoiseThreads) noise_median_kernel(const gb_window_t* __restrict__ wins,
                                                                     const double2* __restrict__ dA,
                                                                     const double2* __restrict__ dE, double T,
                                                                     int debias, double* __restrict__ S,
                                                                     double* __restrict__ wA, double* __restrict__ wE) {
    extern __shared__ double v[];   // P = next power of two >= W
    const int w = blockIdx.x, ch = blockIdx.y;
    const gb_window_t win = wins[w];
    const int W = win.W;
    if (W <= 0) {
        if (threadIdx.x == 0) S[2 * (size_t)w + ch] = nan("");
        return;
    }
    int P = 1;
    while (P < W) P <<= 1;
    const double2* d = (ch == 0 ? dA : dE) + win.data_off;
    for (int i = threadIdx.x; i < P; i += kNoiseThreads) {
        if (i < W) {
            const double2 x = d[i];
            v[i] = __ddiv_rn(__dmul_rn(2.0, __dadd_rn(__dmul_rn(x.x, x.x), __dmul_rn(x.y, x.y))), T);
        } else {
            v[i] = INFINITY;
        }
    }
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += kNoiseThreads) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const double a = v[i], b = v[l];
                    if ((a > b) == up) {
                        v[i] = b;
                        v[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    double m = (W & 1) ? v[W / 2] : (v[W / 2 - 1] + v[W / 2]) / 2.0;
    if (debias) m = m / kLn2;
    if (threadIdx.x == 0) S[2 * (size_t)w + ch] = m;
    double* wt = ch == 0 ? wA : wE;
    if (wt) {
        const double iw = 1.0 / m;
        for (int i = threadIdx.x; i < W; i += kNoiseThreads) wt[win.data_off + i] = iw;
    }
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int gb_noise_median(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win, const double* dA,
                               const double* dE, int64_t n_bins, int32_t debias, double* S, double* wA, double* wE,
                               void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0 || n_bins < 0) return set_error(ctx, GB_EINVAL, "gb_noise_median: negative size");
    if (n_win == 0) return GB_OK;
    if (!win || !dA || !dE || !S) return set_error(ctx, GB_EINVAL, "gb_noise_median: null pointer");
    if ((wA == nullptr) != (wE == nullptr)) return set_error(ctx, GB_EINVAL, "gb_noise_median: wA and wE together");
    for (int32_t i = 0; i < n_win; ++i) {
        const gb_window_t& w = win[i];
        if (w.W < 0 || w.W > kNoiseMaxW || w.data_off < 0 || w.data_off + w.W > n_bins)
            return set_error(ctx, GB_EINVAL,
                             "gb_noise_median: window " + std::to_string(i) + ": W in [0, 4096] inside n_bins");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_noise_median: cudaSetDevice");
    gb_window_t* d_win = nullptr;
    e = cudaMallocAsync((void**)&d_win, sizeof(gb_window_t) * (size_t)n_win, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_noise_median: window upload");
    e = cudaMemcpyAsync(d_win, win, sizeof(gb_window_t) * (size_t)n_win, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) {
        const size_t smem = sizeof(double) * kNoiseMaxW;
        e = cudaFuncSetAttribute(noise_median_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            noise_median_kernel<<<dim3(n_win, 2), kNoiseThreads, smem, (cudaStream_t)stream>>>(
                d_win, (const double2*)dA, (const double2*)dE, ctx->obs.T_obs, debias, S, wA, wE);
            ++ctx->launches;
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaFreeAsync(d_win, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_noise_median launch");
    if (e2 != cudaSuccess) return cuda_error(ctx, e2, "gb_noise_median: free");
    return GB_OK;
}
