// ga.cu -- one generation of the genetic search over every window's population.
//
// The paper's local search (Alg. 2, Sec. III.D) maximises the SNR of Eq. 6 over
// the seven parameters other than A with differential evolution and then sets
// A to the analytic best amplitude of Eq. 7.  The search here is a genetic
// algorithm with the same objective, run on the device so that a whole
// generation (likelihood launch + this kernel) can be replayed from a CUDA
// graph.  Per window (one CTA):
//   * fitness rho = <d|h>/sqrt(<h|h>) of every individual (Eq. 6);
//   * the best individual, with A replaced by A_max = A <d|h>/<h|h> (Eq. 7),
//     goes to slot 0 and to `best`;
//   * optionally the fitness is also maximised over phi0 in closed form: the
//     template carries phi0 only as the common factor exp(i phi0), so with
//     Z = <d|h> + i <d|h>_im (the second the same sum over Im(d conj h)),
//     <d|h(phi0 + delta)> = Re(exp(-i delta) Z); the maximum over delta is |Z|
//     at delta = arg Z, rho = |Z|/sqrt(<h|h>), and the best individual is
//     rotated to phi0 + arg Z with A_max = A |Z|/<h|h>;
//   * with a gradient at the best individual, slots 1..4 take steps of
//     radius 0.3, 0.1, 0.03, 0.01 along the gradient direction in natural
//     units (a line search left to the next generation's selection);
//   * every other slot is a child: two size-k tournaments, blend crossover,
//     Gaussian mutation of each parameter with probability p_mut and scale
//     mut_scale times the box width, then wrapped (longitude, phase,
//     polarisation) or reflected (latitude, inclination, f0, fdot, A) into the
//     window's prior box.
// Random numbers come from Philox-4x32-10 (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), keyed by the seed
// and counted by (generation, window, individual, draw).
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kGaThreads = 256;
constexpr int kGaMaxPop = 32768;   // fitness of the population in shared memory

// Draws of the genetic search.  They only steer a heuristic, so they are taken
// in float where that saves double-precision work: indices by multiply-shift,
// Bernoulli tests as integer thresholds, normals by float Box-Muller.
struct Rng {
    uint32_t k0, k1, gen, win, ind, draw;
    uint4 buf;
    int left = 0;
    __device__ uint32_t next() {
        if (left == 0) {
            buf = philox4x32_10(gen, win, ind, draw++, k0, k1);
            left = 4;
        }
        --left;
        return left == 3 ? buf.x : left == 2 ? buf.y : left == 1 ? buf.z : buf.w;
    }
    __device__ int index(int n) { return (int)(((uint64_t)next() * (uint64_t)n) >> 32); }
    __device__ float uniform_f() { return ((float)(next() >> 8) + 0.5f) * 5.9604644775390625e-08f; }   // 2^-24
    __device__ bool bernoulli(uint32_t thr, bool always) { return always || next() < thr; }
    __device__ float normal_f() {   // Box-Muller
        const float a = uniform_f(), b = uniform_f();
        return sqrtf(-2.0f * logf(a)) * cospif(2.0f * b);
    }
};

// probability p as a threshold on 32 random bits (p >= 1: always)
__device__ __forceinline__ uint32_t prob_threshold(double p, bool& always) {
    always = p >= 1.0;
    return always ? 0u : (uint32_t)(p * 4294967296.0);
}

// reflect / wrap into [lo, hi]; one fold covers a step of up to a box width,
// the remainder form handles any other value
__device__ __forceinline__ double reflect(double x, double lo, double hi) {
    if (x >= lo && x <= hi) return x;
    const double w = hi - lo;
    if (!(w > 0.0)) return lo;
    if (x < lo && x >= lo - w) return 2.0 * lo - x;
    if (x > hi && x <= hi + w) return 2.0 * hi - x;
    double y = fmod(x - lo, 2.0 * w);
    if (y < 0.0) y += 2.0 * w;
    return lo + (y > w ? 2.0 * w - y : y);
}

__device__ __forceinline__ double wrap(double x, double lo, double hi) {
    if (x >= lo && x < hi) return x;
    const double w = hi - lo;
    if (!(w > 0.0)) return lo;
    if (x < lo && x >= lo - w) return x + w;
    if (x >= hi && x < hi + w) return x - w;
    double y = fmod(x - lo, w);
    if (y < 0.0) y += w;
    return lo + y;
}

// rho = <d|h>/sqrt(<h|h>) (Eq. 6), in float: it only ranks individuals
__device__ __forceinline__ float fitness(double dh, double hh) {
    if (!(hh > 0.0) || !isfinite(dh) || !isfinite(hh)) return -INFINITY;
    const float h = (float)hh;
    if (h >= 1e-30f && h <= 1e30f && fabs(dh) < 1e30) return (float)dh * rsqrtf(h);
    return (float)(dh / sqrt(hh));
}

__global__ void __launch_bounds__(kGaThreads) ga_step_kernel(int pop, const double* __restrict__ theta,
                                                             const double* __restrict__ dh,
                                                             const double* __restrict__ hh,
                                                             const double* __restrict__ dh_im,
                                                             const gb_box_t* __restrict__ box, uint64_t seed,
                                                             const uint64_t* __restrict__ gen_in,
                                                             uint64_t* __restrict__ gen_out, gb_ga_params_t prm,
                                                             const double* __restrict__ grad, double T,
                                                             double* __restrict__ out, double* __restrict__ best) {
    extern __shared__ float s_pop_fit[];   // pop
    __shared__ float s_fit[kGaThreads];
    __shared__ int s_idx[kGaThreads];
    __shared__ double s_best[8];
    const int w = blockIdx.x;
    const uint64_t generation = *gen_in;
    if (w == 0 && threadIdx.x == 0) *gen_out = generation + 1;
    const size_t base = (size_t)w * (size_t)pop;
    const double* th = theta + 8 * base;
    double* to = out + 8 * base;
    const gb_box_t bx = box[w];
    // phase maximisation needs the whole circle of phi0 inside the box
    const bool pmax = dh_im != nullptr && bx.hi[7] - bx.lo[7] >= 2.0 * kPi * (1.0 - 1e-12);
    // fitness of every individual, and the best one (lowest index among equals)
    float bf = -INFINITY;
    int bi = 0;
    for (int i = threadIdx.x; i < pop; i += blockDim.x) {
        const float f = pmax ? fitness(hypot(dh[base + i], dh_im[base + i]), hh[base + i])
                             : fitness(dh[base + i], hh[base + i]);
        s_pop_fit[i] = f;
        if (f > bf) {
            bf = f;
            bi = i;
        }
    }
    s_fit[threadIdx.x] = bf;
    s_idx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const float f2 = s_fit[threadIdx.x + s];
            const int i2 = s_idx[threadIdx.x + s];
            if (f2 > s_fit[threadIdx.x] || (f2 == s_fit[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
                s_fit[threadIdx.x] = f2;
                s_idx[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const int ib = s_idx[0];
    if (threadIdx.x < 8) {
        double v = th[8 * ib + threadIdx.x];
        const double di = pmax ? dh_im[base + ib] : 0.0;
        if (threadIdx.x == 4) {   // A_max = A <d|h>/<h|h> (Eq. 7), kept inside the box
            const double d = pmax ? hypot(dh[base + ib], di) : dh[base + ib], h = hh[base + ib];
            if (h > 0.0 && d > 0.0 && isfinite(d)) v = fmin(fmax(v * d / h, bx.lo[4]), bx.hi[4]);
        }
        if (threadIdx.x == 7 && pmax) {   // phi0 + arg Z, back onto the circle of the box
            const double d = dh[base + ib];
            if (isfinite(d) && isfinite(di) && (d != 0.0 || di != 0.0)) v = wrap(v + atan2(di, d), bx.lo[7], bx.hi[7]);
        }
        s_best[threadIdx.x] = v;
        if (best) best[8 * (size_t)w + threadIdx.x] = v;
    }
    __syncthreads();
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double scale[8] = {1.0 / T, 1.0 / (T * T), 1.0, 1.0, s_best[4], 1.0, 1.0, 1.0};
    double gnorm = 0.0;
    if (grad) {
        for (int j = 0; j < 8; ++j) {
            const double g = grad[8 * (size_t)w + j] * scale[j];
            gnorm += g * g;
        }
        gnorm = sqrt(gnorm);
    }
    bool all_c, all_m;
    const uint32_t thr_c = prob_threshold(prm.p_cross, all_c), thr_m = prob_threshold(prm.p_mut, all_m);
    double sigma[8];
    for (int j = 0; j < 8; ++j) sigma[j] = prm.mut_scale * (bx.hi[j] - bx.lo[j]);
    const double radii[4] = {0.3, 0.1, 0.03, 0.01};
    for (int i = threadIdx.x; i < pop; i += blockDim.x) {
        double c[8];
        if (i == 0) {
            for (int j = 0; j < 8; ++j) c[j] = s_best[j];
        } else if (i <= 4 && grad && gnorm > 0.0 && isfinite(gnorm)) {
            for (int j = 0; j < 8; ++j) {
                const double dj = grad[8 * (size_t)w + j] * scale[j] / gnorm;
                c[j] = s_best[j] + radii[i - 1] * scale[j] * dj;
            }
        } else {
            Rng rng{k0, k1, (uint32_t)generation, (uint32_t)w, (uint32_t)i, 0u};
            int par[2];
            for (int p = 0; p < 2; ++p) {
                int win_i = rng.index(pop);
                float win_f = s_pop_fit[win_i];
                for (int t = 1; t < prm.tournament; ++t) {
                    const int j = rng.index(pop);
                    const float f = s_pop_fit[j];
                    if (f > win_f) {
                        win_f = f;
                        win_i = j;
                    }
                }
                par[p] = win_i;
            }
            for (int j = 0; j < 8; ++j) {
                const double a = th[8 * par[0] + j], b = th[8 * par[1] + j];
                const double t = (double)rng.uniform_f();
                double x = rng.bernoulli(thr_c, all_c) ? fma(t, b - a, a) : a;
                if (rng.bernoulli(thr_m, all_m)) x = fma(sigma[j], (double)rng.normal_f(), x);
                c[j] = x;
            }
        }
        // back into the prior box
        c[0] = reflect(c[0], bx.lo[0], bx.hi[0]);
        c[1] = reflect(c[1], bx.lo[1], bx.hi[1]);
        c[2] = reflect(c[2], bx.lo[2], bx.hi[2]);
        c[3] = wrap(c[3], bx.lo[3], bx.hi[3]);
        c[4] = reflect(c[4], bx.lo[4], bx.hi[4]);
        c[5] = reflect(c[5], bx.lo[5], bx.hi[5]);
        c[6] = wrap(c[6], bx.lo[6], bx.hi[6]);
        c[7] = wrap(c[7], bx.lo[7], bx.hi[7]);
        for (int j = 0; j < 8; ++j) to[8 * i + j] = c[j];
    }
}

// Proposals of an independence sampler (Alg. 4: "n samples randomly drawn"),
// one thread per proposal: z_j = Box-Muller normals from Philox counter
// (round, window, proposal, block), theta = mu + L z (L lower triangular),
// log g = -|z|^2/2 - sum_j log L_jj - 4 log(2 pi), log u from one more draw.
__global__ void draw_gaussian_kernel(int n, const double* __restrict__ mu, const double* __restrict__ chol,
                                     uint64_t seed, const uint64_t* __restrict__ round_in,
                                     uint64_t* __restrict__ round_out, double* __restrict__ theta,
                                     double* __restrict__ log_g, double* __restrict__ log_u) {
    const int w = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t rnd = *round_in;
    if (w == 0 && blockIdx.x == 0 && threadIdx.x == 0) *round_out = rnd + 1;
    if (i >= n) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint4 a = philox4x32_10((uint32_t)rnd, (uint32_t)w, (uint32_t)i, 0u, k0, k1);
    const uint4 b = philox4x32_10((uint32_t)rnd, (uint32_t)w, (uint32_t)i, 1u, k0, k1);
    const uint4 c = philox4x32_10((uint32_t)rnd, (uint32_t)w, (uint32_t)i, 2u, k0, k1);
    const uint32_t words[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    double z[8];
    for (int j = 0; j < 4; ++j) {
        const double r = sqrt(-2.0 * log(u01(words[2 * j])));
        double s, co;
        sincospi(2.0 * u01(words[2 * j + 1]), &s, &co);
        z[2 * j] = r * co;
        z[2 * j + 1] = r * s;
    }
    const double* m = mu + 8 * w;
    const double* L = chol + 64 * w;
    const size_t row = (size_t)w * n + i;
    double zz = 0.0, ld = 0.0;
    for (int r = 0; r < 8; ++r) {
        double v = m[r];
        for (int k = 0; k <= r; ++k) v += L[8 * r + k] * z[k];
        theta[8 * row + r] = v;
        zz += z[r] * z[r];
        ld += log(L[8 * r + r]);
    }
    log_g[row] = -0.5 * zz - ld - 4.0 * log(2.0 * kPi);
    log_u[row] = log(u01(c.x));
}

// raw Philox outputs, for tests of the generator against its published definition
__global__ void philox_kernel(uint64_t seed, uint32_t n, uint32_t* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox4x32_10(i, 0u, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    out[4 * i + 0] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int gb_ga_step(gb_ctx_t* ctx, int32_t n_win, int32_t pop, const double* theta, const double* dh,
                          const double* hh, const double* dh_im, const gb_box_t* box, uint64_t seed, const uint64_t* generation_in,
                          uint64_t* generation_out, const gb_ga_params_t* params, const double* grad,
                          double* theta_out, double* best, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0 || pop < 0) return set_error(ctx, GB_EINVAL, "gb_ga_step: negative size");
    if (n_win == 0 || pop == 0) return GB_OK;
    if (!theta || !dh || !hh || !box || !params || !theta_out || !generation_in || !generation_out)
        return set_error(ctx, GB_EINVAL, "gb_ga_step: null pointer");
    if (theta == theta_out) return set_error(ctx, GB_EINVAL, "gb_ga_step: theta_out must not alias theta");
    if (generation_in == generation_out)
        return set_error(ctx, GB_EINVAL, "gb_ga_step: generation_out must not alias generation_in");
    if (params->tournament < 1 || !(params->p_cross >= 0.0 && params->p_cross <= 1.0) ||
        !(params->p_mut >= 0.0 && params->p_mut <= 1.0) || !(params->mut_scale >= 0.0))
        return set_error(ctx, GB_EINVAL, "gb_ga_step: bad parameters");
    if (pop > kGaMaxPop) return set_error(ctx, GB_EINVAL, "gb_ga_step: pop above 32768");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_ga_step: cudaSetDevice");
    const size_t smem = sizeof(float) * (size_t)pop;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(ga_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(ctx, e, "gb_ga_step: smem attribute");
    }
    ga_step_kernel<<<n_win, kGaThreads, smem, (cudaStream_t)stream>>>(pop, theta, dh, hh, dh_im, box, seed, generation_in,
                                                                      generation_out, *params, grad, ctx->obs.T_obs,
                                                                      theta_out, best);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_ga_step launch");
    return GB_OK;
}

extern "C" int gb_draw_gaussian(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* mu, const double* chol,
                                uint64_t seed, const uint64_t* round_in, uint64_t* round_out, double* theta,
                                double* log_g, double* log_u, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0 || n < 0) return set_error(ctx, GB_EINVAL, "gb_draw_gaussian: negative size");
    if (n_win == 0 || n == 0) return GB_OK;
    if (n_win > 65535) return set_error(ctx, GB_EINVAL, "gb_draw_gaussian: more than 65535 windows");
    if (!mu || !chol || !round_in || !round_out || !theta || !log_g || !log_u)
        return set_error(ctx, GB_EINVAL, "gb_draw_gaussian: null pointer");
    if (round_in == round_out) return set_error(ctx, GB_EINVAL, "gb_draw_gaussian: round_out must not alias round_in");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_draw_gaussian: cudaSetDevice");
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_win);
    draw_gaussian_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, mu, chol, seed, round_in, round_out, theta, log_g,
                                                                 log_u);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_draw_gaussian launch");
    return GB_OK;
}

namespace gb {
namespace {

// Gaussian refit of an independence proposal to the states its chain visited
// (Alg. 4 refits the proposal between temperatures).  One CTA per window:
// moments of theta[chain[i]] over all n steps (a state weighs the steps spent
// in it), shifted by the first state, and the number u of accepted moves;
// then one thread blends the sample covariance with the current proposal's
// (weight u/(u + kappa) on the sample), scales it, whitens it with the first
// proposal's factor L0, caps every whitened variance at 1/floor, adds floor
// to the diagonal, factors it and writes L0 L_M.
constexpr int kRefitThreads = 256;

__global__ void __launch_bounds__(kRefitThreads) gauss_refit_kernel(int n, const double* __restrict__ theta,
                                                                    const int32_t* __restrict__ chain,
                                                                    const double* __restrict__ chol0, double ratio,
                                                                    double inflate, double kappa, double floor_,
                                                                    double* __restrict__ mu_out,
                                                                    double* chol_io) {
    __shared__ double x0[8];
    __shared__ double part[kRefitThreads / 32][45];
    const int w = blockIdx.x;
    const double* th = theta + (size_t)w * (size_t)n * 8;
    const int32_t* ch = chain + (size_t)w * (size_t)n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 8) {
        const int c0 = min(max(ch[0], 0), n - 1);
        x0[threadIdx.x] = th[8 * (size_t)c0 + threadIdx.x];
    }
    __syncthreads();
    double s[45];   // 8 first moments, 36 second moments (upper triangle), accepted moves
#pragma unroll
    for (int q = 0; q < 45; ++q) s[q] = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int c = min(max(ch[i], 0), n - 1);
        if (i > 0 && ch[i] == i) s[44] += 1.0;
        double d[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = th[8 * (size_t)c + j] - x0[j];
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] += d[j];
        int q = 8;
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = j; k < 8; ++k) {
                s[q] = fma(d[j], d[k], s[q]);
                ++q;
            }
    }
#pragma unroll
    for (int q = 0; q < 45; ++q) {
        double v = s[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t[45];
    for (int q = 0; q < 45; ++q) {
        t[q] = 0.0;
        for (int k = 0; k < kRefitThreads / 32; ++k) t[q] += part[k][q];
    }
    const double inv_n = 1.0 / (double)n;
    // the current proposal's covariance P = L L^T (read before chol_io is written)
    double* Lio = chol_io + 64 * (size_t)w;
    double P[8][8];
    for (int j = 0; j < 8; ++j)
        for (int k = 0; k <= j; ++k) {
            double v = 0.0;
            for (int m = 0; m <= k; ++m) v += Lio[8 * j + m] * Lio[8 * k + m];
            P[j][k] = v;
            P[k][j] = v;
        }
    const double wgt = t[44] / (t[44] + kappa);
    double C[8][8];
    int q = 8;
    for (int j = 0; j < 8; ++j)
        for (int k = j; k < 8; ++k) {
            const double sc = (t[q] - t[j] * t[k] * inv_n) / (double)(n - 1);
            ++q;
            const double c = ratio * (wgt * inflate * sc + (1.0 - wgt) * P[j][k]);
            C[j][k] = c;
            C[k][j] = c;
        }
    const double* L0 = chol0 + 64 * (size_t)w;
    // Y = L0^-1 C, then M = L0^-1 Y^T (= L0^-1 C L0^-T)
    double Y[8][8], M[8][8];
    for (int col = 0; col < 8; ++col)
        for (int r = 0; r < 8; ++r) {
            double v = C[r][col];
            for (int k = 0; k < r; ++k) v -= L0[8 * r + k] * Y[k][col];
            Y[r][col] = v / L0[8 * r + r];
        }
    for (int col = 0; col < 8; ++col)
        for (int r = 0; r < 8; ++r) {
            double v = Y[col][r];
            for (int k = 0; k < r; ++k) v -= L0[8 * r + k] * M[k][col];
            M[r][col] = v / L0[8 * r + r];
        }
    bool ok = true;
    double dcap[8];
    for (int j = 0; j < 8; ++j) {
        ok = ok && isfinite(M[j][j]);
        dcap[j] = fmax(1.0, sqrt(fmax(M[j][j], 0.0) * floor_));
    }
    for (int j = 0; j < 8; ++j)
        for (int k = 0; k < 8; ++k) {
            ok = ok && isfinite(M[j][k]);
            M[j][k] = 0.5 * (M[j][k] + M[k][j]) / (dcap[j] * dcap[k]);
        }
    if (!ok)
        for (int j = 0; j < 8; ++j)
            for (int k = 0; k < 8; ++k) M[j][k] = j == k ? 1.0 : 0.0;
    for (int j = 0; j < 8; ++j) M[j][j] += floor_;
    // Cholesky of M (positive definite: a covariance plus floor on the diagonal)
    double Lm[8][8];
    for (int j = 0; j < 8; ++j) {
        double dj = M[j][j];
        for (int k = 0; k < j; ++k) dj -= Lm[j][k] * Lm[j][k];
        dj = sqrt(fmax(dj, floor_ * 1e-6));
        Lm[j][j] = dj;
        for (int r = j + 1; r < 8; ++r) {
            double v = M[r][j];
            for (int k = 0; k < j; ++k) v -= Lm[r][k] * Lm[j][k];
            Lm[r][j] = v / dj;
        }
        for (int r = 0; r < j; ++r) Lm[r][j] = 0.0;
    }
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) {
            double v = 0.0;
            for (int k = c; k <= r; ++k) v += L0[8 * r + k] * Lm[k][c];
            Lio[8 * r + c] = c <= r ? v : 0.0;
        }
    for (int j = 0; j < 8; ++j) mu_out[8 * (size_t)w + j] = ok ? x0[j] + t[j] * inv_n : x0[j];
}

}  // namespace
}  // namespace gb

extern "C" int gb_gauss_refit(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* theta, const int32_t* chain,
                              const double* chol0, double ratio, double inflate, double kappa, double floor_,
                              double* mu, double* chol, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0 || n < 0) return set_error(ctx, GB_EINVAL, "gb_gauss_refit: negative size");
    if (n_win == 0) return GB_OK;
    if (n < 2) return set_error(ctx, GB_EINVAL, "gb_gauss_refit: at least two steps per chain");
    if (!theta || !chain || !chol0 || !mu || !chol) return set_error(ctx, GB_EINVAL, "gb_gauss_refit: null pointer");
    if (!(ratio > 0.0) || !(ratio < 1e300) || !(inflate > 0.0) || !(inflate < 1e300) || !(kappa >= 0.0) ||
        !(kappa < 1e300) || !(floor_ > 0.0) || !(floor_ < 1.0))
        return set_error(ctx, GB_EINVAL, "gb_gauss_refit: ratio, inflate > 0, kappa >= 0, 0 < floor < 1");
    if (chol == chol0) return set_error(ctx, GB_EINVAL, "gb_gauss_refit: chol must not alias chol0");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_gauss_refit: cudaSetDevice");
    gauss_refit_kernel<<<n_win, kRefitThreads, 0, (cudaStream_t)stream>>>(n, theta, chain, chol0, ratio, inflate,
                                                                          kappa, floor_, mu, chol);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_gauss_refit launch");
    return GB_OK;
}

extern "C" int gb_philox4x32(gb_ctx_t* ctx, uint64_t seed, uint32_t n, uint32_t* out, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n == 0) return GB_OK;
    if (!out) return set_error(ctx, GB_EINVAL, "gb_philox4x32: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_philox4x32: cudaSetDevice");
    philox_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, n, out);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_philox4x32 launch");
    return GB_OK;
}
