// kde.cu -- paired two-dimensional kernel-density proposals of the annealed
// posterior (Sec. III.G, Alg. 4).
//
// The posterior of a recovered signal is sampled over a reduced box around
// the MLE.  The first temperature draws uniformly from the box; afterwards the
// chain obtained at one temperature, smoothed by a kernel density estimate,
// is the proposal of the next.  The estimates are two-dimensional, one per
// parameter pair: (f0, fdot), (lambda, beta), (A, iota); psi and phi0 stay
// uniform over their narrow ranges.
//
// Each pair's estimate is a G x G grid.  It spans the chain's own range on
// each axis, [max(lo, a - 3h - c0), min(hi, b + 3h + c0)] for entries in
// [a, b], bandwidth h and box cell c0 = (hi - lo)/G, so that its resolution
// follows the posterior (the first temperature's grids span the box):
//   * the chain's n entries are counted per cell, cell index
//     floor((x - lo') / (hi' - lo') * G) clamped to the grid;
//   * the counts are smoothed per axis by a Gaussian kernel of Scott's
//     bandwidth for two dimensions, h = s n_eff^(-1/6) (s the standard
//     deviation of the n entries, n_eff the accepted moves + 1), truncated at
//     min(ceil(3 h / cell), G - 1) cells and normalised to sum one; mass
//     pushed past the grid edge is dropped;
//   * the result is normalised and mixed with a uniform floor eps, and
//     stored as cumulative sums C over the flattened cells c = i G + j.
// A draw takes the first cell with C_c > u and a uniform point in it; its
// density is (C_c - C_(c-1)) / cell area, exactly the probability the draw
// has.  One CTA builds one pair of one window (counts, both smoothing passes
// and the prefix sums in shared memory); one thread draws one proposal.
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kKdeThreads = 256;

__device__ __forceinline__ void pair_dims(int p, int& dx, int& dy) {
    dx = p == 0 ? 0 : p == 1 ? 3 : 4;
    dy = p == 0 ? 1 : p == 1 ? 2 : 5;
}

// cell of value v in [lo, hi] with G cells, clamped (a non-finite value goes to cell 0)
__device__ __forceinline__ int kde_cell(double v, double lo, double hi, int G) {
    const double t = __dmul_rn(__ddiv_rn(__dadd_rn(v, -lo), __dadd_rn(hi, -lo)), (double)G);
    if (!(t >= 0.0)) return 0;
    if (t >= (double)(G - 1)) return G - 1;
    return (int)floor(t);
}

// block-wide sum (OP = 0), minimum (1) or maximum (2) of one double (every thread gets it)
template <int OP>
__device__ double block_reduce(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = OP == 0 ? v + u : OP == 1 ? fmin(v, u) : fmax(v, u);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = red[0];
    for (int w = 1; w < kKdeThreads / 32; ++w) s = OP == 0 ? s + red[w] : OP == 1 ? fmin(s, red[w]) : fmax(s, red[w]);
    return s;
}

// grid extent of one axis: the entries' range [a, b] widened by 3h and a box cell, inside the box
__device__ __forceinline__ void grid_extent(double a, double b, double h, double lo, double hi, int G, double& e0,
                                            double& e1) {
    const double c0 = __ddiv_rn(__dadd_rn(hi, -lo), (double)G), h3 = __dmul_rn(3.0, h);
    e0 = fmax(lo, __dadd_rn(__dadd_rn(a, -h3), -c0));
    e1 = fmin(hi, __dadd_rn(__dadd_rn(b, h3), c0));
}

// Gaussian weights for offsets -r..r (sigma in cells), normalised; r = 0 for
// sigma = 0 or non-finite
__device__ void kernel_weights(double sigma, int G, float* k, int& r) {
    __syncthreads();
    const bool smooth = sigma > 0.0 && isfinite(sigma);
    r = smooth ? (int)fmin(ceil(3.0 * sigma), (double)(G - 1)) : 0;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int d = -r; d <= r; ++d) tot += smooth ? exp(-(double)d * d / (2.0 * sigma * sigma)) : 1.0;
        for (int d = -r; d <= r; ++d)
            k[d + r] = (float)((smooth ? exp(-(double)d * d / (2.0 * sigma * sigma)) : 1.0) / tot);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kKdeThreads) kde_build_kernel(int n, int G, const double* __restrict__ theta,
                                                                const int32_t* __restrict__ chain,
                                                                const double* __restrict__ box, double eps,
                                                                double* __restrict__ cdf, double* __restrict__ ext) {
    const int w = blockIdx.x, p = blockIdx.y, GG = G * G;
    int dx, dy;
    pair_dims(p, dx, dy);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = (double*)smem_raw;                       // kKdeThreads / 32
    double* part = red + kKdeThreads / 32;                 // kKdeThreads
    int* cnt = (int*)(part + kKdeThreads);                 // GG
    float* S1 = (float*)(cnt + GG);                        // GG
    float* S2 = S1 + GG;                                   // GG
    float* kx = S2 + GG;                                   // 2G
    float* ky = kx + 2 * G;                                // 2G
    const double* bx = box + 16 * (size_t)w;
    const double lox = bx[dx], hix = bx[8 + dx], loy = bx[dy], hiy = bx[8 + dy];
    for (int c = threadIdx.x; c < GG; c += kKdeThreads) cnt[c] = 0;
    const double* th = theta + 8 * (size_t)w * n;
    const int32_t* ch = chain + (size_t)w * n;
    // the chain's entries: mean, range and accepted moves, then the spread
    double sx = 0.0, sy = 0.0, acc = 0.0, ax = INFINITY, bx_ = -INFINITY, ay = INFINITY, by_ = -INFINITY;
    for (int i = threadIdx.x; i < n; i += kKdeThreads) {
        int s = ch[i];
        s = s < 0 ? 0 : s >= n ? n - 1 : s;
        if (i >= 1 && s == i) acc += 1.0;
        const double x = th[8 * (size_t)s + dx], y = th[8 * (size_t)s + dy];
        sx += x;
        sy += y;
        ax = fmin(ax, x);
        bx_ = fmax(bx_, x);
        ay = fmin(ay, y);
        by_ = fmax(by_, y);
    }
    const double mx = block_reduce<0>(sx, red) / n, my = block_reduce<0>(sy, red) / n;
    acc = block_reduce<0>(acc, red);
    ax = block_reduce<1>(ax, red);
    bx_ = block_reduce<2>(bx_, red);
    ay = block_reduce<1>(ay, red);
    by_ = block_reduce<2>(by_, red);
    double vx = 0.0, vy = 0.0;
    for (int i = threadIdx.x; i < n; i += kKdeThreads) {
        int s = ch[i];
        s = s < 0 ? 0 : s >= n ? n - 1 : s;
        const double x = th[8 * (size_t)s + dx] - mx, y = th[8 * (size_t)s + dy] - my;
        vx += x * x;
        vy += y * y;
    }
    vx = block_reduce<0>(vx, red) / n;
    vy = block_reduce<0>(vy, red) / n;
    const double bw = pow(acc + 1.0, -1.0 / 6.0);
    const double hx = sqrt(vx) * bw, hy = sqrt(vy) * bw;
    double x0, x1, y0, y1;
    grid_extent(ax, bx_, hx, lox, hix, G, x0, x1);
    grid_extent(ay, by_, hy, loy, hiy, G, y0, y1);
    if (threadIdx.x == 0) {
        double* e = ext + ((size_t)w * 3 + p) * 4;
        e[0] = x0;
        e[1] = x1;
        e[2] = y0;
        e[3] = y1;
    }
    for (int i = threadIdx.x; i < n; i += kKdeThreads) {
        int s = ch[i];
        s = s < 0 ? 0 : s >= n ? n - 1 : s;
        atomicAdd(&cnt[kde_cell(th[8 * (size_t)s + dx], x0, x1, G) * G + kde_cell(th[8 * (size_t)s + dy], y0, y1, G)],
                  1);
    }
    int rx, ry;
    kernel_weights(hx / ((x1 - x0) / G), G, kx, rx);
    kernel_weights(hy / ((y1 - y0) / G), G, ky, ry);
    // smoothing along x (first index), then along y
    for (int c = threadIdx.x; c < GG; c += kKdeThreads) {
        const int i = c / G, j = c - i * G;
        float v = 0.0f;
        for (int d = -rx; d <= rx; ++d) {
            const int i2 = i - d;
            if (i2 >= 0 && i2 < G) v = fmaf(kx[d + rx], (float)cnt[i2 * G + j], v);
        }
        S1[c] = v;
    }
    __syncthreads();
    double tot = 0.0;
    for (int c = threadIdx.x; c < GG; c += kKdeThreads) {
        const int i = c / G, j = c - i * G;
        float v = 0.0f;
        for (int e = -ry; e <= ry; ++e) {
            const int j2 = j - e;
            if (j2 >= 0 && j2 < G) v = fmaf(ky[e + ry], S1[i * G + j2], v);
        }
        S2[c] = v;
        tot += v;
    }
    tot = block_reduce<0>(tot, red);
    // cell probabilities with the floor, cumulative over contiguous chunks
    const double fl = eps / (double)GG, sc = (1.0 - eps) / tot;
    const int per = (GG + kKdeThreads - 1) / kKdeThreads;
    const int c0 = threadIdx.x * per, c1 = min(GG, c0 + per);
    double run = 0.0;
    for (int c = c0; c < c1; ++c) run += (double)S2[c] * sc + fl;
    part[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive scan of the chunk sums
        double a = 0.0;
        for (int t = 0; t < kKdeThreads; ++t) {
            const double v = part[t];
            part[t] = a;
            a += v;
        }
    }
    __syncthreads();
    double* out = cdf + ((size_t)w * 3 + p) * GG;
    run = part[threadIdx.x];
    for (int c = c0; c < c1; ++c) {
        run += (double)S2[c] * sc + fl;
        out[c] = run;
    }
}

// first c with C_c > u, the last cell if none
__device__ __forceinline__ int kde_search(const double* __restrict__ C, int GG, double u) {
    int lo = 0, hi = GG - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (C[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void kde_draw_kernel(int n, int G, const double* __restrict__ box, const double* __restrict__ cdf,
                                const double* __restrict__ ext, uint64_t seed, const uint64_t* __restrict__ round_in, uint64_t* __restrict__ round_out,
                                double* __restrict__ theta, double* __restrict__ log_g, double* __restrict__ log_u) {
    const int w = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t rnd = *round_in;
    if (w == 0 && blockIdx.x == 0 && threadIdx.x == 0) *round_out = rnd + 1;
    if (i >= n) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint4 a = philox4x32_10((uint32_t)rnd, (uint32_t)w, (uint32_t)i, 0u, k0, k1);
    const uint4 b = philox4x32_10((uint32_t)rnd, (uint32_t)w, (uint32_t)i, 1u, k0, k1);
    const uint4 c = philox4x32_10((uint32_t)rnd, (uint32_t)w, (uint32_t)i, 2u, k0, k1);
    const uint32_t words[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    const double* bx = box + 16 * (size_t)w;
    const int GG = G * G;
    double out[8];
    double lg = 0.0;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        int dx, dy;
        pair_dims(p, dx, dy);
        const double* C = cdf + ((size_t)w * 3 + p) * GG;
        const double* e = ext + ((size_t)w * 3 + p) * 4;
        const int cell = kde_search(C, GG, u01(words[3 * p]));
        const double P = C[cell] - (cell > 0 ? C[cell - 1] : 0.0);
        const int ci = cell / G, cj = cell - ci * G;
        const double cx = __ddiv_rn(__dadd_rn(e[1], -e[0]), (double)G);
        const double cy = __ddiv_rn(__dadd_rn(e[3], -e[2]), (double)G);
        out[dx] = __dadd_rn(e[0], __dmul_rn(__dadd_rn((double)ci, u01(words[3 * p + 1])), cx));
        out[dy] = __dadd_rn(e[2], __dmul_rn(__dadd_rn((double)cj, u01(words[3 * p + 2])), cy));
        lg += log(P) - log(__dmul_rn(cx, cy));
    }
#pragma unroll
    for (int d = 6; d < 8; ++d) {
        const double wd = __dadd_rn(bx[8 + d], -bx[d]);
        out[d] = __dadd_rn(bx[d], __dmul_rn(u01(words[d + 3]), wd));
        lg -= log(wd);
    }
    const size_t row = (size_t)w * n + i;
#pragma unroll
    for (int d = 0; d < 8; ++d) theta[8 * row + d] = out[d];
    log_g[row] = lg;
    log_u[row] = log(u01(words[11]));
}

size_t kde_build_smem(int G) {
    const size_t GG = (size_t)G * G;
    return sizeof(double) * (kKdeThreads / 32 + kKdeThreads) + sizeof(int) * GG + 2 * sizeof(float) * GG +
           4 * sizeof(float) * G;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int gb_kde_build(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* theta, const int32_t* chain,
                            const double* box, int32_t grid, double floor_mass, double* cdf, double* ext,
                            void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0 || n < 0) return set_error(ctx, GB_EINVAL, "gb_kde_build: negative size");
    if (n_win == 0) return GB_OK;
    if (n < 1) return set_error(ctx, GB_EINVAL, "gb_kde_build: at least one step per chain");
    if (grid < 2 || grid > 128) return set_error(ctx, GB_EINVAL, "gb_kde_build: grid must be in [2, 128]");
    if (!(floor_mass >= 0.0 && floor_mass <= 1.0)) return set_error(ctx, GB_EINVAL, "gb_kde_build: floor in [0, 1]");
    if (!theta || !chain || !box || !cdf || !ext) return set_error(ctx, GB_EINVAL, "gb_kde_build: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_kde_build: cudaSetDevice");
    const size_t smem = kde_build_smem(grid);
    e = cudaFuncSetAttribute(kde_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_kde_build: smem attribute");
    kde_build_kernel<<<dim3(n_win, 3), kKdeThreads, smem, (cudaStream_t)stream>>>(n, grid, theta, chain, box,
                                                                                  floor_mass, cdf, ext);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_kde_build launch");
    return GB_OK;
}

extern "C" int gb_kde_draw(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* box, int32_t grid,
                           const double* cdf, const double* ext, uint64_t seed, const uint64_t* round_in, uint64_t* round_out,
                           double* theta, double* log_g, double* log_u, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0 || n < 0) return set_error(ctx, GB_EINVAL, "gb_kde_draw: negative size");
    if (n_win == 0 || n == 0) return GB_OK;
    if (n_win > 65535) return set_error(ctx, GB_EINVAL, "gb_kde_draw: more than 65535 windows");
    if (grid < 2 || grid > 128) return set_error(ctx, GB_EINVAL, "gb_kde_draw: grid must be in [2, 128]");
    if (!box || !cdf || !ext || !round_in || !round_out || !theta || !log_g || !log_u)
        return set_error(ctx, GB_EINVAL, "gb_kde_draw: null pointer");
    if (round_in == round_out) return set_error(ctx, GB_EINVAL, "gb_kde_draw: round_out must not alias round_in");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_kde_draw: cudaSetDevice");
    kde_draw_kernel<<<dim3((n + 255) / 256, n_win), 256, 0, (cudaStream_t)stream>>>(
        n, grid, box, cdf, ext, seed, round_in, round_out, theta, log_g, log_u);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_kde_draw launch");
    return GB_OK;
}
