// fp64.cu -- plain IEEE-double path: template by the fast/slow decomposition,
// warp FFT in shared memory, window inner products, log-likelihood (Eq. 2).
//
// Mapping: one CTA per tile (window, <= 32*WARPS candidates).  Each warp owns
// up to 32 consecutive candidates: their per-candidate setup (sky basis,
// polarisation tensor, carrier bin) is computed lane-parallel, one candidate
// per lane, into shared memory; then the warp evaluates them one after the
// other with the N samples strided across the 32 lanes, an in-place radix-2
// FFT in the warp's shared-memory buffer, and the window inner products with
// a warp reduction.
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kWarps64 = 4;

struct C64 {
    double x, y;
};
__device__ __forceinline__ C64 cadd(C64 a, C64 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C64 csub(C64 a, C64 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ C64 cmul(C64 a, C64 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ C64 cscale(C64 a, double s) { return {a.x * s, a.y * s}; }

// Per-candidate constants.
struct Cand64 {
    double k[3];          // propagation direction
    double Hr[6], Hi[6];  // H_xx, H_yy, H_zz, H_xy, H_xz, H_yz
    double f0, fd, delta, phi0, A;
    long long q;
    int bad;
    int pad;
};

struct Geo64 {
    double T, T_over_N, fstar, scale;   // scale = T / (2N)
    int N, logN;
};

// Candidate setup (one lane, one candidate).  The carrier bin uses explicit
// round-to-nearest operations so that q is bit-identical to any IEEE
// evaluation of ((f0*T) + ((0.5*fdot)*T)*T) + 0.5.
__device__ void setup64(const double* th, double T, Cand64& c) {
    const double f0 = th[0], fd = th[1], beta = th[2], lam = th[3];
    const double A = th[4], iota = th[5], psi = th[6], phi0 = th[7];
    bool bad = false;
    for (int i = 0; i < 8; ++i) bad |= !isfinite(th[i]);
    c.bad = bad;
    const double f0T = __dmul_rn(f0, T);
    const double xm = __dadd_rn(f0T, __dmul_rn(__dmul_rn(__dmul_rn(0.5, fd), T), T));
    const double qd = floor(__dadd_rn(xm, 0.5));
    c.q = bad ? 0 : (long long)qd;
    c.delta = __dadd_rn(f0T, -qd);
    c.f0 = f0;
    c.fd = fd;
    c.phi0 = phi0;
    c.A = A;
    double sb, cb, sl, cl, s2, c2;
    sincos(beta, &sb, &cb);
    sincos(lam, &sl, &cl);
    sincos(2.0 * psi, &s2, &c2);
    const double ci = cos(iota);
    c.k[0] = -(cb * cl);
    c.k[1] = -(cb * sl);
    c.k[2] = -sb;
    const double u[3] = {sb * cl, sb * sl, -cb};
    const double v[3] = {sl, -cl, 0.0};
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    const double Ap = A * (1.0 + ci * ci);
    const double Ax = -2.0 * A * ci;
    for (int m = 0; m < 6; ++m) {
        const int a = ia[m], b = ib[m];
        const double ep = u[a] * u[b] - v[a] * v[b];
        const double ex = u[a] * v[b] + v[a] * u[b];
        const double Ep = c2 * ep - s2 * ex;
        const double Ex = s2 * ep + c2 * ex;
        c.Hr[m] = Ap * Ep;
        c.Hi[m] = -(Ax * Ex);
    }
}

// n.H.n for a unit vector n and the symmetric complex H.
__device__ __forceinline__ C64 nHn(const Cand64& c, double nx, double ny, double nz) {
    const double m0 = nx * nx, m1 = ny * ny, m2 = nz * nz;
    const double m3 = 2.0 * nx * ny, m4 = 2.0 * nx * nz, m5 = 2.0 * ny * nz;
    C64 g;
    g.x = c.Hr[0] * m0 + c.Hr[1] * m1 + c.Hr[2] * m2 + c.Hr[3] * m3 + c.Hr[4] * m4 + c.Hr[5] * m5;
    g.y = c.Hi[0] * m0 + c.Hi[1] * m1 + c.Hi[2] * m2 + c.Hi[3] * m3 + c.Hi[4] * m4 + c.Hi[5] * m5;
    return g;
}

// -i a sinc(X) exp(-iX) G exp(i Psi)
__device__ __forceinline__ C64 link64(double a, double X, C64 G, C64 rx) {
    double sX, cX;
    sincos(X, &sX, &cX);
    const double sinc = (X != 0.0) ? sX / X : 1.0;
    const C64 tr = {a * sinc * cX, -(a * sinc * sX)};   // a sinc(X) e^{-iX}
    const C64 z = cmul(cmul(tr, G), rx);
    return {z.y, -z.x};                                    // times -i
}

// Slow part of one candidate into buf{A,E} at bit-reversed positions, then
// an in-place radix-2 FFT -> natural-order DFT S_k, k = 0..N-1.
__device__ void template64(const Cand64& c, const Geo64& g, const OrbitTables64& tab, const C64* tw,
                           C64* bufA, C64* bufE, int lane) {
    const int N = g.N;
    for (int n = lane; n < N; n += 32) {
        const double t = (double)n * g.T_over_N;
        C64 rx[3];
        for (int j = 0; j < 3; ++j) {
            const double kap = (c.k[0] * tab.x[(j * 3 + 0) * N + n] + c.k[1] * tab.x[(j * 3 + 1) * N + n] +
                                c.k[2] * tab.x[(j * 3 + 2) * N + n]) / kC;
            const double ph = 2.0 * kPi *
                                  (c.delta * t / g.T + 0.5 * c.fd * (t * t) - c.f0 * kap - c.fd * t * kap +
                                   0.5 * c.fd * (kap * kap)) +
                              c.phi0;
            double s, co;
            sincos(ph, &s, &co);
            rx[j] = {co, s};
        }
        const double f = c.f0 + c.fd * t;
        const double a = f / (2.0 * g.fstar);
        C64 z01, z10, z12, z21, z20, z02;
        {
            const double nx = tab.arm[0 * N + n], ny = tab.arm[1 * N + n], nz = tab.arm[2 * N + n];
            const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
            const C64 G = nHn(c, nx, ny, nz);
            z01 = link64(a, a * (1.0 - kn), G, rx[1]);
            z10 = link64(a, a * (1.0 + kn), G, rx[0]);
        }
        {
            const double nx = tab.arm[3 * N + n], ny = tab.arm[4 * N + n], nz = tab.arm[5 * N + n];
            const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
            const C64 G = nHn(c, nx, ny, nz);
            z12 = link64(a, a * (1.0 - kn), G, rx[2]);
            z21 = link64(a, a * (1.0 + kn), G, rx[1]);
        }
        {
            const double nx = tab.arm[6 * N + n], ny = tab.arm[7 * N + n], nz = tab.arm[8 * N + n];
            const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
            const C64 G = nHn(c, nx, ny, nz);
            z20 = link64(a, a * (1.0 - kn), G, rx[0]);
            z02 = link64(a, a * (1.0 + kn), G, rx[2]);
        }
        double sD, cD;
        sincos(f / g.fstar, &sD, &cD);
        const C64 D = {cD, -sD};
        const C64 D2 = cmul(D, D);
        const C64 omd = {1.0 - D2.x, -D2.y};
        const C64 X = cmul(omd, csub(cadd(z10, cmul(D, z01)), cadd(z20, cmul(D, z02))));
        const C64 Y = cmul(omd, csub(cadd(z21, cmul(D, z12)), cadd(z01, cmul(D, z10))));
        const C64 Z = cmul(omd, csub(cadd(z02, cmul(D, z20)), cadd(z12, cmul(D, z21))));
        const double r2 = sqrt(2.0), r6 = sqrt(6.0);
        const C64 sA = {(Z.x - X.x) / r2, (Z.y - X.y) / r2};
        const C64 sE = {(X.x - 2.0 * Y.x + Z.x) / r6, (X.y - 2.0 * Y.y + Z.y) / r6};
        const int br = (int)(__brev((unsigned)n) >> (32 - g.logN));
        bufA[br] = sA;
        bufE[br] = sE;
    }
    __syncwarp();
    // radix-2 decimation in time, bit-reversed input, natural-order output
    for (int s = 0; s < g.logN; ++s) {
        const int h = 1 << s;
        const int tstride = kTwiddles >> s;
        for (int b = lane; b < N / 2; b += 32) {
            const int j = b & (h - 1);
            const int i0 = ((b >> s) << (s + 1)) + j;
            const int i1 = i0 + h;
            const C64 w = tw[j * tstride];
            const C64 ua = bufA[i0], va = cmul(w, bufA[i1]);
            bufA[i0] = cadd(ua, va);
            bufA[i1] = csub(ua, va);
            const C64 ue = bufE[i0], ve = cmul(w, bufE[i1]);
            bufE[i0] = cadd(ue, ve);
            bufE[i1] = csub(ue, ve);
        }
        __syncwarp();
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kWarps64 * 32) loglik64_kernel(
    const gb_window_t* __restrict__ wins, const Tile* __restrict__ tiles, TabSet64 tabs,
    const C64* __restrict__ tw_g, double T, double fstar, const C64* __restrict__ dA,
    const C64* __restrict__ dE, const double* __restrict__ wA, const double* __restrict__ wE,
    const double* __restrict__ theta, double* __restrict__ logL, double* __restrict__ dh_out,
    double* __restrict__ hh_out, int* status, int n_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C64* tw = (C64*)smem_raw;                                   // kTwiddles
    double* red = (double*)(tw + kTwiddles);                    // kWarps64
    Cand64* cands = (Cand64*)(red + kWarps64);                  // kWarps64 * 32
    C64* bufs = (C64*)(cands + kWarps64 * 32);                  // kWarps64 * 2 * n_max

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile tile = tiles[blockIdx.x];
    const gb_window_t win = wins[tile.win];
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];

    // <d|d> over the window, block-wide (fixed order -> deterministic)
    double acc = 0.0;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const C64 a = dA[win.data_off + i], e = dE[win.data_off + i];
        acc += wA[win.data_off + i] * (a.x * a.x + a.y * a.y) + wE[win.data_off + i] * (e.x * e.x + e.y * e.y);
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    double dd = 0.0;
    for (int w = 0; w < kWarps64; ++w) dd += red[w];
    dd *= 4.0 / T;

    Geo64 g;
    g.N = win.N;
    g.logN = 31 - __clz(win.N);
    g.T = T;
    g.T_over_N = T / (double)win.N;
    g.fstar = fstar;
    g.scale = T / (2.0 * (double)win.N);
    const OrbitTables64 tab = tabs.t[g.logN - 5];
    C64* bufA = bufs + (size_t)warp * 2 * n_max;
    C64* bufE = bufA + n_max;
    Cand64* mycand = cands + warp * 32;

    const int64_t tlen = tile.c_end - tile.c_begin;
    const int64_t grp = (tlen + kWarps64 - 1) / kWarps64;   // <= 32
    const int64_t c_lo = tile.c_begin + (int64_t)warp * grp;
    const int64_t c_hi = min(tile.c_end, c_lo + grp);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup64(theta + 8 * (c_lo + lane), T, mycand[lane]);
    __syncwarp();
    const int64_t half = win.N / 2;
    for (int64_t cidx = c_lo; cidx < c_hi; ++cidx) {
        const Cand64& c = mycand[cidx - c_lo];
        if (c.bad) {
            if (lane == 0) {
                logL[cidx] = nan("");
                if (dh_out) dh_out[cidx] = nan("");
                if (hh_out) hh_out[cidx] = nan("");
                atomicOr(status, kStatusNonFinite);
            }
            continue;
        }
        template64(c, g, tab, tw, bufA, bufE, lane);
        double sdh = 0.0, shh = 0.0;
        for (int m = lane; m < win.N; m += 32) {
            const int64_t kk = c.q - half + m - win.k0;
            if (kk >= 0 && kk < win.W) {
                const int idx = (m + (int)half) & (win.N - 1);
                const C64 hA = cscale(bufA[idx], g.scale), hE = cscale(bufE[idx], g.scale);
                const C64 a = dA[win.data_off + kk], e = dE[win.data_off + kk];
                const double wa = wA[win.data_off + kk], we = wE[win.data_off + kk];
                sdh += wa * (a.x * hA.x + a.y * hA.y) + we * (e.x * hE.x + e.y * hE.y);
                shh += wa * (hA.x * hA.x + hA.y * hA.y) + we * (hE.x * hE.x + hE.y * hE.y);
            }
        }
        sdh = warp_sum(sdh) * (4.0 / T);
        shh = warp_sum(shh) * (4.0 / T);
        if (lane == 0) {
            logL[cidx] = sdh - 0.5 * shh - 0.5 * dd;
            if (dh_out) dh_out[cidx] = sdh;
            if (hh_out) hh_out[cidx] = shh;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kWarps64 * 32) waveform64_kernel(
    OrbitTables64 tab, const C64* __restrict__ tw_g, double T, double fstar, int N,
    const double* __restrict__ theta, int64_t B, int group, C64* __restrict__ hA, C64* __restrict__ hE,
    int64_t* __restrict__ q_out, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C64* tw = (C64*)smem_raw;
    Cand64* cands = (Cand64*)(tw + kTwiddles);
    C64* bufs = (C64*)(cands + kWarps64 * 32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];
    __syncthreads();
    Geo64 g;
    g.N = N;
    g.logN = 31 - __clz(N);
    g.T = T;
    g.T_over_N = T / (double)N;
    g.fstar = fstar;
    g.scale = T / (2.0 * (double)N);
    C64* bufA = bufs + (size_t)warp * 2 * N;
    C64* bufE = bufA + N;
    Cand64* mycand = cands + warp * 32;
    const int64_t c_lo = ((int64_t)blockIdx.x * kWarps64 + warp) * group;
    const int64_t c_hi = min(B, c_lo + group);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup64(theta + 8 * (c_lo + lane), T, mycand[lane]);
    __syncwarp();
    for (int64_t b = c_lo; b < c_hi; ++b) {
        const Cand64& c = mycand[b - c_lo];
        C64* outA = hA + b * N;
        C64* outE = hE + b * N;
        if (c.bad) {
            for (int m = lane; m < N; m += 32) outA[m] = outE[m] = C64{nan(""), nan("")};
            if (lane == 0) {
                q_out[b] = 0;
                atomicOr(status, kStatusNonFinite);
            }
            continue;
        }
        template64(c, g, tab, tw, bufA, bufE, lane);
        for (int m = lane; m < N; m += 32) {
            const int idx = (m + N / 2) & (N - 1);
            outA[m] = cscale(bufA[idx], g.scale);
            outE[m] = cscale(bufE[idx], g.scale);
        }
        if (lane == 0) q_out[b] = c.q;
        __syncwarp();
    }
}

}  // namespace

static size_t smem64_loglik(int n_max) {
    return sizeof(C64) * kTwiddles + sizeof(double) * kWarps64 + sizeof(Cand64) * kWarps64 * 32 +
           sizeof(C64) * kWarps64 * 2 * (size_t)n_max;
}

int launch_loglik_fp64(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE,
                       const double* wA, const double* wE, const double* theta, double* logL,
                       double* dh, double* hh, cudaStream_t s) {
    if (plan.n_tiles == 0) return GB_OK;
    const size_t smem = smem64_loglik(plan.n_max);
    cudaError_t e = cudaFuncSetAttribute(loglik64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik64: smem attribute");
    loglik64_kernel<<<plan.n_tiles, kWarps64 * 32, smem, s>>>(
        plan.d_win, plan.d_tiles, tabset64(ctx), (const C64*)ctx->d_tw64, ctx->obs.T_obs,
        transfer_frequency(ctx), (const C64*)dA, (const C64*)dE, wA, wE, theta, logL, dh, hh,
        ctx->d_status, plan.n_max);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik64 launch");
    return GB_OK;
}

int launch_waveform_fp64(gb_ctx* ctx, const double* theta, int64_t B, int N, double* hA, double* hE,
                         int64_t* q, cudaStream_t s) {
    if (B == 0) return GB_OK;
    const size_t smem = sizeof(C64) * kTwiddles + sizeof(Cand64) * kWarps64 * 32 +
                        sizeof(C64) * kWarps64 * 2 * (size_t)N;
    cudaError_t e = cudaFuncSetAttribute(waveform64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform64: smem attribute");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int64_t group = (B + (int64_t)sms * kWarps64 * 2 - 1) / ((int64_t)sms * kWarps64 * 2);
    group = group < 1 ? 1 : group > 32 ? 32 : group;
    const int64_t blocks = (B + group * kWarps64 - 1) / (group * kWarps64);
    waveform64_kernel<<<(unsigned)blocks, kWarps64 * 32, smem, s>>>(
        tables64(ctx, N), (const C64*)ctx->d_tw64, ctx->obs.T_obs, transfer_frequency(ctx), N,
        theta, B, (int)group, (C64*)hA, (C64*)hE, q, ctx->d_status);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform64 launch");
    return GB_OK;
}

}  // namespace gb
