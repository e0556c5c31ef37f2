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
    double u[3], v[3];    // polarisation basis (psi = 0)
    double gpr, gxr, gpi, gxi;   // n.H.n = (gpr Fp + gxr Fx) + i (gpi Fp + gxi Fx), Fp = (n.u)^2 - (n.v)^2, Fx = 2 (n.u)(n.v)
    double f0, fd, delta, phi0c, A;   // phi0c = phi0 / (2 pi)
    double D0r, D0i;      // exp(-i f0 / f*)
    double eps;           // fdot / f*
    long long q;
    int bad;
    int J;                // degree of the link-transfer series (0: direct evaluation)
};

struct Geo64 {
    double T, T_over_N, inv_fstar, scale;   // scale = T / (2N)
    int N, logN;
};

// 1/k!, k < 35: the link-transfer series
__constant__ double kInvFact64[35] = {
    1.00000000000000000e+00, 1.00000000000000000e+00, 5.00000000000000000e-01, 1.66666666666666657e-01,
    4.16666666666666644e-02, 8.33333333333333322e-03, 1.38888888888888894e-03, 1.98412698412698413e-04,
    2.48015873015873016e-05, 2.75573192239858925e-06, 2.75573192239858883e-07, 2.50521083854417202e-08,
    2.08767569878681002e-09, 1.60590438368216133e-10, 1.14707455977297245e-11, 7.64716373181981641e-13,
    4.77947733238738525e-14, 2.81145725434552060e-15, 1.56192069685862253e-16, 8.22063524662432950e-18,
    4.11031762331216484e-19, 1.95729410633912626e-20, 8.89679139245057408e-22, 3.86817017063068413e-23,
    1.61173757109611839e-24, 6.44695028438447359e-26, 2.47959626322479759e-27, 9.18368986379554601e-29,
    3.27988923706983776e-30, 1.13099628864477159e-31, 3.76998762881590539e-33, 1.21612504155351789e-34,
    3.80039075485474342e-36, 1.15163356207719509e-37, 3.38715753552116180e-39};

// Candidate setup (one lane, one candidate).  The carrier bin uses explicit
// round-to-nearest operations so that q is bit-identical to any IEEE
// evaluation of ((f0*T) + ((0.5*fdot)*T)*T) + 0.5.
__device__ void setup64(const double* th, double T, double inv_fstar, Cand64& c) {
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
    c.phi0c = phi0 * 0.15915494309189535;   // 1 / (2 pi)
    c.A = A;
    double sb, cb, sl, cl, s2, c2;
    sincos(beta, &sb, &cb);
    sincos(lam, &sl, &cl);
    sincos(2.0 * psi, &s2, &c2);
    const double ci = cos(iota);
    c.k[0] = -(cb * cl);
    c.k[1] = -(cb * sl);
    c.k[2] = -sb;
    c.u[0] = sb * cl;
    c.u[1] = sb * sl;
    c.u[2] = -cb;
    c.v[0] = sl;
    c.v[1] = -cl;
    c.v[2] = 0.0;
    // H = A+ E+(psi) - i Ax Ex(psi) with E+ = u u - v v and Ex = u v + v u rotated
    // by 2 psi: n.H.n = A+ (c2 Fp - s2 Fx) - i Ax (s2 Fp + c2 Fx)
    const double Ap = A * (1.0 + ci * ci);
    const double Ax = -2.0 * A * ci;
    c.gpr = Ap * c2;
    c.gxr = -(Ap * s2);
    c.gpi = -(Ax * s2);
    c.gxi = -(Ax * c2);
    // link-transfer series degree: first omitted term below 1e-17 for the
    // largest argument X = f (1 + |k.n|)/(2 f*) <= f_max / f*
    const double xmax = fmax(fabs(f0), fabs(f0 + fd * T)) * inv_fstar;
    c.J = xmax <= 0.22 ? 6 : xmax <= 0.5 ? 8 : xmax <= 1.3 ? 12 : xmax <= 2.35 ? 16 : 0;
    double sD, cD;
    sincos(f0 * inv_fstar, &sD, &cD);
    c.D0r = cD;
    c.D0i = -sD;
    c.eps = fd * inv_fstar;
}

// n.H.n for a unit arm vector n
__device__ __forceinline__ C64 nHn(const Cand64& c, double nx, double ny, double nz) {
    const double nu = c.u[0] * nx + c.u[1] * ny + c.u[2] * nz;
    const double nv = c.v[0] * nx + c.v[1] * ny;
    const double Fp = (nu - nv) * (nu + nv), Fx = 2.0 * nu * nv;
    return {c.gpr * Fp + c.gxr * Fx, c.gpi * Fp + c.gxi * Fx};
}

// sinc(X) exp(-iX): J+1 terms of the series of (1 - e^{-2iX})/(2iX) split into
// real and imaginary parts (Horner in y = -4X^2); J = 0: direct evaluation
template <int J>
__device__ __forceinline__ C64 transfer64(double X) {
    if constexpr (J == 0) {
        double sX, cX;
        sincos(X, &sX, &cX);
        const double sinc = (X != 0.0) ? sX / X : 1.0;
        return {sinc * cX, -(sinc * sX)};
    } else {
        const double y = -4.0 * X * X;
        double re = kInvFact64[2 * J + 1], im = kInvFact64[2 * J + 2];
#pragma unroll
        for (int j = J - 1; j >= 0; --j) {
            re = fma(re, y, kInvFact64[2 * j + 1]);
            im = fma(im, y, kInvFact64[2 * j + 2]);
        }
        return {re, -2.0 * X * im};
    }
}

// -i a sinc(X) exp(-iX) G exp(i Psi)
template <int J>
__device__ __forceinline__ C64 link64(double a, double X, C64 G, C64 rx) {
    const C64 t = transfer64<J>(X);
    const C64 tr = {a * t.x, a * t.y};
    const C64 z = cmul(cmul(tr, G), rx);
    return {z.y, -z.x};                                    // times -i
}

// Slow part of one candidate into buf{A,E} at bit-reversed positions, then
// an in-place radix-2 FFT -> natural-order DFT S_k, k = 0..N-1.  The receiver
// phases reach ~1e6 rad; taken in cycles and reduced modulo one first, their
// sines come from a short argument.
// bufT (may be null): also T = (X + Y + Z)/sqrt3
// NT threads share the candidate (NT = 32: one warp, `lane` its lane; NT > 32:
// the whole CTA, `lane` the thread index); each sample and each butterfly is
// computed by the same code whichever thread takes it, so the bits do not
// depend on NT.
template <int NT>
__device__ __forceinline__ void sync_nt() {
    if (NT == 32) __syncwarp();
    else __syncthreads();
}

template <int J, int NT>
__device__ void template64(const Cand64& c, const Geo64& g, const OrbitTables64& tab, const C64* tw,
                           C64* bufA, C64* bufE, C64* bufT, int lane) {
    const int N = g.N;
    const double inv_c = 1.0 / kC;
    const double u_step = 1.0 / (double)N;   // t/T = n/N exactly
    for (int n = lane; n < N; n += NT) {
        const double t = (double)n * g.T_over_N;
        C64 rx[3];
        for (int j = 0; j < 3; ++j) {
            const double kap = (c.k[0] * tab.x[(j * 3 + 0) * N + n] + c.k[1] * tab.x[(j * 3 + 1) * N + n] +
                                c.k[2] * tab.x[(j * 3 + 2) * N + n]) * inv_c;
            // receiver phase in cycles, reduced modulo one before the sine and cosine
            double cyc = c.delta * ((double)n * u_step) + 0.5 * c.fd * (t * t) - c.f0 * kap - c.fd * t * kap +
                         0.5 * c.fd * (kap * kap) + c.phi0c;
            cyc -= rint(cyc);
            double s, co;
            sincospi(2.0 * cyc, &s, &co);
            rx[j] = {co, s};
        }
        const double f = c.f0 + c.fd * t;
        const double a = f * (0.5 * g.inv_fstar);
        C64 z01, z10, z12, z21, z20, z02;
        {
            const double nx = tab.arm[0 * N + n], ny = tab.arm[1 * N + n], nz = tab.arm[2 * N + n];
            const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
            const C64 G = nHn(c, nx, ny, nz);
            z01 = link64<J>(a, a * (1.0 - kn), G, rx[1]);
            z10 = link64<J>(a, a * (1.0 + kn), G, rx[0]);
        }
        {
            const double nx = tab.arm[3 * N + n], ny = tab.arm[4 * N + n], nz = tab.arm[5 * N + n];
            const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
            const C64 G = nHn(c, nx, ny, nz);
            z12 = link64<J>(a, a * (1.0 - kn), G, rx[2]);
            z21 = link64<J>(a, a * (1.0 + kn), G, rx[1]);
        }
        {
            const double nx = tab.arm[6 * N + n], ny = tab.arm[7 * N + n], nz = tab.arm[8 * N + n];
            const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
            const C64 G = nHn(c, nx, ny, nz);
            z20 = link64<J>(a, a * (1.0 - kn), G, rx[0]);
            z02 = link64<J>(a, a * (1.0 + kn), G, rx[2]);
        }
        // D = exp(-i f/f*) = exp(-i f0/f*) exp(-i th), th = fdot t / f*: a short
        // series while |th| <= 1/64 (terms to th^7, first omitted below 1e-19)
        C64 D;
        const double th = c.eps * t;
        if (fabs(th) <= 0.015625) {
            const double t2 = th * th;
            const double cs = fma(fma(fma(t2, -1.0 / 720.0, 1.0 / 24.0), t2, -0.5), t2, 1.0);
            const double sn = th * fma(fma(fma(t2, -1.0 / 5040.0, 1.0 / 120.0), t2, -1.0 / 6.0), t2, 1.0);
            D = cmul({c.D0r, c.D0i}, {cs, -sn});
        } else {
            double sD, cD;
            sincos(f * g.inv_fstar, &sD, &cD);
            D = {cD, -sD};
        }
        const C64 D2 = cmul(D, D);
        const C64 omd = {1.0 - D2.x, -D2.y};
        const C64 X = cmul(omd, csub(cadd(z10, cmul(D, z01)), cadd(z20, cmul(D, z02))));
        const C64 Y = cmul(omd, csub(cadd(z21, cmul(D, z12)), cadd(z01, cmul(D, z10))));
        const C64 Z = cmul(omd, csub(cadd(z02, cmul(D, z20)), cadd(z12, cmul(D, z21))));
        const double r2 = 0.70710678118654752, r6 = 0.40824829046386302;   // 1/sqrt(2), 1/sqrt(6)
        const C64 sA = {(Z.x - X.x) * r2, (Z.y - X.y) * r2};
        const C64 sE = {(X.x - 2.0 * Y.x + Z.x) * r6, (X.y - 2.0 * Y.y + Z.y) * r6};
        const int br = (int)(__brev((unsigned)n) >> (32 - g.logN));
        bufA[br] = sA;
        bufE[br] = sE;
        if (bufT) {
            const double r3 = 0.57735026918962576;   // 1/sqrt(3)
            bufT[br] = {(X.x + Y.x + Z.x) * r3, (X.y + Y.y + Z.y) * r3};
        }
    }
    sync_nt<NT>();
    // radix-2 decimation in time, bit-reversed input, natural-order output
    for (int s = 0; s < g.logN; ++s) {
        const int h = 1 << s;
        const int tstride = kTwiddles >> s;
        for (int b = lane; b < N / 2; b += NT) {
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
            if (bufT) {
                const C64 ut = bufT[i0], vt = cmul(w, bufT[i1]);
                bufT[i0] = cadd(ut, vt);
                bufT[i1] = csub(ut, vt);
            }
        }
        sync_nt<NT>();
    }
}

template <int NT = 32>
__device__ void template64_dispatch(const Cand64& c, const Geo64& g, const OrbitTables64& tab, const C64* tw,
                                    C64* bufA, C64* bufE, C64* bufT, int lane) {
    switch (c.J) {
        case 6: template64<6, NT>(c, g, tab, tw, bufA, bufE, bufT, lane); break;
        case 8: template64<8, NT>(c, g, tab, tw, bufA, bufE, bufT, lane); break;
        case 12: template64<12, NT>(c, g, tab, tw, bufA, bufE, bufT, lane); break;
        case 16: template64<16, NT>(c, g, tab, tw, bufA, bufE, bufT, lane); break;
        default: template64<0, NT>(c, g, tab, tw, bufA, bufE, bufT, lane); break;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// <d|d> of window `win` over the whole block, in a fixed order (deterministic);
// every thread returns the same value.  `red` holds kWarps64 doubles.
__device__ __forceinline__ double window_dd64(const gb_window_t& win, bool useT, const C64* __restrict__ dA,
                                              const C64* __restrict__ dE, const double* __restrict__ wA,
                                              const double* __restrict__ wE, const C64* __restrict__ dT,
                                              const double* __restrict__ wT, double T, double* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const C64 a = dA[win.data_off + i], e = dE[win.data_off + i];
        acc += wA[win.data_off + i] * (a.x * a.x + a.y * a.y) + wE[win.data_off + i] * (e.x * e.x + e.y * e.y);
        if (useT) {
            const C64 t = dT[win.data_off + i];
            acc += wT[win.data_off + i] * (t.x * t.x + t.y * t.y);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    double dd = 0.0;
    for (int w = 0; w < kWarps64; ++w) dd += red[w];
    return dd * (4.0 / T);
}

// Window inner products of one computed template (one warp, in a fixed
// order) and Eq. 2; lane 0 writes output row `row`.
__device__ __forceinline__ void ip64(const Cand64& c, int64_t row, const Geo64& g, const C64* bufA, const C64* bufE,
                                     const C64* bufT, const gb_window_t& win, double dd, const C64* __restrict__ dA,
                                     const C64* __restrict__ dE, const double* __restrict__ wA,
                                     const double* __restrict__ wE, const C64* __restrict__ dT,
                                     const double* __restrict__ wT, double* __restrict__ logL,
                                     double* __restrict__ dh_out, double* __restrict__ hh_out,
                                     double* __restrict__ dhi_out, int lane) {
    const double T = g.T;
    const int64_t half = win.N / 2;
    double sdh = 0.0, shh = 0.0, sdhi = 0.0;
    for (int m = lane; m < win.N; m += 32) {
        const int64_t kk = c.q - half + m - win.k0;
        if (kk >= 0 && kk < win.W) {
            const int idx = (m + (int)half) & (win.N - 1);
            const C64 hA = cscale(bufA[idx], g.scale), hE = cscale(bufE[idx], g.scale);
            const C64 a = dA[win.data_off + kk], e = dE[win.data_off + kk];
            const double wa = wA[win.data_off + kk], we = wE[win.data_off + kk];
            sdh += wa * (a.x * hA.x + a.y * hA.y) + we * (e.x * hE.x + e.y * hE.y);
            shh += wa * (hA.x * hA.x + hA.y * hA.y) + we * (hE.x * hE.x + hE.y * hE.y);
            if (dhi_out) sdhi += wa * (a.y * hA.x - a.x * hA.y) + we * (e.y * hE.x - e.x * hE.y);
            if (bufT) {
                const C64 hT = cscale(bufT[idx], g.scale), t = dT[win.data_off + kk];
                const double wt = wT[win.data_off + kk];
                sdh += wt * (t.x * hT.x + t.y * hT.y);
                shh += wt * (hT.x * hT.x + hT.y * hT.y);
                if (dhi_out) sdhi += wt * (t.y * hT.x - t.x * hT.y);
            }
        }
    }
    sdh = warp_sum(sdh) * (4.0 / T);
    shh = warp_sum(shh) * (4.0 / T);
    if (dhi_out) sdhi = warp_sum(sdhi) * (4.0 / T);
    if (lane == 0) {
        logL[row] = sdh - 0.5 * shh - 0.5 * dd;
        if (dh_out) dh_out[row] = sdh;
        if (hh_out) hh_out[row] = shh;
        if (dhi_out) dhi_out[row] = sdhi;
    }
}

// NaN outputs of a candidate with a non-finite parameter (one thread)
__device__ __forceinline__ void bad64(int64_t row, double* logL, double* dh_out, double* hh_out, double* dhi_out,
                                      int* status) {
    logL[row] = nan("");
    if (dh_out) dh_out[row] = nan("");
    if (hh_out) hh_out[row] = nan("");
    if (dhi_out) dhi_out[row] = nan("");
    atomicOr(status, kStatusNonFinite);
}

// One candidate (one warp): template, window inner products and Eq. 2; lane 0
// writes output row `row`.
__device__ __forceinline__ void eval64(const Cand64& c, int64_t row, const Geo64& g, const OrbitTables64& tab,
                                       const C64* tw, C64* bufA, C64* bufE, C64* bufT, const gb_window_t& win,
                                       double dd, const C64* __restrict__ dA, const C64* __restrict__ dE,
                                       const double* __restrict__ wA, const double* __restrict__ wE,
                                       const C64* __restrict__ dT, const double* __restrict__ wT,
                                       double* __restrict__ logL, double* __restrict__ dh_out,
                                       double* __restrict__ hh_out, double* __restrict__ dhi_out, int* status,
                                       int lane) {
    if (c.bad) {
        if (lane == 0) bad64(row, logL, dh_out, hh_out, dhi_out, status);
        return;
    }
    template64_dispatch(c, g, tab, tw, bufA, bufE, bufT, lane);
    ip64(c, row, g, bufA, bufE, bufT, win, dd, dA, dE, wA, wE, dT, wT, logL, dh_out, hh_out, dhi_out, lane);
    __syncwarp();
}

__device__ __forceinline__ Geo64 geometry64(int N, double T, double fstar) {
    Geo64 g;
    g.N = N;
    g.logN = 31 - __clz(N);
    g.T = T;
    g.T_over_N = T / (double)N;
    g.inv_fstar = 1.0 / fstar;
    g.scale = T / (2.0 * (double)N);
    return g;
}

// ROWS = false: one CTA per plan tile, the tile's candidates split over the
// warps.  ROWS = true: blockIdx.x is a window and its candidates are the rows
// listed in rows[cand_off + j], j in [row_lo[w], row_hi[w]) (device lists);
// the gridDim.y CTAs of a window take them one at a time (few rows, each
// spread over a CTA, for latency).
template <bool ROWS>
__global__ void __launch_bounds__(kWarps64 * 32) loglik64_kernel(
    const gb_window_t* __restrict__ wins, const Tile* __restrict__ tiles, TabSet64 tabs,
    const C64* __restrict__ tw_g, double T, double fstar, const C64* __restrict__ dA,
    const C64* __restrict__ dE, const double* __restrict__ wA, const double* __restrict__ wE,
    const double* __restrict__ theta, double* __restrict__ logL, double* __restrict__ dh_out,
    double* __restrict__ hh_out, double* __restrict__ dhi_out, const C64* __restrict__ dT,
    const double* __restrict__ wT, int* status, int n_max, const int32_t* __restrict__ rows,
    const int32_t* __restrict__ row_lo, const int32_t* __restrict__ row_hi, const int* __restrict__ gate) {
    if (ROWS && gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C64* tw = (C64*)smem_raw;                                   // kTwiddles
    double* red = (double*)(tw + kTwiddles);                    // kWarps64
    Cand64* cands = (Cand64*)(red + kWarps64);                  // kWarps64 * 32
    C64* bufs = (C64*)(cands + kWarps64 * 32);                  // kWarps64 * (2 or 3) * n_max
    const int nch = dT ? 3 : 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Tile tile{};
    int lo = 0, hi = 0;
    if (ROWS) {
        tile.win = blockIdx.x;
    } else {
        tile = tiles[blockIdx.x];
    }
    const gb_window_t win = wins[tile.win];
    if (ROWS) {
        lo = max(row_lo[tile.win], 0);
        hi = min(row_hi[tile.win], win.n_cand);
        if (lo >= hi) return;                                   // nothing listed (block-uniform)
    }
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];

    // T enters windows whose lowest frequency is at least f*/2
    const bool useT = dT != nullptr && (double)win.k0 / T >= 0.5 * fstar;
    const double dd = window_dd64(win, useT, dA, dE, wA, wE, dT, wT, T, red);

    const Geo64 g = geometry64(win.N, T, fstar);
    const OrbitTables64 tab = tabs.t[g.logN - 5];
    C64* bufA = bufs + (size_t)warp * nch * n_max;
    C64* bufE = bufA + n_max;
    C64* bufT = useT ? bufE + n_max : nullptr;
    Cand64* mycand = cands + warp * 32;

    if (!ROWS) {
        const int64_t tlen = tile.c_end - tile.c_begin;
        const int64_t grp = (tlen + kWarps64 - 1) / kWarps64;   // <= 32
        const int64_t c_lo = tile.c_begin + (int64_t)warp * grp;
        const int64_t c_hi = min(tile.c_end, c_lo + grp);
        if (c_lo >= c_hi) return;
        if (c_lo + lane < c_hi) setup64(theta + 8 * (c_lo + lane), T, g.inv_fstar, mycand[lane]);
        __syncwarp();
        for (int64_t cidx = c_lo; cidx < c_hi; ++cidx)
            eval64(mycand[cidx - c_lo], cidx, g, tab, tw, bufA, bufE, bufT, win, dd, dA, dE, wA, wE, dT, wT, logL,
                   dh_out, hh_out, dhi_out, status, lane);
    } else {
        // one listed row at a time for the whole CTA (entries lo + y, lo + y
        // + Y, ... for CTA y of the window's Y): the template over all the
        // CTA's threads, the inner products in warp 0 in a warp's order
        C64* cA = bufs;
        C64* cE = bufs + n_max;
        for (int slot = lo + (int)blockIdx.y; slot < hi; slot += (int)gridDim.y) {
            const int64_t row = rows[win.cand_off + slot];
            if (row < win.cand_off || row >= win.cand_off + win.n_cand) continue;   // not this window's row
            if (threadIdx.x == 0) setup64(theta + 8 * row, T, g.inv_fstar, cands[0]);
            __syncthreads();
            if (cands[0].bad) {
                if (threadIdx.x == 0) bad64(row, logL, dh_out, hh_out, dhi_out, status);
            } else {
                template64_dispatch<kWarps64 * 32>(cands[0], g, tab, tw, cA, cE, nullptr, threadIdx.x);
                if (warp == 0)
                    ip64(cands[0], row, g, cA, cE, nullptr, win, dd, dA, dE, wA, wE, nullptr, nullptr, logL, dh_out,
                         hh_out, dhi_out, lane);
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kWarps64 * 32) waveform64_kernel(
    OrbitTables64 tab, const C64* __restrict__ tw_g, double T, double fstar, int N,
    const double* __restrict__ theta, int64_t B, int group, C64* __restrict__ hA, C64* __restrict__ hE,
    C64* __restrict__ hT, int64_t* __restrict__ q_out, int* status) {
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
    g.inv_fstar = 1.0 / fstar;
    g.scale = T / (2.0 * (double)N);
    C64* bufA = bufs + (size_t)warp * (hT ? 3 : 2) * N;
    C64* bufE = bufA + N;
    C64* bufT = hT ? bufE + N : nullptr;
    Cand64* mycand = cands + warp * 32;
    const int64_t c_lo = ((int64_t)blockIdx.x * kWarps64 + warp) * group;
    const int64_t c_hi = min(B, c_lo + group);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup64(theta + 8 * (c_lo + lane), T, g.inv_fstar, mycand[lane]);
    __syncwarp();
    for (int64_t b = c_lo; b < c_hi; ++b) {
        const Cand64& c = mycand[b - c_lo];
        C64* outA = hA + b * N;
        C64* outE = hE + b * N;
        if (c.bad) {
            for (int m = lane; m < N; m += 32) {
                outA[m] = outE[m] = C64{nan(""), nan("")};
                if (hT) hT[b * N + m] = C64{nan(""), nan("")};
            }
            if (lane == 0) {
                q_out[b] = 0;
                atomicOr(status, kStatusNonFinite);
            }
            continue;
        }
        template64_dispatch(c, g, tab, tw, bufA, bufE, bufT, lane);
        for (int m = lane; m < N; m += 32) {
            const int idx = (m + N / 2) & (N - 1);
            outA[m] = cscale(bufA[idx], g.scale);
            outE[m] = cscale(bufE[idx], g.scale);
            if (hT) hT[b * N + m] = cscale(bufT[idx], g.scale);
        }
        if (lane == 0) q_out[b] = c.q;
        __syncwarp();
    }
}

// Window inner product <x|y> = (4/T) Re sum_k w_k x_k y_k* of two templates
// (or data, y) over the window's bins, block-wide in a fixed order.  A
// template is given by its natural-order buffers (scaled by `sc`) and carrier
// bin; bins it does not reach count zero.  `red` holds kWarps64 doubles.
struct WinTpl {
    const C64* A;
    const C64* E;
    long long q;
    double sc;
};
__device__ __forceinline__ C64 tpl_at(const WinTpl& t, int N, long long k) {
    const long long m = k - (t.q - N / 2);
    if (m < 0 || m >= N) return {0.0, 0.0};
    const int idx = (int)((m + N / 2) & (N - 1));
    return {t.sc * t.A[idx].x, t.sc * t.A[idx].y};
}
__device__ __forceinline__ C64 tpl_at_e(const WinTpl& t, int N, long long k) {
    const long long m = k - (t.q - N / 2);
    if (m < 0 || m >= N) return {0.0, 0.0};
    const int idx = (int)((m + N / 2) & (N - 1));
    return {t.sc * t.E[idx].x, t.sc * t.E[idx].y};
}
__device__ double block_sum64(double v, double* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kWarps64; ++w) s += red[w];
    return s;
}
// <x|y> with x a template and y a template (yt) or the data (yt == nullptr)
__device__ double win_inner(const WinTpl& x, const WinTpl* yt, const gb_window_t& win, const C64* __restrict__ dA,
                            const C64* __restrict__ dE, const double* __restrict__ wA, const double* __restrict__ wE,
                            double T, double* red) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const long long k = win.k0 + i;
        const C64 xa = tpl_at(x, win.N, k), xe = tpl_at_e(x, win.N, k);
        C64 ya, ye;
        if (yt) {
            ya = tpl_at(*yt, win.N, k);
            ye = tpl_at_e(*yt, win.N, k);
        } else {
            ya = dA[win.data_off + i];
            ye = dE[win.data_off + i];
        }
        acc += wA[win.data_off + i] * (xa.x * ya.x + xa.y * ya.y) + wE[win.data_off + i] * (xe.x * ye.x + xe.y * ye.y);
    }
    return block_sum64(acc, red) * (4.0 / T);
}

// Gram matrix G_ij = <s_i|s_j>, b_i = <d|s_i> and the multi-signal SNR
// rho = sum_i b_i / sqrt(sum_ij G_ij) (Eq. 11) of each window's sources (one
// CTA per window; the sources are the window's candidate rows).  Template i
// is held in buffer P while the templates j > i pass through buffer Q.
__global__ void __launch_bounds__(kWarps64 * 32) multi_gram_kernel(
    const gb_window_t* __restrict__ wins, TabSet64 tabs, const C64* __restrict__ tw_g, double T, double fstar,
    const C64* __restrict__ dA, const C64* __restrict__ dE, const double* __restrict__ wA,
    const double* __restrict__ wE, const double* __restrict__ theta, int kmax, double* __restrict__ gram,
    double* __restrict__ dh_out, double* __restrict__ rho_out, int* status, int n_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C64* tw = (C64*)smem_raw;                   // kTwiddles
    double* red = (double*)(tw + kTwiddles);    // kWarps64
    Cand64* cand = (Cand64*)(red + kWarps64);   // 2
    C64* PA = (C64*)(cand + 2);                 // 4 buffers of n_max
    C64* PE = PA + n_max;
    C64* QA = PE + n_max;
    C64* QE = QA + n_max;
    const gb_window_t win = wins[blockIdx.x];
    const int K = win.n_cand;
    double* G = gram + (size_t)blockIdx.x * kmax * kmax;
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];
    const Geo64 g = geometry64(win.N, T, fstar);
    const OrbitTables64 tab = tabs.t[g.logN - 5];
    const bool data = dA != nullptr;
    double sum_b = 0.0, sum_g = 0.0;
    bool bad_any = false;
    for (int i = 0; i < K; ++i) {
        __syncthreads();
        if (threadIdx.x == 0) setup64(theta + 8 * (win.cand_off + i), T, g.inv_fstar, cand[0]);
        __syncthreads();
        const bool bad_i = cand[0].bad;
        if (!bad_i) template64_dispatch<kWarps64 * 32>(cand[0], g, tab, tw, PA, PE, nullptr, threadIdx.x);
        __syncthreads();
        const WinTpl P{PA, PE, cand[0].q, g.scale};
        const double gii = bad_i ? nan("") : win_inner(P, &P, win, dA, dE, wA, wE, T, red);
        const double bi = bad_i || !data ? nan("") : win_inner(P, nullptr, win, dA, dE, wA, wE, T, red);
        if (threadIdx.x == 0) {
            G[i * kmax + i] = gii;
            if (dh_out) dh_out[win.cand_off + i] = bi;
            if (bad_i) atomicOr(status, kStatusNonFinite);
            sum_b += bi;
            sum_g += gii;
            bad_any |= bad_i;
        }
        for (int j = i + 1; j < K; ++j) {
            __syncthreads();
            if (threadIdx.x == 0) setup64(theta + 8 * (win.cand_off + j), T, g.inv_fstar, cand[1]);
            __syncthreads();
            const bool bad_j = cand[1].bad;
            if (!bad_j) template64_dispatch<kWarps64 * 32>(cand[1], g, tab, tw, QA, QE, nullptr, threadIdx.x);
            __syncthreads();
            const WinTpl Q{QA, QE, cand[1].q, g.scale};
            const double gij = bad_i || bad_j ? nan("") : win_inner(P, &Q, win, dA, dE, wA, wE, T, red);
            if (threadIdx.x == 0) {
                G[i * kmax + j] = gij;
                G[j * kmax + i] = gij;
                sum_g += 2.0 * gij;
            }
        }
    }
    if (threadIdx.x == 0 && rho_out)
        rho_out[blockIdx.x] = (K == 0 || bad_any || !data) ? nan("") : sum_b / sqrt(sum_g);
}

}  // namespace

static size_t smem64_loglik(int n_max, int nch) {
    return sizeof(C64) * kTwiddles + sizeof(double) * kWarps64 + sizeof(Cand64) * kWarps64 * 32 +
           sizeof(C64) * kWarps64 * nch * (size_t)n_max;
}

int launch_loglik_fp64(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE,
                       const double* wA, const double* wE, const double* theta, double* logL,
                       double* dh, double* hh, double* dh_im, const double* dT, const double* wT,
                       cudaStream_t s) {
    if (plan.n_tiles == 0) return GB_OK;
    const size_t smem = smem64_loglik(plan.n_max, dT ? 3 : 2);
    cudaError_t e = cudaFuncSetAttribute(loglik64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik64: smem attribute");
    loglik64_kernel<false><<<plan.n_tiles, kWarps64 * 32, smem, s>>>(
        plan.d_win, plan.d_tiles, tabset64(ctx), (const C64*)ctx->d_tw64, ctx->obs.T_obs,
        transfer_frequency(ctx), (const C64*)dA, (const C64*)dE, wA, wE, theta, logL, dh, hh,
        dh_im, (const C64*)dT, wT, ctx->d_status, plan.n_max, nullptr, nullptr, nullptr, nullptr);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik64 launch");
    return GB_OK;
}

int launch_loglik_rows64(gb_ctx* ctx, const gb_window_t* d_win, int n_win, int n_max, int ctas_per_win,
                         const double* dA, const double* dE, const double* wA, const double* wE, const double* theta,
                         const int32_t* rows, const int32_t* row_lo, const int32_t* row_hi, double* logL,
                         double* dh, double* hh, const int* gate, cudaStream_t s) {
    if (n_win == 0) return GB_OK;
    const size_t smem = smem64_loglik(n_max, 2);
    cudaError_t e = cudaFuncSetAttribute(loglik64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik64 rows: smem attribute");
    const dim3 grid((unsigned)n_win, (unsigned)(ctas_per_win < 1 ? 1 : ctas_per_win));
    loglik64_kernel<true><<<grid, kWarps64 * 32, smem, s>>>(
        d_win, nullptr, tabset64(ctx), (const C64*)ctx->d_tw64, ctx->obs.T_obs, transfer_frequency(ctx),
        (const C64*)dA, (const C64*)dE, wA, wE, theta, logL, dh, hh, nullptr, nullptr, nullptr, ctx->d_status,
        n_max, rows, row_lo, row_hi, gate);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik64 rows launch");
    return GB_OK;
}

int launch_waveform_fp64(gb_ctx* ctx, const double* theta, int64_t B, int N, double* hA, double* hE,
                         double* hT, int64_t* q, cudaStream_t s) {
    if (B == 0) return GB_OK;
    const size_t smem = sizeof(C64) * kTwiddles + sizeof(Cand64) * kWarps64 * 32 +
                        sizeof(C64) * kWarps64 * (hT ? 3 : 2) * (size_t)N;
    cudaError_t e = cudaFuncSetAttribute(waveform64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform64: smem attribute");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int64_t group = (B + (int64_t)sms * kWarps64 * 2 - 1) / ((int64_t)sms * kWarps64 * 2);
    group = group < 1 ? 1 : group > 32 ? 32 : group;
    const int64_t blocks = (B + group * kWarps64 - 1) / (group * kWarps64);
    waveform64_kernel<<<(unsigned)blocks, kWarps64 * 32, smem, s>>>(
        tables64(ctx, N), (const C64*)ctx->d_tw64, ctx->obs.T_obs, transfer_frequency(ctx), N,
        theta, B, (int)group, (C64*)hA, (C64*)hE, (C64*)hT, q, ctx->d_status);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform64 launch");
    return GB_OK;
}

int launch_multi_gram(gb_ctx* ctx, const gb_window_t* d_win, int n_win, int n_max, const double* dA,
                      const double* dE, const double* wA, const double* wE, const double* theta, int kmax,
                      double* gram, double* dh, double* rho, cudaStream_t s) {
    if (n_win == 0) return GB_OK;
    const size_t smem = sizeof(C64) * kTwiddles + sizeof(double) * kWarps64 + sizeof(Cand64) * 2 +
                        sizeof(C64) * 4 * (size_t)n_max;
    cudaError_t e = cudaFuncSetAttribute(multi_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "multi_gram: smem attribute");
    multi_gram_kernel<<<n_win, kWarps64 * 32, smem, s>>>(d_win, tabset64(ctx), (const C64*)ctx->d_tw64, ctx->obs.T_obs,
                                                         transfer_frequency(ctx), (const C64*)dA, (const C64*)dE, wA,
                                                         wE, theta, kmax, gram, dh, rho, ctx->d_status, n_max);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "multi_gram launch");
    return GB_OK;
}

}  // namespace gb
