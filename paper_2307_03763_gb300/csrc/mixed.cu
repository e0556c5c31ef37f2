// mixed.cu -- mixed-precision path: the carrier phase and the bin offset keep
// double-precision accuracy (double-word float arithmetic), while the detector
// response, the FFT and the window inner products run in float with
// compensated sums.  Inputs, the per-window <d|d> and every output are double.
//
// Why double-word instead of native double: on GB300 the FP64 pipe issues at
// 1/64 of the FP32 rate, so a native-double phase (about ten operations per
// sample) would cost more than the whole float response.  A double-word
// product with an exact FMA error term costs two or three float operations.
//
// Phase of the receiver-j link, in cycles, at u = t/T = n/N (reading R5):
//   P_j = phi0/2pi + delta u + (fdot T^2/2) u^2 - f0 K(n) - fdot T u K(n)
//         - f rho_j(n) + (fdot/2) (K + rho_j)^2,
//   K(n) = k.x_centre/c = Kc cos(alpha_n) + Ks sin(alpha_n),
//   rho_j = k.(x_j - x_centre)/c,  f = f0 + fdot T u.
// The first four terms can reach hundreds of cycles and are formed in
// double-word arithmetic, each product reduced modulo one exactly; the rest
// are below 0.1 cycle and are float.  exp(2 pi i P_j) is the common factor
// exp(2 pi i P_c) (one accurate sincospi) times exp(2 pi i dP_j) for the
// small per-spacecraft remainder (short Taylor series).
//
// Link transfer a sinc(X) exp(-iX) = a sum_k (-2iX)^k/(k+1)! is evaluated as
// two Horner polynomials in y = -4X^2 (even and odd k), with the number of
// terms chosen per candidate from the largest X = f/f* it can reach.
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kWarpsMx = 4;

struct CandMix {
    float c0h, c0l;     // phi0 / 2pi mod 1
    float c1h, c1l;     // delta
    float c2h, c2l;     // fdot T^2 / 2
    float Fch, Fcl;     // f0 Kc   (cycles)
    float Fsh, Fsl;     // f0 Ks
    float Kc, Ks;       // s
    float k0, k1, k2;   // propagation direction
    float u0, u1, u2;   // polarisation basis
    float v0, v1, v2;
    float gpr, gxr, gpi, gxi;   // G = (gpr F+ + gxr Fx) + i (gpi F+ + gxi Fx), unit amplitude
    float f0, fdT, fdh; // Hz, fdot T [Hz], fdot/2 [Hz/s]
    float a0, a1;       // a = f/(2 f*) = a0 + a1 u
    float D0r, D0i;     // exp(-i f0/f*)
    float eps;          // fdot T / f*
    int J;              // Horner length of the link transfer polynomial (0: direct)
    int bad;
    long long q;
    double A;
};

struct Win32 {
    float2 dA, dE;   // data scaled by sigma
    float wA, wE;    // 1/S scaled by 1/sigma^2
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ void split(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

// 1/k! for the link transfer series (Taylor coefficients of (e^w - 1)/w)
__constant__ float kInvFact[24] = {
    1.0f, 1.0f, 0.5f, 1.6666666666666666e-01f, 4.1666666666666664e-02f, 8.3333333333333332e-03f,
    1.3888888888888889e-03f, 1.9841269841269841e-04f, 2.4801587301587302e-05f, 2.7557319223985893e-06f,
    2.7557319223985888e-07f, 2.5052108385441720e-08f, 2.0876756987868100e-09f, 1.6059043836821613e-10f,
    1.1470745597729725e-11f, 7.6471637318198164e-13f, 4.7794773323873853e-14f, 2.8114572543455206e-15f,
    1.5619206968586225e-16f, 8.2206352466243295e-18f, 4.1103176233121648e-19f, 1.9572941063391263e-20f,
    8.8967913924505741e-22f, 3.8681701706306835e-23f};

__device__ void setup_mixed(const double* th, double T, double fstar, CandMix& c) {
    const double f0 = th[0], fd = th[1], beta = th[2], lam = th[3];
    const double A = th[4], iota = th[5], psi = th[6], phi0 = th[7];
    bool bad = false;
    for (int i = 0; i < 8; ++i) bad |= !isfinite(th[i]);
    c.bad = bad;
    c.A = A;
    const double f0T = __dmul_rn(f0, T);
    const double xm = __dadd_rn(f0T, __dmul_rn(__dmul_rn(__dmul_rn(0.5, fd), T), T));
    const double qd = floor(__dadd_rn(xm, 0.5));
    c.q = bad ? 0 : (long long)qd;
    const double delta = __dadd_rn(f0T, -qd);
    const double inv2pi = 0.15915494309189535;
    double p0 = phi0 * inv2pi;
    p0 -= rint(p0);
    split(p0, c.c0h, c.c0l);
    split(delta, c.c1h, c.c1l);
    split(0.5 * fd * T * T, c.c2h, c.c2l);
    double sb, cb, sl, cl;
    sincos(beta, &sb, &cb);
    sincos(lam, &sl, &cl);
    const double r = kAU / kC;
    const double Kc = -r * cb * cl, Ks = -r * cb * sl;
    c.Kc = (float)Kc;
    c.Ks = (float)Ks;
    split(f0 * Kc, c.Fch, c.Fcl);
    split(f0 * Ks, c.Fsh, c.Fsl);
    const float fsb = (float)sb, fcb = (float)cb, fsl = (float)sl, fcl = (float)cl;
    c.k0 = -fcb * fcl;
    c.k1 = -fcb * fsl;
    c.k2 = -fsb;
    c.u0 = fsb * fcl;
    c.u1 = fsb * fsl;
    c.u2 = -fcb;
    c.v0 = fsl;
    c.v1 = -fcl;
    c.v2 = 0.0f;
    float s2, c2;
    sincosf(2.0f * (float)psi, &s2, &c2);
    const float ci = cosf((float)iota);
    const float Ap = 1.0f + ci * ci, Ax = -2.0f * ci;
    c.gpr = Ap * c2;
    c.gxr = -Ap * s2;
    c.gpi = -Ax * s2;
    c.gxi = -Ax * c2;
    c.f0 = (float)f0;
    c.fdT = (float)(fd * T);
    c.fdh = (float)(0.5 * fd);
    c.a0 = (float)(f0 / (2.0 * fstar));
    c.a1 = (float)(fd * T / (2.0 * fstar));
    float sD, cD;
    sincosf((float)(f0 / fstar), &sD, &cD);
    c.D0r = cD;
    c.D0i = -sD;
    c.eps = (float)(fd * T / fstar);
    // largest link argument X = f (1 + |k.n|)/(2 f*) <= f_max / f*
    const double xmax = fmax(fabs(f0), fabs(f0 + fd * T)) / fstar;
    c.J = xmax <= 0.489 ? 4 : xmax <= 1.34 ? 7 : xmax <= 2.35 ? 10 : 0;
}

// a-free link transfer sinc(X) exp(-iX), J+1 terms of each series
template <int J>
__device__ __forceinline__ float2 link_transfer(float X) {
    if (J == 0) {
        float s, co;
        sincosf(X, &s, &co);
        const float sc = X != 0.0f ? s / X : 1.0f;
        return make_float2(sc * co, -sc * s);
    }
    const float y = -4.0f * X * X;
    float re = kInvFact[2 * J + 1], im = kInvFact[2 * J + 2];
#pragma unroll
    for (int j = J - 1; j >= 0; --j) {
        re = fmaf(re, y, kInvFact[2 * j + 1]);
        im = fmaf(im, y, kInvFact[2 * j + 2]);
    }
    return make_float2(re, -2.0f * X * im);
}

// exp(2 pi i x) for |x| <= 0.125, Taylor series of sin and cos of 2 pi x
__device__ __forceinline__ float2 cis_small(float x) {
    const float t = 6.2831853071795865f * x;
    const float t2 = t * t;
    float s = fmaf(t2, 2.7557319223985893e-06f, -1.9841269841269841e-04f);
    s = fmaf(s, t2, 8.3333333333333332e-03f);
    s = fmaf(s, t2, -1.6666666666666666e-01f);
    s = fmaf(s * t2, t, t);
    float co = fmaf(t2, -2.7557319223985888e-07f, 2.4801587301587302e-05f);
    co = fmaf(co, t2, -1.3888888888888889e-03f);
    co = fmaf(co, t2, 4.1666666666666664e-02f);
    co = fmaf(co, t2, -0.5f);
    co = fmaf(co, t2, 1.0f);
    return make_float2(co, s);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int J>
__device__ void slow_part_mixed(const CandMix& c, const OrbitTables32& tab, int N, int logN, float2* bufA,
                                float2* bufE, int lane) {
    const float invN = 1.0f / (float)N;
    const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f;
    for (int n = lane; n < N; n += 32) {
        const float u = (float)n * invN;
        const float uu = u * u;
        const float cah = __ldg(tab.calpha + n), cal = __ldg(tab.calpha + N + n);
        const float sah = __ldg(tab.salpha + n), sal = __ldg(tab.salpha + N + n);
        // double-word products, reduced modulo one
        float p1 = c.c1h * u;
        const float e1 = fmaf(c.c1h, u, -p1) + c.c1l * u;
        float p2 = c.c2h * uu;
        const float e2 = fmaf(c.c2h, uu, -p2) + c.c2l * uu;
        float p3 = c.Fch * cah;
        const float e3 = fmaf(c.Fch, cah, -p3) + fmaf(c.Fch, cal, c.Fcl * cah);
        float p4 = c.Fsh * sah;
        const float e4 = fmaf(c.Fsh, sah, -p4) + fmaf(c.Fsh, sal, c.Fsl * sah);
        p1 -= rintf(p1);
        p2 -= rintf(p2);
        p3 -= rintf(p3);
        p4 -= rintf(p4);
        float s, e, ea, eb, ec;
        two_sum(c.c0h, p1, s, ea);
        two_sum(s, p2, s, eb);
        two_sum(s, -p3, s, ec);
        two_sum(s, -p4, s, e);
        s -= rintf(s);
        const float K = fmaf(c.Kc, cah, c.Ks * sah);
        const float small = ((c.c0l + e1 + e2 - e3 - e4) + (ea + eb + ec + e)) - c.fdT * u * K;
        // P_c = hi + lo exactly; exp(2 pi i P_c) = exp(2 pi i hi) (1 + 2 pi i lo)
        float Pc, Pl;
        two_sum(s, small, Pc, Pl);
        Pc -= rintf(Pc);
        float sPc, cPc;
        sincospif(2.0f * Pc, &sPc, &cPc);
        const float tl = 6.2831853071795865f * Pl;
        const float2 ePc = make_float2(fmaf(-tl, sPc, cPc), fmaf(tl, cPc, sPc));
        const float f = fmaf(c.fdT, u, c.f0);
        float2 rx[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float rho = fmaf(c.k0, __ldg(tab.rho + (j * 3 + 0) * N + n),
                                   fmaf(c.k1, __ldg(tab.rho + (j * 3 + 1) * N + n),
                                        c.k2 * __ldg(tab.rho + (j * 3 + 2) * N + n)));
            const float kap = K + rho;
            const float dP = fmaf(-f, rho, c.fdh * kap * kap);
            rx[j] = cis_small(dP);   // the common factor exp(2 pi i P_c) is applied once, below
        }
        const float a = fmaf(c.a1, u, c.a0);
        float2 zp[3], zm[3];   // arm a: link along +n (receiver rc[a]) and -n (receiver em[a])
#pragma unroll
        for (int arm = 0; arm < 3; ++arm) {
            const float nx = __ldg(tab.arm + (arm * 3 + 0) * N + n);
            const float ny = __ldg(tab.arm + (arm * 3 + 1) * N + n);
            const float nz = __ldg(tab.arm + (arm * 3 + 2) * N + n);
            const float kn = fmaf(c.k0, nx, fmaf(c.k1, ny, c.k2 * nz));
            const float nu = fmaf(c.u0, nx, fmaf(c.u1, ny, c.u2 * nz));
            const float nv = fmaf(c.v0, nx, fmaf(c.v1, ny, c.v2 * nz));
            const float Fp = (nu - nv) * (nu + nv);
            const float Fx = 2.0f * nu * nv;
            const float2 G = make_float2(fmaf(c.gpr, Fp, c.gxr * Fx), fmaf(c.gpi, Fp, c.gxi * Fx));
            const int rp = arm == 2 ? 0 : arm + 1;   // receiver of the +n link
            const int rm = arm;                      // receiver of the -n link
            zp[arm] = cmulf(cmulf(link_transfer<J>(a * (1.0f - kn)), G), rx[rp]);
            zm[arm] = cmulf(cmulf(link_transfer<J>(a * (1.0f + kn)), G), rx[rm]);
        }
        // links: z01 = zp[0], z10 = zm[0], z12 = zp[1], z21 = zm[1], z20 = zp[2], z02 = zm[2]
        const float du = c.eps * u;
        const float2 Dc = make_float2(fmaf(-0.5f * du, du, 1.0f), -du);
        const float2 D = cmulf(make_float2(c.D0r, c.D0i), Dc);
        const float2 Xp = caddf(csubf(zm[0], zp[2]), cmulf(D, csubf(zp[0], zm[2])));
        const float2 Yp = caddf(csubf(zm[1], zp[0]), cmulf(D, csubf(zp[1], zm[0])));
        const float2 Zp = caddf(csubf(zm[2], zp[1]), cmulf(D, csubf(zp[2], zm[1])));
        // F = -i a (1 - D^2) = 2 a sin(f/f*) D with sin(f/f*) = -Im D: no
        // cancellation in 1 - D^2 at low frequency
        const float sa2 = -2.0f * a * D.y;
        const float2 F = cmulf(make_float2(sa2 * D.x, sa2 * D.y), ePc);
        const float2 Ap = make_float2((Zp.x - Xp.x) * r2, (Zp.y - Xp.y) * r2);
        const float2 Ep = make_float2((Xp.x - 2.0f * Yp.x + Zp.x) * r6, (Xp.y - 2.0f * Yp.y + Zp.y) * r6);
        const int br = (int)(__brev((unsigned)n) >> (32 - logN));
        bufA[br] = cmulf(F, Ap);
        bufE[br] = cmulf(F, Ep);
    }
}

__device__ void fft_mixed(int N, int logN, const float2* tw, float2* bufA, float2* bufE, int lane) {
    __syncwarp();
    for (int s = 0; s < logN; ++s) {
        const int h = 1 << s;
        const int tstride = kTwiddles >> s;
        for (int b = lane; b < N / 2; b += 32) {
            const int j = b & (h - 1);
            const int i0 = ((b >> s) << (s + 1)) + j;
            const int i1 = i0 + h;
            const float2 w = tw[j * tstride];
            const float2 ua = bufA[i0], va = cmulf(w, bufA[i1]);
            bufA[i0] = caddf(ua, va);
            bufA[i1] = csubf(ua, va);
            const float2 ue = bufE[i0], ve = cmulf(w, bufE[i1]);
            bufE[i0] = caddf(ue, ve);
            bufE[i1] = csubf(ue, ve);
        }
        __syncwarp();
    }
}

__device__ void template_mixed(const CandMix& c, const OrbitTables32& tab, int N, int logN, const float2* tw,
                               float2* bufA, float2* bufE, int lane) {
    switch (c.J) {
        case 4: slow_part_mixed<4>(c, tab, N, logN, bufA, bufE, lane); break;
        case 7: slow_part_mixed<7>(c, tab, N, logN, bufA, bufE, lane); break;
        case 10: slow_part_mixed<10>(c, tab, N, logN, bufA, bufE, lane); break;
        default: slow_part_mixed<0>(c, tab, N, logN, bufA, bufE, lane); break;
    }
    fft_mixed(N, logN, tw, bufA, bufE, lane);
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__global__ void __launch_bounds__(kWarpsMx * 32) loglik_mixed_kernel(
    const gb_window_t* __restrict__ wins, const Tile* __restrict__ tiles, TabSet32 tabs,
    const float2* __restrict__ tw_g, double T, double fstar, const double2* __restrict__ dA,
    const double2* __restrict__ dE, const double* __restrict__ wA, const double* __restrict__ wE,
    const double* __restrict__ theta, double* __restrict__ logL, double* __restrict__ dh_out,
    double* __restrict__ hh_out, int* status, int n_max, int w_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = (float2*)smem_raw;                               // kTwiddles
    double* red = (double*)(tw + kTwiddles);                      // 2 * kWarpsMx
    CandMix* cands = (CandMix*)(red + 2 * kWarpsMx);              // kWarpsMx * 32
    Win32* ws = (Win32*)(cands + kWarpsMx * 32);                  // w_max
    float2* bufs = (float2*)(ws + w_max);                         // kWarpsMx * 2 * n_max

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile tile = tiles[blockIdx.x];
    const gb_window_t win = wins[tile.win];
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];

    // <d|d> and the window scale sigma^2 = max w (block-wide, fixed order)
    double acc = 0.0, wmax = 0.0;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const double2 a = dA[win.data_off + i], e = dE[win.data_off + i];
        const double wa = wA[win.data_off + i], we = wE[win.data_off + i];
        acc += wa * (a.x * a.x + a.y * a.y) + we * (e.x * e.x + e.y * e.y);
        wmax = fmax(wmax, fmax(wa, we));
    }
    acc = warp_sum_d(acc);
    for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (lane == 0) {
        red[warp] = acc;
        red[kWarpsMx + warp] = wmax;
    }
    __syncthreads();
    double dd = 0.0, sig2 = 0.0;
    for (int w = 0; w < kWarpsMx; ++w) {
        dd += red[w];
        sig2 = fmax(sig2, red[kWarpsMx + w]);
    }
    dd *= 4.0 / T;
    if (!(sig2 > 0.0) || !isfinite(sig2)) sig2 = 1.0;
    const double sig = sqrt(sig2), isig2 = 1.0 / sig2;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const double2 a = dA[win.data_off + i], e = dE[win.data_off + i];
        Win32 v;
        v.dA = make_float2((float)(a.x * sig), (float)(a.y * sig));
        v.dE = make_float2((float)(e.x * sig), (float)(e.y * sig));
        v.wA = (float)(wA[win.data_off + i] * isig2);
        v.wE = (float)(wE[win.data_off + i] * isig2);
        ws[i] = v;
    }
    __syncthreads();

    const int N = win.N;
    const int logN = 31 - __clz(N);
    const OrbitTables32 tab = tabs.t[logN - 5];
    float2* bufA = bufs + (size_t)warp * 2 * n_max;
    float2* bufE = bufA + n_max;
    CandMix* mycand = cands + warp * 32;
    const int64_t tlen = tile.c_end - tile.c_begin;
    const int64_t grp = (tlen + kWarpsMx - 1) / kWarpsMx;
    const int64_t c_lo = tile.c_begin + (int64_t)warp * grp;
    const int64_t c_hi = min(tile.c_end, c_lo + grp);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup_mixed(theta + 8 * (c_lo + lane), T, fstar, mycand[lane]);
    __syncwarp();
    const double s_dh = 2.0 * sig / (double)N;
    const double s_hh = T * sig2 / ((double)N * (double)N);
    for (int64_t cidx = c_lo; cidx < c_hi; ++cidx) {
        const CandMix& c = mycand[cidx - c_lo];
        if (c.bad) {
            if (lane == 0) {
                logL[cidx] = nan("");
                if (dh_out) dh_out[cidx] = nan("");
                if (hh_out) hh_out[cidx] = nan("");
                atomicOr(status, 1);
            }
            continue;
        }
        template_mixed(c, tab, N, logN, tw, bufA, bufE, lane);
        const int64_t off64 = c.q - N / 2 - win.k0;
        float sdh = 0.0f, cdh = 0.0f, shh = 0.0f, chh = 0.0f;
        if (off64 > -(int64_t)N && off64 < (int64_t)win.W) {
            const int off = (int)off64;
            for (int m = lane; m < N; m += 32) {
                const int kk = off + m;
                if (kk >= 0 && kk < win.W) {
                    const int idx = (m + N / 2) & (N - 1);
                    const float2 hA = bufA[idx], hE = bufE[idx];
                    const Win32 v = ws[kk];
                    kahan_add(sdh, cdh, fmaf(v.wA, fmaf(v.dA.x, hA.x, v.dA.y * hA.y),
                                             v.wE * fmaf(v.dE.x, hE.x, v.dE.y * hE.y)));
                    kahan_add(shh, chh, fmaf(v.wA, fmaf(hA.x, hA.x, hA.y * hA.y),
                                             v.wE * fmaf(hE.x, hE.x, hE.y * hE.y)));
                }
            }
        }
        const double Sdh = warp_sum_d((double)sdh - (double)cdh);
        const double Shh = warp_sum_d((double)shh - (double)chh);
        if (lane == 0) {
            const double dh = c.A * s_dh * Sdh;
            const double hh = c.A * c.A * s_hh * Shh;
            logL[cidx] = dh - 0.5 * hh - 0.5 * dd;
            if (dh_out) dh_out[cidx] = dh;
            if (hh_out) hh_out[cidx] = hh;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kWarpsMx * 32) waveform_mixed_kernel(
    OrbitTables32 tab, const float2* __restrict__ tw_g, double T, double fstar, int N,
    const double* __restrict__ theta, int64_t B, int group, double2* __restrict__ hA,
    double2* __restrict__ hE, int64_t* __restrict__ q_out, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = (float2*)smem_raw;
    CandMix* cands = (CandMix*)(tw + kTwiddles);
    float2* bufs = (float2*)(cands + kWarpsMx * 32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];
    __syncthreads();
    const int logN = 31 - __clz(N);
    float2* bufA = bufs + (size_t)warp * 2 * N;
    float2* bufE = bufA + N;
    CandMix* mycand = cands + warp * 32;
    const int64_t c_lo = ((int64_t)blockIdx.x * kWarpsMx + warp) * group;
    const int64_t c_hi = min(B, c_lo + group);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup_mixed(theta + 8 * (c_lo + lane), T, fstar, mycand[lane]);
    __syncwarp();
    const double scale = T / (2.0 * (double)N);
    for (int64_t b = c_lo; b < c_hi; ++b) {
        const CandMix& c = mycand[b - c_lo];
        double2* outA = hA + b * N;
        double2* outE = hE + b * N;
        if (c.bad) {
            for (int m = lane; m < N; m += 32) outA[m] = outE[m] = make_double2(nan(""), nan(""));
            if (lane == 0) {
                q_out[b] = 0;
                atomicOr(status, 1);
            }
            continue;
        }
        template_mixed(c, tab, N, logN, tw, bufA, bufE, lane);
        const double s = scale * c.A;
        for (int m = lane; m < N; m += 32) {
            const int idx = (m + N / 2) & (N - 1);
            const float2 a = bufA[idx], e = bufE[idx];
            outA[m] = make_double2(s * a.x, s * a.y);
            outE[m] = make_double2(s * e.x, s * e.y);
        }
        if (lane == 0) q_out[b] = c.q;
        __syncwarp();
    }
}

}  // namespace

int launch_loglik_mixed(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                        const double* wE, const double* theta, double* logL, double* dh, double* hh,
                        cudaStream_t s) {
    if (plan.n_tiles == 0) return GB_OK;
    const size_t smem = sizeof(float2) * kTwiddles + sizeof(double) * 2 * kWarpsMx +
                        sizeof(CandMix) * kWarpsMx * 32 + sizeof(Win32) * (size_t)plan.w_max +
                        sizeof(float2) * kWarpsMx * 2 * (size_t)plan.n_max;
    cudaError_t e = cudaFuncSetAttribute(loglik_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik_mixed: smem attribute");
    loglik_mixed_kernel<<<plan.n_tiles, kWarpsMx * 32, smem, s>>>(
        plan.d_win, plan.d_tiles, tabset32(ctx), (const float2*)ctx->d_tw32, ctx->obs.T_obs,
        transfer_frequency(ctx), (const double2*)dA, (const double2*)dE, wA, wE, theta, logL, dh, hh,
        ctx->d_status, plan.n_max, plan.w_max);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik_mixed launch");
    return GB_OK;
}

int launch_waveform_mixed(gb_ctx* ctx, const double* theta, int64_t B, int N, double* hA, double* hE,
                          int64_t* q, cudaStream_t s) {
    if (B == 0) return GB_OK;
    const size_t smem =
        sizeof(float2) * kTwiddles + sizeof(CandMix) * kWarpsMx * 32 + sizeof(float2) * kWarpsMx * 2 * (size_t)N;
    cudaError_t e = cudaFuncSetAttribute(waveform_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform_mixed: smem attribute");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int64_t group = (B + (int64_t)sms * kWarpsMx * 2 - 1) / ((int64_t)sms * kWarpsMx * 2);
    group = group < 1 ? 1 : group > 32 ? 32 : group;
    const int64_t blocks = (B + group * kWarpsMx - 1) / (group * kWarpsMx);
    waveform_mixed_kernel<<<(unsigned)blocks, kWarpsMx * 32, smem, s>>>(
        tables32(ctx, N), (const float2*)ctx->d_tw32, ctx->obs.T_obs, transfer_frequency(ctx), N, theta, B,
        (int)group, (double2*)hA, (double2*)hE, q, ctx->d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform_mixed launch");
    return GB_OK;
}

}  // namespace gb
