// grad64.cu -- gradient of the window log-likelihood, plain IEEE double.
//
// With h_k = (T/2N) S_m and r_m = w_k (d_k - h_k) on window bins (0 elsewhere),
//   d logL / d theta_i = (4/T) sum_k w_k Re[(d_k - h_k) conj(d h_k/d theta_i)]
//                      = (2/N) Re sum_n  c_n conj(d s_n / d theta_i),
//   c_n = sum_m r_m exp(+2 pi i m n / N)        (the adjoint of the DFT).
// Per candidate the kernel (1) recomputes the template, (2) forms the
// residual r and logL, (3) runs the adjoint FFT to get c_n, and (4) sweeps the
// samples again carrying the slow-part response with eight tangents (one per
// parameter, forward mode) and contracts them with c_n.  Nothing is stored
// between candidates beyond the warp's shared-memory buffers.
//
// Tangents in closed form (k = propagation direction, u, v the polarisation
// basis, kappa_j = k.x_j/c, f = f0 + fdot t):
//   dPsi_j/df0 = 2 pi (t - kappa_j),  dPsi_j/dfdot = pi (t - kappa_j)^2,
//   dPsi_j/dbeta = -2 pi (f - fdot kappa_j) u.x_j/c,
//   dPsi_j/dlambda = -2 pi (f - fdot kappa_j) cos(beta) v.x_j/c,  dPsi_j/dphi0 = 1,
//   dk/dbeta = u, dk/dlambda = cos(beta) v, du/dbeta = -k, du/dlambda = -sin(beta) v,
//   dv/dlambda = (cos lambda, sin lambda, 0),
//   H = alpha e+ + gamma ex with alpha = A+ cos2psi - i Ax sin2psi,
//   gamma = -A+ sin2psi - i Ax cos2psi (linear in A, simple in iota and psi),
//   d/dX [sinc(X) e^{-iX}] = (e^{-2iX} - sinc(X) e^{-iX}) / X.
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kWarpsG = 2;
constexpr int K = 8;   // f0, fdot, beta, lambda, A, iota, psi, phi0

struct C {
    double x, y;
};
__device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ C cmul(C a, C b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ C cscale(C a, double s) { return {a.x * s, a.y * s}; }

struct DR {
    double v, d[K];
};
struct DC {
    C v, d[K];
};

__device__ __forceinline__ DC dmul(const DC& a, const DC& b) {
    DC o;
    o.v = cmul(a.v, b.v);
#pragma unroll
    for (int k = 0; k < K; ++k) o.d[k] = cadd(cmul(a.d[k], b.v), cmul(a.v, b.d[k]));
    return o;
}
__device__ __forceinline__ DC dadd(const DC& a, const DC& b) {
    DC o;
    o.v = cadd(a.v, b.v);
#pragma unroll
    for (int k = 0; k < K; ++k) o.d[k] = cadd(a.d[k], b.d[k]);
    return o;
}
__device__ __forceinline__ DC dsub(const DC& a, const DC& b) {
    DC o;
    o.v = csub(a.v, b.v);
#pragma unroll
    for (int k = 0; k < K; ++k) o.d[k] = csub(a.d[k], b.d[k]);
    return o;
}
__device__ __forceinline__ DC dscale(const DC& a, double s) {
    DC o;
    o.v = cscale(a.v, s);
#pragma unroll
    for (int k = 0; k < K; ++k) o.d[k] = cscale(a.d[k], s);
    return o;
}

struct CandG {
    double k[3], u[3], v[3], w[3];   // w = dv/dlambda
    double cb, sb;
    C al, ga, al_i[3], ga_i[3];      // alpha, gamma and their derivatives wrt A, iota, psi
    double f0, fd, delta, phi0, A;
    long long q;
    int bad, pad;
};

__device__ void setup_grad(const double* th, double T, CandG& c) {
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
    double sb, cb, sl, cl, s2, c2, si, ci;
    sincos(beta, &sb, &cb);
    sincos(lam, &sl, &cl);
    sincos(2.0 * psi, &s2, &c2);
    sincos(iota, &si, &ci);
    c.cb = cb;
    c.sb = sb;
    c.k[0] = -(cb * cl);
    c.k[1] = -(cb * sl);
    c.k[2] = -sb;
    c.u[0] = sb * cl;
    c.u[1] = sb * sl;
    c.u[2] = -cb;
    c.v[0] = sl;
    c.v[1] = -cl;
    c.v[2] = 0.0;
    c.w[0] = cl;
    c.w[1] = sl;
    c.w[2] = 0.0;
    const double Ap = A * (1.0 + ci * ci), Ax = -2.0 * A * ci;
    c.al = {Ap * c2, -(Ax * s2)};
    c.ga = {-(Ap * s2), -(Ax * c2)};
    // d/dA
    const double Ap1 = 1.0 + ci * ci, Ax1 = -2.0 * ci;
    c.al_i[0] = {Ap1 * c2, -(Ax1 * s2)};
    c.ga_i[0] = {-(Ap1 * s2), -(Ax1 * c2)};
    // d/diota: dA+ = -2 A cos(iota) sin(iota), dAx = 2 A sin(iota)
    const double dAp = -2.0 * A * ci * si, dAx = 2.0 * A * si;
    c.al_i[1] = {dAp * c2, -(dAx * s2)};
    c.ga_i[1] = {-(dAp * s2), -(dAx * c2)};
    // d/dpsi
    c.al_i[2] = {-2.0 * Ap * s2, -2.0 * Ax * c2};
    c.ga_i[2] = {-2.0 * Ap * c2, 2.0 * Ax * s2};
}

// sinc(X) e^{-iX} and its derivative in X
__device__ __forceinline__ void transfer(double X, C& Tv, C& Td) {
    if (fabs(X) < 0.25) {
        // series of (e^w - 1)/w, w = -2iX, and its derivative, 18 terms
        C t = {0.0, 0.0}, td = {0.0, 0.0};
        C wk = {1.0, 0.0};   // (-2i)^k X^k
        double inv = 1.0;    // 1/(k+1)!
        C wkm1 = {0.0, 0.0}; // (-2i)^k X^(k-1) * k
        for (int k = 0; k < 18; ++k) {
            inv /= (double)(k + 1);
            t = cadd(t, cscale(wk, inv));
            if (k >= 1) td = cadd(td, cscale(wkm1, inv));
            // advance: wkm1 for k+1 = (k+1) (-2i)^(k+1) X^k
            const C m2i = {0.0, -2.0};
            wkm1 = cscale(cmul(wk, m2i), (double)(k + 1));
            wk = cmul(cscale(wk, X), m2i);
        }
        Tv = t;
        Td = td;
        return;
    }
    double s, co;
    sincos(X, &s, &co);
    const double sc = s / X;
    Tv = {sc * co, -(sc * s)};
    const C e2 = {co * co - s * s, -2.0 * s * co};
    Td = cscale(csub(e2, Tv), 1.0 / X);
}

struct Geo {
    double T, T_over_N, fstar, scale;
    int N, logN;
};

// Slow-part response of one sample with eight tangents: returns A and E, and
// T = (X + Y + Z)/sqrt3 when Tout is not null.
__device__ void sample_dual(const CandG& c, const Geo& g, const OrbitTables64& tab, int n, DC& Aout, DC& Eout,
                            DC* Tout = nullptr) {
    const int N = g.N;
    const double t = (double)n * g.T_over_N;
    const double f = c.f0 + c.fd * t;
    DC rx[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double x0 = tab.x[(j * 3 + 0) * N + n], x1 = tab.x[(j * 3 + 1) * N + n],
                     x2 = tab.x[(j * 3 + 2) * N + n];
        const double kap = (c.k[0] * x0 + c.k[1] * x1 + c.k[2] * x2) / kC;
        const double ux = (c.u[0] * x0 + c.u[1] * x1 + c.u[2] * x2) / kC;
        const double vx = (c.v[0] * x0 + c.v[1] * x1 + c.v[2] * x2) / kC;
        const double ph = 2.0 * kPi *
                              (c.delta * t / g.T + 0.5 * c.fd * (t * t) - c.f0 * kap - c.fd * t * kap +
                               0.5 * c.fd * (kap * kap)) +
                          c.phi0;
        double dph[K];
        const double tk = t - kap;
        const double fk = f - c.fd * kap;
        dph[0] = 2.0 * kPi * tk;
        dph[1] = kPi * tk * tk;
        dph[2] = -2.0 * kPi * fk * ux;
        dph[3] = -2.0 * kPi * fk * c.cb * vx;
        dph[4] = 0.0;
        dph[5] = 0.0;
        dph[6] = 0.0;
        dph[7] = 1.0;
        double s, co;
        sincos(ph, &s, &co);
        rx[j].v = {co, s};
#pragma unroll
        for (int k = 0; k < K; ++k) rx[j].d[k] = {-s * dph[k], co * dph[k]};
    }
    const double a = f / (2.0 * g.fstar);
    double da[K] = {1.0 / (2.0 * g.fstar), t / (2.0 * g.fstar), 0, 0, 0, 0, 0, 0};
    DC zp[3], zm[3];
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        const double nx = tab.arm[(arm * 3 + 0) * N + n], ny = tab.arm[(arm * 3 + 1) * N + n],
                     nz = tab.arm[(arm * 3 + 2) * N + n];
        const double kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
        const double nu = c.u[0] * nx + c.u[1] * ny + c.u[2] * nz;
        const double nv = c.v[0] * nx + c.v[1] * ny + c.v[2] * nz;
        const double nw = c.w[0] * nx + c.w[1] * ny + c.w[2] * nz;
        double dkn[K] = {0, 0, nu, c.cb * nv, 0, 0, 0, 0};
        const double Fp = nu * nu - nv * nv, Fx = 2.0 * nu * nv;
        const double dFp_b = -2.0 * nu * kn, dFx_b = -2.0 * kn * nv;
        const double dFp_l = -2.0 * c.sb * nu * nv - 2.0 * nv * nw;
        const double dFx_l = -2.0 * c.sb * nv * nv + 2.0 * nu * nw;
        DC G;
        G.v = cadd(cscale(c.al, Fp), cscale(c.ga, Fx));
        G.d[0] = {0.0, 0.0};
        G.d[1] = {0.0, 0.0};
        G.d[2] = cadd(cscale(c.al, dFp_b), cscale(c.ga, dFx_b));
        G.d[3] = cadd(cscale(c.al, dFp_l), cscale(c.ga, dFx_l));
        G.d[4] = cadd(cscale(c.al_i[0], Fp), cscale(c.ga_i[0], Fx));
        G.d[5] = cadd(cscale(c.al_i[1], Fp), cscale(c.ga_i[1], Fx));
        G.d[6] = cadd(cscale(c.al_i[2], Fp), cscale(c.ga_i[2], Fx));
        G.d[7] = {0.0, 0.0};
        const int rp = arm == 2 ? 0 : arm + 1, rm = arm;
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double sdir = sgn == 0 ? 1.0 : -1.0;   // +n link: X = a(1 - kn); -n link: X = a(1 + kn)
            const double X = a * (1.0 - sdir * kn);
            C Tv, Td;
            transfer(X, Tv, Td);
            DC Tl;
            Tl.v = Tv;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const double dX = da[k] * (1.0 - sdir * kn) - sdir * a * dkn[k];
                Tl.d[k] = cscale(Td, dX);
            }
            const DC z = dmul(dmul(Tl, G), rx[sgn == 0 ? rp : rm]);
            if (sgn == 0)
                zp[arm] = z;
            else
                zm[arm] = z;
        }
    }
    // D = exp(-i f/f*)
    DC D;
    {
        double s, co;
        sincos(f / g.fstar, &s, &co);
        D.v = {co, -s};
        const double df[K] = {1.0 / g.fstar, t / g.fstar, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < K; ++k) D.d[k] = {-s * df[k], -co * df[k]};   // -i D df
    }
    const DC Xp = dadd(dsub(zm[0], zp[2]), dmul(D, dsub(zp[0], zm[2])));
    const DC Yp = dadd(dsub(zm[1], zp[0]), dmul(D, dsub(zp[1], zm[0])));
    const DC Zp = dadd(dsub(zm[2], zp[1]), dmul(D, dsub(zp[2], zm[1])));
    // F = -i a (1 - D^2)
    const DC D2 = dmul(D, D);
    DC F;
    F.v = {-a * D2.v.y, -a * (1.0 - D2.v.x)};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        // d[-i a (1 - D2)] = -i [da (1 - D2) - a dD2]
        const C q = {da[k] * (1.0 - D2.v.x) - a * D2.d[k].x, -da[k] * D2.v.y - a * D2.d[k].y};
        F.d[k] = {q.y, -q.x};
    }
    const double r2 = sqrt(2.0), r6 = sqrt(6.0);
    const DC Ap = dscale(dsub(Zp, Xp), 1.0 / r2);
    const DC Ep = dscale(dadd(dsub(Xp, dscale(Yp, 2.0)), Zp), 1.0 / r6);
    Aout = dmul(F, Ap);
    Eout = dmul(F, Ep);
    if (Tout) *Tout = dmul(F, dscale(dadd(dadd(Xp, Yp), Zp), 1.0 / sqrt(3.0)));
}

// forward template (value only), used for the residual
__device__ void template_value(const CandG& c, const Geo& g, const OrbitTables64& tab, const C* tw, C* bufA,
                               C* bufE, C* bufT, int lane) {
    const int N = g.N;
    for (int n = lane; n < N; n += 32) {
        DC Ad, Ed, Td;
        sample_dual(c, g, tab, n, Ad, Ed, bufT ? &Td : nullptr);
        const int br = (int)(__brev((unsigned)n) >> (32 - g.logN));
        bufA[br] = Ad.v;
        bufE[br] = Ed.v;
        if (bufT) bufT[br] = Td.v;
    }
    __syncwarp();
}

__device__ void fft_inplace(int N, int logN, const C* tw, C* bufA, C* bufE, C* bufT, int lane) {
    for (int s = 0; s < logN; ++s) {
        const int h = 1 << s;
        const int tstride = kTwiddles >> s;
        for (int b = lane; b < N / 2; b += 32) {
            const int j = b & (h - 1);
            const int i0 = ((b >> s) << (s + 1)) + j;
            const int i1 = i0 + h;
            const C w = tw[j * tstride];
            const C ua = bufA[i0], va = cmul(w, bufA[i1]);
            bufA[i0] = cadd(ua, va);
            bufA[i1] = csub(ua, va);
            const C ue = bufE[i0], ve = cmul(w, bufE[i1]);
            bufE[i0] = cadd(ue, ve);
            bufE[i1] = csub(ue, ve);
            if (bufT) {
                const C ut = bufT[i0], vt = cmul(w, bufT[i1]);
                bufT[i0] = cadd(ut, vt);
                bufT[i1] = csub(ut, vt);
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kWarpsG * 32) grad64_kernel(
    const gb_window_t* __restrict__ wins, const Tile* __restrict__ tiles, TabSet64 tabs, const C* __restrict__ tw_g,
    double T, double fstar, const C* __restrict__ dA, const C* __restrict__ dE, const double* __restrict__ wA,
    const double* __restrict__ wE, const double* __restrict__ theta, double* __restrict__ logL_out,
    double* __restrict__ grad_out, const C* __restrict__ dT, const double* __restrict__ wT, int* status,
    int n_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = (C*)smem_raw;
    double* red = (double*)(tw + kTwiddles);
    CandG* cands = (CandG*)(red + kWarpsG);
    C* bufs = (C*)(cands + kWarpsG * 32);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile tile = tiles[blockIdx.x];
    const gb_window_t win = wins[tile.win];
    for (int i = threadIdx.x; i < kTwiddles; i += blockDim.x) tw[i] = tw_g[i];
    // T enters windows whose lowest frequency is at least f*/2 (dT given)
    const bool useT = dT != nullptr && (double)win.k0 / T >= 0.5 * fstar;
    double acc = 0.0;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const C a = dA[win.data_off + i], e = dE[win.data_off + i];
        acc += wA[win.data_off + i] * (a.x * a.x + a.y * a.y) + wE[win.data_off + i] * (e.x * e.x + e.y * e.y);
        if (useT) {
            const C t = dT[win.data_off + i];
            acc += wT[win.data_off + i] * (t.x * t.x + t.y * t.y);
        }
    }
    acc = wsum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    double dd = 0.0;
    for (int w = 0; w < kWarpsG; ++w) dd += red[w];
    dd *= 4.0 / T;

    Geo g;
    g.N = win.N;
    g.logN = 31 - __clz(win.N);
    g.T = T;
    g.T_over_N = T / (double)win.N;
    g.fstar = fstar;
    g.scale = T / (2.0 * (double)win.N);
    const OrbitTables64 tab = tabs.t[g.logN - 5];
    const int N = g.N;
    C* bufA = bufs + (size_t)warp * (dT ? 3 : 2) * n_max;
    C* bufE = bufA + n_max;
    C* bufT = useT ? bufE + n_max : nullptr;
    CandG* mycand = cands + warp * 32;
    const int64_t tlen = tile.c_end - tile.c_begin;
    const int64_t grp = (tlen + kWarpsG - 1) / kWarpsG;
    const int64_t c_lo = tile.c_begin + (int64_t)warp * grp;
    const int64_t c_hi = min(tile.c_end, c_lo + grp);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup_grad(theta + 8 * (c_lo + lane), T, mycand[lane]);
    __syncwarp();
    for (int64_t cidx = c_lo; cidx < c_hi; ++cidx) {
        const CandG& c = mycand[cidx - c_lo];
        if (c.bad) {
            if (lane == 0) {
                if (logL_out) logL_out[cidx] = nan("");
                for (int k = 0; k < K; ++k) grad_out[8 * cidx + k] = nan("");
                atomicOr(status, kStatusNonFinite);
            }
            continue;
        }
        // (1) template
        template_value(c, g, tab, tw, bufA, bufE, bufT, lane);
        fft_inplace(N, g.logN, tw, bufA, bufE, bufT, lane);
        // (2) logL and residual r_m = w (d - h) at DFT index m mod N, in place
        double sdh = 0.0, shh = 0.0;
        for (int idx = lane; idx < N; idx += 32) {
            const int m = idx < N / 2 ? idx : idx - N;      // signed frequency offset
            const int64_t kk = c.q + m - win.k0;
            const C hA = cscale(bufA[idx], g.scale), hE = cscale(bufE[idx], g.scale);
            C rA = {0.0, 0.0}, rE = {0.0, 0.0};
            if (kk >= 0 && kk < win.W) {
                const C a = dA[win.data_off + kk], e = dE[win.data_off + kk];
                const double wa = wA[win.data_off + kk], we = wE[win.data_off + kk];
                sdh += wa * (a.x * hA.x + a.y * hA.y) + we * (e.x * hE.x + e.y * hE.y);
                shh += wa * (hA.x * hA.x + hA.y * hA.y) + we * (hE.x * hE.x + hE.y * hE.y);
                rA = {wa * (a.x - hA.x), wa * (a.y - hA.y)};
                rE = {we * (e.x - hE.x), we * (e.y - hE.y)};
            }
            // conjugate for the adjoint transform: c = conj(FFT(conj(r)))
            bufA[idx] = {rA.x, -rA.y};
            bufE[idx] = {rE.x, -rE.y};
            if (useT) {
                const C hT = cscale(bufT[idx], g.scale);
                C rT = {0.0, 0.0};
                if (kk >= 0 && kk < win.W) {
                    const C t = dT[win.data_off + kk];
                    const double wt = wT[win.data_off + kk];
                    sdh += wt * (t.x * hT.x + t.y * hT.y);
                    shh += wt * (hT.x * hT.x + hT.y * hT.y);
                    rT = {wt * (t.x - hT.x), wt * (t.y - hT.y)};
                }
                bufT[idx] = {rT.x, -rT.y};
            }
        }
        sdh = wsum(sdh) * (4.0 / T);
        shh = wsum(shh) * (4.0 / T);
        __syncwarp();
        // (3) bit-reversal permutation in place, then the same forward FFT
        for (int i = lane; i < N; i += 32) {
            const int j = (int)(__brev((unsigned)i) >> (32 - g.logN));
            if (i < j) {
                const C ta = bufA[i];
                bufA[i] = bufA[j];
                bufA[j] = ta;
                const C te = bufE[i];
                bufE[i] = bufE[j];
                bufE[j] = te;
                if (useT) {
                    const C tt = bufT[i];
                    bufT[i] = bufT[j];
                    bufT[j] = tt;
                }
            }
        }
        __syncwarp();
        fft_inplace(N, g.logN, tw, bufA, bufE, bufT, lane);
        // (4) tangent sweep: g_i += Re(c_n conj(ds_n/dtheta_i)), c_n = conj(buf[n])
        double gacc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) gacc[k] = 0.0;
        for (int n = lane; n < N; n += 32) {
            DC Ad, Ed, Td;
            sample_dual(c, g, tab, n, Ad, Ed, useT ? &Td : nullptr);
            const C cA = {bufA[n].x, -bufA[n].y}, cE = {bufE[n].x, -bufE[n].y};
#pragma unroll
            for (int k = 0; k < K; ++k)
                gacc[k] += cA.x * Ad.d[k].x + cA.y * Ad.d[k].y + cE.x * Ed.d[k].x + cE.y * Ed.d[k].y;
            if (useT) {
                const C cT = {bufT[n].x, -bufT[n].y};
#pragma unroll
                for (int k = 0; k < K; ++k) gacc[k] += cT.x * Td.d[k].x + cT.y * Td.d[k].y;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) gacc[k] = wsum(gacc[k]) * (2.0 / (double)N);
        if (lane == 0) {
            if (logL_out) logL_out[cidx] = sdh - 0.5 * shh - 0.5 * dd;
#pragma unroll
            for (int k = 0; k < K; ++k) grad_out[8 * cidx + k] = gacc[k];
        }
        __syncwarp();
    }
}

}  // namespace

int launch_grad_fp64(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                     const double* wE, const double* theta, double* logL, double* grad, const double* dT,
                     const double* wT, cudaStream_t s) {
    if (plan.n_tiles == 0) return GB_OK;
    const size_t smem = sizeof(C) * kTwiddles + sizeof(double) * kWarpsG + sizeof(CandG) * kWarpsG * 32 +
                        sizeof(C) * kWarpsG * (dT ? 3 : 2) * (size_t)plan.n_max;
    cudaError_t e = cudaFuncSetAttribute(grad64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "grad64: smem attribute");
    grad64_kernel<<<plan.n_tiles, kWarpsG * 32, smem, s>>>(plan.d_win, plan.d_tiles, tabset64(ctx),
                                                           (const C*)ctx->d_tw64, ctx->obs.T_obs,
                                                           transfer_frequency(ctx), (const C*)dA, (const C*)dE,
                                                           wA, wE, theta, logL, grad, (const C*)dT, wT,
                                                           ctx->d_status, plan.n_max);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "grad64 launch");
    return GB_OK;
}

}  // namespace gb
