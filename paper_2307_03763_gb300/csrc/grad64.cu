// grad64.cu -- gradient of the window log-likelihood, plain IEEE double.
//
// With h_k = (T/2N) S_m and r_m = w_k (d_k - h_k) on window bins (0 elsewhere),
//   d logL / d theta_i = (4/T) sum_k w_k Re[(d_k - h_k) conj(d h_k/d theta_i)]
//                      = (2/N) Re sum_n  conj(c_n) d s_n / d theta_i,
//   c_n = conj(sum_m conj(r_m) exp(-2 pi i m n / N))   (the adjoint of the DFT).
// Per candidate the kernel (1) computes the template, (2) forms the residual
// r and logL, (3) runs the adjoint FFT to get c_n, and (4) sweeps the samples
// in reverse mode: each sample's forward values (the fast/slow response of
// Sec. II, in the same link form as the FP64 likelihood), then the adjoints
// of the channel samples c_n propagated back through the TDI combination,
// the six links and the three receiver phases to the parameters.  The
// amplitude, inclination and polarisation enter only through the two complex
// polarisation coefficients alpha, gamma (n.H.n = alpha Fp + gamma Fx); their
// adjoints are summed over the samples and contracted with d alpha/d theta,
// d gamma/d theta once per candidate.
//
// Derivatives used (k = propagation direction, u, v the polarisation basis,
// kappa_j = k.x_j/c, f = f0 + fdot t, receiver phase 2 pi cyc_j):
//   d cyc_j/d f0 = t - kappa_j,  d cyc_j/d fdot = (t - kappa_j)^2 / 2,
//   d cyc_j/d beta = -(f - fdot kappa_j) u.x_j/c,
//   d cyc_j/d lambda = -(f - fdot kappa_j) cos(beta) v.x_j/c,  d cyc_j/d phi0 = 1/(2 pi),
//   dk/dbeta = u, dk/dlambda = cos(beta) v, du/dbeta = -k, du/dlambda = -sin(beta) v,
//   dv/dlambda = (cos lambda, sin lambda, 0),
//   d/dX [sinc(X) e^{-iX}] from the derivative of its series (or, evaluated
//   directly, (e^{-2iX} - sinc(X) e^{-iX}) / X).
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
// a conj(b)
__device__ __forceinline__ C cmulc(C a, C b) { return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }
__device__ __forceinline__ C cscale(C a, double s) { return {a.x * s, a.y * s}; }
// Re(conj(a) b)
__device__ __forceinline__ double redot(C a, C b) { return a.x * b.x + a.y * b.y; }

// Series of the link transfer V(X) = sinc(X) e^{-iX} in y = -4 X^2:
//   Re V = sum_j y^j/(2j+1)!,          Im V = -2X sum_j y^j/(2j+2)!,
//   d Re V/dX = X sum_j y^j (-8(j+1))/(2j+3)!,   d Im V/dX = sum_j y^j (-2(2j+1))/(2j+2)!
// (each coefficient the double nearest its exact rational value)
struct Series4 {
    double re, im, dre, dim;
};
__constant__ Series4 kTransferSeries[17] = {
    {1.0, 0.5, -1.3333333333333333, -1.0},
    {0.16666666666666666, 0.041666666666666664, -0.13333333333333333, -0.25},
    {0.008333333333333333, 0.001388888888888889, -0.004761904761904762, -0.013888888888888888},
    {0.0001984126984126984, 2.48015873015873e-05, -8.818342151675486e-05, -0.00034722222222222224},
    {2.7557319223985893e-06, 2.755731922398589e-07, -1.0020843354176687e-06, -4.96031746031746e-06},
    {2.505210838544172e-08, 2.08767569878681e-09, -7.708341041674375e-09, -4.592886537330982e-08},
    {1.6059043836821613e-10, 1.1470745597729725e-11, -4.282411689819097e-11, -2.9823938554097286e-10},
    {7.647163731819816e-13, 4.779477332387385e-14, -1.7993326427811332e-13, -1.4338431997162156e-12},
    {2.8114572543455206e-15, 1.5619206968586225e-16, -5.918857377569517e-16, -5.310530369319317e-15},
    {8.22063524662433e-18, 4.110317623312165e-19, -1.565835285071301e-18, -1.5619206968586227e-17},
    {1.9572941063391263e-20, 8.896791392450574e-22, -3.403989750155002e-21, -3.7366523848292405e-20},
    {3.868170170630684e-23, 1.6117375710961184e-24, -6.189072273009094e-24, -7.413992827042144e-23},
    {6.446950284384474e-26, 2.4795962632247976e-27, -9.551037458347369e-27, -1.2397981316123987e-25},
    {9.183689863795546e-29, 3.279889237069838e-30, -1.2667158432821444e-29, -1.7711401880177124e-28},
    {1.1309962886447716e-31, 3.7699876288159054e-33, -1.4593500498642214e-32, -2.1865928247132253e-31},
    {1.216125041553518e-34, 3.8003907548547434e-36, -1.4740909594588097e-35, -2.356242268009941e-34},
    {1.151633562077195e-37, 3.387157535521162e-39, -1.3161526423739371e-38, -2.235523973443967e-37},
};

struct CandG {
    double k[3], u[3], v[3], w[3];   // w = dv/dlambda
    double cb, sb;
    C al, ga, al_i[3], ga_i[3];      // alpha, gamma and their derivatives wrt A, iota, psi
    double f0, fd, delta, phi0c;
    double D0r, D0i, eps;            // exp(-i f0/f*), fdot/f*
    long long q;
    int bad, J;
};

__device__ void setup_grad(const double* th, double T, double inv_fstar, CandG& c) {
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
    // series degree of the link transfer: first omitted term (of the
    // transfer and of its derivative) below 1e-15 for the largest argument
    // X = f (1 + |k.n|)/(2 f*) <= f_max / f*
    const double xmax = fmax(fabs(f0), fabs(f0 + fd * T)) * inv_fstar;
    c.J = xmax <= 0.22 ? 6 : xmax <= 0.5 ? 8 : xmax <= 1.3 ? 12 : xmax <= 2.35 ? 16 : 0;
    double sD, cD;
    sincos(f0 * inv_fstar, &sD, &cD);
    c.D0r = cD;
    c.D0i = -sD;
    c.eps = fd * inv_fstar;
}

// V = sinc(X) e^{-iX} and, with DER, dV/dX
template <bool DER>
__device__ __forceinline__ void transfer(double X, int J, C& V, C& Vd) {
    if (J == 0) {
        double s, co;
        sincos(X, &s, &co);
        const double sinc = X != 0.0 ? s / X : 1.0;
        V = {sinc * co, -(sinc * s)};
        if (DER) {
            const C e2 = {co * co - s * s, -2.0 * s * co};
            Vd = X != 0.0 ? cscale(csub(e2, V), 1.0 / X) : C{0.0, -1.0};
        }
        return;
    }
    const double y = -4.0 * X * X;
    const Series4 cJ = kTransferSeries[J];
    double re = cJ.re, im = cJ.im, dim = cJ.dim, dre = kTransferSeries[J - 1].dre;
    for (int j = J - 1; j >= 0; --j) {
        const Series4 cj = kTransferSeries[j];
        re = fma(re, y, cj.re);
        im = fma(im, y, cj.im);
        if (DER) {
            dim = fma(dim, y, cj.dim);
            if (j > 0) dre = fma(dre, y, kTransferSeries[j - 1].dre);
        }
    }
    V = {re, -2.0 * X * im};
    if (DER) Vd = {X * dre, dim};
}

struct Geo {
    double T, T_over_N, inv_fstar, scale;
    int N, logN;
};

// Forward values of one sample (Sec. II): receiver phasors, the six links
// z_ij = -i a V(a (1 -+ k.n)) (n.H.n) exp(2 pi i cyc), D = exp(-i f/f*) and
// the combinations P of X = (1 - D^2) P (Y, Z likewise).  Link order:
// 01, 10, 12, 21, 20, 02 (arm 0: 01, 10; arm 1: 12, 21; arm 2: 20, 02).
struct Fwd {
    double t, f, a, kap[3];
    C rx[3], z[6], D, omd, PX, PY, PZ;
};

__device__ __forceinline__ void arm_geometry(const CandG& c, const OrbitTables64& tab, int arm, int N, int n,
                                             double& kn, double& nu, double& nv, double& nw) {
    const double nx = tab.arm[(arm * 3 + 0) * N + n], ny = tab.arm[(arm * 3 + 1) * N + n],
                 nz = tab.arm[(arm * 3 + 2) * N + n];
    kn = c.k[0] * nx + c.k[1] * ny + c.k[2] * nz;
    nu = c.u[0] * nx + c.u[1] * ny + c.u[2] * nz;
    nv = c.v[0] * nx + c.v[1] * ny;
    nw = c.w[0] * nx + c.w[1] * ny;
}

// receiver of link l: 01 -> 1, 10 -> 0, 12 -> 2, 21 -> 1, 20 -> 0, 02 -> 2
__device__ __forceinline__ int link_rx(int l) { return l == 0 ? 1 : l == 1 ? 0 : l == 2 ? 2 : l == 3 ? 1 : l == 4 ? 0 : 2; }

__device__ void forward(const CandG& c, const Geo& g, const OrbitTables64& tab, int n, Fwd& fw) {
    const int N = g.N;
    const double inv_c = 1.0 / kC;
    fw.t = (double)n * g.T_over_N;
    const double t = fw.t;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double kap = (c.k[0] * tab.x[(j * 3 + 0) * N + n] + c.k[1] * tab.x[(j * 3 + 1) * N + n] +
                            c.k[2] * tab.x[(j * 3 + 2) * N + n]) * inv_c;
        fw.kap[j] = kap;
        double cyc = c.delta * ((double)n / (double)N) + 0.5 * c.fd * (t * t) - c.f0 * kap - c.fd * t * kap +
                     0.5 * c.fd * (kap * kap) + c.phi0c;
        cyc -= rint(cyc);
        double s, co;
        sincospi(2.0 * cyc, &s, &co);
        fw.rx[j] = {co, s};
    }
    fw.f = c.f0 + c.fd * t;
    fw.a = fw.f * (0.5 * g.inv_fstar);
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        double kn, nu, nv, nw;
        arm_geometry(c, tab, arm, N, n, kn, nu, nv, nw);
        const double Fp = (nu - nv) * (nu + nv), Fx = 2.0 * nu * nv;
        const C G = cadd(cscale(c.al, Fp), cscale(c.ga, Fx));
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int l = 2 * arm + s;
            C V, Vd;
            transfer<false>(fw.a * (s == 0 ? 1.0 - kn : 1.0 + kn), c.J, V, Vd);
            const C q = cmul(cmul(cscale(V, fw.a), G), fw.rx[link_rx(l)]);
            fw.z[l] = {q.y, -q.x};   // times -i
        }
    }
    // D = exp(-i f/f*) = exp(-i f0/f*) exp(-i th), th = fdot t/f*: a short
    // series while |th| <= 1/64
    const double th = c.eps * t;
    if (fabs(th) <= 0.015625) {
        const double t2 = th * th;
        const double cs = fma(fma(fma(t2, -1.0 / 720.0, 1.0 / 24.0), t2, -0.5), t2, 1.0);
        const double sn = th * fma(fma(fma(t2, -1.0 / 5040.0, 1.0 / 120.0), t2, -1.0 / 6.0), t2, 1.0);
        fw.D = cmul({c.D0r, c.D0i}, {cs, -sn});
    } else {
        double sD, cD;
        sincos(fw.f * g.inv_fstar, &sD, &cD);
        fw.D = {cD, -sD};
    }
    const C D2 = cmul(fw.D, fw.D);
    fw.omd = {1.0 - D2.x, -D2.y};
    const C* z = fw.z;
    fw.PX = csub(cadd(z[1], cmul(fw.D, z[0])), cadd(z[4], cmul(fw.D, z[5])));
    fw.PY = csub(cadd(z[3], cmul(fw.D, z[2])), cadd(z[0], cmul(fw.D, z[1])));
    fw.PZ = csub(cadd(z[5], cmul(fw.D, z[4])), cadd(z[2], cmul(fw.D, z[3])));
}

constexpr double kR2 = 0.70710678118654752, kR6 = 0.40824829046386302, kR3 = 0.57735026918962576;

// template samples (values) at bit-reversed positions
__device__ void template_value(const CandG& c, const Geo& g, const OrbitTables64& tab, C* bufA, C* bufE, C* bufT,
                               int lane) {
    const int N = g.N;
    for (int n = lane; n < N; n += 32) {
        Fwd fw;
        forward(c, g, tab, n, fw);
        const C X = cmul(fw.omd, fw.PX), Y = cmul(fw.omd, fw.PY), Z = cmul(fw.omd, fw.PZ);
        const int br = (int)(__brev((unsigned)n) >> (32 - g.logN));
        bufA[br] = cscale(csub(Z, X), kR2);
        bufE[br] = cscale(cadd(csub(X, cscale(Y, 2.0)), Z), kR6);
        if (bufT) bufT[br] = cscale(cadd(cadd(X, Y), Z), kR3);
    }
    __syncwarp();
}

// Per-lane gradient accumulators: f0, fdot, beta, lambda, phi0 directly;
// A, iota, psi through the adjoints of alpha and gamma.
struct Acc {
    double f0, fd, beta, lam, phi0;
    C al, ga;
};

// Reverse-mode step of one sample: the adjoints cA, cE (and cT) of the
// channel samples s_n give Re(conj(c) d s_n/d theta) summed into acc.
__device__ void sample_adjoint(const CandG& c, const Geo& g, const OrbitTables64& tab, int n, C cA, C cE, C cT,
                               bool useT, Acc& acc) {
    const int N = g.N;
    Fwd fw;
    forward(c, g, tab, n, fw);
    // A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6, T = (X + Y + Z)/sqrt3
    C Xb = cadd(cscale(cA, -kR2), cscale(cE, kR6)), Yb = cscale(cE, -2.0 * kR6), Zb = cadd(cscale(cA, kR2),
                                                                                        cscale(cE, kR6));
    if (useT) {
        Xb = cadd(Xb, cscale(cT, kR3));
        Yb = cadd(Yb, cscale(cT, kR3));
        Zb = cadd(Zb, cscale(cT, kR3));
    }
    // X = omd PX, ...
    const C omdb = cadd(cadd(cmulc(Xb, fw.PX), cmulc(Yb, fw.PY)), cmulc(Zb, fw.PZ));
    const C PXb = cmulc(Xb, fw.omd), PYb = cmulc(Yb, fw.omd), PZb = cmulc(Zb, fw.omd);
    // PX = z10 + D z01 - z20 - D z02, PY = z21 + D z12 - z01 - D z10, PZ = z02 + D z20 - z12 - D z21
    const C* z = fw.z;
    C zb[6];
    zb[0] = csub(cmulc(PXb, fw.D), PYb);   // z01
    zb[1] = csub(PXb, cmulc(PYb, fw.D));   // z10
    zb[2] = csub(cmulc(PYb, fw.D), PZb);   // z12
    zb[3] = csub(PYb, cmulc(PZb, fw.D));   // z21
    zb[4] = csub(cmulc(PZb, fw.D), PXb);   // z20
    zb[5] = csub(PZb, cmulc(PXb, fw.D));   // z02
    // D enters the combinations and omd = 1 - D^2
    C Db = cadd(cadd(cmulc(PXb, csub(z[0], z[5])), cmulc(PYb, csub(z[2], z[1]))), cmulc(PZb, csub(z[4], z[3])));
    Db = csub(Db, cmulc(omdb, cscale(fw.D, 2.0)));
    // D = exp(-i f/f*): dD = -i D df/f*
    double fb = (Db.x * fw.D.y - Db.y * fw.D.x) * g.inv_fstar;
    double ab = 0.0;
    C rxb[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        double kn, nu, nv, nw;
        arm_geometry(c, tab, arm, N, n, kn, nu, nv, nw);
        const double Fp = (nu - nv) * (nu + nv), Fx = 2.0 * nu * nv;
        const C G = cadd(cscale(c.al, Fp), cscale(c.ga, Fx));
        C Gb = {0.0, 0.0};
        double knb = 0.0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int l = 2 * arm + s;
            const int j = link_rx(l);
            const double sg = s == 0 ? -1.0 : 1.0;   // X = a (1 + sg kn)
            const double Xa = fw.a * (1.0 + sg * kn);
            C V, Vd;
            transfer<true>(Xa, c.J, V, Vd);
            // z = -i a V W, W = G rx: with zz = i zbar and P = conj(zz) W,
            // abar += Re(P V), Xbar = a Re(P V'), Wbar = a zz conj(V)
            const C zz = {-zb[l].y, zb[l].x};
            const C W = cmul(G, fw.rx[j]);
            const C P = cmulc(W, zz);
            ab += P.x * V.x - P.y * V.y;
            const double Xb_ = fw.a * (P.x * Vd.x - P.y * Vd.y);
            const C Wb = cscale(cmulc(zz, V), fw.a);
            Gb = cadd(Gb, cmulc(Wb, fw.rx[j]));
            rxb[j] = cadd(rxb[j], cmulc(Wb, G));
            ab += Xb_ * (1.0 + sg * kn);
            knb += sg * fw.a * Xb_;
        }
        // G = alpha Fp + gamma Fx
        acc.al = cadd(acc.al, cscale(Gb, Fp));
        acc.ga = cadd(acc.ga, cscale(Gb, Fx));
        const double Fpb = redot(Gb, c.al), Fxb = redot(Gb, c.ga);
        const double nub = 2.0 * (nu * Fpb + nv * Fxb), nvb = 2.0 * (nu * Fxb - nv * Fpb);
        acc.beta += knb * nu - nub * kn;
        acc.lam += knb * c.cb * nv - nub * c.sb * nv + nvb * nw;
    }
    // receiver phases rx_j = exp(2 pi i cyc_j)
    const double inv_c = 1.0 / kC;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double pb = fw.rx[j].x * rxb[j].y - fw.rx[j].y * rxb[j].x;   // Re(conj(rxbar) i rx)
        const double cycb = 2.0 * kPi * pb;
        const double x0 = tab.x[(j * 3 + 0) * N + n], x1 = tab.x[(j * 3 + 1) * N + n],
                     x2 = tab.x[(j * 3 + 2) * N + n];
        const double ux = (c.u[0] * x0 + c.u[1] * x1 + c.u[2] * x2) * inv_c;
        const double vx = (c.v[0] * x0 + c.v[1] * x1) * inv_c;
        const double tk = fw.t - fw.kap[j], fk = fw.f - c.fd * fw.kap[j];
        acc.f0 += cycb * tk;
        acc.fd += 0.5 * cycb * (tk * tk);
        acc.beta -= cycb * fk * ux;
        acc.lam -= cycb * fk * c.cb * vx;
        acc.phi0 += pb;
    }
    // a = f/(2 f*), f = f0 + fdot t
    fb += ab * (0.5 * g.inv_fstar);
    acc.f0 += fb;
    acc.fd += fb * fw.t;
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
    g.inv_fstar = 1.0 / fstar;
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
    if (c_lo + lane < c_hi) setup_grad(theta + 8 * (c_lo + lane), T, g.inv_fstar, mycand[lane]);
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
        template_value(c, g, tab, bufA, bufE, bufT, lane);
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
        // (4) reverse-mode sweep: the adjoint of sample n is c_n = conj(buf[n])
        Acc acc = {0.0, 0.0, 0.0, 0.0, 0.0, {0.0, 0.0}, {0.0, 0.0}};
        for (int n = lane; n < N; n += 32) {
            const C cA = {bufA[n].x, -bufA[n].y}, cE = {bufE[n].x, -bufE[n].y};
            const C cT = useT ? C{bufT[n].x, -bufT[n].y} : C{0.0, 0.0};
            sample_adjoint(c, g, tab, n, cA, cE, cT, useT, acc);
        }
        double gacc[K];
        gacc[0] = acc.f0;
        gacc[1] = acc.fd;
        gacc[2] = acc.beta;
        gacc[3] = acc.lam;
#pragma unroll
        for (int k = 0; k < 3; ++k) gacc[4 + k] = redot(acc.al, c.al_i[k]) + redot(acc.ga, c.ga_i[k]);
        gacc[7] = acc.phi0;
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
