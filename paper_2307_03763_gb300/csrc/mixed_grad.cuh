// mixed_grad.cuh -- the mixed-precision adjoint gradient's device code
// (shared by mixed_grad.cu and mixed_grad_t.cu, which instantiate the kernel
// without and with the T channel).
// ---------------------------------------------------------------------------
// Gradient of the window log-likelihood, mixed precision.
//
// With the unit-amplitude slow part s^ (s = A s^), the float window copy
// (d^ = sigma d, w^ = w / sigma^2) and the unit-amplitude DFT S,
//   r^_k = w^_k (d^_k - kappa S_k),  kappa = sigma A T / (2N),
//   c^_n = sum_k r^_k exp(+2 pi i k n / N)                (adjoint DFT),
//   d logL / d theta_i = (2 sigma A / N) Re sum_n c^_n conj(d s^_n / d theta_i)
// (for theta_i = A the derivative of s = A s^ is s^, without the factor A).
// s^ is linear in the polarisation coefficients: s^ = gp P + gx Q, where P and
// Q are the responses with n.H.n replaced by F+ = n.e+.n and Fx = n.ex.n and
// gp = gpr + i gpi, gx = gxr + i gxi.  So A, iota, psi and phi0 need only the
// two sums V_P = sum c^ conj(P), V_Q = sum c^ conj(Q):
//   d/dA     = (2 sigma/N)   Re(conj(gp) V_P + conj(gx) V_Q)
//   d/diota  = (2 sigma A/N) Re(conj(d_iota gp) V_P + conj(d_iota gx) V_Q), psi alike
//   d/dphi0  = (2 sigma A/N) Im(conj(gp) V_P + conj(gx) V_Q)   (s^ ~ exp(i phi0)).
// f0, fdot, beta, lambda come from the reverse mode of each sample's
// computation (sample_adjoint): the sample's cotangent is propagated back
// through F, the TDI combination and the six links to the receiver phases,
// the transfer functions and the arms' polarisation responses, whose
// parameter derivatives are closed forms.
// ---------------------------------------------------------------------------
#pragma once
#include "mixed_common.cuh"

namespace gb {
namespace {

constexpr int KT = 4;   // f0, fdot, beta, lambda

struct CandGx {
    CandMix m;
    float Uc, Us, Vc, Vs;   // (AU/c)(u.e_x, u.e_y), (AU/c)(v.e_x, v.e_y): guiding-centre parts of u.x/c, v.x/c
    float cb, sb, cl, sl;
    float2 gp, gx, gp_i, gx_i, gp_p, gx_p;   // coefficients and their iota, psi derivatives
};

__device__ void setup_grad_mixed(const double* th, double T, double fstar, CandGx& g) {
    setup_mixed(th, T, 1.0 / fstar, g.m);
    const float beta = (float)th[2], lam = (float)th[3], iota = (float)th[5], psi = (float)th[6];
    float sb, cb, sl, cl, si, ci, s2, c2;
    sincosf(beta, &sb, &cb);
    sincosf(lam, &sl, &cl);
    sincosf(iota, &si, &ci);
    sincosf(2.0f * psi, &s2, &c2);
    const float r = (float)(kAU / kC);
    g.Uc = r * sb * cl;
    g.Us = r * sb * sl;
    g.Vc = r * sl;
    g.Vs = -r * cl;
    g.cb = cb;
    g.sb = sb;
    g.cl = cl;
    g.sl = sl;
    const float Ap = 1.0f + ci * ci, Ax = -2.0f * ci;
    g.gp = make_float2(Ap * c2, -Ax * s2);
    g.gx = make_float2(-Ap * s2, -Ax * c2);
    const float dAp = -2.0f * ci * si, dAx = 2.0f * si;
    g.gp_i = make_float2(dAp * c2, -dAx * s2);
    g.gx_i = make_float2(-dAp * s2, -dAx * c2);
    g.gp_p = make_float2(-2.0f * Ap * s2, -2.0f * Ax * c2);
    g.gx_p = make_float2(-2.0f * Ap * c2, 2.0f * Ax * s2);
}

// sinc(X) exp(-iX) and its derivative in X (Horner with derivative in y = -4X^2)
template <int J>
__device__ __forceinline__ void link_transfer_d(float X, float2& Tv, float2& Td) {
    if (J == 0) {
        float s, co;
        sincosf(X, &s, &co);
        const float sc = X != 0.0f ? s / X : 1.0f;
        Tv = make_float2(sc * co, -sc * s);
        const float iX = X != 0.0f ? 1.0f / X : 0.0f;
        Td = make_float2((co * co - s * s - Tv.x) * iX, (-2.0f * s * co - Tv.y) * iX);
        return;
    }
    const float y = -4.0f * X * X;
    float a = kInvFact[2 * J + 1], da = 0.0f, b = kInvFact[2 * J + 2], db = 0.0f;
#pragma unroll
    for (int j = J - 1; j >= 0; --j) {
        da = fmaf(da, y, a);
        a = fmaf(a, y, kInvFact[2 * j + 1]);
        db = fmaf(db, y, b);
        b = fmaf(b, y, kInvFact[2 * j + 2]);
    }
    // Re T = a(y), Im T = -2X b(y); dy/dX = -8X
    Tv = make_float2(a, -2.0f * X * b);
    Td = make_float2(-8.0f * X * da, -2.0f * b + 16.0f * X * X * db);
}

// One sample's share of the four phase-side derivatives, by reverse mode
// through the sample computation.  With the sample's cotangents cA, cE (cT)
// of the unit-amplitude A, E (T) values, it adds
//   Re sum_ch conj(c_ch) dS_ch / dtheta_k,   k = f0, fdot, beta, lambda,
// to dth[k], and U_P = sum_ch conj(c_ch) P_ch, U_Q likewise, to up, uq.
//
// S_ch = F sum_links mu_ch,l z_l, where z_l = T(X_l) G_arm rx_recv is one
// link (transfer function, polarisation response of its arm, phase at its
// receiver), F = -i a (1 - D^2) and the TDI coefficients mu hold 1, -1 and
// the delay factor D.  So with omega_X,Y,Z = F times the channel weights of
// X, Y, Z, the link cotangent is mu_l = D omega_a - omega_a+1 (the link
// towards arm a+1's end) or omega_a - D omega_a+1 (the other), and
//   d/dtheta Re(mu z) = Re(mu G rx T') dX/dtheta + Re(mu rx T dG/dtheta)
//                       - 2 pi Im(mu z) dphase_recv/dtheta,
// plus the derivatives of F and D themselves (f0 and fdot only).  P and Q are
// S with G replaced by F+ and Fx: U_P = sum_arms Gamma_arm F+, with Gamma the
// arm's sum of mu rx T.
template <int J, bool T3 = false>
__device__ __forceinline__ void sample_adjoint(const CandGx& g, const OrbitTables32& tab, int N, int n, float Tf,
                                               float inv_fstar, float2 cA, float2 cE, float2 cT, float (&dth)[KT],
                                               float2& up, float2& uq) {
    const CandMix& c = g.m;
    const int R = N >> 5;
    const int p = (n % R) * 32 + brev5(n / R);
    const float u = (float)n / (float)N;
    const float uu = u * u;
    const float4 g0 = __ldg(tab.g + p), g1 = __ldg(tab.g + N + p);
    const float4 g2 = __ldg(tab.g + 2 * N + p), g3 = __ldg(tab.g + 3 * N + p);
    const float cah = g3.x, cal = g3.y, sah = g3.z, sal = g3.w;
    // common phase in double-word arithmetic (as in the likelihood kernel)
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
    float Pc, Pl;
    two_sum(s, small, Pc, Pl);
    Pc -= rintf(Pc);
    float sPc, cPc;
    sincospif(2.0f * Pc, &sPc, &cPc);
    const float tl = 6.2831853071795865f * Pl;
    const float2 ePc = make_float2(fmaf(-tl, sPc, cPc), fmaf(tl, cPc, sPc));
    const float f = fmaf(c.fdT, u, c.f0);
    const float fd = 2.0f * c.fdh;
    const float tu = Tf * u;
    float krho[3], urho[3], vrho[3];
    krho[0] = fmaf(c.k0, g0.x, fmaf(c.k1, g0.y, c.k2 * g0.z));
    krho[1] = fmaf(c.k0, g0.w, fmaf(c.k1, g1.x, c.k2 * g1.y));
    urho[0] = fmaf(c.u0, g0.x, fmaf(c.u1, g0.y, c.u2 * g0.z));
    urho[1] = fmaf(c.u0, g0.w, fmaf(c.u1, g1.x, c.u2 * g1.y));
    vrho[0] = fmaf(c.v0, g0.x, c.v1 * g0.y);
    vrho[1] = fmaf(c.v0, g0.w, c.v1 * g1.x);
    krho[2] = -krho[0] - krho[1];
    urho[2] = -urho[0] - urho[1];
    vrho[2] = -vrho[0] - vrho[1];
    // phase factor at each receiver
    float2 rx[3];
    float kap[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        kap[j] = K + krho[j];
        const float dP = fmaf(-f, krho[j], c.fdh * kap[j] * kap[j]);
        rx[j] = cmulf(ePc, cis_rx<J>(dP));
    }
    const float a = fmaf(c.a1, u, c.a0);
    float kn_[3], nu_[3], nv_[3], nw_[3];
    kn_[0] = fmaf(c.k0, g1.z, fmaf(c.k1, g1.w, c.k2 * g2.x));
    nu_[0] = fmaf(c.u0, g1.z, fmaf(c.u1, g1.w, c.u2 * g2.x));
    nv_[0] = fmaf(c.v0, g1.z, c.v1 * g1.w);
    nw_[0] = fmaf(g.cl, g1.z, g.sl * g1.w);
    kn_[1] = fmaf(c.k0, g2.y, fmaf(c.k1, g2.z, c.k2 * g2.w));
    nu_[1] = fmaf(c.u0, g2.y, fmaf(c.u1, g2.z, c.u2 * g2.w));
    nv_[1] = fmaf(c.v0, g2.y, c.v1 * g2.z);
    nw_[1] = fmaf(g.cl, g2.y, g.sl * g2.z);
    kn_[2] = -kn_[0] - kn_[1];
    nu_[2] = -nu_[0] - nu_[1];
    nv_[2] = -nv_[0] - nv_[1];
    nw_[2] = -nw_[0] - nw_[1];
    // links: [arm][0] towards arm+1's end (+n, receiver arm+1), [arm][1] the
    // other (-n, receiver arm); transfer value and derivative, link value
    float2 G[3], Tv[3][2], Td[3][2], z[3][2];
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        const float nu = nu_[arm], nv = nv_[arm];
        const float Fp = (nu - nv) * (nu + nv), Fx = 2.0f * nu * nv;
        G[arm] = make_float2(fmaf(g.gp.x, Fp, g.gx.x * Fx), fmaf(g.gp.y, Fp, g.gx.y * Fx));
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const float X = a * (sgn == 0 ? 1.0f - kn_[arm] : 1.0f + kn_[arm]);
            link_transfer_d<J>(X, Tv[arm][sgn], Td[arm][sgn]);
            const int j = sgn == 0 ? (arm == 2 ? 0 : arm + 1) : arm;
            z[arm][sgn] = cmulf(cmulf(Tv[arm][sgn], G[arm]), rx[j]);
        }
    }
    // delay factor D = exp(-i f/f*) and F = -i a (1 - D^2) = 2 a sin(f/f*) D
    const float du = c.eps * u;
    const float2 D = cmulf(make_float2(c.D0r, c.D0i), make_float2(fmaf(-0.5f * du, du, 1.0f), -du));
    const float sa2 = -2.0f * a * D.y;
    const float2 F = make_float2(sa2 * D.x, sa2 * D.y);
    // first-generation Michelson X, Y, Z (without F)
    const float2 Xp = caddf(csubf(z[0][1], z[2][0]), cmulf(D, csubf(z[0][0], z[2][1])));
    const float2 Yp = caddf(csubf(z[1][1], z[0][0]), cmulf(D, csubf(z[1][0], z[0][1])));
    const float2 Zp = caddf(csubf(z[2][1], z[1][0]), cmulf(D, csubf(z[2][0], z[1][1])));
    // channel weights of X, Y, Z: A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6,
    // T = (X + Y + Z)/sqrt3, each with conj(c)
    const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f;
    const float2 ca = make_float2(cA.x * r2, -cA.y * r2), ce = make_float2(cE.x * r6, -cE.y * r6);
    float2 w[3] = {csubf(ce, ca), make_float2(-2.0f * ce.x, -2.0f * ce.y), caddf(ca, ce)};
    if constexpr (T3) {
        const float r3 = 0.57735026918962576f;
        const float2 ct = make_float2(cT.x * r3, -cT.y * r3);
#pragma unroll
        for (int q = 0; q < 3; ++q) w[q] = caddf(w[q], ct);
    }
    // F and D depend on f0 and fdot: dD = -i D dphi, dphi = (1, t)/f*,
    // d(sa2) = -2 (da D.y + a dD.y), da = (1, t)/(2 f*)
    const float2 Wsum = caddf(caddf(cmulf(w[0], Xp), cmulf(w[1], Yp)), cmulf(w[2], Zp));
    float2 om[3], Dom[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        om[q] = cmulf(F, w[q]);
        Dom[q] = cmulf(D, om[q]);
    }
    const float2 Qd = caddf(caddf(cmulf(om[0], csubf(z[0][0], z[2][1])), cmulf(om[1], csubf(z[1][0], z[0][1]))),
                            cmulf(om[2], csubf(z[2][0], z[1][1])));
    {
        // per unit dphi: dD = -i D, so Re(Qd dD) = Im(Qd D); da = 1/2 and
        // d(sa2) = -2 (D.y / 2 + a (-D.x)) = 2 a D.x - D.y
        const float2 QD = cmulf(Qd, D);
        const float dsa2 = fmaf(2.0f * a, D.x, -D.y);
        const float2 dF = make_float2(fmaf(dsa2, D.x, sa2 * D.y), fmaf(dsa2, D.y, -sa2 * D.x));
        const float fdf = fmaf(dF.x, Wsum.x, -dF.y * Wsum.y) + QD.y;   // per unit dphi
        dth[0] = fmaf(fdf, inv_fstar, dth[0]);
        dth[1] = fmaf(fdf, tu * inv_fstar, dth[1]);
    }
    float A1 = 0.0f;                           // sum of Re(mu G rx T') (1 -+ kn)
    float Phi[3] = {0.0f, 0.0f, 0.0f};         // sum over the receiver's links of Im(mu z)
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        const int an = arm == 2 ? 0 : arm + 1;
        float B = 0.0f;                        // sum of -+ Re(mu G rx T')
        float2 Gam = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int j = sgn == 0 ? an : arm;
            const float2 mu = sgn == 0 ? csubf(Dom[arm], om[an]) : csubf(om[arm], Dom[an]);
            const float2 nu_l = cmulf(mu, rx[j]);
            const float2 nuG = cmulf(nu_l, G[arm]);
            const float rho = fmaf(nuG.x, Td[arm][sgn].x, -nuG.y * Td[arm][sgn].y);
            Phi[j] += fmaf(nuG.x, Tv[arm][sgn].y, nuG.y * Tv[arm][sgn].x);
            Gam = caddf(Gam, cmulf(nu_l, Tv[arm][sgn]));
            const float kf = sgn == 0 ? 1.0f - kn_[arm] : 1.0f + kn_[arm];
            A1 = fmaf(rho, kf, A1);
            B += sgn == 0 ? -rho : rho;
        }
        const float nu = nu_[arm], nv = nv_[arm], nw = nw_[arm], kn = kn_[arm];
        const float Fp = (nu - nv) * (nu + nv), Fx = 2.0f * nu * nv;
        // Re(Gamma dG) = Re(Gamma gp) dF+ + Re(Gamma gx) dFx
        const float gpr = fmaf(Gam.x, g.gp.x, -Gam.y * g.gp.y), gxr = fmaf(Gam.x, g.gx.x, -Gam.y * g.gx.y);
        // beta: dn.u = -k.n, dn.v = 0; lambda: dn.u = -sin(beta) n.v, dn.v = n.w;
        // dX = -+ a dk.n with dk.n = n.u (beta), cos(beta) n.v (lambda)
        const float dnu_l = -g.sb * nv;
        const float dFp_b = -2.0f * nu * kn, dFx_b = -2.0f * kn * nv;
        const float dFp_l = 2.0f * fmaf(nu, dnu_l, -nv * nw), dFx_l = 2.0f * fmaf(dnu_l, nv, nu * nw);
        dth[2] += fmaf(gpr, dFp_b, fmaf(gxr, dFx_b, a * B * nu));
        dth[3] += fmaf(gpr, dFp_l, fmaf(gxr, dFx_l, a * B * g.cb * nv));
        up = caddf(up, make_float2(Gam.x * Fp, Gam.y * Fp));
        uq = caddf(uq, make_float2(Gam.x * Fx, Gam.y * Fx));
    }
    // transfer functions: dX = da (1 -+ kn), da = (1, t)/(2 f*)
    dth[0] = fmaf(A1, 0.5f * inv_fstar, dth[0]);
    dth[1] = fmaf(A1, 0.5f * tu * inv_fstar, dth[1]);
    // receiver phases: d phase_j = (t - kap, (t - kap)^2/2, -(f - fdot kap) u.x_j/c,
    // -(f - fdot kap) cos(beta) v.x_j/c) cycles
    const float ux0 = fmaf(g.Uc, cah, g.Us * sah), vx0 = fmaf(g.Vc, cah, g.Vs * sah);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float ph = -6.2831853071795865f * Phi[j];
        const float tk = tu - kap[j];
        const float fk = fmaf(-fd, kap[j], f);
        dth[0] = fmaf(ph, tk, dth[0]);
        dth[1] = fmaf(ph, 0.5f * tk * tk, dth[1]);
        dth[2] = fmaf(ph, -fk * (ux0 + urho[j]), dth[2]);
        dth[3] = fmaf(ph, -fk * g.cb * (vx0 + vrho[j]), dth[3]);
    }
}

// The sample adjoints of one candidate: lane l takes samples l, l + 32, ...
// (cA, cE, cT: the adjoint transform's output c^_n; cT may be null in the T
// instantiation, for windows without T).  Sums are compensated per lane.
template <int J, bool T3 = false>
__device__ void adjoint_sweep(const CandGx& g, const OrbitTables32& tab, int N, float Tf, float inv_fstar,
                              const float2* cA, const float2* cE, int lane, float (&tacc)[KT][2],
                              float (&vp)[2][2], float (&vq)[2][2], const float2* cT = nullptr) {
    for (int n = lane; n < N; n += 32) {
        float dth[KT] = {0.0f, 0.0f, 0.0f, 0.0f};
        float2 up = make_float2(0.0f, 0.0f), uq = make_float2(0.0f, 0.0f);
        const float2 t = (T3 && cT) ? cT[n] : make_float2(0.0f, 0.0f);
        sample_adjoint<J, T3>(g, tab, N, n, Tf, inv_fstar, cA[n], cE[n], t, dth, up, uq);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            f2 sum = make_float2(tacc[2 * p][0], tacc[2 * p + 1][0]), comp = make_float2(tacc[2 * p][1], tacc[2 * p + 1][1]);
            kahan_add2(sum, comp, make_float2(dth[2 * p], dth[2 * p + 1]));
            tacc[2 * p][0] = sum.x;
            tacc[2 * p + 1][0] = sum.y;
            tacc[2 * p][1] = comp.x;
            tacc[2 * p + 1][1] = comp.y;
        }
        // V = sum c conj(P) = conj(U_P)
        kahan_add(vp[0][0], vp[0][1], up.x);
        kahan_add(vp[1][0], vp[1][1], -up.y);
        kahan_add(vq[0][0], vq[0][1], uq.x);
        kahan_add(vq[1][0], vq[1][1], -uq.y);
    }
}

// Forward FFT of R register values per lane: on entry lane l holds input
// index R brev5(l) + r in x[r]; on exit it holds output index l + 32 r.
template <int R>
__device__ __forceinline__ void fft_regs(float2 (&x)[R], const OrbitTables32& tab, const float2* tw1024,
                                         const LaneTw& ltw, int lane) {
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = lane_fft(x[r], ltw, lane);
#pragma unroll
    for (int r = 1; r < R; ++r) x[r] = cmulf(x[r], __ldg(tab.ltw + r * 32 + lane));
    reg_fft<R>(x, tw1024);
}

// Per-candidate sums left for the epilogue (compensated float pairs).
struct EpiG {
    float dh[2], hh[2];
    float t[KT][2];
    float vp[2][2], vq[2][2];   // [re, im][hi, lo]
};

// Forward FFT of one channel, window inner products, residual (conjugated) in
// natural bin order in buf, then the adjoint FFT leaving c^_n = buf[n].
template <int R>
__device__ void residual_adjoint(float2* buf, int ch, const OrbitTables32& tab, const float2* tw1024,
                                 const LaneTw& ltw, int lane, int off, int W, const Win32* __restrict__ pw,
                                 float kappa, float& sdh, float& cdh, float& shh, float& chh) {
    constexpr int N = 32 * R;
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = buf[r * 32 + lane];
    fft_regs<R>(x, tab, tw1024, ltw, lane);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
        const int k = lane + 32 * k1;
        const int m = k < N / 2 ? k : k - N;
        const int kk = off + m;
        float2 rc = make_float2(0.0f, 0.0f);
        if (kk >= 0 && kk < W) {
            const Win32 v = pw[kk];
            const float2 d = ch == 0 ? make_float2(v.dre.x, v.dim.x) : make_float2(v.dre.y, v.dim.y);
            const float w = ch == 0 ? v.w.x : v.w.y;
            kahan_add(sdh, cdh, __fmul_rn(w, fmaf(d.x, x[k1].x, d.y * x[k1].y)));
            kahan_add(shh, chh, __fmul_rn(w, fmaf(x[k1].x, x[k1].x, x[k1].y * x[k1].y)));
            rc = make_float2(w * fmaf(-kappa, x[k1].x, d.x), -(w * fmaf(-kappa, x[k1].y, d.y)));   // conj(r)
        }
        buf[k] = rc;
    }
    __syncwarp();
    const int nb = R * brev5(lane);
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = buf[nb + r];
    fft_regs<R>(x, tab, tw1024, ltw, lane);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) buf[lane + 32 * k1] = make_float2(x[k1].x, -x[k1].y);   // c^_n
    __syncwarp();
}

// resident CTAs per SM the N <= 256 instantiation is compiled for (register cap)
#ifndef GB_GRAD_MINB
#define GB_GRAD_MINB 2
#endif

template <int RMAX, bool T3>
__global__ void __launch_bounds__(kWarpsMx * 32, RMAX <= 8 ? GB_GRAD_MINB : 1) grad_mixed_kernel(
    const gb_window_t* __restrict__ wins, const WinMeta* __restrict__ meta, const Win32* __restrict__ prep,
    const Tile* __restrict__ items, int n_items, int* head, TabSet32 tabs, const float2* __restrict__ tw1024,
    double T, double fstar, const double* __restrict__ theta, double* __restrict__ logL,
    double* __restrict__ grad, int* status, int n_max, unsigned long long budget_ns, long long n_prep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CandGx* cands = (CandGx*)smem_raw + warp * 32;
    EpiG* epi = (EpiG*)((CandGx*)smem_raw + kWarpsMx * 32) + warp * 32;
    float2* bufA = (float2*)((EpiG*)((CandGx*)smem_raw + kWarpsMx * 32) + kWarpsMx * 32) + (size_t)warp * 2 * n_max;
    float2* bufE = bufA + n_max;
    // T3: one more buffer per warp, for T
    float2* bufT = T3 ? (float2*)((EpiG*)((CandGx*)smem_raw + kWarpsMx * 32) + kWarpsMx * 32) +
                            (size_t)kWarpsMx * 2 * n_max + (size_t)warp * n_max
                      : nullptr;
    const LaneTw ltw = lane_twiddles(lane);
    const float Tf = (float)T, inv_fstar = (float)(1.0 / fstar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        // a warp past the time budget takes no further item and flags it
        int item = 0;
        if (lane == 0) {
            if (budget_ns != 0ULL && global_ns() - t0 > budget_ns) {
                atomicOr(status, kStatusBudget);
                item = n_items;
            } else {
                item = atomicAdd(head, 1);
            }
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const Tile t = items[item];
        const gb_window_t win = wins[t.win];
        const WinMeta wm = meta[t.win];
        const Win32* pw = prep + wm.prep_off;
        const int N = win.N;
        const OrbitTables32 tab = tabs.t[__ffs(N) - 6];
        const int cnt = (int)(t.c_end - t.c_begin);
        const bool useT = T3 && wm.use_t;
        const Win32* pwT = prep + n_prep + wm.prep_off;
        if (lane < cnt) setup_grad_mixed(theta + 8 * (t.c_begin + lane), T, fstar, cands[lane]);
        __syncwarp();
        for (int i = 0; i < cnt; ++i) {
            const CandGx& g = cands[i];
            float sdh = 0.0f, cdh = 0.0f, shh = 0.0f, chh = 0.0f;
            float tacc[KT][2] = {}, vp[2][2] = {}, vq[2][2] = {};
            if (!g.m.bad) {
                slow_part_dispatch<false, T3>(g.m, tab, N, bufA, bufE, lane, useT ? bufT : nullptr);
                __syncwarp();
                const long long off64 = g.m.q - win.k0;
                const int off = (off64 > -(long long)N && off64 < (long long)win.W + N) ? (int)off64 : -4 * N;
                const float kappa = (float)(wm.sig * g.m.A * T / (2.0 * (double)N));
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    float2* buf = ch == 0 ? bufA : bufE;
                    if constexpr (RMAX <= 8) {
                        switch (N) {
                            case 32: residual_adjoint<1>(buf, ch, tab, tw1024, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                            case 64: residual_adjoint<2>(buf, ch, tab, tw1024, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                            case 128: residual_adjoint<4>(buf, ch, tab, tw1024, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                            default: residual_adjoint<8>(buf, ch, tab, tw1024, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                        }
                    } else {
                        if (N == 512)
                            residual_adjoint<16>(buf, ch, tab, tw1024, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh);
                        else
                            residual_adjoint<32>(buf, ch, tab, tw1024, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh);
                    }
                }
                if constexpr (T3) {
                    if (useT) {   // T's data sit in the first slot of each pair of its float copy
                        if constexpr (RMAX <= 8) {
                            switch (N) {
                                case 32: residual_adjoint<1>(bufT, 0, tab, tw1024, ltw, lane, off, win.W, pwT, kappa, sdh, cdh, shh, chh); break;
                                case 64: residual_adjoint<2>(bufT, 0, tab, tw1024, ltw, lane, off, win.W, pwT, kappa, sdh, cdh, shh, chh); break;
                                case 128: residual_adjoint<4>(bufT, 0, tab, tw1024, ltw, lane, off, win.W, pwT, kappa, sdh, cdh, shh, chh); break;
                                default: residual_adjoint<8>(bufT, 0, tab, tw1024, ltw, lane, off, win.W, pwT, kappa, sdh, cdh, shh, chh); break;
                            }
                        } else {
                            if (N == 512)
                                residual_adjoint<16>(bufT, 0, tab, tw1024, ltw, lane, off, win.W, pwT, kappa, sdh, cdh, shh, chh);
                            else
                                residual_adjoint<32>(bufT, 0, tab, tw1024, ltw, lane, off, win.W, pwT, kappa, sdh, cdh, shh, chh);
                        }
                    }
                }
                const float2* cT = useT ? bufT : nullptr;
                switch (g.m.J) {
                    case 4: adjoint_sweep<4, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                    case 7: adjoint_sweep<7, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                    case 10: adjoint_sweep<10, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                    default: adjoint_sweep<0, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                }
                __syncwarp();
            }
            EpiG s;
            warp_sum2(sdh, cdh, s.dh[0], s.dh[1]);
            warp_sum2(shh, chh, s.hh[0], s.hh[1]);
#pragma unroll
            for (int k = 0; k < KT; ++k) warp_sum2(tacc[k][0], tacc[k][1], s.t[k][0], s.t[k][1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                warp_sum2(vp[q][0], vp[q][1], s.vp[q][0], s.vp[q][1]);
                warp_sum2(vq[q][0], vq[q][1], s.vq[q][0], s.vq[q][1]);
            }
            if (lane == 0) epi[i] = s;
        }
        __syncwarp();
        if (lane < cnt) {
            const CandGx& g = cands[lane];
            const int64_t cidx = t.c_begin + lane;
            if (g.m.bad) {
                if (logL) logL[cidx] = nan("");
                for (int k = 0; k < 8; ++k) grad[8 * cidx + k] = nan("");
                atomicOr(status, kStatusNonFinite);
            } else {
                const EpiG& s = epi[lane];
                const double A = g.m.A, sig = wm.sig;
                const double dh = A * (2.0 * sig / (double)N) * ((double)s.dh[0] + (double)s.dh[1]);
                const double hh = A * A * (T * sig * sig / ((double)N * (double)N)) * ((double)s.hh[0] + (double)s.hh[1]);
                if (logL) logL[cidx] = dh - 0.5 * hh - 0.5 * wm.dd;
                const double sc = 2.0 * sig / (double)N;
                const double VPr = (double)s.vp[0][0] + s.vp[0][1], VPi = (double)s.vp[1][0] + s.vp[1][1];
                const double VQr = (double)s.vq[0][0] + s.vq[0][1], VQi = (double)s.vq[1][0] + s.vq[1][1];
                // Re(conj(a) V) = a.x V.x + a.y V.y ; Im(conj(a) V) = a.x V.y - a.y V.x
                auto re_c = [&](float2 a, float2 b) { return (double)a.x * VPr + (double)a.y * VPi + (double)b.x * VQr + (double)b.y * VQi; };
                const double im0 = (double)g.gp.x * VPi - (double)g.gp.y * VPr + (double)g.gx.x * VQi - (double)g.gx.y * VQr;
                double out[8];
                for (int k = 0; k < KT; ++k) out[k] = sc * A * ((double)s.t[k][0] + (double)s.t[k][1]);
                out[4] = sc * re_c(g.gp, g.gx);
                out[5] = sc * A * re_c(g.gp_i, g.gx_i);
                out[6] = sc * A * re_c(g.gp_p, g.gx_p);
                out[7] = sc * A * im0;
                for (int k = 0; k < 8; ++k) grad[8 * cidx + k] = out[k];
            }
        }
        __syncwarp();
    }
}

}  // namespace
}  // namespace gb
