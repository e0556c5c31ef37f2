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

// sinc(X) exp(-iX) and its X derivative for a pair (see link_transfer_d)
template <int J>
__device__ __forceinline__ void plink_transfer_d(f2 X, cpair& Tv, cpair& Td) {
    if constexpr (J == 0) {
        float2 a, da, b, db;
        link_transfer_d<0>(X.x, a, da);
        link_transfer_d<0>(X.y, b, db);
        Tv = cpair{make_float2(a.x, b.x), make_float2(a.y, b.y)};
        Td = cpair{make_float2(da.x, db.x), make_float2(da.y, db.y)};
    } else {
        const f2 y = pmul(bc(-4.0f), pmul(X, X));
        const float4 cJ = kLinkPair[J];
        f2 a = make_float2(cJ.x, cJ.y), b = make_float2(cJ.z, cJ.w), da = bc(0.0f), db = bc(0.0f);
#pragma unroll
        for (int j = J - 1; j >= 0; --j) {
            const float4 cj = kLinkPair[j];
            da = pfma(da, y, a);
            a = pfma(a, y, make_float2(cj.x, cj.y));
            db = pfma(db, y, b);
            b = pfma(b, y, make_float2(cj.z, cj.w));
        }
        // Re T = a(y), Im T = -2X b(y); dy/dX = -8X
        Tv = cpair{a, pmul(pmul(bc(-2.0f), X), b)};
        Td = cpair{pmul(pmul(bc(-8.0f), X), da), pfma(pmul(bc(16.0f), pmul(X, X)), db, pmul(bc(-2.0f), b))};
    }
}

__device__ __forceinline__ cpair pcbc(float2 v) { return cpair{bc(v.x), bc(v.y)}; }
__device__ __forceinline__ cpair pcscale(cpair a, f2 s) { return cpair{pmul(a.re, s), pmul(a.im, s)}; }
// Re(a b) and Im(a b) of a pair
__device__ __forceinline__ f2 pcre(cpair a, cpair b) { return pfma(a.re, b.re, pneg(pmul(a.im, b.im))); }
__device__ __forceinline__ f2 pcim(cpair a, cpair b) { return pfma(a.re, b.im, pmul(a.im, b.re)); }

// One sample's share of the four phase-side derivatives, by reverse mode
// through the sample computation, for the two samples n0 and n0 + 32 at once
// (packed FP32; a second sample past N has zero cotangents).  With the
// samples' cotangents cA, cE (cT) of the unit-amplitude A, E (T) values, it
// adds
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
__device__ __forceinline__ void sample_adjoint(const CandGx& g, const OrbitTables32& tab, int N, int n0, int n1,
                                               unsigned pha, unsigned phb, float Tf, float inv_fstar, cpair cA,
                                               cpair cE, cpair cT, f2 (&dth)[KT], cpair& up, cpair& uq) {
    const CandMix& c = g.m;
    const int R = N >> 5;
    const int pa = (n0 % R) * 32 + brev5(n0 / R), pb = (n1 % R) * 32 + brev5(n1 / R);
    const float4 a0 = __ldg(tab.g + pa), a1 = __ldg(tab.g + N + pa);
    const float4 a2 = __ldg(tab.g + 2 * N + pa), a3 = __ldg(tab.g + 3 * N + pa);
    const float4 b0 = __ldg(tab.g + pb), b1 = __ldg(tab.g + N + pb);
    const float4 b2 = __ldg(tab.g + 2 * N + pb), b3 = __ldg(tab.g + 3 * N + pb);
    const f2 u = pmul(make_float2((float)n0, (float)n1), bc(1.0f / (float)N));
    const f2 uu = pmul(u, u);
    const f2 cah = make_float2(a3.x, b3.x), cal = make_float2(a3.y, b3.y);
    const f2 sah = make_float2(a3.z, b3.z), sal = make_float2(a3.w, b3.w);
    const f2 K = pfma(bc(c.Kc), cah, pmul(bc(c.Ks), sah));
    f2 Pc, tl;   // the common phase: Pc + tl / (2 pi) cycles
    if (!c.wide) {
        // common phase in fixed point, as in the likelihood kernel (pha, phb:
        // the recurrence's top words for n0, n1)
        const int2 qa = __ldg(tab.gq + n0), qb = __ldg(tab.gq + n1);
        phase_fix(c, pha, phb, qa.x, qa.y, qb.x, qb.y, pmul(pneg(pmul(bc(c.fdT), u)), K), Pc, tl);
    } else {
        // outside the fixed-point ranges: double-word arithmetic
        f2 p1 = pmul(bc(c.c1h), u);
        const f2 e1 = pfma(bc(c.c1l), u, pfma(bc(c.c1h), u, pneg(p1)));
        f2 p2 = pmul(bc(c.c2h), uu);
        const f2 e2 = pfma(bc(c.c2l), uu, pfma(bc(c.c2h), uu, pneg(p2)));
        f2 p3 = pmul(bc(c.Fch), cah);
        const f2 e3 = padd(pfma(bc(c.Fch), cah, pneg(p3)), pfma(bc(c.Fch), cal, pmul(bc(c.Fcl), cah)));
        f2 p4 = pmul(bc(c.Fsh), sah);
        const f2 e4 = padd(pfma(bc(c.Fsh), sah, pneg(p4)), pfma(bc(c.Fsh), sal, pmul(bc(c.Fsl), sah)));
        p1 = psub(p1, print(p1));
        p2 = psub(p2, print(p2));
        p3 = psub(p3, print(p3));
        p4 = psub(p4, print(p4));
        f2 s, e, ea, eb, ec;
        ptwo_sum(bc(c.c0h), p1, s, ea);
        ptwo_sum(s, p2, s, eb);
        ptwo_sum(s, pneg(p3), s, ec);
        ptwo_sum(s, pneg(p4), s, e);
        s = psub(s, print(s));
        const f2 lo = padd(psub(psub(padd(padd(bc(c.c0l), e1), e2), e3), e4), padd(padd(padd(ea, eb), ec), e));
        const f2 small = pfma(pneg(pmul(bc(c.fdT), u)), K, lo);
        f2 Pl;
        ptwo_sum(s, small, Pc, Pl);
        Pc = psub(Pc, print(Pc));
        tl = pmul(bc(6.2831853071795865f), Pl);
    }
    float sx, cx, sy, cy;
    sincospif(2.0f * Pc.x, &sx, &cx);
    sincospif(2.0f * Pc.y, &sy, &cy);
    const f2 sP = make_float2(sx, sy), cP = make_float2(cx, cy);
    const cpair ePc{pfma(pneg(tl), sP, cP), pfma(tl, cP, sP)};
    const f2 f = pfma(bc(c.fdT), u, bc(c.f0));
    const f2 tu = pmul(bc(Tf), u);
    // geometry: spacecraft offsets rho_0, rho_1 and arm vectors n_0, n_1
    const f2 r0x = make_float2(a0.x, b0.x), r0y = make_float2(a0.y, b0.y), r0z = make_float2(a0.z, b0.z);
    const f2 r1x = make_float2(a0.w, b0.w), r1y = make_float2(a1.x, b1.x), r1z = make_float2(a1.y, b1.y);
    const f2 n0x = make_float2(a1.z, b1.z), n0y = make_float2(a1.w, b1.w), n0z = make_float2(a2.x, b2.x);
    const f2 n1x = make_float2(a2.y, b2.y), n1y = make_float2(a2.z, b2.z), n1z = make_float2(a2.w, b2.w);
    f2 krho[3], urho[3], vrho[3];
    krho[0] = pfma(bc(c.k0), r0x, pfma(bc(c.k1), r0y, pmul(bc(c.k2), r0z)));
    krho[1] = pfma(bc(c.k0), r1x, pfma(bc(c.k1), r1y, pmul(bc(c.k2), r1z)));
    urho[0] = pfma(bc(c.u0), r0x, pfma(bc(c.u1), r0y, pmul(bc(c.u2), r0z)));
    urho[1] = pfma(bc(c.u0), r1x, pfma(bc(c.u1), r1y, pmul(bc(c.u2), r1z)));
    vrho[0] = pfma(bc(c.v0), r0x, pmul(bc(c.v1), r0y));
    vrho[1] = pfma(bc(c.v0), r1x, pmul(bc(c.v1), r1y));
    krho[2] = psub(pneg(krho[0]), krho[1]);
    urho[2] = psub(pneg(urho[0]), urho[1]);
    vrho[2] = psub(pneg(vrho[0]), vrho[1]);
    // phase factor at each receiver
    cpair rx[3];
    f2 kap[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        kap[j] = padd(K, krho[j]);
        const f2 dP = pfma(pneg(f), krho[j], pmul(pmul(bc(c.fdh), kap[j]), kap[j]));
        rx[j] = pcmul(ePc, pcis_rx<J>(dP));
    }
    const f2 a = pfma(bc(c.a1), u, bc(c.a0));
    f2 kn_[3], nu_[3], nv_[3], nw_[3];
    kn_[0] = pfma(bc(c.k0), n0x, pfma(bc(c.k1), n0y, pmul(bc(c.k2), n0z)));
    nu_[0] = pfma(bc(c.u0), n0x, pfma(bc(c.u1), n0y, pmul(bc(c.u2), n0z)));
    nv_[0] = pfma(bc(c.v0), n0x, pmul(bc(c.v1), n0y));
    nw_[0] = pfma(bc(g.cl), n0x, pmul(bc(g.sl), n0y));
    kn_[1] = pfma(bc(c.k0), n1x, pfma(bc(c.k1), n1y, pmul(bc(c.k2), n1z)));
    nu_[1] = pfma(bc(c.u0), n1x, pfma(bc(c.u1), n1y, pmul(bc(c.u2), n1z)));
    nv_[1] = pfma(bc(c.v0), n1x, pmul(bc(c.v1), n1y));
    nw_[1] = pfma(bc(g.cl), n1x, pmul(bc(g.sl), n1y));
    kn_[2] = psub(pneg(kn_[0]), kn_[1]);
    nu_[2] = psub(pneg(nu_[0]), nu_[1]);
    nv_[2] = psub(pneg(nv_[0]), nv_[1]);
    nw_[2] = psub(pneg(nw_[0]), nw_[1]);
    // links: [arm][0] towards arm+1's end (+n, receiver arm+1), [arm][1] the
    // other (-n, receiver arm); transfer value and derivative, link value
    cpair G[3], Tv[3][2], Td[3][2], z[3][2];
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        const f2 nu = nu_[arm], nv = nv_[arm];
        const f2 Fp = pmul(psub(nu, nv), padd(nu, nv)), Fx = pmul(pmul(bc(2.0f), nu), nv);
        G[arm] = cpair{pfma(bc(g.gp.x), Fp, pmul(bc(g.gx.x), Fx)), pfma(bc(g.gp.y), Fp, pmul(bc(g.gx.y), Fx))};
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const f2 X = pmul(a, sgn == 0 ? psub(bc(1.0f), kn_[arm]) : padd(bc(1.0f), kn_[arm]));
            plink_transfer_d<J>(X, Tv[arm][sgn], Td[arm][sgn]);
            const int j = sgn == 0 ? (arm == 2 ? 0 : arm + 1) : arm;
            z[arm][sgn] = pcmul(pcmul(Tv[arm][sgn], G[arm]), rx[j]);
        }
    }
    // delay factor D = exp(-i f/f*) and F = -i a (1 - D^2) = 2 a sin(f/f*) D
    const f2 du = pmul(bc(c.eps), u);
    const cpair D = pcmul(cpair{bc(c.D0r), bc(c.D0i)}, cpair{pfma(pmul(bc(-0.5f), du), du, bc(1.0f)), pneg(du)});
    const f2 sa2 = pmul(pmul(bc(-2.0f), a), D.im);
    const cpair F = pcscale(D, sa2);
    // first-generation Michelson X, Y, Z (without F)
    const cpair Xp = pcadd(pcsub(z[0][1], z[2][0]), pcmul(D, pcsub(z[0][0], z[2][1])));
    const cpair Yp = pcadd(pcsub(z[1][1], z[0][0]), pcmul(D, pcsub(z[1][0], z[0][1])));
    const cpair Zp = pcadd(pcsub(z[2][1], z[1][0]), pcmul(D, pcsub(z[2][0], z[1][1])));
    // channel weights of X, Y, Z: A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6,
    // T = (X + Y + Z)/sqrt3, each with conj(c)
    const f2 r2 = bc(0.70710678118654752f), r6 = bc(0.40824829046386302f);
    const cpair ca{pmul(cA.re, r2), pneg(pmul(cA.im, r2))}, ce{pmul(cE.re, r6), pneg(pmul(cE.im, r6))};
    cpair w[3] = {pcsub(ce, ca), pcscale(ce, bc(-2.0f)), pcadd(ca, ce)};
    if constexpr (T3) {
        const f2 r3 = bc(0.57735026918962576f);
        const cpair ct{pmul(cT.re, r3), pneg(pmul(cT.im, r3))};
#pragma unroll
        for (int q = 0; q < 3; ++q) w[q] = pcadd(w[q], ct);
    }
    const cpair Wsum = pcadd(pcadd(pcmul(w[0], Xp), pcmul(w[1], Yp)), pcmul(w[2], Zp));
    cpair om[3], Dom[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        om[q] = pcmul(F, w[q]);
        Dom[q] = pcmul(D, om[q]);
    }
    const cpair Qd = pcadd(pcadd(pcmul(om[0], pcsub(z[0][0], z[2][1])), pcmul(om[1], pcsub(z[1][0], z[0][1]))),
                           pcmul(om[2], pcsub(z[2][0], z[1][1])));
    {
        // F and D depend on f0 and fdot through dphi = (1, t)/f*: per unit
        // dphi, dD = -i D, so Re(Qd dD) = Im(Qd D); da = 1/2 and
        // d(sa2) = -2 (D.y / 2 + a (-D.x)) = 2 a D.x - D.y
        const f2 dsa2 = pfma(pmul(bc(2.0f), a), D.re, pneg(D.im));
        const cpair dF{pfma(dsa2, D.re, pmul(sa2, D.im)), pfma(dsa2, D.im, pneg(pmul(sa2, D.re)))};
        const f2 fdf = padd(pcre(dF, Wsum), pcim(Qd, D));   // per unit dphi
        dth[0] = pfma(fdf, bc(inv_fstar), dth[0]);
        dth[1] = pfma(fdf, pmul(tu, bc(inv_fstar)), dth[1]);
    }
    f2 A1 = bc(0.0f);                          // sum of Re(mu G rx T') (1 -+ kn)
    f2 Phi[3] = {bc(0.0f), bc(0.0f), bc(0.0f)};   // sum over the receiver's links of Im(mu z)
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        const int an = arm == 2 ? 0 : arm + 1;
        f2 B = bc(0.0f);                       // sum of -+ Re(mu G rx T')
        cpair Gam{bc(0.0f), bc(0.0f)};
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int j = sgn == 0 ? an : arm;
            const cpair mu = sgn == 0 ? pcsub(Dom[arm], om[an]) : pcsub(om[arm], Dom[an]);
            const cpair nl = pcmul(mu, rx[j]);
            const cpair nG = pcmul(nl, G[arm]);
            const f2 rho = pcre(nG, Td[arm][sgn]);
            Phi[j] = padd(Phi[j], pcim(nG, Tv[arm][sgn]));
            Gam = pcadd(Gam, pcmul(nl, Tv[arm][sgn]));
            const f2 kf = sgn == 0 ? psub(bc(1.0f), kn_[arm]) : padd(bc(1.0f), kn_[arm]);
            A1 = pfma(rho, kf, A1);
            B = sgn == 0 ? psub(B, rho) : padd(B, rho);
        }
        const f2 nu = nu_[arm], nv = nv_[arm], nw = nw_[arm], kn = kn_[arm];
        const f2 Fp = pmul(psub(nu, nv), padd(nu, nv)), Fx = pmul(pmul(bc(2.0f), nu), nv);
        // Re(Gamma dG) = Re(Gamma gp) dF+ + Re(Gamma gx) dFx
        const f2 gpr = pcre(Gam, pcbc(g.gp)), gxr = pcre(Gam, pcbc(g.gx));
        // beta: dn.u = -k.n, dn.v = 0; lambda: dn.u = -sin(beta) n.v, dn.v = n.w;
        // dX = -+ a dk.n with dk.n = n.u (beta), cos(beta) n.v (lambda)
        const f2 dnu_l = pmul(bc(-g.sb), nv);
        const f2 dFp_b = pmul(pmul(bc(-2.0f), nu), kn), dFx_b = pmul(pmul(bc(-2.0f), kn), nv);
        const f2 dFp_l = pmul(bc(2.0f), pfma(nu, dnu_l, pneg(pmul(nv, nw))));
        const f2 dFx_l = pmul(bc(2.0f), pfma(dnu_l, nv, pmul(nu, nw)));
        const f2 aB = pmul(a, B);
        dth[2] = padd(dth[2], pfma(gpr, dFp_b, pfma(gxr, dFx_b, pmul(aB, nu))));
        dth[3] = padd(dth[3], pfma(gpr, dFp_l, pfma(gxr, dFx_l, pmul(pmul(aB, bc(g.cb)), nv))));
        up = pcadd(up, pcscale(Gam, Fp));
        uq = pcadd(uq, pcscale(Gam, Fx));
    }
    // transfer functions: dX = da (1 -+ kn), da = (1, t)/(2 f*)
    dth[0] = pfma(A1, bc(0.5f * inv_fstar), dth[0]);
    dth[1] = pfma(A1, pmul(tu, bc(0.5f * inv_fstar)), dth[1]);
    // receiver phases: d phase_j = (t - kap, (t - kap)^2/2, -(f - fdot kap) u.x_j/c,
    // -(f - fdot kap) cos(beta) v.x_j/c) cycles
    const f2 ux0 = pfma(bc(g.Uc), cah, pmul(bc(g.Us), sah)), vx0 = pfma(bc(g.Vc), cah, pmul(bc(g.Vs), sah));
    const float fd = 2.0f * c.fdh;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const f2 ph = pmul(bc(-6.2831853071795865f), Phi[j]);
        const f2 tk = psub(tu, kap[j]);
        const f2 mfk = pfma(bc(fd), kap[j], pneg(f));   // -(f - fdot kap)
        dth[0] = pfma(ph, tk, dth[0]);
        dth[1] = pfma(pmul(ph, bc(0.5f)), pmul(tk, tk), dth[1]);
        dth[2] = pfma(pmul(ph, mfk), padd(ux0, urho[j]), dth[2]);
        dth[3] = pfma(pmul(ph, mfk), pmul(bc(g.cb), padd(vx0, vrho[j])), dth[3]);
    }
}

// The sample adjoints of one candidate: lane l takes the sample pairs
// (l + 64 m, l + 64 m + 32) (cA, cE, cT: the adjoint transform's output c^_n;
// cT may be null in the T instantiation, for windows without T).  Sums are
// per lane and sample slot, then merged exactly (two-sum of the slots).
// PACKED: the cotangents of both channels come from one array of
// channel-pair elements (A re, E re, A im, E im) at nat_sw(n, N) (cA; cE
// unused).
template <int J, bool T3 = false, bool PACKED = false>
__device__ void adjoint_sweep(const CandGx& g, const OrbitTables32& tab, int N, float Tf, float inv_fstar,
                              const float2* cA, const float2* cE, int lane, float (&tacc)[KT][2],
                              float (&vp)[2][2], float (&vq)[2][2], const float2* cT = nullptr) {
    // per-lane plain sums: a lane adds N/64 terms; the warp reduction after
    // the sweep is compensated
    f2 sum[KT + 4];
#pragma unroll
    for (int k = 0; k < KT + 4; ++k) sum[k] = bc(0.0f);
    PhaseRec rec(g.m, N, lane);
    for (int n0 = lane; n0 < N; n0 += 64) {
        // N = 32: the second slot repeats sample n0 with zero cotangents
        const bool two = n0 + 32 < N;
        const int n1 = two ? n0 + 32 : n0;
        auto ld = [&](const float2* b) {
            const float2 x = b[n0], y = two ? b[n1] : make_float2(0.0f, 0.0f);
            return cpair{make_float2(x.x, y.x), make_float2(x.y, y.y)};
        };
        cpair a, e;
        if constexpr (PACKED) {
            const float4* b4 = (const float4*)cA;
            const float4 x = b4[nat_sw(n0, N)], y = two ? b4[nat_sw(n1, N)] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            a = cpair{make_float2(x.x, y.x), make_float2(x.z, y.z)};
            e = cpair{make_float2(x.y, y.y), make_float2(x.w, y.w)};
        } else {
            a = ld(cA);
            e = ld(cE);
        }
        const cpair t = (T3 && cT) ? ld(cT) : cpair{bc(0.0f), bc(0.0f)};
        f2 dth[KT] = {bc(0.0f), bc(0.0f), bc(0.0f), bc(0.0f)};
        cpair up{bc(0.0f), bc(0.0f)}, uq{bc(0.0f), bc(0.0f)};
        unsigned pha, phb;
        rec.next(pha, phb);
        sample_adjoint<J, T3>(g, tab, N, n0, n1, pha, phb, Tf, inv_fstar, a, e, t, dth, up, uq);
#pragma unroll
        for (int k = 0; k < KT; ++k) sum[k] = padd(sum[k], dth[k]);
        // V = sum c conj(P) = conj(U_P)
        sum[KT] = padd(sum[KT], up.re);
        sum[KT + 1] = psub(sum[KT + 1], up.im);
        sum[KT + 2] = padd(sum[KT + 2], uq.re);
        sum[KT + 3] = psub(sum[KT + 3], uq.im);
    }
    const f2 z = bc(0.0f);
#pragma unroll
    for (int k = 0; k < KT; ++k) kahan_merge(sum[k], z, tacc[k][0], tacc[k][1]);
    kahan_merge(sum[KT], z, vp[0][0], vp[0][1]);
    kahan_merge(sum[KT + 1], z, vp[1][0], vp[1][1]);
    kahan_merge(sum[KT + 2], z, vq[0][0], vq[0][1]);
    kahan_merge(sum[KT + 3], z, vq[1][0], vq[1][1]);
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
    // the residual is stored swizzled, entry e at e ^ ((e >> SH) & 15): both
    // the natural-order writes and the transform's transposed reads (lane l,
    // entries R brev5(l) + r) then touch 16 distinct bank pairs per half warp
    constexpr int SH = (R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5) + 1;
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
        buf[k ^ ((k >> SH) & 15)] = rc;
    }
    __syncwarp();
    const int nb = R * brev5(lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = nb + r;
        x[r] = buf[e ^ ((e >> SH) & 15)];
    }
    fft_regs<R>(x, tab, tw1024, ltw, lane);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) buf[lane + 32 * k1] = make_float2(x[k1].x, -x[k1].y);   // c^_n
    __syncwarp();
}

// lane_fft of a channel pair (packed FP32)
__device__ __forceinline__ cpair lane_fft2(cpair x, const LaneTw& tw, int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int h = 1 << s;
        const cpair u = s == 0 ? x : pcmul(x, pcbc(tw.w[s - 1]));
        const cpair v = shfl_xor4(u, h);
        x = (lane & h) ? pcsub(v, u) : pcadd(u, v);
    }
    return x;
}

// fft_regs of a channel pair
template <int R>
__device__ __forceinline__ void fft_regs2(cpair (&x)[R], const OrbitTables32& tab, const LaneTw& ltw, int lane) {
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = lane_fft2(x[r], ltw, lane);
#pragma unroll
    for (int r = 1; r < R; ++r) x[r] = pcmul(x[r], ldg4(tab.ltw4 + r * 32 + lane));
    reg_fft2<R>(x);
}

// residual_adjoint of both channels at once (A, E in the two halves of each
// packed register pair), for N <= 256; the sums of both channels are added
// into (sdh, cdh) and (shh, chh).
template <int R>
__device__ void residual_adjoint2(float2* bufA, float2* bufE, const OrbitTables32& tab, const LaneTw& ltw, int lane,
                                  int off, int W, const Win32* __restrict__ pw, float kappa, float& sdh, float& cdh,
                                  float& shh, float& chh) {
    constexpr int N = 32 * R;
    constexpr int SH = (R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5) + 1;
    cpair x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 a = bufA[r * 32 + lane], e = bufE[r * 32 + lane];
        x[r] = cpair{make_float2(a.x, e.x), make_float2(a.y, e.y)};
    }
    fft_regs2<R>(x, tab, ltw, lane);
    __syncwarp();
    f2 s_dh = bc(0.0f), c_dh = bc(0.0f), s_hh = bc(0.0f), c_hh = bc(0.0f);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
        const int k = lane + 32 * k1;
        const int m = k < N / 2 ? k : k - N;
        const int kk = off + m;
        cpair rc{bc(0.0f), bc(0.0f)};
        if (kk >= 0 && kk < W) {
            const Win32 v = pw[kk];
            const cpair d{v.dre, v.dim};
            kahan_add2(s_dh, c_dh, pmul(v.w, pfma(d.re, x[k1].re, pmul(d.im, x[k1].im))));
            kahan_add2(s_hh, c_hh, pmul(v.w, pfma(x[k1].re, x[k1].re, pmul(x[k1].im, x[k1].im))));
            rc = cpair{pmul(v.w, pfma(bc(-kappa), x[k1].re, d.re)),
                       pneg(pmul(v.w, pfma(bc(-kappa), x[k1].im, d.im)))};   // conj(r)
        }
        const int ks = k ^ ((k >> SH) & 15);   // the swizzle of residual_adjoint
        bufA[ks] = make_float2(rc.re.x, rc.im.x);
        bufE[ks] = make_float2(rc.re.y, rc.im.y);
    }
    float ps, pc;
    kahan_merge(s_dh, c_dh, ps, pc);
    kahan_join(sdh, cdh, ps, pc);
    kahan_merge(s_hh, c_hh, ps, pc);
    kahan_join(shh, chh, ps, pc);
    __syncwarp();
    const int nb = R * brev5(lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = nb + r, es = e ^ ((e >> SH) & 15);
        const float2 a = bufA[es], b = bufE[es];
        x[r] = cpair{make_float2(a.x, b.x), make_float2(a.y, b.y)};
    }
    fft_regs2<R>(x, tab, ltw, lane);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {   // c^_n
        bufA[lane + 32 * k1] = make_float2(x[k1].re.x, -x[k1].im.x);
        bufE[lane + 32 * k1] = make_float2(x[k1].re.y, -x[k1].im.y);
    }
    __syncwarp();
}

// Both channels at once in natural order, with the likelihood kernel's
// transform (buf: N channel-pair elements, sample n at n, from the packed
// slow part): forward transform and window inner products as the likelihood
// kernel forms them, the conjugated residual conj(w^ (d^ - kappa S)) stored at
// its DFT index, the same transform again (the adjoint, conjugated), and
// c^_n left at sample n, each as a channel-pair element; both stores and the
// second transform's reads go through nat_sw, which keeps the scattered bin
// stores free of bank conflicts.  Sums are joined into (sdh, cdh) and
// (shh, chh).
template <int R>
__device__ void residual_adjoint_nat(float4* buf, const OrbitTables32& tab, const LaneTw& ltw, int lane, int off,
                                     int W, const Win32* __restrict__ pw, float kappa, float& sdh, float& cdh,
                                     float& shh, float& chh) {
    constexpr int N = 32 * R;
    cpair x[R];
    int kbase = nat_transform<R>(buf, tab, ltw, lane, x);
    f2 s_dh = bc(0.0f), c_dh = bc(0.0f), s_hh = bc(0.0f), c_hh = bc(0.0f);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int K = bin_of<R>(kbase, q);
        const int m = K < N / 2 ? K : K - N;
        const int kk = off + m;
        cpair rc{bc(0.0f), bc(0.0f)};
        if (kk >= 0 && kk < W) {
            const Win32 v = pw[kk];
            kahan_add2(s_dh, c_dh, pmul(v.w, pfma(v.dre, x[q].re, pmul(v.dim, x[q].im))));
            kahan_add2(s_hh, c_hh, pmul(v.w, pfma(x[q].re, x[q].re, pmul(x[q].im, x[q].im))));
            rc = cpair{pmul(v.w, pfma(bc(-kappa), x[q].re, v.dre)), pneg(pmul(v.w, pfma(bc(-kappa), x[q].im, v.dim)))};
        }
        st4(buf + nat_sw(K, N), rc);
    }
    float ps, pc;
    kahan_merge(s_dh, c_dh, ps, pc);
    kahan_join(sdh, cdh, ps, pc);
    kahan_merge(s_hh, c_hh, ps, pc);
    kahan_join(shh, chh, ps, pc);
    __syncwarp();
    kbase = nat_transform<R, false, true>(buf, tab, ltw, lane, x);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < R; ++q) st4(buf + nat_sw(bin_of<R>(kbase, q), N), cpair{x[q].re, pneg(x[q].im)});   // c^_n
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
            // N <= 256 without T data (every window of the plain instantiation): the
            // packed slow part in natural order and the likelihood kernel's transform
            bool packed_done = false;
            if constexpr (RMAX <= 8) {
              if (!g.m.bad && !useT) {
                packed_done = true;
                slow_part_dispatch<true>(g.m, tab, N, bufA, bufE, lane);
                __syncwarp();
                const long long off64 = g.m.q - win.k0;
                const int off = (off64 > -(long long)N && off64 < (long long)win.W + N) ? (int)off64 : -4 * N;
                const float kappa = (float)(wm.sig * g.m.A * T / (2.0 * (double)N));
                float4* buf4 = (float4*)bufA;
                switch (N) {
                    case 32: residual_adjoint_nat<1>(buf4, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                    case 64: residual_adjoint_nat<2>(buf4, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                    case 128: residual_adjoint_nat<4>(buf4, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                    default: residual_adjoint_nat<8>(buf4, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                }
                switch (g.m.J) {
                    case 4: adjoint_sweep<4, false, true>(g, tab, N, Tf, inv_fstar, bufA, nullptr, lane, tacc, vp, vq); break;
                    case 7: adjoint_sweep<7, false, true>(g, tab, N, Tf, inv_fstar, bufA, nullptr, lane, tacc, vp, vq); break;
                    case 10: adjoint_sweep<10, false, true>(g, tab, N, Tf, inv_fstar, bufA, nullptr, lane, tacc, vp, vq); break;
                    default: adjoint_sweep<0, false, true>(g, tab, N, Tf, inv_fstar, bufA, nullptr, lane, tacc, vp, vq); break;
                }
                __syncwarp();
              }
            }
            if (!T3 && RMAX <= 8) {
              // no other path in the plain N <= 256 instantiation
            } else {
              if (!g.m.bad && !packed_done) {
                slow_part_dispatch<false, T3>(g.m, tab, N, bufA, bufE, lane, useT ? bufT : nullptr);
                __syncwarp();
                const long long off64 = g.m.q - win.k0;
                const int off = (off64 > -(long long)N && off64 < (long long)win.W + N) ? (int)off64 : -4 * N;
                const float kappa = (float)(wm.sig * g.m.A * T / (2.0 * (double)N));
                if constexpr (RMAX <= 8) {   // both channels at once
                    switch (N) {
                        case 32: residual_adjoint2<1>(bufA, bufE, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                        case 64: residual_adjoint2<2>(bufA, bufE, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                        case 128: residual_adjoint2<4>(bufA, bufE, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                        default: residual_adjoint2<8>(bufA, bufE, tab, ltw, lane, off, win.W, pw, kappa, sdh, cdh, shh, chh); break;
                    }
                }
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    float2* buf = ch == 0 ? bufA : bufE;
                    if constexpr (RMAX > 8) {
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
