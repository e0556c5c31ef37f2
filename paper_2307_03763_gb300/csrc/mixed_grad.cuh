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
// f0, fdot, beta, lambda are carried as forward-mode tangents through the
// sample computation.
// ---------------------------------------------------------------------------
#pragma once
#include "mixed_common.cuh"

namespace gb {
namespace {

constexpr int KT = 4;   // f0, fdot, beta, lambda

// A complex value with its KT = 4 forward tangents.  The tangents are kept
// as two pairs, k = (0, 1) and (2, 3), of real parts dr and imaginary parts
// di, so that every tangent operation is one packed FP32 instruction per pair.
struct DCf {
    float2 v;
    f2 dr[2], di[2];
};
__device__ __forceinline__ DCf dmulf(const DCf& a, const DCf& b) {
    DCf o;
    o.v = cmulf(a.v, b.v);
#pragma unroll
    for (int p = 0; p < 2; ++p) {   // a.d b.v + a.v b.d
        const f2 re1 = pfma(a.dr[p], bc(b.v.x), pneg(pmul(a.di[p], bc(b.v.y))));
        const f2 im1 = pfma(a.dr[p], bc(b.v.y), pmul(a.di[p], bc(b.v.x)));
        const f2 re2 = pfma(bc(a.v.x), b.dr[p], pneg(pmul(bc(a.v.y), b.di[p])));
        const f2 im2 = pfma(bc(a.v.x), b.di[p], pmul(bc(a.v.y), b.dr[p]));
        o.dr[p] = padd(re1, re2);
        o.di[p] = padd(im1, im2);
    }
    return o;
}
__device__ __forceinline__ DCf daddf(const DCf& a, const DCf& b) {
    DCf o;
    o.v = caddf(a.v, b.v);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        o.dr[p] = padd(a.dr[p], b.dr[p]);
        o.di[p] = padd(a.di[p], b.di[p]);
    }
    return o;
}
__device__ __forceinline__ DCf dsubf(const DCf& a, const DCf& b) {
    DCf o;
    o.v = csubf(a.v, b.v);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        o.dr[p] = psub(a.dr[p], b.dr[p]);
        o.di[p] = psub(a.di[p], b.di[p]);
    }
    return o;
}
__device__ __forceinline__ DCf dscalef(const DCf& a, float s) {
    DCf o;
    o.v = make_float2(a.v.x * s, a.v.y * s);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        o.dr[p] = pmul(a.dr[p], bc(s));
        o.di[p] = pmul(a.di[p], bc(s));
    }
    return o;
}

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

// the T channel's sample with its tangents and P, Q responses
struct TOut {
    DCf S;
    float2 P, Q;
};

// One sample of the unit-amplitude slow part at sample n: A and E with the
// four forward tangents, and the P and Q responses (values); with T3 also T
// = (X + Y + Z)/sqrt3 into *to.
template <int J, bool T3 = false>
__device__ __forceinline__ void sample_grad(const CandGx& g, const OrbitTables32& tab, int N, int n, float Tf,
                                            float inv_fstar, DCf& SA, DCf& SE, float2& PA, float2& PE, float2& QA,
                                            float2& QE, TOut* to = nullptr) {
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
    const float ux0 = fmaf(g.Uc, cah, g.Us * sah), vx0 = fmaf(g.Vc, cah, g.Vs * sah);
    DCf rx[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float kap = K + krho[j];
        const float dP = fmaf(-f, krho[j], c.fdh * kap * kap);
        const float2 v = cmulf(ePc, cis_rx<J>(dP));
        const float tk = tu - kap;
        const float fk = fmaf(-fd, kap, f);
        float dph[KT];
        dph[0] = tk;
        dph[1] = 0.5f * tk * tk;
        dph[2] = -fk * (ux0 + urho[j]);
        dph[3] = -fk * g.cb * (vx0 + vrho[j]);
        rx[j].v = v;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const f2 t = pmul(bc(6.2831853071795865f), make_float2(dph[2 * p], dph[2 * p + 1]));
            rx[j].dr[p] = pmul(pneg(t), bc(v.y));
            rx[j].di[p] = pmul(t, bc(v.x));
        }
    }
    const float a = fmaf(c.a1, u, c.a0);
    const float da[KT] = {0.5f * inv_fstar, 0.5f * tu * inv_fstar, 0.0f, 0.0f};
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
    DCf zp[3], zm[3];
    float2 zpP[3], zmP[3], zpQ[3], zmQ[3];
#pragma unroll
    for (int arm = 0; arm < 3; ++arm) {
        const float kn = kn_[arm], nu = nu_[arm], nv = nv_[arm], nw = nw_[arm];
        const float dkn[KT] = {0.0f, 0.0f, nu, g.cb * nv};
        const float dnu[KT] = {0.0f, 0.0f, -kn, -g.sb * nv};
        const float dnv[KT] = {0.0f, 0.0f, 0.0f, nw};
        const float Fp = (nu - nv) * (nu + nv), Fx = 2.0f * nu * nv;
        DCf G;
        G.v = make_float2(fmaf(g.gp.x, Fp, g.gx.x * Fx), fmaf(g.gp.y, Fp, g.gx.y * Fx));
        float dFp[KT], dFx[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            dFp[k] = 2.0f * (nu * dnu[k] - nv * dnv[k]);
            dFx[k] = 2.0f * (dnu[k] * nv + nu * dnv[k]);
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const f2 fp = make_float2(dFp[2 * p], dFp[2 * p + 1]), fx = make_float2(dFx[2 * p], dFx[2 * p + 1]);
            G.dr[p] = pfma(bc(g.gp.x), fp, pmul(bc(g.gx.x), fx));
            G.di[p] = pfma(bc(g.gp.y), fp, pmul(bc(g.gx.y), fx));
        }
        const int rp = arm == 2 ? 0 : arm + 1, rm = arm;
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const float sd = sgn == 0 ? 1.0f : -1.0f;   // +n link: X = a(1 - kn); -n link: X = a(1 + kn)
            const float X = a * fmaf(-sd, kn, 1.0f);
            float2 Tv, Td;
            link_transfer_d<J>(X, Tv, Td);
            DCf Tl;
            Tl.v = Tv;
            float dX[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) dX[k] = da[k] * fmaf(-sd, kn, 1.0f) - sd * a * dkn[k];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const f2 x = make_float2(dX[2 * p], dX[2 * p + 1]);
                Tl.dr[p] = pmul(bc(Td.x), x);
                Tl.di[p] = pmul(bc(Td.y), x);
            }
            const DCf& rr = rx[sgn == 0 ? rp : rm];
            const DCf z = dmulf(dmulf(Tl, G), rr);
            const float2 Tr = cmulf(Tv, rr.v);
            const float2 zP = make_float2(Tr.x * Fp, Tr.y * Fp), zQ = make_float2(Tr.x * Fx, Tr.y * Fx);
            if (sgn == 0) {
                zp[arm] = z;
                zpP[arm] = zP;
                zpQ[arm] = zQ;
            } else {
                zm[arm] = z;
                zmP[arm] = zP;
                zmQ[arm] = zQ;
            }
        }
    }
    // delay factor D = exp(-i f/f*) and F = -i a (1 - D^2) = 2 a sin(f/f*) D
    DCf D;
    {
        const float du = c.eps * u;
        D.v = cmulf(make_float2(c.D0r, c.D0i), make_float2(fmaf(-0.5f * du, du, 1.0f), -du));
        const float dphi[KT] = {inv_fstar, tu * inv_fstar, 0.0f, 0.0f};
#pragma unroll
        for (int p = 0; p < 2; ++p) {   // -i D dphi
            const f2 x = make_float2(dphi[2 * p], dphi[2 * p + 1]);
            D.dr[p] = pmul(bc(D.v.y), x);
            D.di[p] = pmul(bc(-D.v.x), x);
        }
    }
    DCf F;
    {
        const float sa2 = -2.0f * a * D.v.y;
        F.v = make_float2(sa2 * D.v.x, sa2 * D.v.y);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const f2 dsa2 = pmul(bc(-2.0f), pfma(make_float2(da[2 * p], da[2 * p + 1]), bc(D.v.y), pmul(bc(a), D.di[p])));
            F.dr[p] = pfma(dsa2, bc(D.v.x), pmul(bc(sa2), D.dr[p]));
            F.di[p] = pfma(dsa2, bc(D.v.y), pmul(bc(sa2), D.di[p]));
        }
    }
    const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f;
    {
        const DCf Xp = daddf(dsubf(zm[0], zp[2]), dmulf(D, dsubf(zp[0], zm[2])));
        const DCf Yp = daddf(dsubf(zm[1], zp[0]), dmulf(D, dsubf(zp[1], zm[0])));
        const DCf Zp = daddf(dsubf(zm[2], zp[1]), dmulf(D, dsubf(zp[2], zm[1])));
        SA = dmulf(F, dscalef(dsubf(Zp, Xp), r2));
        SE = dmulf(F, dscalef(daddf(dsubf(Xp, dscalef(Yp, 2.0f)), Zp), r6));
        if constexpr (T3) to->S = dmulf(F, dscalef(daddf(daddf(Xp, Yp), Zp), 0.57735026918962576f));
    }
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const float2* zpv = w == 0 ? zpP : zpQ;
        const float2* zmv = w == 0 ? zmP : zmQ;
        const float2 Xp = caddf(csubf(zmv[0], zpv[2]), cmulf(D.v, csubf(zpv[0], zmv[2])));
        const float2 Yp = caddf(csubf(zmv[1], zpv[0]), cmulf(D.v, csubf(zpv[1], zmv[0])));
        const float2 Zp = caddf(csubf(zmv[2], zpv[1]), cmulf(D.v, csubf(zpv[2], zmv[1])));
        const float2 Av = cmulf(F.v, make_float2((Zp.x - Xp.x) * r2, (Zp.y - Xp.y) * r2));
        const float2 Ev =
            cmulf(F.v, make_float2((Xp.x - 2.0f * Yp.x + Zp.x) * r6, (Xp.y - 2.0f * Yp.y + Zp.y) * r6));
        if (w == 0) {
            PA = Av;
            PE = Ev;
        } else {
            QA = Av;
            QE = Ev;
        }
        if constexpr (T3) {
            const float r3 = 0.57735026918962576f;
            const float2 Tv = cmulf(F.v, make_float2((Xp.x + Yp.x + Zp.x) * r3, (Xp.y + Yp.y + Zp.y) * r3));
            if (w == 0)
                to->P = Tv;
            else
                to->Q = Tv;
        }
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

// cT (T3, may be null): the T channel's adjoint
template <int J, bool T3 = false>
__device__ void tangent_sweep(const CandGx& g, const OrbitTables32& tab, int N, float Tf, float inv_fstar,
                              const float2* cA, const float2* cE, int lane, float (&tacc)[KT][2],
                              float (&vp)[2][2], float (&vq)[2][2], const float2* cT = nullptr) {
    for (int n = lane; n < N; n += 32) {
        DCf SA, SE;
        float2 PA, PE, QA, QE;
        TOut to;
        if (T3 && cT)
            sample_grad<J, true>(g, tab, N, n, Tf, inv_fstar, SA, SE, PA, PE, QA, QE, &to);
        else
            sample_grad<J, false>(g, tab, N, n, Tf, inv_fstar, SA, SE, PA, PE, QA, QE);
        const float2 a = cA[n], e = cE[n];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            f2 sum = make_float2(tacc[2 * p][0], tacc[2 * p + 1][0]), comp = make_float2(tacc[2 * p][1], tacc[2 * p + 1][1]);
            kahan_add2(sum, comp, pfma(bc(a.x), SA.dr[p], pfma(bc(a.y), SA.di[p], pfma(bc(e.x), SE.dr[p],
                                                                                       pmul(bc(e.y), SE.di[p])))));
            tacc[2 * p][0] = sum.x;
            tacc[2 * p + 1][0] = sum.y;
            tacc[2 * p][1] = comp.x;
            tacc[2 * p + 1][1] = comp.y;
        }
        // c conj(P) = (c.x P.x + c.y P.y) + i (c.y P.x - c.x P.y)
        kahan_add(vp[0][0], vp[0][1], fmaf(a.x, PA.x, fmaf(a.y, PA.y, fmaf(e.x, PE.x, e.y * PE.y))));
        kahan_add(vp[1][0], vp[1][1], fmaf(a.y, PA.x, fmaf(-a.x, PA.y, fmaf(e.y, PE.x, -e.x * PE.y))));
        kahan_add(vq[0][0], vq[0][1], fmaf(a.x, QA.x, fmaf(a.y, QA.y, fmaf(e.x, QE.x, e.y * QE.y))));
        kahan_add(vq[1][0], vq[1][1], fmaf(a.y, QA.x, fmaf(-a.x, QA.y, fmaf(e.y, QE.x, -e.x * QE.y))));
        if constexpr (T3) {
            if (cT) {
                const float2 t = cT[n];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    f2 sum = make_float2(tacc[2 * p][0], tacc[2 * p + 1][0]);
                    f2 comp = make_float2(tacc[2 * p][1], tacc[2 * p + 1][1]);
                    kahan_add2(sum, comp, pfma(bc(t.x), to.S.dr[p], pmul(bc(t.y), to.S.di[p])));
                    tacc[2 * p][0] = sum.x;
                    tacc[2 * p + 1][0] = sum.y;
                    tacc[2 * p][1] = comp.x;
                    tacc[2 * p + 1][1] = comp.y;
                }
                kahan_add(vp[0][0], vp[0][1], fmaf(t.x, to.P.x, t.y * to.P.y));
                kahan_add(vp[1][0], vp[1][1], fmaf(t.y, to.P.x, -t.x * to.P.y));
                kahan_add(vq[0][0], vq[0][1], fmaf(t.x, to.Q.x, t.y * to.Q.y));
                kahan_add(vq[1][0], vq[1][1], fmaf(t.y, to.Q.x, -t.x * to.Q.y));
            }
        }
    }
}

template <int RMAX, bool T3>
__global__ void __launch_bounds__(kWarpsMx * 32, RMAX <= 8 ? 2 : 1) grad_mixed_kernel(
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
                    case 4: tangent_sweep<4, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                    case 7: tangent_sweep<7, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                    case 10: tangent_sweep<10, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
                    default: tangent_sweep<0, T3>(g, tab, N, Tf, inv_fstar, bufA, bufE, lane, tacc, vp, vq, cT); break;
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
