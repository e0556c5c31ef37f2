// mixed_common.cuh -- device code shared by the mixed-precision translation
// units (likelihood, its variants, waveform, gradient): the per-candidate
// set-up, the slow part, the transforms, the window preparation and the
// persistent likelihood kernel template.  Every definition sits in an
// anonymous namespace, so each translation unit instantiates what it uses.
//
// The mixed-precision path: the carrier phase and the bin offset keep
// double-precision accuracy, while the detector response, the FFT and the
// window inner products run in float with compensated sums.  Inputs, the
// per-window <d|d> and every output are double.
//
// Why not native double for the phase: on GB300 the FP64 pipe issues at 1/64
// of the FP32 rate, so a native-double phase (about ten operations per
// sample) would cost more than the whole float response.  The paired slow
// part takes the phase in fixed point (64-bit integer fractions of a cycle,
// whose sums wrap modulo one exactly: PhaseRec, phase_fix); the scalar slow
// part and candidates outside the fixed-point ranges take it in double-word
// float arithmetic (a product with an exact FMA error term costs two or three
// float operations).
//
// Phase of the receiver-j link, in cycles, at u = t/T = n/N (reading R5):
//   P_j = phi0/2pi + delta u + (fdot T^2/2) u^2 - f0 K(n) - fdot T u K(n)
//         - f rho_j(n) + (fdot/2) (K + rho_j)^2,
//   K(n) = k.x_centre/c = Kc cos(alpha_n) + Ks sin(alpha_n),
//   rho_j = k.(x_j - x_centre)/c,  f = f0 + fdot T u.
// The first four terms can reach hundreds of cycles and are formed modulo one
// exactly (fixed point, or double-word arithmetic with each product reduced
// modulo one); the rest are below 0.1 cycle and are float.  exp(2 pi i P_j) is the common factor
// exp(2 pi i P_c) (one accurate sincospi, applied once per sample to A and E)
// times exp(2 pi i dP_j) for the small per-spacecraft remainder.
//
// Link transfer sinc(X) exp(-iX) = sum_k (-2iX)^k/(k+1)! is evaluated as two
// Horner polynomials in y = -4X^2 (even and odd k), with the number of terms
// chosen per candidate from the largest X = f/f* it can reach.
//
// Execution: a persistent kernel whose warps take work items (a window and up
// to 32 of its candidates, 16 by default) from a global queue, most expensive
// first.  Per item the warp sets the candidates up one per lane, then
// evaluates them one after the other.  In the likelihood kernel lane l
// computes samples n = l + 32 r (R = N/32), for N >= 64 two at a time (n and
// n + 32) with packed two-wide FP32 instructions (sm_100 and later: one FFMA2
// does the FMAs of both samples), reading the orbit tables in a layout that
// gives both samples' values as one register pair; the transform is R-point
// register DFTs around skewed shared-memory transposes, both channels packed
// together (see fft_inner_ch).
// The waveform and gradient kernels keep the earlier order n = R brev5(l) + r
// with a 32-point stage across lanes (shuffles, bit-reversed input, natural
// output), a lane twiddle and an R-point register FFT, after which lane l
// holds bins l + 32 k1.  A preparation kernel forms <d|d>, the scale sigma
// and the float copy of every window once per launch.
#pragma once
#include <cmath>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int kWarpsMx = 4;
// candidates per work item of the T-channel likelihood: a smaller candidate
// array keeps two CTAs of the N = 1,024 instantiation resident per SM
constexpr int kCapT = 16;

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
    float gpr, gxr2, gpi, gxi2;   // G = (gpr F+ + gxr Fx) + i (gpi F+ + gxi Fx), unit amplitude, with
                                  // gxr2 = 2 gxr and gxi2 = 2 gxi (Fx = 2 n.u n.v)
    float f0, fdT, fdh; // Hz, fdot T [Hz], fdot/2 [Hz/s]
    float a0, a1;       // a = f/(2 f*) = a0 + a1 u
    float D0r, D0i;     // exp(-i f0/f*)
    float eps;          // fdot T / f*
    int J;              // Horner length of the link transfer polynomial (0: direct)
    int bad;
    long long q;
    double A;
    // The carrier phase in fixed point for the paired slow part (cycles as
    // unsigned fractions, so that sums wrap modulo one exactly): phi0/2pi in
    // units of 2^-64; delta mod 1024 in units of 2^-54 and fdot T^2/2 mod 2^20
    // in units of 2^-44, which shifts by 10 - log2 N and 20 - 2 log2 N bring
    // to 2^-64 per unit of n and n^2; f0 Kc and f0 Ks in units of 2^-26
    // (|f0 K| < 31 cycles, else wide).
    unsigned long long C0, K1, K2;
    int Fc, Fs;
    int wide;           // outside the fixed-point ranges: the scalar slow part
};

// per-candidate sums left by the warp for the lane-parallel epilogue
template <bool IM>
struct Epi {
    float dh_hi, dh_lo, hh_hi, hh_lo;
};
template <>
struct Epi<true> {
    float dh_hi, dh_lo, hh_hi, hh_lo, im_hi, im_lo;
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

// exp(-2 pi i m / 32), m < 16: the twiddles of the register DFTs (R <= 32),
// read with compile-time indices as constant operands
__constant__ float2 kW32[16] = {
    {1.000000000e+00f, 0.0f}, {9.807852804e-01f, -1.950903220e-01f},
    {9.238795325e-01f, -3.826834324e-01f}, {8.314696123e-01f, -5.555702330e-01f},
    {7.071067812e-01f, -7.071067812e-01f}, {5.555702330e-01f, -8.314696123e-01f},
    {3.826834324e-01f, -9.238795325e-01f}, {1.950903220e-01f, -9.807852804e-01f},
    {0.0f, -1.000000000e+00f}, {-1.950903220e-01f, -9.807852804e-01f},
    {-3.826834324e-01f, -9.238795325e-01f}, {-5.555702330e-01f, -8.314696123e-01f},
    {-7.071067812e-01f, -7.071067812e-01f}, {-8.314696123e-01f, -5.555702330e-01f},
    {-9.238795325e-01f, -3.826834324e-01f}, {-9.807852804e-01f, -1.950903220e-01f}};

// 1/k! for the link transfer series (Taylor coefficients of (e^w - 1)/w)
__constant__ float kInvFact[24] = {
    1.0f, 1.0f, 0.5f, 1.6666666666666666e-01f, 4.1666666666666664e-02f, 8.3333333333333332e-03f,
    1.3888888888888889e-03f, 1.9841269841269841e-04f, 2.4801587301587302e-05f, 2.7557319223985893e-06f,
    2.7557319223985888e-07f, 2.5052108385441720e-08f, 2.0876756987868100e-09f, 1.6059043836821613e-10f,
    1.1470745597729725e-11f, 7.6471637318198164e-13f, 4.7794773323873853e-14f, 2.8114572543455206e-15f,
    1.5619206968586225e-16f, 8.2206352466243295e-18f, 4.1103176233121648e-19f, 1.9572941063391263e-20f,
    8.8967913924505741e-22f, 3.8681701706306835e-23f};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// sin(k pi/64), cos(k pi/64) for k = 0 .. 127 as double-word float pairs
// (sin hi, sin lo, cos hi, cos lo), from 50-digit values
__device__ const float4 kSinCosDW[128] = {
    {0.000000000e+00f, 0.000000000e+00f, 1.000000000e+00f, 0.000000000e+00f},
    {4.906767607e-02f, -1.739934308e-09f, 9.987954497e-01f, 6.471438052e-09f},
    {9.801714122e-02f, -8.933931928e-10f, 9.951847196e-01f, 7.109666189e-09f},
    {1.467304677e-01f, 6.778245520e-09f, 9.891765118e-01f, -1.799745353e-09f},
    {1.950903237e-01f, -1.670471428e-09f, 9.807852507e-01f, 2.973947311e-08f},
    {2.429801822e-01f, -2.267604104e-09f, 9.700312614e-01f, -8.249547712e-09f},
    {2.902846634e-01f, 1.381566506e-08f, 9.569403529e-01f, -1.718450804e-08f},
    {3.368898630e-01f, -9.622000974e-09f, 9.415440559e-01f, 9.244300436e-09f},
    {3.826834261e-01f, 6.223350724e-09f, 9.238795042e-01f, 2.830748969e-08f},
    {4.275550842e-01f, 9.201766460e-09f, 9.039893150e-01f, -2.190951598e-08f},
    {4.713967443e-01f, -7.425253745e-09f, 8.819212914e-01f, -2.700296342e-08f},
    {5.141027570e-01f, -1.278385930e-08f, 8.577286005e-01f, 9.498258180e-09f},
    {5.555702448e-01f, -1.176952136e-08f, 8.314695954e-01f, 1.687026341e-08f},
    {5.956993103e-01f, -5.810301129e-09f, 8.032075167e-01f, 1.481041778e-08f},
    {6.343932748e-01f, 9.379557575e-09f, 7.730104327e-01f, 2.064255256e-08f},
    {6.715589762e-01f, -2.132638244e-08f, 7.409511209e-01f, 4.501535145e-09f},
    {7.071067691e-01f, 1.210161749e-08f, 7.071067691e-01f, 1.210161749e-08f},
    {7.409511209e-01f, 4.501535145e-09f, 6.715589762e-01f, -2.132638244e-08f},
    {7.730104327e-01f, 2.064255256e-08f, 6.343932748e-01f, 9.379557575e-09f},
    {8.032075167e-01f, 1.481041778e-08f, 5.956993103e-01f, -5.810301129e-09f},
    {8.314695954e-01f, 1.687026341e-08f, 5.555702448e-01f, -1.176952136e-08f},
    {8.577286005e-01f, 9.498258180e-09f, 5.141027570e-01f, -1.278385930e-08f},
    {8.819212914e-01f, -2.700296342e-08f, 4.713967443e-01f, -7.425253745e-09f},
    {9.039893150e-01f, -2.190951598e-08f, 4.275550842e-01f, 9.201766460e-09f},
    {9.238795042e-01f, 2.830748969e-08f, 3.826834261e-01f, 6.223350724e-09f},
    {9.415440559e-01f, 9.244300436e-09f, 3.368898630e-01f, -9.622000974e-09f},
    {9.569403529e-01f, -1.718450804e-08f, 2.902846634e-01f, 1.381566506e-08f},
    {9.700312614e-01f, -8.249547712e-09f, 2.429801822e-01f, -2.267604104e-09f},
    {9.807852507e-01f, 2.973947311e-08f, 1.950903237e-01f, -1.670471428e-09f},
    {9.891765118e-01f, -1.799745353e-09f, 1.467304677e-01f, 6.778245520e-09f},
    {9.951847196e-01f, 7.109666189e-09f, 9.801714122e-02f, -8.933931928e-10f},
    {9.987954497e-01f, 6.471438052e-09f, 4.906767607e-02f, -1.739934308e-09f},
    {1.000000000e+00f, 0.000000000e+00f, -0.000000000e+00f, -0.000000000e+00f},
    {9.987954497e-01f, 6.471438052e-09f, -4.906767607e-02f, 1.739934308e-09f},
    {9.951847196e-01f, 7.109666189e-09f, -9.801714122e-02f, 8.933931928e-10f},
    {9.891765118e-01f, -1.799745353e-09f, -1.467304677e-01f, -6.778245520e-09f},
    {9.807852507e-01f, 2.973947311e-08f, -1.950903237e-01f, 1.670471428e-09f},
    {9.700312614e-01f, -8.249547712e-09f, -2.429801822e-01f, 2.267604104e-09f},
    {9.569403529e-01f, -1.718450804e-08f, -2.902846634e-01f, -1.381566506e-08f},
    {9.415440559e-01f, 9.244300436e-09f, -3.368898630e-01f, 9.622000974e-09f},
    {9.238795042e-01f, 2.830748969e-08f, -3.826834261e-01f, -6.223350724e-09f},
    {9.039893150e-01f, -2.190951598e-08f, -4.275550842e-01f, -9.201766460e-09f},
    {8.819212914e-01f, -2.700296342e-08f, -4.713967443e-01f, 7.425253745e-09f},
    {8.577286005e-01f, 9.498258180e-09f, -5.141027570e-01f, 1.278385930e-08f},
    {8.314695954e-01f, 1.687026341e-08f, -5.555702448e-01f, 1.176952136e-08f},
    {8.032075167e-01f, 1.481041778e-08f, -5.956993103e-01f, 5.810301129e-09f},
    {7.730104327e-01f, 2.064255256e-08f, -6.343932748e-01f, -9.379557575e-09f},
    {7.409511209e-01f, 4.501535145e-09f, -6.715589762e-01f, 2.132638244e-08f},
    {7.071067691e-01f, 1.210161749e-08f, -7.071067691e-01f, -1.210161749e-08f},
    {6.715589762e-01f, -2.132638244e-08f, -7.409511209e-01f, -4.501535145e-09f},
    {6.343932748e-01f, 9.379557575e-09f, -7.730104327e-01f, -2.064255256e-08f},
    {5.956993103e-01f, -5.810301129e-09f, -8.032075167e-01f, -1.481041778e-08f},
    {5.555702448e-01f, -1.176952136e-08f, -8.314695954e-01f, -1.687026341e-08f},
    {5.141027570e-01f, -1.278385930e-08f, -8.577286005e-01f, -9.498258180e-09f},
    {4.713967443e-01f, -7.425253745e-09f, -8.819212914e-01f, 2.700296342e-08f},
    {4.275550842e-01f, 9.201766460e-09f, -9.039893150e-01f, 2.190951598e-08f},
    {3.826834261e-01f, 6.223350724e-09f, -9.238795042e-01f, -2.830748969e-08f},
    {3.368898630e-01f, -9.622000974e-09f, -9.415440559e-01f, -9.244300436e-09f},
    {2.902846634e-01f, 1.381566506e-08f, -9.569403529e-01f, 1.718450804e-08f},
    {2.429801822e-01f, -2.267604104e-09f, -9.700312614e-01f, 8.249547712e-09f},
    {1.950903237e-01f, -1.670471428e-09f, -9.807852507e-01f, -2.973947311e-08f},
    {1.467304677e-01f, 6.778245520e-09f, -9.891765118e-01f, 1.799745353e-09f},
    {9.801714122e-02f, -8.933931928e-10f, -9.951847196e-01f, -7.109666189e-09f},
    {4.906767607e-02f, -1.739934308e-09f, -9.987954497e-01f, -6.471438052e-09f},
    {0.000000000e+00f, 0.000000000e+00f, -1.000000000e+00f, -0.000000000e+00f},
    {-4.906767607e-02f, 1.739934308e-09f, -9.987954497e-01f, -6.471438052e-09f},
    {-9.801714122e-02f, 8.933931928e-10f, -9.951847196e-01f, -7.109666189e-09f},
    {-1.467304677e-01f, -6.778245520e-09f, -9.891765118e-01f, 1.799745353e-09f},
    {-1.950903237e-01f, 1.670471428e-09f, -9.807852507e-01f, -2.973947311e-08f},
    {-2.429801822e-01f, 2.267604104e-09f, -9.700312614e-01f, 8.249547712e-09f},
    {-2.902846634e-01f, -1.381566506e-08f, -9.569403529e-01f, 1.718450804e-08f},
    {-3.368898630e-01f, 9.622000974e-09f, -9.415440559e-01f, -9.244300436e-09f},
    {-3.826834261e-01f, -6.223350724e-09f, -9.238795042e-01f, -2.830748969e-08f},
    {-4.275550842e-01f, -9.201766460e-09f, -9.039893150e-01f, 2.190951598e-08f},
    {-4.713967443e-01f, 7.425253745e-09f, -8.819212914e-01f, 2.700296342e-08f},
    {-5.141027570e-01f, 1.278385930e-08f, -8.577286005e-01f, -9.498258180e-09f},
    {-5.555702448e-01f, 1.176952136e-08f, -8.314695954e-01f, -1.687026341e-08f},
    {-5.956993103e-01f, 5.810301129e-09f, -8.032075167e-01f, -1.481041778e-08f},
    {-6.343932748e-01f, -9.379557575e-09f, -7.730104327e-01f, -2.064255256e-08f},
    {-6.715589762e-01f, 2.132638244e-08f, -7.409511209e-01f, -4.501535145e-09f},
    {-7.071067691e-01f, -1.210161749e-08f, -7.071067691e-01f, -1.210161749e-08f},
    {-7.409511209e-01f, -4.501535145e-09f, -6.715589762e-01f, 2.132638244e-08f},
    {-7.730104327e-01f, -2.064255256e-08f, -6.343932748e-01f, -9.379557575e-09f},
    {-8.032075167e-01f, -1.481041778e-08f, -5.956993103e-01f, 5.810301129e-09f},
    {-8.314695954e-01f, -1.687026341e-08f, -5.555702448e-01f, 1.176952136e-08f},
    {-8.577286005e-01f, -9.498258180e-09f, -5.141027570e-01f, 1.278385930e-08f},
    {-8.819212914e-01f, 2.700296342e-08f, -4.713967443e-01f, 7.425253745e-09f},
    {-9.039893150e-01f, 2.190951598e-08f, -4.275550842e-01f, -9.201766460e-09f},
    {-9.238795042e-01f, -2.830748969e-08f, -3.826834261e-01f, -6.223350724e-09f},
    {-9.415440559e-01f, -9.244300436e-09f, -3.368898630e-01f, 9.622000974e-09f},
    {-9.569403529e-01f, 1.718450804e-08f, -2.902846634e-01f, -1.381566506e-08f},
    {-9.700312614e-01f, 8.249547712e-09f, -2.429801822e-01f, 2.267604104e-09f},
    {-9.807852507e-01f, -2.973947311e-08f, -1.950903237e-01f, 1.670471428e-09f},
    {-9.891765118e-01f, 1.799745353e-09f, -1.467304677e-01f, -6.778245520e-09f},
    {-9.951847196e-01f, -7.109666189e-09f, -9.801714122e-02f, 8.933931928e-10f},
    {-9.987954497e-01f, -6.471438052e-09f, -4.906767607e-02f, 1.739934308e-09f},
    {-1.000000000e+00f, -0.000000000e+00f, -0.000000000e+00f, -0.000000000e+00f},
    {-9.987954497e-01f, -6.471438052e-09f, 4.906767607e-02f, -1.739934308e-09f},
    {-9.951847196e-01f, -7.109666189e-09f, 9.801714122e-02f, -8.933931928e-10f},
    {-9.891765118e-01f, 1.799745353e-09f, 1.467304677e-01f, 6.778245520e-09f},
    {-9.807852507e-01f, -2.973947311e-08f, 1.950903237e-01f, -1.670471428e-09f},
    {-9.700312614e-01f, 8.249547712e-09f, 2.429801822e-01f, -2.267604104e-09f},
    {-9.569403529e-01f, 1.718450804e-08f, 2.902846634e-01f, 1.381566506e-08f},
    {-9.415440559e-01f, -9.244300436e-09f, 3.368898630e-01f, -9.622000974e-09f},
    {-9.238795042e-01f, -2.830748969e-08f, 3.826834261e-01f, 6.223350724e-09f},
    {-9.039893150e-01f, 2.190951598e-08f, 4.275550842e-01f, 9.201766460e-09f},
    {-8.819212914e-01f, 2.700296342e-08f, 4.713967443e-01f, -7.425253745e-09f},
    {-8.577286005e-01f, -9.498258180e-09f, 5.141027570e-01f, -1.278385930e-08f},
    {-8.314695954e-01f, -1.687026341e-08f, 5.555702448e-01f, -1.176952136e-08f},
    {-8.032075167e-01f, -1.481041778e-08f, 5.956993103e-01f, -5.810301129e-09f},
    {-7.730104327e-01f, -2.064255256e-08f, 6.343932748e-01f, 9.379557575e-09f},
    {-7.409511209e-01f, -4.501535145e-09f, 6.715589762e-01f, -2.132638244e-08f},
    {-7.071067691e-01f, -1.210161749e-08f, 7.071067691e-01f, 1.210161749e-08f},
    {-6.715589762e-01f, 2.132638244e-08f, 7.409511209e-01f, 4.501535145e-09f},
    {-6.343932748e-01f, -9.379557575e-09f, 7.730104327e-01f, 2.064255256e-08f},
    {-5.956993103e-01f, 5.810301129e-09f, 8.032075167e-01f, 1.481041778e-08f},
    {-5.555702448e-01f, 1.176952136e-08f, 8.314695954e-01f, 1.687026341e-08f},
    {-5.141027570e-01f, 1.278385930e-08f, 8.577286005e-01f, 9.498258180e-09f},
    {-4.713967443e-01f, 7.425253745e-09f, 8.819212914e-01f, -2.700296342e-08f},
    {-4.275550842e-01f, -9.201766460e-09f, 9.039893150e-01f, -2.190951598e-08f},
    {-3.826834261e-01f, -6.223350724e-09f, 9.238795042e-01f, 2.830748969e-08f},
    {-3.368898630e-01f, 9.622000974e-09f, 9.415440559e-01f, 9.244300436e-09f},
    {-2.902846634e-01f, -1.381566506e-08f, 9.569403529e-01f, -1.718450804e-08f},
    {-2.429801822e-01f, 2.267604104e-09f, 9.700312614e-01f, -8.249547712e-09f},
    {-1.950903237e-01f, 1.670471428e-09f, 9.807852507e-01f, 2.973947311e-08f},
    {-1.467304677e-01f, -6.778245520e-09f, 9.891765118e-01f, -1.799745353e-09f},
    {-9.801714122e-02f, 8.933931928e-10f, 9.951847196e-01f, 7.109666189e-09f},
    {-4.906767607e-02f, 1.739934308e-09f, 9.987954497e-01f, 6.471438052e-09f}};

// sin and cos of a double argument to about 1e-12 absolute with little FP64
// work (on GB300 the FP64 pipe issues at 1/64 of the FP32 rate): the
// reduction x = k pi/64 + r (|r| <= pi/128) in double with a two-part pi/64,
// then double-word float arithmetic: sin r = r - r^3/6 + r^5/120 and
// cos r = 1 - r^2/2 + r^4/24 - r^6/720 with r and r^2 as double-word values
// and the smaller terms (below 3e-6 of the leading one) in float, and
//   sin x = S_k cos r + C_k sin r,  cos x = C_k cos r - S_k sin r
// with the table's S_k, C_k.
__device__ __forceinline__ void dw_mul_acc(float ah, float al, float bh, float bl, float& p, float& e) {
    p = ah * bh;
    e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
}
__device__ void sincos_dw(double x, double& sn, double& cs) {
    const double k = rint(x * 20.371832715762604);                  // 64/pi
    double r = fma(-k, 0.04908738521234052, x);                     // pi/64, high part
    r = fma(-k, 1.9135106236677394e-18, r);                         // low part
    const float4 t = kSinCosDW[((int)(long long)k) & 127];
    const float rh = (float)r, rl = (float)(r - (double)rh);
    const float z = rh * rh;
    float s1, e1, s2, e2;
    const float ts = -(rh * z) * (0.16666667f - z * 0.0083333333f);
    two_sum(rh, ts, s1, e1);
    const float srh = s1, srl = e1 + rl;                            // sin r
    const float p = rh * rh;
    const float ep = fmaf(rh, rh, -p) + 2.0f * (rh * rl);
    const float tc = (z * z) * (0.041666668f - z * 0.0013888889f);
    two_sum(1.0f, -0.5f * p, s2, e2);
    const float crh = s2, crl = (e2 - 0.5f * ep) + tc;             // cos r
    float a, ae, b, be, sh, se, ch, ce;
    dw_mul_acc(t.x, t.y, crh, crl, a, ae);
    dw_mul_acc(t.z, t.w, srh, srl, b, be);
    two_sum(a, b, sh, se);
    se += ae + be;
    dw_mul_acc(t.z, t.w, crh, crl, a, ae);
    dw_mul_acc(t.x, t.y, srh, srl, b, be);
    two_sum(a, -b, ch, ce);
    ce += ae - be;
    sn = (double)sh + (double)se;
    cs = (double)ch + (double)ce;
}

// ifs = 1/f*, formed once per thread by the caller
// dw: also the double-word phase fields (c0h .. Fsl), which the scalar slow
// part reads; the paired one reads them only for a candidate outside the
// fixed-point ranges (wide), so the likelihood kernel skips them for N >= 64
__device__ void setup_mixed(const double* th, double T, double ifs, CandMix& c, bool dw = true) {
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
    double sb, cb, sl, cl;
    sincos_dw(beta, sb, cb);
    sincos_dw(lam, sl, cl);
    const double r = kAU / kC;
    const double Kc = -r * cb * cl, Ks = -r * cb * sl;
    c.Kc = (float)Kc;
    c.Ks = (float)Ks;
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
    c.gxr2 = 2.0f * (-Ap * s2);
    c.gpi = -Ax * s2;
    c.gxi2 = 2.0f * (-Ax * c2);
    c.f0 = (float)f0;
    c.fdT = (float)(fd * T);
    c.fdh = (float)(0.5 * fd);
    c.a0 = (float)(0.5 * f0 * ifs);
    c.a1 = (float)(0.5 * fd * T * ifs);
    float sD, cD;
    sincosf((float)(f0 * ifs), &sD, &cD);
    c.D0r = cD;
    c.D0i = -sD;
    c.eps = (float)(fd * T * ifs);
    // fixed-point phase coefficients (reductions exact in double)
    c.C0 = (unsigned long long)__double2ll_rn(p0 * 0x1p62) << 2;
    const double dr = delta - 1024.0 * rint(delta * (1.0 / 1024.0));
    const double cq2 = 0.5 * fd * T * T;
    const double c2r = cq2 - 0x1p20 * rint(cq2 * 0x1p-20);
    c.K1 = (unsigned long long)__double2ll_rn(dr * 0x1p54);
    c.K2 = (unsigned long long)__double2ll_rn(c2r * 0x1p44);
    const double Fc = f0 * Kc, Fs = f0 * Ks;
    // the paired slow part also drops (fdot/2) (k.rho)^2 from the receiver
    // phases: below 2^-32 cycles while |fdot| (L/c)^2 / 6 is, with
    // |k.rho| <= L/(sqrt3 c) and L/c = 1/(2 pi f*)
    const bool fd_ok = fabs(fd) * (ifs * ifs) < 0x1p-32 * 24.0 * kPi * kPi;
    c.wide = !(fabs(Fc) < 31.0 && fabs(Fs) < 31.0 && fabs(c2r) < 0x1p19 && fabs(dr) < 512.0 && fd_ok);
    c.Fc = c.wide ? 0 : __double2int_rn(Fc * 0x1p26);
    c.Fs = c.wide ? 0 : __double2int_rn(Fs * 0x1p26);
    if (dw || c.wide) {
        split(p0, c.c0h, c.c0l);
        split(delta, c.c1h, c.c1l);
        split(cq2, c.c2h, c.c2l);
        split(Fc, c.Fch, c.Fcl);
        split(Fs, c.Fsh, c.Fsl);
    }
    // largest link argument X = f (1 + |k.n|)/(2 f*) <= f_max / f*; the
    // tier keeps the first omitted series term below 2e-8 (few tiers: every
    // tier is a separate copy of the slow part in the instruction cache)
    const double xmax = fmax(fabs(f0), fabs(f0 + fd * T)) * ifs;
    c.J = xmax <= 0.489 ? 4 : xmax <= 1.34 ? 7 : xmax <= 2.35 ? 10 : 0;
}

// sinc(X) exp(-iX), J+1 terms of each series (J = 0: direct evaluation)
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

// exp(2 pi i x) for a receiver phase x = -f k.rho + ..., |x| <= xmax/(2 pi sqrt 3)
// (each spacecraft is L/sqrt 3 from the guiding centre, and f L/c = xmax/(2 pi)):
// Taylor series of sin and cos of t = 2 pi x, truncated where the first
// omitted term is below 2e-8 for the tier's bound on t (J = 4: t <= 0.282,
// 7: 0.774); sincospif above the J = 7 tier.
template <int J>
__device__ __forceinline__ float2 cis_rx(float x) {
    if constexpr (J == 0 || J >= 10) {
        float sn, cs;
        sincospif(2.0f * x, &sn, &cs);
        return make_float2(cs, sn);
    } else {
        // the Taylor series in x (cycles) with the powers of 2 pi folded into
        // the coefficients: sin to x^7 and cos to x^6 (J <= 4), one more term
        // each above
        const float x2 = x * x;
        float s, co;
        if constexpr (J <= 4) {
            s = fmaf(x2, -76.70585975306136f, 81.60524927607504f);
            s = fmaf(s, x2, -41.341702240399755f);
            s = fmaf(s, x2, 6.283185307179586f) * x;
            co = fmaf(x2, -85.45681720669371f, 64.93939402266828f);
            co = fmaf(co, x2, -19.739208802178716f);
            co = fmaf(co, x2, 1.0f);
        } else {
            s = fmaf(x2, 42.058693944897634f, -76.70585975306136f);
            s = fmaf(s, x2, 81.60524927607504f);
            s = fmaf(s, x2, -41.341702240399755f);
            s = fmaf(s, x2, 6.283185307179586f) * x;
            co = fmaf(x2, -26.426256783374388f, 60.24464137187664f);
            co = fmaf(co, x2, -85.45681720669371f);
            co = fmaf(co, x2, 64.93939402266828f);
            co = fmaf(co, x2, -19.739208802178716f);
            co = fmaf(co, x2, 1.0f);
        }
        return make_float2(co, s);
    }
}


// Slow part of one candidate: lane l, step r computes sample n and writes A, E
// to buf{A,E}[r*32 + l] (conflict-free), with n = l + 32 r (NAT: natural
// order, for the transform of the likelihood kernel) or n = R brev5(l) + r
// (for the across-lane transform of the waveform and gradient kernels).
template <int J, bool NAT>
__device__ void slow_part_mixed(const CandMix& c, const OrbitTables32& tab, int N, float2* bufA, float2* bufE,
                                int lane, float2* bufT) {
    const int R = N >> 5;
    const float invN = 1.0f / (float)N;
    const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f;
    const int nb = NAT ? lane : R * brev5(lane);
    const float4* tg = NAT ? tab.gn : tab.g;
    for (int r = 0; r < R; ++r) {
        const int p = r * 32 + lane;
        const float u = (float)(NAT ? nb + 32 * r : nb + r) * invN;
        const float uu = u * u;
        const float4 g0 = __ldg(tg + p), g1 = __ldg(tg + N + p);
        const float4 g2 = __ldg(tg + 2 * N + p), g3 = __ldg(tg + 3 * N + p);
        const float cah = g3.x, cal = g3.y, sah = g3.z, sal = g3.w;
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
        // k.rho_j: the third from the other two (the centroid is the guiding centre)
        float krho[3];
        krho[0] = fmaf(c.k0, g0.x, fmaf(c.k1, g0.y, c.k2 * g0.z));
        krho[1] = fmaf(c.k0, g0.w, fmaf(c.k1, g1.x, c.k2 * g1.y));
        krho[2] = -krho[0] - krho[1];
        // dP_j = -f k.rho_j + (fdot/2) (K + k.rho_j)^2 as a quadratic in k.rho_j
        const float q1 = fmaf(2.0f * c.fdh, K, -f), q0 = c.fdh * K * K;
        float2 rx[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)   // the common factor exp(2 pi i P_c) is applied once, below
            rx[j] = cis_rx<J>(fmaf(fmaf(c.fdh, krho[j], q1), krho[j], q0));
        const float a = fmaf(c.a1, u, c.a0);
        // projections of the arms on k, u, v; arm 2->0 closes the triangle
        float kn_[3], nu_[3], nv_[3];
        kn_[0] = fmaf(c.k0, g1.z, fmaf(c.k1, g1.w, c.k2 * g2.x));
        nu_[0] = fmaf(c.u0, g1.z, fmaf(c.u1, g1.w, c.u2 * g2.x));
        nv_[0] = fmaf(c.v0, g1.z, c.v1 * g1.w);   // v has no z component
        kn_[1] = fmaf(c.k0, g2.y, fmaf(c.k1, g2.z, c.k2 * g2.w));
        nu_[1] = fmaf(c.u0, g2.y, fmaf(c.u1, g2.z, c.u2 * g2.w));
        nv_[1] = fmaf(c.v0, g2.y, c.v1 * g2.z);
        kn_[2] = -kn_[0] - kn_[1];
        nu_[2] = -nu_[0] - nu_[1];
        nv_[2] = -nv_[0] - nv_[1];
        float2 zp[3], zm[3];   // arm a: link along +n (receiver rc[a]) and -n (receiver em[a])
#pragma unroll
        for (int arm = 0; arm < 3; ++arm) {
            const float kn = kn_[arm], nu = nu_[arm], nv = nv_[arm];
            const float Fp = fmaf(nu, nu, -(nv * nv));
            const float Fx1 = nu * nv;   // Fx / 2
            const float2 G = make_float2(fmaf(c.gpr, Fp, c.gxr2 * Fx1), fmaf(c.gpi, Fp, c.gxi2 * Fx1));
            const int rp = arm == 2 ? 0 : arm + 1;   // receiver of the +n link
            const int rm = arm;                      // receiver of the -n link
            zp[arm] = cmulf(cmulf(link_transfer<J>(fmaf(-a, kn, a)), G), rx[rp]);   // a (1 - kn)
            zm[arm] = cmulf(cmulf(link_transfer<J>(fmaf(a, kn, a)), G), rx[rm]);    // a (1 + kn)
        }
        // links: z01 = zp[0], z10 = zm[0], z12 = zp[1], z21 = zm[1], z20 = zp[2], z02 = zm[2]
        const float du = c.eps * u;
        const float2 Dc = make_float2(fmaf(-0.5f * du, du, 1.0f), -du);
        const float2 D = cmulf(make_float2(c.D0r, c.D0i), Dc);
        const float2 Xp = caddf(csubf(zm[0], zp[2]), cmulf(D, csubf(zp[0], zm[2])));
        const float2 Yp = caddf(csubf(zm[1], zp[0]), cmulf(D, csubf(zp[1], zm[0])));
        const float2 Zp = caddf(csubf(zm[2], zp[1]), cmulf(D, csubf(zp[2], zm[1])));
        // -i a (1 - D^2) = 2 a sin(f/f*) D with sin(f/f*) = -Im D (no
        // cancellation at low frequency), times the common phase factor
        const float sa2 = -2.0f * a * D.y;
        const float2 F = cmulf(make_float2(sa2 * D.x, sa2 * D.y), ePc);
        const float2 Ap = make_float2((Zp.x - Xp.x) * r2, (Zp.y - Xp.y) * r2);
        const float2 Ep = make_float2((Xp.x - 2.0f * Yp.x + Zp.x) * r6, (Xp.y - 2.0f * Yp.y + Zp.y) * r6);
        const float2 oA = cmulf(F, Ap), oE = cmulf(F, Ep);
        if constexpr (NAT) {   // channel-pair elements for the likelihood transform
            ((float4*)bufA)[p] = make_float4(oA.x, oE.x, oA.y, oE.y);
        } else {
            bufA[p] = oA;
            bufE[p] = oE;
        }
        if (bufT) {   // T = (X + Y + Z)/sqrt3, one complex float per sample
            const float r3 = 0.57735026918962576f;
            bufT[p] = cmulf(F, make_float2((Xp.x + Yp.x + Zp.x) * r3, (Xp.y + Yp.y + Zp.y) * r3));
        }
    }
}

// ---------------------------------------------------------------------------
// The slow part two samples at a time.  Lane l takes the samples n = l + 32 r
// and n + 32 of one step together; every float operation acts on the pair
// (x = sample n, y = sample n + 32) as one packed FP32 instruction, and a
// complex value of the pair is kept as two pairs (real parts, imaginary
// parts).  The arithmetic is that of slow_part_mixed, operation by operation.
// ---------------------------------------------------------------------------
using f2 = float2;
__device__ __forceinline__ f2 bc(float x) { return make_float2(x, x); }
__device__ __forceinline__ f2 padd(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 pmul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 pfma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 pneg(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 psub(f2 a, f2 b) { return __fadd2_rn(a, pneg(b)); }
__device__ __forceinline__ f2 print(f2 a) { return make_float2(rintf(a.x), rintf(a.y)); }

__device__ __forceinline__ void ptwo_sum(f2 a, f2 b, f2& s, f2& e) {
    s = padd(a, b);
    const f2 bb = psub(s, a);
    e = padd(psub(a, psub(s, bb)), psub(b, bb));
}

struct cpair {   // two complex numbers: re = (re_x, re_y), im = (im_x, im_y)
    f2 re, im;
};
__device__ __forceinline__ cpair pcmul(cpair a, cpair b) {
    return cpair{pfma(a.re, b.re, pneg(pmul(a.im, b.im))), pfma(a.re, b.im, pmul(a.im, b.re))};
}
__device__ __forceinline__ cpair pcadd(cpair a, cpair b) { return cpair{padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ cpair pcsub(cpair a, cpair b) { return cpair{psub(a.re, b.re), psub(a.im, b.im)}; }

// coefficient pairs (1/(2j+1)!, 1/(2j+2)!) of the link series, each value
// duplicated for the two samples
__constant__ float4 kLinkPair[11] = {
    {1.0f, 1.0f, 0.5f, 0.5f},
    {1.6666666666666666e-01f, 1.6666666666666666e-01f, 4.1666666666666664e-02f, 4.1666666666666664e-02f},
    {8.3333333333333332e-03f, 8.3333333333333332e-03f, 1.3888888888888889e-03f, 1.3888888888888889e-03f},
    {1.9841269841269841e-04f, 1.9841269841269841e-04f, 2.4801587301587302e-05f, 2.4801587301587302e-05f},
    {2.7557319223985893e-06f, 2.7557319223985893e-06f, 2.7557319223985888e-07f, 2.7557319223985888e-07f},
    {2.5052108385441720e-08f, 2.5052108385441720e-08f, 2.0876756987868100e-09f, 2.0876756987868100e-09f},
    {1.6059043836821613e-10f, 1.6059043836821613e-10f, 1.1470745597729725e-11f, 1.1470745597729725e-11f},
    {7.6471637318198164e-13f, 7.6471637318198164e-13f, 4.7794773323873853e-14f, 4.7794773323873853e-14f},
    {2.8114572543455206e-15f, 2.8114572543455206e-15f, 1.5619206968586225e-16f, 1.5619206968586225e-16f},
    {8.2206352466243295e-18f, 8.2206352466243295e-18f, 4.1103176233121648e-19f, 4.1103176233121648e-19f},
    {1.9572941063391263e-20f, 1.9572941063391263e-20f, 8.8967913924505741e-22f, 8.8967913924505741e-22f}};

// The link series of a pair in x2 = X^2 with the powers of y = -4 X^2 and the
// factor -2 of Im folded into the coefficients: (1/(2j+1)!, -2/(2j+2)!) times
// (-4)^j.  Scalings by powers of two are exact, so every intermediate equals
// the plain Horner value in y times (-4)^j and the results are those of
// link_transfer<J> bit for bit, with two operations fewer per link.
__constant__ float4 kLinkPairS[11] = {
    {1.000000000e+00f, 1.000000000e+00f, -1.000000000e+00f, -1.000000000e+00f},
    {-6.666666865e-01f, -6.666666865e-01f, 3.333333433e-01f, 3.333333433e-01f},
    {1.333333403e-01f, 1.333333403e-01f, -4.444444552e-02f, -4.444444552e-02f},
    {-1.269841287e-02f, -1.269841287e-02f, 3.174603218e-03f, 3.174603218e-03f},
    {7.054673624e-04f, 7.054673624e-04f, -1.410934783e-04f, -1.410934783e-04f},
    {-2.565335853e-05f, -2.565335853e-05f, 4.275559604e-06f, 4.275559604e-06f},
    {6.577784575e-07f, 6.577784575e-07f, -9.396834599e-08f, -9.396834599e-08f},
    {-1.252911286e-08f, -1.252911286e-08f, 1.566139107e-09f, 1.566139107e-09f},
    {1.842516695e-10f, 1.842516695e-10f, -2.047240676e-11f, -2.047240676e-11f},
    {-2.154990162e-12f, -2.154990162e-12f, 2.154990189e-13f, 2.154990189e-13f},
    {2.052371673e-14f, 2.052371673e-14f, -1.865792295e-15f, -1.865792295e-15f}};

// link_transfer<J> of a pair
template <int J>
__device__ __forceinline__ cpair plink_transfer(f2 X) {
    if constexpr (J == 0) {
        const float2 a = link_transfer<0>(X.x), b = link_transfer<0>(X.y);
        return cpair{make_float2(a.x, b.x), make_float2(a.y, b.y)};
    } else {
        const f2 x2 = pmul(X, X);
        f2 re, im;
        if constexpr (J <= 4) {
            // the same coefficients as literals (measured faster for the
            // short series, slower for the longer ones)
            constexpr float cre[5] = {1.000000000e+00f, -6.666666865e-01f, 1.333333403e-01f, -1.269841287e-02f,
                                      7.054673624e-04f};
            constexpr float cim[5] = {-1.000000000e+00f, 3.333333433e-01f, -4.444444552e-02f, 3.174603218e-03f,
                                      -1.410934783e-04f};
            re = bc(cre[J]);
            im = bc(cim[J]);
#pragma unroll
            for (int j = J - 1; j >= 0; --j) {
                re = pfma(re, x2, bc(cre[j]));
                im = pfma(im, x2, bc(cim[j]));
            }
        } else {
            const float4 cJ = kLinkPairS[J];
            re = make_float2(cJ.x, cJ.y);
            im = make_float2(cJ.z, cJ.w);
#pragma unroll
            for (int j = J - 1; j >= 0; --j) {
                const float4 cj = kLinkPairS[j];
                re = pfma(re, x2, make_float2(cj.x, cj.y));
                im = pfma(im, x2, make_float2(cj.z, cj.w));
            }
        }
        return cpair{re, pmul(X, im)};
    }
}

// cis_rx<J> of a pair
template <int J>
__device__ __forceinline__ cpair pcis_rx(f2 x) {
    if constexpr (J == 0 || J >= 10) {
        const float2 a = cis_rx<J>(x.x), b = cis_rx<J>(x.y);
        return cpair{make_float2(a.x, b.x), make_float2(a.y, b.y)};
    } else {
        f2 s, co;
        if constexpr (J <= 4) {
            // the Taylor series in x (cycles) with the powers of 2 pi folded
            // into the coefficients: sin to x^7, cos to x^6
            const f2 x2 = pmul(x, x);
            s = pfma(x2, bc(-76.70585975306136f), bc(81.60524927607504f));
            s = pfma(s, x2, bc(-41.341702240399755f));
            s = pmul(pfma(s, x2, bc(6.283185307179586f)), x);
            co = pfma(x2, bc(-85.45681720669371f), bc(64.93939402266828f));
            co = pfma(co, x2, bc(-19.739208802178716f));
            co = pfma(co, x2, bc(1.0f));
        } else {
            // the same with one more term each: sin to x^9, cos to x^10
            const f2 x2 = pmul(x, x);
            s = pfma(x2, bc(42.058693944897634f), bc(-76.70585975306136f));
            s = pfma(s, x2, bc(81.60524927607504f));
            s = pfma(s, x2, bc(-41.341702240399755f));
            s = pmul(pfma(s, x2, bc(6.283185307179586f)), x);
            co = pfma(x2, bc(-26.426256783374388f), bc(60.24464137187664f));
            co = pfma(co, x2, bc(-85.45681720669371f));
            co = pfma(co, x2, bc(64.93939402266828f));
            co = pfma(co, x2, bc(-19.739208802178716f));
            co = pfma(co, x2, bc(1.0f));
        }
        return cpair{co, s};
    }
}

// f0 (Kc cos a + Ks sin a) modulo one in units of 2^-32 of a cycle (rounded
// down), from the Q1.31 cos a, sin a of a sample: the products are in units
// of 2^-57, and |f0 K| < 31 keeps their sum inside 64 bits
__device__ __forceinline__ unsigned dop_fix(const CandMix& c, int cq, int sq) {
    const long long d = (long long)c.Fc * cq + (long long)c.Fs * sq;
    return (unsigned)((unsigned long long)d >> 25);
}

// Recurrence of c0 + c1 u + c2 u^2 (u = n/N) in units of 2^-64 of a cycle
// over a lane's sample pairs (n, n + 32), n = lane + 64 h: exact modulo one
struct PhaseRec {
    unsigned long long ph, dph, e32, ddph, de32;
    __device__ __forceinline__ PhaseRec(const CandMix& c, int N, int lane) {
        const int lg = __ffs(N) - 1;
        const unsigned long long k1 = c.K1 << (10 - lg), k2 = c.K2 << (20 - 2 * lg);
        const unsigned long long l = (unsigned long long)lane;
        ph = c.C0 + k1 * l + k2 * (l * l);
        dph = 64ull * k1 + k2 * (128ull * l + 4096ull);
        e32 = 32ull * k1 + k2 * (64ull * l + 1024ull);
        ddph = 8192ull * k2;
        de32 = 4096ull * k2;
    }
    // top words of the phases of n and n + 32, then advance to n + 64
    __device__ __forceinline__ void next(unsigned& a, unsigned& b) {
        a = (unsigned)(ph >> 32);
        b = (unsigned)((ph + e32) >> 32);
        ph += dph;
        dph += ddph;
        e32 += de32;
    }
};

// The common phase P_c = Pc + Pl of a sample pair (Pc in [-1/2, 1/2] up to
// small, |Pl| < 2^-19; returned as Pc and 2 pi Pl): the recurrence's top words pa, pb minus
// f0 (Kc cos a + Ks sin a), modulo one in 32 bits, split into its top 20
// and low 12 bits (both exact in float), plus small = -fdot T u K in float
__device__ __forceinline__ void phase_fix(const CandMix& c, unsigned pa, unsigned pb, int cqa, int sqa, int cqb,
                                          int sqb, f2 small, f2& Pc, f2& tl) {
    pa -= dop_fix(c, cqa, sqa);
    pb -= dop_fix(c, cqb, sqb);
    const f2 xh = make_float2(__int_as_float(0x4B400000 + ((int)pa >> 12)),
                              __int_as_float(0x4B400000 + ((int)pb >> 12)));
    const f2 xl = make_float2(__uint_as_float(0x4B000000u | (pa & 0xFFFu)),
                              __uint_as_float(0x4B000000u | (pb & 0xFFFu)));
    const f2 Ph = pfma(xh, bc(0x1p-20f), bc(-12.0f));     // in [-1/2, 1/2)
    // 2 pi times the low bits' value (in [0, 2^-20) cycles)
    const f2 Pt = pfma(xl, bc(6.2831853071795865f * 0x1p-32f), bc(-6.2831853071795865f * 0x1p-9f));
    // Ph + small with its exact rounding error by Fast2Sum: Ph is a multiple
    // of 2^-20 and so of ulp(small) (|small| < 8), so Ph + small - RN(...) is
    // exact whichever is larger; the result is TwoSum's
    Pc = padd(Ph, small);
    const f2 e = psub(small, psub(Pc, Ph));
    tl = pfma(bc(6.2831853071795865f), e, Pt);
}

// natural sample order (the likelihood kernel's transform), N >= 64; with
// T3 and bufT also T = (X + Y + Z)/sqrt3, one complex float per sample.  The
// carrier phase is taken in 64-bit fixed point (CandMix), where the sums
// wrap modulo one exactly; the rest follows slow_part_mixed operation by
// operation.
template <int J, bool T3>
__device__ void slow_part_pair(const CandMix& c, const OrbitTables32& tab, int N, float2* bufA, float2* bufE,
                               int lane, float2* bufT) {
    const int R = N >> 5, H = N >> 1;
    const float invN = 1.0f / (float)N;
    // 1/sqrt2, 1/sqrt6 times the factor -2 of F (exact: a power of two)
    const f2 r2 = bc(-2.0f * 0.70710678118654752f), r6 = bc(-2.0f * 0.40824829046386302f);
    PhaseRec rec(c, N, lane);
    for (int r = 0; r < R; r += 2) {
        const int m = (r >> 1) * 32 + lane;
        const int n = lane + 32 * r;
        const f2 u = pmul(make_float2((float)n, (float)(n + 32)), bc(invN));
        float4 t[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) t[f] = __ldg(tab.gp + f * H + m);
        const f2 rho0x = make_float2(t[0].x, t[0].y), rho0y = make_float2(t[0].z, t[0].w);
        const f2 rho0z = make_float2(t[1].x, t[1].y), rho1x = make_float2(t[1].z, t[1].w);
        const f2 rho1y = make_float2(t[2].x, t[2].y), rho1z = make_float2(t[2].z, t[2].w);
        const f2 n0x = make_float2(t[3].x, t[3].y), n0y = make_float2(t[3].z, t[3].w);
        const f2 n0z = make_float2(t[4].x, t[4].y), n1x = make_float2(t[4].z, t[4].w);
        const f2 n1y = make_float2(t[5].x, t[5].y), n1z = make_float2(t[5].z, t[5].w);
        // cos a, sin a (float) and the same in Q1.31 (int bits) for both samples
        const f2 cah = make_float2(t[6].x, t[6].y), sah = make_float2(t[6].z, t[6].w);
        const int cqa = __float_as_int(t[7].x), cqb = __float_as_int(t[7].y);
        const int sqa = __float_as_int(t[7].z), sqb = __float_as_int(t[7].w);
        // carrier phase modulo one in fixed point (PhaseRec, phase_fix)
        unsigned pa, pb;
        rec.next(pa, pb);
        const f2 K = pfma(bc(c.Kc), cah, pmul(bc(c.Ks), sah));
        f2 Pc, tl;
        phase_fix(c, pa, pb, cqa, sqa, cqb, sqb, pmul(pneg(pmul(bc(c.fdT), u)), K), Pc, tl);
        float sx, cx, sy, cy;
        sincospif(2.0f * Pc.x, &sx, &cx);
        sincospif(2.0f * Pc.y, &sy, &cy);
        const f2 sP = make_float2(sx, sy), cP = make_float2(cx, cy);
        const cpair ePc{pfma(pneg(tl), sP, cP), pfma(tl, cP, sP)};
        const f2 fr = pfma(bc(c.fdT), u, bc(c.f0));
        f2 krho[3];
        krho[0] = pfma(bc(c.k0), rho0x, pfma(bc(c.k1), rho0y, pmul(bc(c.k2), rho0z)));
        krho[1] = pfma(bc(c.k0), rho1x, pfma(bc(c.k1), rho1y, pmul(bc(c.k2), rho1z)));
        krho[2] = psub(pneg(krho[0]), krho[1]);
        // dP_j = -f k.rho_j + (fdot/2) (K + k.rho_j)^2 to first order in
        // k.rho_j: (fdot K - f) k.rho_j + (fdot/2) K^2; the (fdot/2) (k.rho_j)^2
        // left out is below 2^-32 cycles for every candidate this path takes
        // (setup_mixed sends the others to the scalar slow part)
        const f2 g1 = pfma(bc(2.0f * c.fdh), K, pneg(fr));
        const f2 g0 = pmul(pmul(bc(c.fdh), K), K);
        cpair rx[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) rx[j] = pcis_rx<J>(pfma(g1, krho[j], g0));
        const f2 a = pfma(bc(c.a1), u, bc(c.a0));
        f2 kn_[3], nu_[3], nv_[3];
        kn_[0] = pfma(bc(c.k0), n0x, pfma(bc(c.k1), n0y, pmul(bc(c.k2), n0z)));
        nu_[0] = pfma(bc(c.u0), n0x, pfma(bc(c.u1), n0y, pmul(bc(c.u2), n0z)));
        nv_[0] = pfma(bc(c.v0), n0x, pmul(bc(c.v1), n0y));   // v has no z component
        kn_[1] = pfma(bc(c.k0), n1x, pfma(bc(c.k1), n1y, pmul(bc(c.k2), n1z)));
        nu_[1] = pfma(bc(c.u0), n1x, pfma(bc(c.u1), n1y, pmul(bc(c.u2), n1z)));
        nv_[1] = pfma(bc(c.v0), n1x, pmul(bc(c.v1), n1y));
        kn_[2] = psub(pneg(kn_[0]), kn_[1]);
        nu_[2] = psub(pneg(nu_[0]), nu_[1]);
        nv_[2] = psub(pneg(nv_[0]), nv_[1]);
        cpair zp[3], zm[3];
#pragma unroll
        for (int arm = 0; arm < 3; ++arm) {
            const f2 kn = kn_[arm], nu = nu_[arm], nv = nv_[arm];
            const f2 Fp = pfma(nu, nu, pneg(pmul(nv, nv)));
            // Fx = 2 nu nv with the exact factor 2 on the x coefficients
            const f2 Fx1 = pmul(nu, nv);
            const cpair G{pfma(bc(c.gpr), Fp, pmul(bc(c.gxr2), Fx1)), pfma(bc(c.gpi), Fp, pmul(bc(c.gxi2), Fx1))};
            const int rp = arm == 2 ? 0 : arm + 1;
            const int rm = arm;
            zp[arm] = pcmul(pcmul(plink_transfer<J>(pfma(pneg(a), kn, a)), G), rx[rp]);   // a (1 - kn)
            zm[arm] = pcmul(pcmul(plink_transfer<J>(pfma(a, kn, a)), G), rx[rm]);         // a (1 + kn)
        }
        const f2 du = pmul(bc(c.eps), u);
        const cpair Dc{pfma(pmul(bc(-0.5f), du), du, bc(1.0f)), pneg(du)};
        const cpair D = pcmul(cpair{bc(c.D0r), bc(c.D0i)}, Dc);
        const cpair Xp = pcadd(pcsub(zm[0], zp[2]), pcmul(D, pcsub(zp[0], zm[2])));
        const cpair Yp = pcadd(pcsub(zm[1], zp[0]), pcmul(D, pcsub(zp[1], zm[0])));
        const cpair Zp = pcadd(pcsub(zm[2], zp[1]), pcmul(D, pcsub(zp[2], zm[1])));
        // F / -2 (its -2 is in r2, r6, r3)
        const f2 sa = pmul(a, D.im);
        const cpair F = pcmul(cpair{pmul(sa, D.re), pmul(sa, D.im)}, ePc);
        const cpair Ap{pmul(psub(Zp.re, Xp.re), r2), pmul(psub(Zp.im, Xp.im), r2)};
        // X - 2Y in one fused operation (2Y is exact)
        const cpair Ep{pmul(padd(pfma(bc(-2.0f), Yp.re, Xp.re), Zp.re), r6),
                       pmul(padd(pfma(bc(-2.0f), Yp.im, Xp.im), Zp.im), r6)};
        const cpair oA = pcmul(F, Ap), oE = pcmul(F, Ep);
        // channel-pair elements (A re, E re, A im, E im) for the transform
        const int p = r * 32 + lane;
        float4* buf = (float4*)bufA;
        buf[p] = make_float4(oA.re.x, oE.re.x, oA.im.x, oE.im.x);
        buf[p + 32] = make_float4(oA.re.y, oE.re.y, oA.im.y, oE.im.y);
        if constexpr (T3) {
            if (bufT) {
                const f2 r3 = bc(-2.0f * 0.57735026918962576f);
                const cpair Tp{pmul(padd(padd(Xp.re, Yp.re), Zp.re), r3), pmul(padd(padd(Xp.im, Yp.im), Zp.im), r3)};
                const cpair oT = pcmul(F, Tp);
                bufT[p] = make_float2(oT.re.x, oT.im.x);
                bufT[p + 32] = make_float2(oT.re.y, oT.im.y);
            }
        }
    }
}

template <bool NAT, bool T3 = false>
__device__ void slow_part_dispatch(const CandMix& c, const OrbitTables32& tab, int N, float2* bufA, float2* bufE,
                                   int lane, float2* bufT = nullptr) {
    if constexpr (NAT) {
        if (N >= 64 && !c.wide) {
            switch (c.J) {
                case 4: slow_part_pair<4, T3>(c, tab, N, bufA, bufE, lane, bufT); break;
                case 7: slow_part_pair<7, T3>(c, tab, N, bufA, bufE, lane, bufT); break;
                case 10: slow_part_pair<10, T3>(c, tab, N, bufA, bufE, lane, bufT); break;
                default: slow_part_pair<0, T3>(c, tab, N, bufA, bufE, lane, bufT); break;
            }
            return;
        }
    }
    float2* bt = T3 ? bufT : nullptr;
    switch (c.J) {
        case 4: slow_part_mixed<4, NAT>(c, tab, N, bufA, bufE, lane, bt); break;
        case 7: slow_part_mixed<7, NAT>(c, tab, N, bufA, bufE, lane, bt); break;
        case 10: slow_part_mixed<10, NAT>(c, tab, N, bufA, bufE, lane, bt); break;
        default: slow_part_mixed<0, NAT>(c, tab, N, bufA, bufE, lane, bt); break;
    }
}

// Per-lane twiddles of the across-lane radix-2 stages (half size h = 2^s):
// the upper lane of a pair multiplies its value by exp(-i pi (l mod h)/h).
struct LaneTw {
    float2 w[4];   // stages h = 2, 4, 8, 16 (h = 1 has twiddle 1)
};

__device__ __forceinline__ LaneTw lane_twiddles(int lane) {
    LaneTw t;
#pragma unroll
    for (int s = 1; s < 5; ++s) {
        const int h = 1 << s;
        if (lane & h) {
            float sn, cs;
            sincospif((float)(lane & (h - 1)) / (float)h, &sn, &cs);
            t.w[s - 1] = make_float2(cs, -sn);
        } else {
            t.w[s - 1] = make_float2(1.0f, 0.0f);
        }
    }
    return t;
}

// 32-point DFT across the lanes: lane l holds element brev5(l) of the
// sequence on entry and element l of its transform on exit (radix-2 DIT).
__device__ __forceinline__ float2 lane_fft(float2 x, const LaneTw& tw, int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int h = 1 << s;
        const float2 u = s == 0 ? x : cmulf(x, tw.w[s - 1]);
        const float2 v = make_float2(__shfl_xor_sync(0xffffffffu, u.x, h), __shfl_xor_sync(0xffffffffu, u.y, h));
        x = (lane & h) ? csubf(v, u) : caddf(u, v);
    }
    return x;
}

// R-point DFT in registers, natural order in and out (radix-2 DIT with a
// compile-time bit reversal); twiddles exp(-2 pi i j / R) from the table of
// exp(-2 pi i k / 1024), k < 512.
template <int R>
__device__ __forceinline__ void reg_fft(float2 (&x)[R], const float2* __restrict__ tw1024) {
    if constexpr (R > 1) {
        constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
        float2 y[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            int b = 0;
#pragma unroll
            for (int k = 0; k < LR; ++k) b |= ((i >> k) & 1) << (LR - 1 - k);
            y[b] = x[i];
        }
#pragma unroll
        for (int s = 0; s < LR; ++s) {
            const int h = 1 << s;
#pragma unroll
            for (int b = 0; b < R / 2; ++b) {
                const int j = b & (h - 1);
                const int i0 = ((b >> s) << (s + 1)) + j;
                const int i1 = i0 + h;
                float2 t;
                if (j == 0) {
                    t = y[i1];
                } else if (4 * j == 2 * h) {   // exp(-i pi/2) = -i
                    t = make_float2(y[i1].y, -y[i1].x);
                } else {
                    t = cmulf(kW32[j * (16 / h)], y[i1]);
                }
                y[i1] = csubf(y[i0], t);
                y[i0] = caddf(y[i0], t);
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = y[i];
    }
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Transform one channel (R values per lane in buf[r*32 + lane]) into bins
// l + 32 k1 held in x[k1].
template <int R>
__device__ __forceinline__ void channel_fft(const float2* buf, const OrbitTables32& tab, const float2* tw1024,
                                            const LaneTw& ltw, int lane, float2 (&x)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = lane_fft(buf[r * 32 + lane], ltw, lane);
#pragma unroll
    for (int r = 1; r < R; ++r) x[r] = cmulf(x[r], __ldg(tab.ltw + r * 32 + lane));
    reg_fft<R>(x, tw1024);
}

// ---------------------------------------------------------------------------
// Transform of the likelihood kernel.  Input: lane l holds samples
// n = l + 32 r, r < R (R = N/32).  With n = l + 32 r and bin K = k1 + R k2,
//   S[K] = sum_l w32^(l k2) [ wN^(l k1) sum_r s[l + 32 r] wR^(r k1) ],
// so each lane first takes an R-point DFT of its own samples and a twiddle;
// a transpose through shared memory then gives each group of G = 32/R lanes
// one of the R 32-point DFTs, factored as 32 = R x G over l = j + G m:
//   sum_l y_l w32^(l k2) = sum_j w32^(j ka) wG^(j kb) sum_m y_(j+Gm) wR^(m ka),
//   k2 = ka + R kb:
// an R-point DFT in registers, a twiddle, and a G-point DFT across the
// group's lanes -- by a second transpose and register DFTs when R >= G, by
// radix-2 decimation-in-frequency shuffles otherwise.  Both transposes are
// skewed so that every half-warp access touches 16 distinct banks.
// ---------------------------------------------------------------------------

// element (k1, l) of the first transpose: row k1 of 32, rotated by G k1
template <int R>
__device__ __forceinline__ int t1_addr(int k1, int l) {
    return 32 * k1 + ((l + (32 / R) * k1) & 31);
}

// element (group g, ka, u, v) of the second transpose for R = 4 (G = 8):
// lane j = u + 2v of group g holds ka; lane 2 ka + u collects v = 0..3
__device__ __forceinline__ int t2_addr4(int g, int ka, int u, int v) {
    const int h = g >> 1, gp = g & 1;
    return 64 * h + 16 * ka + ((8 * gp + 4 * u + v + ka) & 15);
}

// element (group g, lane j of the group, ka) of the second transpose (R >= 8),
// in 16-byte elements: row g G + j of R elements, the low three index bits
// rotated so that every quarter-warp access touches 8 distinct 16-byte bank
// groups (rotation constants found by checking all accesses of each R)
template <int R>
__device__ __forceinline__ int t2_addr(int g, int j, int ka) {
    constexpr int G = 32 / R;
    constexpr int a = R == 8 ? 2 : R == 16 ? 1 : 0, b = R == 16 ? 2 : 1, c = R == 16 ? 1 : 0;
    return (g * G + j) * R + (ka & ~7) + ((ka + a * j + b * g + c * (ka >> 3)) & 7);
}

// bit reversal of the low b bits
__device__ __forceinline__ int brev_bits(int x, int b) { return b == 0 ? 0 : (int)(__brev((unsigned)x) >> (32 - b)); }

// The transform works on both channels at once: a value is a cpair with
// channel A in .x and channel E in .y of its real and imaginary pairs, kept in
// shared memory as one 16-byte element (A re, E re, A im, E im).
__device__ __forceinline__ cpair ld4(const float4* p) {
    const float4 v = *p;
    return cpair{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ cpair ldg4(const float4* p) {
    const float4 v = __ldg(p);
    return cpair{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st4(float4* p, cpair v) { *p = make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }
__device__ __forceinline__ cpair pmul_mi(cpair v) { return cpair{v.im, pneg(v.re)}; }   // times -i

// exp(-2 pi i m / 32), m < 16, each part duplicated for the two channels
__constant__ float4 kW32d[16] = {
    {1.000000000e+00f, 1.000000000e+00f, 0.0f, 0.0f},
    {9.807852804e-01f, 9.807852804e-01f, -1.950903220e-01f, -1.950903220e-01f},
    {9.238795325e-01f, 9.238795325e-01f, -3.826834324e-01f, -3.826834324e-01f},
    {8.314696123e-01f, 8.314696123e-01f, -5.555702330e-01f, -5.555702330e-01f},
    {7.071067812e-01f, 7.071067812e-01f, -7.071067812e-01f, -7.071067812e-01f},
    {5.555702330e-01f, 5.555702330e-01f, -8.314696123e-01f, -8.314696123e-01f},
    {3.826834324e-01f, 3.826834324e-01f, -9.238795325e-01f, -9.238795325e-01f},
    {1.950903220e-01f, 1.950903220e-01f, -9.807852804e-01f, -9.807852804e-01f},
    {0.0f, 0.0f, -1.000000000e+00f, -1.000000000e+00f},
    {-1.950903220e-01f, -1.950903220e-01f, -9.807852804e-01f, -9.807852804e-01f},
    {-3.826834324e-01f, -3.826834324e-01f, -9.238795325e-01f, -9.238795325e-01f},
    {-5.555702330e-01f, -5.555702330e-01f, -8.314696123e-01f, -8.314696123e-01f},
    {-7.071067812e-01f, -7.071067812e-01f, -7.071067812e-01f, -7.071067812e-01f},
    {-8.314696123e-01f, -8.314696123e-01f, -5.555702330e-01f, -5.555702330e-01f},
    {-9.238795325e-01f, -9.238795325e-01f, -3.826834324e-01f, -3.826834324e-01f},
    {-9.807852804e-01f, -9.807852804e-01f, -1.950903220e-01f, -1.950903220e-01f}};

// reg_fft<R> on channel pairs
template <int R>
__device__ __forceinline__ void reg_fft2(cpair (&x)[R]) {
    if constexpr (R > 1) {
        constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
        cpair y[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            int b = 0;
#pragma unroll
            for (int k = 0; k < LR; ++k) b |= ((i >> k) & 1) << (LR - 1 - k);
            y[b] = x[i];
        }
#pragma unroll
        for (int s = 0; s < LR; ++s) {
            const int h = 1 << s;
#pragma unroll
            for (int b = 0; b < R / 2; ++b) {
                const int j = b & (h - 1);
                const int i0 = ((b >> s) << (s + 1)) + j;
                const int i1 = i0 + h;
                cpair t;
                if (j == 0) {
                    t = y[i1];
                } else if (4 * j == 2 * h) {   // exp(-i pi/2) = -i
                    t = pmul_mi(y[i1]);
                } else {
                    const float4 w = kW32d[j * (16 / h)];
                    t = pcmul(cpair{make_float2(w.x, w.y), make_float2(w.z, w.w)}, y[i1]);
                }
                y[i1] = pcsub(y[i0], t);
                y[i0] = pcadd(y[i0], t);
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = y[i];
    }
}

// G-point DFT of v[0..G) in registers, natural order in and out (G = 1, 2, 4)
template <int G>
__device__ __forceinline__ void dft_small2(cpair* v) {
    if constexpr (G == 2) {
        const cpair a = v[0], b = v[1];
        v[0] = pcadd(a, b);
        v[1] = pcsub(a, b);
    } else if constexpr (G == 4) {
        const cpair s02 = pcadd(v[0], v[2]), d02 = pcsub(v[0], v[2]);
        const cpair s13 = pcadd(v[1], v[3]), d13 = pcsub(v[1], v[3]);
        v[0] = pcadd(s02, s13);
        v[2] = pcsub(s02, s13);
        v[1] = cpair{padd(d02.re, d13.im), psub(d02.im, d13.re)};   // d02 - i d13
        v[3] = cpair{psub(d02.re, d13.im), padd(d02.im, d13.re)};   // d02 + i d13
    }
}

__device__ __forceinline__ cpair shfl_xor4(cpair v, int m) {
    return cpair{make_float2(__shfl_xor_sync(0xffffffffu, v.re.x, m), __shfl_xor_sync(0xffffffffu, v.re.y, m)),
                 make_float2(__shfl_xor_sync(0xffffffffu, v.im.x, m), __shfl_xor_sync(0xffffffffu, v.im.y, m))};
}

__device__ __forceinline__ void kahan_add2(f2& sum, f2& comp, f2 x) {
    const f2 y = psub(x, comp);
    const f2 t = padd(sum, y);
    comp = psub(psub(t, sum), y);
    sum = t;
}

// the two channels' Kahan pairs as one: the sum is s - c
__device__ __forceinline__ void kahan_merge(f2 sum, f2 comp, float& s, float& c) {
    float e;
    two_sum(sum.x, sum.y, s, e);
    c = (comp.x + comp.y) - e;
}

// Swizzled position of element e of an N-element channel-pair buffer: the
// low three index bits XORed with higher ones, chosen (by exhaustive search
// over such maps) so that both the reads in sample order (r 32 + lane) and
// the stores at the bins bin_of<R>(kbase, q) leave the eight lanes of each
// quarter-warp in eight different 16-byte bank groups.
__device__ __forceinline__ int nat_sw(int e, int N) {
    if (N == 32) return e ^ ((e >> 3) & 3);
    if (N == 64) return e ^ ((e >> 3) & 7);
    if (N == 128) return e ^ ((e >> 3) & 1) ^ ((e >> 5) & 2);
    return e ^ ((e >> 3) & 6);
}

// Transform of both channels of one candidate (buf: N channel-pair elements,
// sample n at n, or at nat_sw(n) with SWIN; with ONE the samples are read
// from src, one complex float each, the second channel zero, and buf is only
// the workspace).  On return x[q] holds the DFT at index K(q) =
// bin_of<R>(kbase, q) (returned: kbase), and the transform is done with buf.
template <int R, bool ONE = false, bool SWIN = false>
__device__ __forceinline__ int nat_transform(float4* buf, const OrbitTables32& tab, const LaneTw& ltw, int lane,
                                             cpair (&x)[R], const float2* src = nullptr) {
    constexpr int N = 32 * R, G = 32 / R;
    constexpr int LG = G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : G == 16 ? 4 : 5;
    (void)N;
    const int g = lane / G, j = lane % G;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if constexpr (ONE) {
            const float2 v = src[r * 32 + lane];
            x[r] = cpair{make_float2(v.x, 0.0f), make_float2(v.y, 0.0f)};
        } else {
            x[r] = ld4(buf + (SWIN ? nat_sw(r * 32 + lane, N) : r * 32 + lane));
        }
    }
    reg_fft2<R>(x);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) x[k1] = pcmul(x[k1], ldg4(tab.ltw4 + k1 * 32 + lane));
    if constexpr (R > 1) {
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) st4(buf + t1_addr<R>(k1, lane), x[k1]);
        __syncwarp();
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = ld4(buf + t1_addr<R>(g, j + G * m));
        reg_fft2<R>(x);
        if constexpr (G > 1) {
            // exp(-2 pi i j ka / 32) = exp(-2 pi i (R j) ka / N): the lane-twiddle table
#pragma unroll
            for (int ka = 1; ka < R; ++ka) x[ka] = pcmul(x[ka], ldg4(tab.ltw4 + ka * 32 + R * j));
        }
    }
    // x[q] is the value of bin K(q): the G-point stage, then the bin map
    int kbase;   // K(q) = g + R*(ka(q) + R*kb(q)) with ka, kb per branch below
    if constexpr (R == 4) {
        // 8 = 4 x 2 over j = u + 2v: lane 2 ka + u gathers v = 0..3, a 4-point
        // DFT over v, twiddle exp(-2 pi i u kv / 8), a 2-point DFT over u
        // across the lane pair; it then holds kb = kv + 4 u, kv = 0..3
        const int u = j & 1, ka = j >> 1;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; ++q) st4(buf + t2_addr4(g, q, j & 1, j >> 1), x[q]);
        __syncwarp();
#pragma unroll
        for (int v = 0; v < 4; ++v) x[v] = ld4(buf + t2_addr4(g, ka, u, v));
        dft_small2<4>(x);
        if (u) {
            const f2 r = bc(0.70710678118654752f);
            x[1] = cpair{pmul(r, padd(x[1].re, x[1].im)), pmul(r, psub(x[1].im, x[1].re))};     // * exp(-i pi/4)
            x[2] = pmul_mi(x[2]);                                                                  // * -i
            x[3] = cpair{pmul(r, psub(x[3].im, x[3].re)), pneg(pmul(r, padd(x[3].re, x[3].im)))};  // * exp(-3 i pi/4)
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const cpair v = shfl_xor4(x[q], 1);
            x[q] = u ? pcsub(v, x[q]) : pcadd(x[q], v);
        }
        kbase = g + 4 * ka + 64 * u;   // + 16 kv for x[kv]: K = g + 4 (ka + 4 (kv + 4 u))
    } else if constexpr (R >= G && G > 1) {
        __syncwarp();
#pragma unroll
        for (int ka = 0; ka < R; ++ka) st4(buf + t2_addr<R>(g, j, ka), x[ka]);
        __syncwarp();
        // lane j now takes ka = (R/G) j + t for t < R/G, all G lanes of the group
#pragma unroll
        for (int t = 0; t < R / G; ++t) {
#pragma unroll
            for (int j2 = 0; j2 < G; ++j2) x[t * G + j2] = ld4(buf + t2_addr<R>(g, j2, (R / G) * j + t));
            dft_small2<G>(x + t * G);
        }
        kbase = g + R * (R / G) * j;   // + R t + R^2 kb for x[t G + kb]
    } else if constexpr (G > 1) {
        // radix-2 decimation in frequency across the group's lanes
#pragma unroll
        for (int s = LG - 1; s >= 0; --s) {
            const int h = 1 << s;
            const bool upper = (lane & h) != 0;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const cpair v = shfl_xor4(x[q], h);
                if (!upper) {
                    x[q] = pcadd(x[q], v);
                } else {
                    const cpair d = pcsub(v, x[q]);
                    x[q] = s == 0 ? d : pcmul(d, cpair{bc(ltw.w[s - 1].x), bc(ltw.w[s - 1].y)});
                }
            }
        }
        kbase = g + R * R * brev_bits(j, LG);   // + R ka for x[ka]
    } else {
        kbase = g;   // G = 1: + R ka for x[ka]
    }
    return kbase;
}

// DFT index of x[q] after nat_transform
template <int R>
__device__ __forceinline__ int bin_of(int kbase, int q) {
    constexpr int G = 32 / R;
    if constexpr (R == 4) return kbase + 16 * q;
    else if constexpr (R >= G && G > 1) return kbase + R * (q / G) + R * R * (q % G);
    else return kbase + R * q;
}

// Both channels of one candidate (buf: N channel-pair elements, sample n at
// n): transform, then the window inner products (with IM also the imaginary
// part of sum w d conj(h)); each sum is returned as s - c.  With ONE, the
// samples are read from src (one complex float each, the second channel
// zero) and buf is only the transform's workspace.
template <int R, bool IM, bool ONE = false>
__device__ void fft_inner_ch(float4* buf, const OrbitTables32& tab, const LaneTw& ltw, int lane, int off, int W,
                             const Win32* __restrict__ pw, float& sdh, float& cdh, float& shh, float& chh, float& sim,
                             float& cim, const float2* src = nullptr) {
    constexpr int N = 32 * R;
    cpair x[R];
    const int kbase = nat_transform<R, ONE>(buf, tab, ltw, lane, x, src);
    const f2 z = bc(0.0f);
    f2 s_dh = z, c_dh = z, s_hh = z, c_hh = z, s_im = z, c_im = z;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int K = bin_of<R>(kbase, q);
        const int m = K < N / 2 ? K : K - N;
        const int kk = off + m;
        if (kk >= 0 && kk < W) {
            const Win32 v = pw[kk];
            // explicit products: the same rounding in every kernel that forms these sums
            kahan_add2(s_dh, c_dh, pmul(v.w, pfma(v.dre, x[q].re, pmul(v.dim, x[q].im))));
            kahan_add2(s_hh, c_hh, pmul(v.w, pfma(x[q].re, x[q].re, pmul(x[q].im, x[q].im))));
            if constexpr (IM) kahan_add2(s_im, c_im, pmul(v.w, pfma(v.dim, x[q].re, pneg(pmul(v.dre, x[q].im)))));
        }
    }
    kahan_merge(s_dh, c_dh, sdh, cdh);
    kahan_merge(s_hh, c_hh, shh, chh);
    if constexpr (IM) kahan_merge(s_im, c_im, sim, cim);
}

// The T channel of one candidate, N = 32 R >= 64 points, without an idle
// half: T's even and odd samples form one channel pair (T_2m, T_2m+1) of an
// N/2-point transform (tabh: the N/2 tables; buf: workspace of N/2
// channel-pair elements), whose bins K < N/2 are E_K, O_K, and the radix-2
// step X_K = E_K + w^K O_K, X_K+N/2 = E_K - w^K O_K (w = exp(-2 pi i/N),
// from the 1024-point twiddles) gives T's N bins; then T's window inner
// products (its data in the first slot of each element of its float copy),
// compensated per lane, returned as s - c.
__device__ __forceinline__ void kahan_add1(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}
template <int R, bool IM>
__device__ void fft_inner_t_half(float4* buf, const float2* srcT, const OrbitTables32& tabh, const float2* tw1024,
                                 const LaneTw& ltw, int lane, int off, int W, const Win32* __restrict__ pw, float& sdh,
                                 float& cdh, float& shh, float& chh, float& sim, float& cim) {
    static_assert(R >= 2, "N >= 64");
    constexpr int N = 32 * R, H = R / 2;
    const float4* t4 = (const float4*)srcT;   // element m: (T_2m re, T_2m im, T_2m+1 re, T_2m+1 im)
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float4 v = t4[lane + 32 * j];
        buf[lane + 32 * j] = make_float4(v.x, v.z, v.y, v.w);
    }
    cpair x[H];
    const int kbase = nat_transform<H>(buf, tabh, ltw, lane, x);
    sdh = cdh = shh = chh = sim = cim = 0.0f;
#pragma unroll
    for (int q = 0; q < H; ++q) {
        const int K = bin_of<H>(kbase, q);                 // 0 <= K < N/2
        const float2 w = __ldg(tw1024 + K * (1024 / N));
        const float ore = x[q].re.y, oim = x[q].im.y;
        const float tre = fmaf(w.x, ore, -w.y * oim), tim = fmaf(w.x, oim, w.y * ore);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const float hre = half == 0 ? x[q].re.x + tre : x[q].re.x - tre;
            const float him = half == 0 ? x[q].im.x + tim : x[q].im.x - tim;
            const int m = half == 0 ? K : K - N / 2;       // bin q_c + m
            const int kk = off + m;
            if (kk >= 0 && kk < W) {
                const Win32 v = pw[kk];
                kahan_add1(sdh, cdh, __fmul_rn(v.w.x, fmaf(v.dre.x, hre, __fmul_rn(v.dim.x, him))));
                kahan_add1(shh, chh, __fmul_rn(v.w.x, fmaf(hre, hre, __fmul_rn(him, him))));
                if constexpr (IM) kahan_add1(sim, cim, __fmul_rn(v.w.x, fmaf(v.dim.x, hre, -__fmul_rn(v.dre.x, him))));
            }
        }
    }
}

// Compensated warp sums of two Kahan pairs a and b at once (reduce-scatter):
// at the first level the lower half-warp keeps a and the upper half keeps b,
// each sending the other value to its partner, so that the four remaining
// levels move one pair per lane instead of two.  Every value is combined by
// the same tree as in warp_sum2 (TwoSum is exact and symmetric), so the
// results are warp_sum2's bit for bit.  a's total is returned in (ah, al)
// and b's in (bh, bl) on every lane.
__device__ __forceinline__ void warp_sum2x2(float as, float ac, float bs, float bc_, float& ah, float& al, float& bh,
                                            float& bl, int lane) {
    const bool upper = (lane & 16) != 0;
    float kh = upper ? bs : as, kl = upper ? -bc_ : -ac;      // the value this half keeps
    const float sh = upper ? as : bs, sl = upper ? -ac : -bc_;
    const float rh = __shfl_xor_sync(0xffffffffu, sh, 16), rl = __shfl_xor_sync(0xffffffffu, sl, 16);
    float s, e;
    two_sum(kh, rh, s, e);
    kh = s;
    kl = kl + rl + e;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, kh, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, kl, o);
        two_sum(kh, h2, s, e);
        kh = s;
        kl = kl + l2 + e;
    }
    const float oh = __shfl_xor_sync(0xffffffffu, kh, 16), ol = __shfl_xor_sync(0xffffffffu, kl, 16);
    ah = upper ? oh : kh;
    al = upper ? ol : kl;
    bh = upper ? kh : oh;
    bl = upper ? kl : ol;
}

// Compensated warp sum of Kahan pairs: returns hi + lo on every lane.
__device__ __forceinline__ void warp_sum2(float sum, float comp, float& hi, float& lo) {
    hi = sum;
    lo = -comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo = lo + l2 + e;
    }
}

// dT, wT (may be null): the T channel, used in windows whose lowest frequency
// k0/T is at least f*/2; its float copy goes n_prep entries after A and E's.
__global__ void prep_mixed_kernel(const gb_window_t* __restrict__ wins, WinMeta* __restrict__ meta,
                                  Win32* __restrict__ prep, const double2* __restrict__ dA,
                                  const double2* __restrict__ dE, const double* __restrict__ wA,
                                  const double* __restrict__ wE, const double2* __restrict__ dT,
                                  const double* __restrict__ wT, long long n_prep, double T, double fstar,
                                  int* head) {
    __shared__ double s_acc[32], s_max[32];
    const int w = blockIdx.x;
    if (w == 0 && threadIdx.x < 2) head[threadIdx.x] = 0;   // both work queues
    const gb_window_t win = wins[w];
    const bool useT = dT != nullptr && (double)win.k0 / T >= 0.5 * fstar;
    double acc = 0.0, wmax = 0.0;
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const double2 a = dA[win.data_off + i], e = dE[win.data_off + i];
        const double wa = wA[win.data_off + i], we = wE[win.data_off + i];
        acc += wa * (a.x * a.x + a.y * a.y) + we * (e.x * e.x + e.y * e.y);
        wmax = fmax(wmax, fmax(wa, we));
        if (useT) {
            const double2 t = dT[win.data_off + i];
            const double wt = wT[win.data_off + i];
            acc += wt * (t.x * t.x + t.y * t.y);
            wmax = fmax(wmax, wt);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        s_acc[warp] = acc;
        s_max[warp] = wmax;
    }
    __syncthreads();
    double dd = 0.0, sig2 = 0.0;
    for (int i = 0; i < nw; ++i) {
        dd += s_acc[i];
        sig2 = fmax(sig2, s_max[i]);
    }
    if (!(sig2 > 0.0) || !isfinite(sig2)) sig2 = 1.0;
    const double sig = sqrt(sig2), isig2 = 1.0 / sig2;
    const long long po = meta[w].prep_off;
    if (threadIdx.x == 0) {
        meta[w].dd = dd * (4.0 / T);
        meta[w].sig = sig;
        meta[w].use_t = useT ? 1 : 0;
    }
    for (int i = threadIdx.x; i < win.W; i += blockDim.x) {
        const double2 a = dA[win.data_off + i], e = dE[win.data_off + i];
        Win32 v;
        v.dre = make_float2((float)(a.x * sig), (float)(e.x * sig));
        v.dim = make_float2((float)(a.y * sig), (float)(e.y * sig));
        v.w = make_float2((float)(wA[win.data_off + i] * isig2), (float)(wE[win.data_off + i] * isig2));
        prep[po + i] = v;
        if (useT) {   // T in the first slot of each pair, zero in the second
            const double2 t = dT[win.data_off + i];
            Win32 u;
            u.dre = make_float2((float)(t.x * sig), 0.0f);
            u.dim = make_float2((float)(t.y * sig), 0.0f);
            u.w = make_float2((float)(wT[win.data_off + i] * isig2), 0.0f);
            prep[n_prep + po + i] = u;
        }
    }
}

// resident CTAs per SM the small-N instantiation is compiled for (register cap)
#ifndef GB_MIXED_MINB
#define GB_MIXED_MINB 4
#endif

// RMAX: largest R = N/32 this instantiation handles (8: N <= 256; 32: N = 512, 1024)
// the two channels' compensated sums added into one (true sums s - c)
__device__ __forceinline__ void kahan_join(float& s, float& c, float s2, float c2) {
    float hi, e;
    two_sum(s, s2, hi, e);
    s = hi;
    c = (c + c2) - e;
}

template <int RMAX, bool IM, bool T3>
__global__ void __launch_bounds__(kWarpsMx * 32, RMAX <= 8 ? GB_MIXED_MINB : 2) loglik_mixed_kernel(
    const gb_window_t* __restrict__ wins, const WinMeta* __restrict__ meta, const Win32* __restrict__ prep,
    const Tile* __restrict__ items, int n_items, int* head, TabSet32 tabs, const float2* __restrict__ tw1024,
    double T, double fstar, const double* __restrict__ theta, double* __restrict__ logL,
    double* __restrict__ dh_out, double* __restrict__ hh_out, double* __restrict__ dhi_out, int* status, int n_max,
    unsigned long long budget_ns, long long n_prep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int CAP = T3 ? kCapT : 32;   // candidates of one work item
    CandMix* cands = (CandMix*)smem_raw + warp * CAP;
    Epi<IM>* epi = (Epi<IM>*)((CandMix*)smem_raw + kWarpsMx * CAP) + warp * CAP;
    float2* bufA =
        (float2*)((Epi<IM>*)((CandMix*)smem_raw + kWarpsMx * CAP) + kWarpsMx * CAP) + (size_t)warp * 2 * n_max;
    float2* bufE = bufA + n_max;
    // T3: T's samples per warp, one complex float each (the transform then
    // runs in bufA once A and E are done)
    float2* bufT = T3 ? (float2*)((Epi<IM>*)((CandMix*)smem_raw + kWarpsMx * CAP) + kWarpsMx * CAP) +
                            (size_t)kWarpsMx * 2 * n_max + (size_t)warp * n_max
                      : nullptr;
    const LaneTw ltw = lane_twiddles(lane);
    const double ifs = 1.0 / fstar;   // the float results do not see the reciprocal's rounding

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
        const bool useT = T3 && wm.use_t;
        const Win32* pwT = prep + n_prep + wm.prep_off;
        const int N = win.N;
        const OrbitTables32 tab = tabs.t[__ffs(N) - 6];
        const int cnt = (int)(t.c_end - t.c_begin);
        if (lane < cnt) setup_mixed(theta + 8 * (t.c_begin + lane), T, ifs, cands[lane], N < 64);
        __syncwarp();
        for (int i = 0; i < cnt; ++i) {
            const CandMix& c = cands[i];
            float sdh = 0.0f, cdh = 0.0f, shh = 0.0f, chh = 0.0f, sim = 0.0f, cim = 0.0f;
            if (!c.bad) {
                slow_part_dispatch<true, T3>(c, tab, N, bufA, bufE, lane, useT ? bufT : nullptr);
                __syncwarp();
                const long long off64 = c.q - win.k0;
                if (off64 > -(long long)N && off64 < (long long)win.W + N) {
                    const int off = (int)off64;
#define GB_FFT_INNER(R) \
    fft_inner_ch<R, IM>((float4*)bufA, tab, ltw, lane, off, win.W, pw, sdh, cdh, shh, chh, sim, cim)
                    if constexpr (RMAX <= 8) {
                        switch (N) {
                            case 32: GB_FFT_INNER(1); break;
                            case 64: GB_FFT_INNER(2); break;
                            case 128: GB_FFT_INNER(4); break;
                            default: GB_FFT_INNER(8); break;
                        }
                    } else {
                        if (N == 512)
                            GB_FFT_INNER(16);
                        else
                            GB_FFT_INNER(32);
                    }
#undef GB_FFT_INNER
                    if constexpr (T3) {
                        if (useT) {   // the T channel (a half-length transform), then into the sums
                            float tdh = 0.0f, tcdh = 0.0f, thh = 0.0f, tchh = 0.0f, tim = 0.0f, tcim = 0.0f;
                            __syncwarp();
#define GB_FFT_INNER_T(R)                                                                                    \
    fft_inner_t_half<R, IM>((float4*)bufA, bufT, tabs.t[__ffs(N) - 7], tw1024, ltw, lane, off, win.W, pwT, tdh, \
                            tcdh, thh, tchh, tim, tcim)
                            if constexpr (RMAX <= 8) {
                                switch (N) {
                                    case 32:
                                        fft_inner_ch<1, IM, true>((float4*)bufA, tab, ltw, lane, off, win.W, pwT, tdh,
                                                                  tcdh, thh, tchh, tim, tcim, bufT);
                                        break;
                                    case 64: GB_FFT_INNER_T(2); break;
                                    case 128: GB_FFT_INNER_T(4); break;
                                    default: GB_FFT_INNER_T(8); break;
                                }
                            } else {
                                if (N == 512)
                                    GB_FFT_INNER_T(16);
                                else
                                    GB_FFT_INNER_T(32);
                            }
#undef GB_FFT_INNER_T
                            kahan_join(sdh, cdh, tdh, tcdh);
                            kahan_join(shh, chh, thh, tchh);
                            if constexpr (IM) kahan_join(sim, cim, tim, tcim);
                        }
                    }
                }
                __syncwarp();
            }
            float dhh, dhl, hhh, hhl, imh = 0.0f, iml = 0.0f;
            warp_sum2x2(sdh, cdh, shh, chh, dhh, dhl, hhh, hhl, lane);
            if constexpr (IM) warp_sum2(sim, cim, imh, iml);
            if (lane == 0) {
                if constexpr (IM)
                    epi[i] = Epi<IM>{dhh, dhl, hhh, hhl, imh, iml};
                else
                    epi[i] = Epi<IM>{dhh, dhl, hhh, hhl};
            }
        }
        __syncwarp();
        // lane-parallel epilogue in double, coalesced stores
        if (lane < cnt) {
            const CandMix& c = cands[lane];
            const int64_t cidx = t.c_begin + lane;
            if (c.bad) {
                logL[cidx] = nan("");
                if (dh_out) dh_out[cidx] = nan("");
                if (hh_out) hh_out[cidx] = nan("");
                if (IM && dhi_out) dhi_out[cidx] = nan("");
                atomicOr(status, kStatusNonFinite);
            } else {
                const Epi<IM> s = epi[lane];
                const double Sdh = (double)s.dh_hi + (double)s.dh_lo;
                const double Shh = (double)s.hh_hi + (double)s.hh_lo;
                const double dh = c.A * (2.0 * wm.sig / (double)N) * Sdh;
                const double hh = (c.A * c.A) * (T * wm.sig * wm.sig / ((double)N * (double)N)) * Shh;
                logL[cidx] = dh - 0.5 * hh - 0.5 * wm.dd;
                if (dh_out) dh_out[cidx] = dh;
                if (hh_out) hh_out[cidx] = hh;
                if constexpr (IM) {
                    if (dhi_out) dhi_out[cidx] = c.A * (2.0 * wm.sig / (double)N) * ((double)s.im_hi + (double)s.im_lo);
                }
            }
        }
        __syncwarp();
    }
}

int resident_blocks(const void* kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}cudaError_t launch_mixed_part(const void* kfn, int grid, size_t smem, cudaStream_t s, const gb_window_t* wins,
                              const WinMeta* meta, const Win32* prep, const Tile* items, int n_items, int* head,
                              TabSet32 tabs, const float2* tw1024, double T, double fstar, const double* theta,
                              double* logL, double* dh, double* hh, double* dhi, int* status, int n_max,
                              unsigned long long budget_ns, long long n_prep) {
    void* args[] = {&wins, &meta, &prep, &items, &n_items, &head,  &tabs,      &tw1024, &T,     &fstar,
                    &theta, &logL, &dh,  &hh,    &dhi,     &status, &n_max,    &budget_ns, &n_prep};
    return cudaLaunchKernel(kfn, dim3(grid), dim3(kWarpsMx * 32), args, smem, s);
}

}  // namespace
}  // namespace gb
