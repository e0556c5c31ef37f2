// gb_internal.cuh -- types and helpers shared by the libgb translation units.
//
// Physical model (the paper cites, but does not print, the waveform and the
// detector response; Sec. III first paragraph and Sec. III.G):
//   * rigid equal-arm triangle of arm L on the first-order heliocentric orbit,
//     spacecraft i at beta_i = 2 pi i / 3, alpha = 2 pi t / yr;
//   * plane wave h_ab = Re[H_ab exp(i Phi(t - k.x/c))], H = A+ E+ - i Ax Ex,
//     Phi = 2 pi f0 xi + pi fdot xi^2 + phi0;
//   * link i -> j:  z_ij = -i (f/2f*) sinc(X) exp(-iX) (n.H.n) exp(i Psi_j),
//     X = (f/2f*)(1 - k.n), Psi_j the receiver's phase heterodyned by q;
//   * first-generation equal-arm TDI X, Y, Z with D = exp(-i f/f*), then
//     A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6 (Eq. 5).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gb.h"

namespace gb {

constexpr double kC = 299792458.0;           // m/s
constexpr double kAU = 1.495978707e11;       // m
constexpr double kYear = 31557600.0;         // s (Julian year)
constexpr double kPi = 3.14159265358979323846;
constexpr int kNumSizes = 6;                 // N = 32 .. 1024
constexpr int kTwiddles = 512;               // exp(-2 pi i k / 1024), k < 512

inline int log2_size(int N) {
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}
inline bool valid_size(int N) {
    return N >= GB_N_MIN && N <= GB_N_MAX && (N & (N - 1)) == 0;
}
inline int size_index(int N) { return log2_size(N) - 5; }

// Per-N geometry tables (device).  Layout: component-major, N entries each.
struct OrbitTables64 {
    const double* x;     // [3 craft][3 xyz][N]    positions, m
    const double* arm;   // [3 arms][3 xyz][N]     unit vectors of arms 0->1, 1->2, 2->0
};
// Float tables are stored lane-permuted: with R = N/32, entry p = r*32 + l
// holds sample n = R*brev5(l) + r, which is the sample lane l evaluates in its
// r-th step (the bit reversal feeds the across-lane FFT stage).
// Four float4 per sample (group-major, [4][N]); with rho_j = (x_j - x_centre)/c
// and n_01, n_12 the unit vectors of arms 0->1 and 1->2:
//   g[0] = (rho_0.xyz, rho_1.x)   g[1] = (rho_1.yz, n_01.xy)
//   g[2] = (n_01.z, n_12.xyz)     g[3] = (cos a hi, cos a lo, sin a hi, sin a lo)
// The third spacecraft and arm follow exactly from the rigid triangle:
// rho_2 = -rho_0 - rho_1 (the centroid is the guiding centre) and
// n_20 = -n_01 - n_12 (the arms close).
struct OrbitTables32 {
    const float4* g;     // [4][N], lane-permuted order (see the table kernel)
    const float2* ltw;   // [R][32]                exp(-2 pi i r l / N), lane twiddles
    const float4* gn;    // [4][N], the same values in natural sample order
    const float4* gp;    // [8][N/2], sample pairs (n, n + 32) of each lane, component pairs
                         // (components 0..11 as g[0..2]; 12, 13 cos a, sin a hi; 14, 15
                         // cos a, sin a in Q1.31 as int bits)
    const float4* ltw4;  // [R][32]                the lane twiddles as (re, re, im, im)
    const int2* gq;      // [N]                    (cos a, sin a) in Q1.31, natural order
};

constexpr int kTab64PerN = 18;   // doubles per sample
// floats per sample: 4 float4 (permuted) + lane twiddles + 4 float4 (natural) + 4 float4 (pairs)
// + duplicated lane twiddles + the Q1.31 cos a, sin a
constexpr int kTab32PerN = 56;

__host__ __device__ inline int brev5(int l) {
    return ((l & 1) << 4) | ((l & 2) << 2) | (l & 4) | ((l & 8) >> 2) | ((l & 16) >> 4);
}

// Tables of every size, passed by value as a kernel argument.
struct TabSet64 {
    OrbitTables64 t[kNumSizes];
};
struct TabSet32 {
    OrbitTables32 t[kNumSizes];
};

// Work item: candidates [c_begin, c_end) of window `win`.
struct Tile {
    int32_t win;
    int32_t pad;
    int64_t c_begin;
    int64_t c_end;
};

// Per-window values the mixed-precision kernels derive once per launch:
// <d|d>, the scale sigma = sqrt(max w) of the float copy of the window, and
// where that copy starts in the plan's scratch buffer.
struct WinMeta {
    double dd;
    double sig;
    long long prep_off;
    int use_t;   // the window's <.|.> includes the T channel (float copy at prep_off + n_prep)
    int pad;
};

// Float copy of one window bin: data times sigma, weights over sigma^2.
struct Win32 {
    float2 dre;   // (Re dA, Re dE)
    float2 dim;   // (Im dA, Im dE)
    float2 w;     // (wA, wE)
};

struct Plan {
    uint64_t key = 0;
    int prec = -1;
    int n_win = 0;
    int n_tiles = 0;
    int n_max = 0;
    int w_max = 0;
    long long n_prep = 0;           // total window bins (scratch entries)
    int n_large = 0;                // mixed plans: items with N >= 512 come first
    int tile_cands = 0;             // candidates per work item at most
    std::vector<gb_window_t> win;   // host copy of the layout: a lookup compares it, not only the hash
    gb_window_t* d_win = nullptr;
    Tile* d_tiles = nullptr;
    // scratch of the mixed-precision path (owned by the plan)
    WinMeta* d_meta = nullptr;
    Win32* d_prep = nullptr;
    int* d_head = nullptr;          // work-queue head
    uint64_t last_use = 0;
};

}  // namespace gb

struct gb_ctx {
    int device = 0;
    gb_obs_t obs{};
    std::string err;
    // tables, one allocation per N
    double* d_tab64[gb::kNumSizes] = {};
    float* d_tab32[gb::kNumSizes] = {};
    double* d_tw64 = nullptr;   // kTwiddles complex
    float* d_tw32 = nullptr;
    int* d_status = nullptr;    // device status word (GB_OK or GB_EINVAL)
    std::vector<gb::Plan> plans;
    uint64_t clock = 0;
    // launch shapes chosen by gb_autotune (0: built-in heuristics)
    int tune_item = 0;        // mixed: candidates per work item
    int tune_bpsm = 0;        // mixed: resident CTAs per SM of the persistent kernels
    int tune_tile64 = 0;      // FP64: candidates per CTA tile
    // chunk summaries of the MH scan (grown on demand)
    void* d_mh = nullptr;
    size_t mh_bytes = 0;
    // certified chains: exact flags, re-evaluation queues, counters (grown on demand)
    void* d_cert = nullptr;
    size_t cert_bytes = 0;
    // kernels launched by this context's calls
    uint64_t launches = 0;
    // work budget of the persistent kernels, nanoseconds per warp (0: none)
    unsigned long long budget_ns = 0;
    // events recorded around the next mixed likelihood launch, then cleared
    cudaEvent_t kev_start = nullptr, kev_end = nullptr;
};

namespace gb {

// bits of the device status word
constexpr int kStatusNonFinite = 1;   // a candidate had a non-finite parameter
constexpr int kStatusBudget = 2;      // a persistent kernel stopped at its time budget

// Nanoseconds since an arbitrary origin, from the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Philox-4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC 2011): ten rounds of two 32x32 -> 64-bit products
// with the Weyl key schedule.
__device__ __forceinline__ void philox_round(uint32_t (&c)[4], const uint32_t (&k)[2]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

// four 32-bit outputs for counter (a, b, cc, d) under key (k0, k1)
__device__ __forceinline__ uint4 philox4x32_10(uint32_t a, uint32_t b, uint32_t cc, uint32_t d, uint32_t k0,
                                               uint32_t k1) {
    uint32_t c[4] = {a, b, cc, d};
    uint32_t k[2] = {k0, k1};
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    return make_uint4(c[0], c[1], c[2], c[3]);
}

// uniform in (0, 1) from 32 bits
__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

int set_error(gb_ctx* ctx, int code, const std::string& msg);
// MH scratch: bytes for `chunk_slots` (chain, chunk) summaries and the keys
// of `proposals` proposals; grow the buffer
int ensure_mh_scratch(gb_ctx* ctx, size_t bytes);
size_t mh_scratch_bytes(size_t chunk_slots, size_t proposals);
int cuda_error(gb_ctx* ctx, cudaError_t e, const char* what);

cudaError_t build_tables_into(double T, double L, double* const tab64[kNumSizes], float* const tab32[kNumSizes],
                              double* tw64, float* tw32, cudaStream_t s);
OrbitTables64 tables64(const gb_ctx* ctx, int N);
OrbitTables32 tables32(const gb_ctx* ctx, int N);
TabSet64 tabset64(const gb_ctx* ctx);
TabSet32 tabset32(const gb_ctx* ctx);
inline double transfer_frequency(const gb_ctx* ctx) { return kC / (2.0 * kPi * ctx->obs.arm_L); }

// Validate windows and return (creating and uploading if needed) the launch
// plan for this layout; tiles hold at most `tile_cands` candidates.
int get_plan(gb_ctx* ctx, int prec, const gb_window_t* win, int32_t n_win, int tile_cands,
             const Plan** out);

// launchers implemented per precision
int launch_loglik_fp64(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE,
                       const double* wA, const double* wE, const double* theta, double* logL,
                       double* dh, double* hh, double* dh_im, const double* dT, const double* wT,
                       cudaStream_t s);
// FP64 likelihood of listed rows: window w's entries are rows[cand_off + j],
// j in [row_lo[w], row_hi[w]) (device), each a row of that window; results
// bit-identical to launch_loglik_fp64's for the same rows; gate (device, may
// be null): skip the launch when *gate == 0
int launch_loglik_rows64(gb_ctx* ctx, const gb_window_t* d_win, int n_win, int n_max, int ctas_per_win,
                         const double* dA, const double* dE, const double* wA, const double* wE, const double* theta,
                         const int32_t* rows, const int32_t* row_lo, const int32_t* row_hi, double* logL,
                         double* dh, double* hh, const int* gate, cudaStream_t s);
// chains (mh.cu); gate (device, may be null): skip the launch when *gate == 0
int launch_mh(gb_ctx* ctx, int32_t n_chains, int32_t n, const double* logL, const double* log_g, const double* log_u,
              const double* temperature, int32_t literal, int32_t* chain_idx, int32_t* n_accept, const int* gate,
              cudaStream_t st);
// Scratch of the certified chains (device): per row the bound (float), the
// queued mark, the re-evaluation queue and the unsettled steps; per chain the
// queue range of the last pass; per pass and chain the rows queued, the steps
// recorded and the finished CTAs; per pass the rows queued and the flips.
struct CertScratch {
    float* err;
    int32_t* mark;
    int32_t* queue;
    int32_t* steps;
    int32_t* q_lo;
    int32_t* q_hi;
    int* cnt;
    int* scnt;
    int* done;
    int* n_new;
    int* n_flip;
};
// one certification pass over chains built from bounded values (mh.cu); pass
// 0 also computes the bounds from the mixed outputs
int launch_mh_certify(gb_ctx* ctx, const CertScratch& cs, int32_t n_chains, int32_t n, const double* logL,
                      const double* dh, const double* hh, const double* log_g, const double* log_u,
                      const double* temperature, int32_t literal, double eps, const int32_t* chain_idx, int pass,
                      const int* gate, cudaStream_t st);
// after pass `pass`'s rows are re-evaluated: their bounds to 0, and the flips
// of the pass's unsettled steps counted into n_flip[pass] (mh.cu)
int launch_mh_flip(gb_ctx* ctx, const CertScratch& cs, int32_t n_chains, int32_t n, const double* logL,
                   const double* log_g, const double* log_u, const double* temperature, int32_t literal,
                   const int32_t* chain_idx, int pass, cudaStream_t st);
// out[r] = sum of cnt[p][r] over the first n_pass passes (mh.cu)
int launch_sum_rows(gb_ctx* ctx, const int* cnt, int32_t n_chains, int n_pass, int32_t* out, cudaStream_t st);
// Gram matrices, <d|s_i> and multi-signal SNRs of each window's sources (fp64.cu)
int launch_multi_gram(gb_ctx* ctx, const gb_window_t* d_win, int n_win, int n_max, const double* dA,
                      const double* dE, const double* wA, const double* wE, const double* theta, int kmax,
                      double* gram, double* dh, double* rho, cudaStream_t s);
int launch_waveform_fp64(gb_ctx* ctx, const double* theta, int64_t B, int N, double* hA,
                         double* hE, double* hT, int64_t* q, cudaStream_t s);
int launch_loglik_mixed(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE,
                        const double* wA, const double* wE, const double* theta, double* logL,
                        double* dh, double* hh, double* dh_im, const double* dT, const double* wT,
                        cudaStream_t s);
// the persistent likelihood kernel with the phase output and/or the T channel
// (part 0: N >= 512, part 1: N <= 256), compiled in mixed_variants.cu
const void* mixed_kernel_fn_variant(int part, bool im, bool t3);
const void* mixed_kernel_fn_t(int part, bool im);            // mixed_variants_t.cu
const void* grad_mixed_kernel_fn_t(int part);                // mixed_grad_t.cu, the gradient with T
int launch_waveform_mixed(gb_ctx* ctx, const double* theta, int64_t B, int N, double* hA,
                          double* hE, double* hT, int64_t* q, cudaStream_t s);
int launch_grad_fp64(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                     const double* wE, const double* theta, double* logL, double* grad, const double* dT,
                     const double* wT, cudaStream_t s);
int launch_grad_mixed(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                      const double* wE, const double* theta, double* logL, double* grad, const double* dT,
                      const double* wT, cudaStream_t s);

}  // namespace gb
