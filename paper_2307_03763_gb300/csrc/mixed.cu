// mixed.cu -- the mixed-precision likelihood (A and E), the waveform, and
// their launchers; the shared device code is in mixed_common.cuh, the
// likelihood's variants with the phase output or the T channel in
// mixed_variants.cu, the gradient in mixed_grad.cu.
#include "mixed_common.cuh"

namespace gb {
namespace {

__global__ void __launch_bounds__(kWarpsMx * 32) waveform_mixed_kernel(
    OrbitTables32 tab, const float2* __restrict__ tw1024, double T, double fstar, int N,
    const double* __restrict__ theta, int64_t B, int group, double2* __restrict__ hA, double2* __restrict__ hE,
    double2* __restrict__ hT, int64_t* __restrict__ q_out, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = hT ? 3 : 2;
    CandMix* cands = (CandMix*)smem_raw + warp * 32;
    float2* bufA = (float2*)((CandMix*)smem_raw + kWarpsMx * 32) + (size_t)warp * nch * N;
    float2* bufE = bufA + N;
    float2* bufT = hT ? bufE + N : nullptr;
    const LaneTw ltw = lane_twiddles(lane);
    const int64_t c_lo = ((int64_t)blockIdx.x * kWarpsMx + warp) * group;
    const int64_t c_hi = min(B, c_lo + group);
    if (c_lo >= c_hi) return;
    if (c_lo + lane < c_hi) setup_mixed(theta + 8 * (c_lo + lane), T, 1.0 / fstar, cands[lane]);
    __syncwarp();
    const int R = N / 32;
    const double scale = T / (2.0 * (double)N);
    for (int64_t b = c_lo; b < c_hi; ++b) {
        const CandMix& c = cands[b - c_lo];
        double2* outA = hA + b * N;
        double2* outE = hE + b * N;
        if (c.bad) {
            for (int m = lane; m < N; m += 32) {
                outA[m] = outE[m] = make_double2(nan(""), nan(""));
                if (hT) hT[b * N + m] = make_double2(nan(""), nan(""));
            }
            if (lane == 0) {
                q_out[b] = 0;
                atomicOr(status, kStatusNonFinite);
            }
            continue;
        }
        slow_part_dispatch<false, true>(c, tab, N, bufA, bufE, lane, bufT);
        __syncwarp();
        const double s = scale * c.A;
        for (int ch = 0; ch < nch; ++ch) {
            float2 x[32];
            const float2* buf = ch == 0 ? bufA : ch == 1 ? bufE : bufT;
            double2* out = ch == 0 ? outA : ch == 1 ? outE : hT + b * N;
            switch (R) {
                case 1: channel_fft<1>(buf, tab, tw1024, ltw, lane, *(float2(*)[1])x); break;
                case 2: channel_fft<2>(buf, tab, tw1024, ltw, lane, *(float2(*)[2])x); break;
                case 4: channel_fft<4>(buf, tab, tw1024, ltw, lane, *(float2(*)[4])x); break;
                case 8: channel_fft<8>(buf, tab, tw1024, ltw, lane, *(float2(*)[8])x); break;
                case 16: channel_fft<16>(buf, tab, tw1024, ltw, lane, *(float2(*)[16])x); break;
                default: channel_fft<32>(buf, tab, tw1024, ltw, lane, *(float2(*)[32])x); break;
            }
            for (int k1 = 0; k1 < R; ++k1) {
                const int k = lane + 32 * k1;
                const int m = (k + N / 2) & (N - 1);   // entry m stands for bin q - N/2 + m
                out[m] = make_double2(s * x[k1].x, s * x[k1].y);
            }
        }
        if (lane == 0) q_out[b] = c.q;
        __syncwarp();
    }
}

// Part 0 drains the N >= 512 queue, part 1 the N <= 256 queue; the variants
// with the phase output or the T channel are compiled in mixed_variants.cu.
const void* mixed_kernel_fn(int part, bool im, bool t3) {
    if (im || t3) return mixed_kernel_fn_variant(part, im, t3);
    return part == 0 ? (const void*)loglik_mixed_kernel<32, false, false> : (const void*)loglik_mixed_kernel<8, false, false>;
}

}  // namespace

int launch_loglik_mixed(gb_ctx* ctx, const Plan& plan, const double* dA, const double* dE, const double* wA,
                        const double* wE, const double* theta, double* logL, double* dh, double* hh,
                        double* dh_im, const double* dT, const double* wT, cudaStream_t s) {
    if (plan.n_tiles == 0) return GB_OK;
    const bool t3 = dT != nullptr;
    if (t3 && plan.tile_cands > kCapT) return set_error(ctx, GB_EINVAL, "loglik_mixed: T-channel items hold at most 16");
    prep_mixed_kernel<<<plan.n_win, 256, 0, s>>>(plan.d_win, plan.d_meta, plan.d_prep, (const double2*)dA,
                                                 (const double2*)dE, wA, wE, (const double2*)dT, wT, plan.n_prep,
                                                 ctx->obs.T_obs, transfer_frequency(ctx), plan.d_head);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "prep_mixed launch");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    // the caller's events, if set, bracket the likelihood kernels (once)
    const cudaEvent_t ev_start = ctx->kev_start, ev_end = ctx->kev_end;
    ctx->kev_start = ctx->kev_end = nullptr;
    if (ev_start) {
        e = cudaEventRecord(ev_start, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "loglik_mixed: kernel start event");
    }
    // two persistent launches drain the two queues: N >= 512 items, then N <= 256
    const int n_small = plan.n_tiles - plan.n_large;
    for (int part = 0; part < 2; ++part) {
        const int n_items = part == 0 ? plan.n_large : n_small;
        if (n_items == 0) continue;
        const int nmax = part == 0 ? 1024 : (plan.n_max < 256 ? plan.n_max : 256);
        const size_t epi_bytes = dh_im ? sizeof(Epi<true>) : sizeof(Epi<false>);
        const size_t cap = t3 ? kCapT : 32;
        const size_t smem = (sizeof(CandMix) + epi_bytes) * kWarpsMx * cap + sizeof(float2) * kWarpsMx * 2 * (size_t)nmax +
                            (t3 ? sizeof(float2) * kWarpsMx * (size_t)nmax : 0);
        const void* kfn = mixed_kernel_fn(part, dh_im != nullptr, t3);
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(ctx, e, "loglik_mixed: smem attribute");
        int bpsm = resident_blocks(kfn, kWarpsMx * 32, smem);
        if (ctx->tune_bpsm > 0 && ctx->tune_bpsm < bpsm) bpsm = ctx->tune_bpsm;
        int grid = sms * bpsm;
        const int need = (n_items + kWarpsMx - 1) / kWarpsMx;
        if (grid > need) grid = need;
        const Tile* items = plan.d_tiles + (part == 0 ? 0 : plan.n_large);
        int* head = plan.d_head + (part == 0 ? 1 : 0);
        e = launch_mixed_part(kfn, grid, smem, s, plan.d_win, plan.d_meta, plan.d_prep, items, n_items, head,
                              tabset32(ctx), (const float2*)ctx->d_tw32, ctx->obs.T_obs, transfer_frequency(ctx),
                              theta, logL, dh, hh, dh_im, ctx->d_status, nmax, ctx->budget_ns, plan.n_prep);
        ++ctx->launches;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(ctx, e, "loglik_mixed launch");
    }
    if (ev_end) {
        e = cudaEventRecord(ev_end, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "loglik_mixed: kernel end event");
    }
    return GB_OK;
}

int launch_waveform_mixed(gb_ctx* ctx, const double* theta, int64_t B, int N, double* hA, double* hE,
                          double* hT, int64_t* q, cudaStream_t s) {
    if (B == 0) return GB_OK;
    const size_t smem = sizeof(CandMix) * kWarpsMx * 32 + sizeof(float2) * kWarpsMx * (hT ? 3 : 2) * (size_t)N;
    cudaError_t e = cudaFuncSetAttribute(waveform_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform_mixed: smem attribute");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int64_t group = (B + (int64_t)sms * kWarpsMx * 2 - 1) / ((int64_t)sms * kWarpsMx * 2);
    group = group < 1 ? 1 : group > 32 ? 32 : group;
    const int64_t blocks = (B + group * kWarpsMx - 1) / (group * kWarpsMx);
    waveform_mixed_kernel<<<(unsigned)blocks, kWarpsMx * 32, smem, s>>>(
        tables32(ctx, N), (const float2*)ctx->d_tw32, ctx->obs.T_obs, transfer_frequency(ctx), N, theta, B,
        (int)group, (double2*)hA, (double2*)hE, (double2*)hT, q, ctx->d_status);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "waveform_mixed launch");
    return GB_OK;
}

}  // namespace gb

// ---------------------------------------------------------------------------
// Allocation-free variant of the mixed-precision likelihood.
//
// Everything the kernels above need beyond the caller's inputs and outputs --
// geometry tables and twiddles, the window descriptors and work items, the
// per-window values and float copies, the work-queue heads -- lives in one
// file-scope device array, so a call allocates no memory at all.
// ---------------------------------------------------------------------------
#include <cuda.h>

#include <cstring>
#include <mutex>

namespace gb {
namespace {

constexpr int kNaMaxWindows = 4096;
constexpr long long kNaMaxBins = 262144;
constexpr int kNaMaxItems = 65536;
constexpr size_t kNaAlign = 256;
constexpr size_t na_round(size_t x) { return (x + kNaAlign - 1) / kNaAlign * kNaAlign; }
constexpr size_t kNaSamples = 32 + 64 + 128 + 256 + 512 + 1024;
constexpr size_t kNaOffTab64 = 0;
constexpr size_t kNaOffTab32 = na_round(kNaOffTab64 + sizeof(double) * kTab64PerN * kNaSamples);
constexpr size_t kNaOffTw64 = na_round(kNaOffTab32 + sizeof(float) * kTab32PerN * kNaSamples);
constexpr size_t kNaOffTw32 = na_round(kNaOffTw64 + sizeof(double) * 2 * kTwiddles);
constexpr size_t kNaOffWin = na_round(kNaOffTw32 + sizeof(float) * 2 * kTwiddles);
constexpr size_t kNaOffItems = na_round(kNaOffWin + sizeof(gb_window_t) * kNaMaxWindows);
constexpr size_t kNaOffMeta = na_round(kNaOffItems + sizeof(Tile) * kNaMaxItems);
constexpr size_t kNaOffPrep = na_round(kNaOffMeta + sizeof(WinMeta) * kNaMaxWindows);
constexpr size_t kNaOffHead = na_round(kNaOffPrep + sizeof(Win32) * kNaMaxBins);
constexpr size_t kNaBytes = na_round(kNaOffHead + 4 * sizeof(int));   // two queue heads, status

// 8.7 MB per device, kept until the process exits
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// What the tables in a device's array were built for: the array's address,
// the CUDA context it lives in and the observation.  A new context (after a
// device reset, say) reloads the module, so the tables are built again.
struct NaDevice {
    bool built = false;
    unsigned char* base = nullptr;
    unsigned long long ctx_id = 0;
    double T = 0.0, L = 0.0;
};
constexpr int kNaMaxDevices = 64;
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mutex;
Tile g_na_items[kNaMaxItems];          // host staging of the work items
WinMeta g_na_meta[kNaMaxWindows];

int na_fail(char* err, int err_len, int code, const char* msg) {
    if (err && err_len > 0) {
        std::strncpy(err, msg, (size_t)err_len - 1);
        err[err_len - 1] = '\0';
    }
    return code;
}

// Unique id of the current CUDA context (cuCtxGetId through the runtime's
// driver entry points, so no link against the driver library); 0 if the
// driver does not provide it.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrent)f1;
            get_id = (GetId)f2;
        }
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int gb_loglik_mixed_noalloc(const gb_obs_t* obs, const gb_window_t* win, int32_t n_win,
                                       const double* dA, const double* dE, const double* wA, const double* wE,
                                       int64_t n_bins, const double* theta, int64_t n_rows, double* logL,
                                       double* dh, double* hh, int32_t* status, void* stream, char* err,
                                       int32_t err_len) {
    if (err && err_len > 0) err[0] = '\0';
    if (!obs || !(obs->T_obs > 0.0) || !(obs->arm_L > 0.0) || obs->orbit_model != 0)
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: bad observation");
    if (n_win < 0 || n_bins < 0 || n_rows < 0 || (n_win > 0 && !win))
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: bad sizes");
    if (n_win > kNaMaxWindows)
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: more than 4096 windows");
    long long total = 0, bins = 0, items = 0;
    int n_max = 0;
    for (int i = 0; i < n_win; ++i) {
        const gb_window_t& w = win[i];
        if (!valid_size(w.N) || w.W < 0 || w.n_cand < 0 || w.data_off < 0 || w.cand_off < 0 ||
            w.data_off + (int64_t)w.W > n_bins || w.cand_off + (int64_t)w.n_cand > n_rows)
            return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: invalid window descriptor");
        total += w.n_cand;
        bins += w.W;
        n_max = w.N > n_max ? w.N : n_max;
    }
    if (bins > kNaMaxBins)
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: more than 262144 window bins in total");
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    // the uploads below read host staging that the next call overwrites, so a
    // captured copy of this call would replay another call's work items
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return na_fail(err, err_len, GB_ECUDA, "gb_loglik_mixed_noalloc: stream query failed");
    if (cap != cudaStreamCaptureStatusNone)
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: the stream is capturing a graph; "
                                                "this entry point cannot be captured");
    if (total == 0) {
        if (status && cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess)
            return na_fail(err, err_len, GB_ECUDA, "gb_loglik_mixed_noalloc: status reset failed");
        return GB_OK;
    }
    if (!dA || !dE || !wA || !wE || !theta || !logL)
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: null pointer");
    int dev = 0, sms = 152;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return na_fail(err, err_len, GB_ECUDA, "gb_loglik_mixed_noalloc: no current device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per = (int)std::min<long long>(32, std::max<long long>(1, (total + sms * 16 - 1) / (sms * 16)));
    for (int i = 0; i < n_win; ++i) items += (win[i].n_cand + per - 1) / per;
    if (items > kNaMaxItems)
        return na_fail(err, err_len, GB_EINVAL, "gb_loglik_mixed_noalloc: more than 65536 work items "
                                                "(about 2 million candidates)");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    // the array's device address, taken on every call (this allocates nothing)
    unsigned char* b = nullptr;
    e = cudaGetSymbolAddress((void**)&b, g_noalloc_scratch);
    if (e != cudaSuccess || !b)
        return na_fail(err, err_len, GB_ECUDA, "gb_loglik_mixed_noalloc: cudaGetSymbolAddress failed");
    const unsigned long long ctx_id = current_context_id();
    NaDevice& d = g_na_dev[dev];
    double* t64[kNumSizes];
    float* t32[kNumSizes];
    TabSet32 tabs;
    size_t o64 = kNaOffTab64, o32 = kNaOffTab32;
    for (int i = 0; i < kNumSizes; ++i) {
        const int N = 32 << i;
        t64[i] = (double*)(b + o64);
        t32[i] = (float*)(b + o32);
        tabs.t[i] = OrbitTables32{(const float4*)t32[i], (const float2*)(t32[i] + 16 * N),
                                  (const float4*)(t32[i] + 18 * N), (const float4*)(t32[i] + 34 * N),
                                  (const float4*)(t32[i] + 50 * N), (const int2*)(t32[i] + 54 * N)};
        o64 += sizeof(double) * kTab64PerN * N;
        o32 += sizeof(float) * kTab32PerN * N;
    }
    double* tw64 = (double*)(b + kNaOffTw64);
    float* tw32 = (float*)(b + kNaOffTw32);
    if (!d.built || d.base != b || d.ctx_id != ctx_id || d.T != obs->T_obs || d.L != obs->arm_L) {
        d.built = false;
        e = build_tables_into(obs->T_obs, obs->arm_L, t64, t32, tw64, tw32, s);
        if (e != cudaSuccess) return na_fail(err, err_len, GB_ECUDA, "gb_loglik_mixed_noalloc: table build failed");
        d.built = true;
        d.base = b;
        d.ctx_id = ctx_id;
        d.T = obs->T_obs;
        d.L = obs->arm_L;
    }
    // work items (windows with N >= 512 first) and window offsets, staged on the host
    int n_large = 0, k = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < n_win; ++i) {
            if ((win[i].N >= 512) != (pass == 0)) continue;
            for (int64_t c = 0; c < win[i].n_cand; c += per) {
                Tile t;
                t.win = i;
                t.pad = 0;
                t.c_begin = win[i].cand_off + c;
                t.c_end = win[i].cand_off + std::min<int64_t>(win[i].n_cand, c + per);
                g_na_items[k++] = t;
                if (pass == 0) ++n_large;
            }
        }
    long long off = 0;
    for (int i = 0; i < n_win; ++i) {
        g_na_meta[i].dd = 0.0;
        g_na_meta[i].sig = 1.0;
        g_na_meta[i].prep_off = off;
        g_na_meta[i].use_t = 0;
        g_na_meta[i].pad = 0;
        off += win[i].W;
    }
    gb_window_t* d_win = (gb_window_t*)(b + kNaOffWin);
    Tile* d_items = (Tile*)(b + kNaOffItems);
    WinMeta* d_meta = (WinMeta*)(b + kNaOffMeta);
    Win32* d_prep = (Win32*)(b + kNaOffPrep);
    int* d_head = (int*)(b + kNaOffHead);
    int* d_status = d_head + 2;
    e = cudaMemcpyAsync(d_win, win, sizeof(gb_window_t) * (size_t)n_win, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, g_na_items, sizeof(Tile) * (size_t)k, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_meta, g_na_meta, sizeof(WinMeta) * (size_t)n_win, cudaMemcpyHostToDevice, s);
    // this call's status starts clear (the queue heads are reset by the preparation kernel)
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
    if (e != cudaSuccess) return na_fail(err, err_len, GB_ECUDA, "gb_loglik_mixed_noalloc: upload failed");
    const double fstar = kC / (2.0 * kPi * obs->arm_L);
    prep_mixed_kernel<<<n_win, 256, 0, s>>>(d_win, d_meta, d_prep, (const double2*)dA, (const double2*)dE, wA, wE,
                                            nullptr, nullptr, 0LL, obs->T_obs, fstar, d_head);
    e = cudaGetLastError();
    for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
        const int n_items = part == 0 ? n_large : k - n_large;
        if (n_items == 0) continue;
        const int nmax = part == 0 ? 1024 : (n_max < 256 ? n_max : 256);
        const size_t smem =
            (sizeof(CandMix) + sizeof(Epi<false>)) * kWarpsMx * 32 + sizeof(float2) * kWarpsMx * 2 * (size_t)nmax;
        const void* kfn = mixed_kernel_fn(part, false, false);
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) break;
        int grid = sms * resident_blocks(kfn, kWarpsMx * 32, smem);
        const int need = (n_items + kWarpsMx - 1) / kWarpsMx;
        if (grid > need) grid = need;
        const Tile* it = d_items + (part == 0 ? 0 : n_large);
        int* head = d_head + (part == 0 ? 1 : 0);
        e = launch_mixed_part(kfn, grid, smem, s, d_win, d_meta, d_prep, it, n_items, head, tabs, (const float2*)tw32,
                              obs->T_obs, fstar, theta, logL, dh, hh, nullptr, d_status, nmax, 0ULL, 0LL);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, d_status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return na_fail(err, err_len, GB_ECUDA, cudaGetErrorString(e));
    return GB_OK;
}
