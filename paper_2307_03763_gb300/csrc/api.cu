// api.cu -- host entry points: argument checks, launch plans, dispatch by precision.
#include <algorithm>
#include <climits>
#include <string>

#include "gb_internal.cuh"

using namespace gb;

namespace {

int check_windows(gb_ctx* ctx, const char* fn, const gb_window_t* win, int32_t n_win, int64_t n_bins,
                  int64_t n_rows, int64_t* total) {
    *total = 0;
    if (n_win < 0) return set_error(ctx, GB_EINVAL, std::string(fn) + ": n_win < 0");
    if (n_win > 0 && !win) return set_error(ctx, GB_EINVAL, std::string(fn) + ": null window array");
    if (n_bins < 0 || n_rows < 0) return set_error(ctx, GB_EINVAL, std::string(fn) + ": negative extent");
    for (int i = 0; i < n_win; ++i) {
        const gb_window_t& w = win[i];
        const std::string at = std::string(fn) + ": window " + std::to_string(i) + ": ";
        if (!valid_size(w.N)) return set_error(ctx, GB_EINVAL, at + "N must be a power of two in [32, 1024]");
        if (w.W < 0 || w.n_cand < 0 || w.data_off < 0 || w.cand_off < 0)
            return set_error(ctx, GB_EINVAL, at + "negative size or offset");
        if (w.data_off + (int64_t)w.W > n_bins) return set_error(ctx, GB_EINVAL, at + "data_off + W > n_bins");
        if (w.cand_off + (int64_t)w.n_cand > n_rows) return set_error(ctx, GB_EINVAL, at + "cand_off + n_cand > n_rows");
        *total += w.n_cand;
    }
    return GB_OK;
}

int sm_count(gb_ctx* ctx) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || n <= 0) n = 152;
    return n;
}

// candidates per tile: at most 32 per warp; fewer when the batch is small so
// that every SM gets work
int tile_size(gb_ctx* ctx, int64_t total, int warps) {
    const int64_t target = (int64_t)sm_count(ctx) * 2;
    int64_t t = (total + target - 1) / target;
    if (t > 32 * warps) t = 32 * warps;
    if (t < warps) t = warps;
    return (int)t;
}

int loglik_impl(gb_ctx_t* ctx, const char* name, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                const double* dE, const double* wA, const double* wE, int64_t n_bins, const double* theta,
                int64_t n_rows, double* logL, double* dh, double* dh_im, double* hh, void* stream,
                const double* dT = nullptr, const double* wT = nullptr) {
    if (!ctx) return GB_EINVAL;
    if (prec != GB_FP64 && prec != GB_MIXED) return set_error(ctx, GB_EINVAL, std::string(name) + ": unknown precision");
    int64_t total = 0;
    int rc = check_windows(ctx, name, win, n_win, n_bins, n_rows, &total);
    if (rc != GB_OK) return rc;
    if (total == 0) return GB_OK;
    if (!dA || !dE || !wA || !wE || !theta || !logL) return set_error(ctx, GB_EINVAL, std::string(name) + ": null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "loglik: cudaSetDevice");
    const Plan* plan = nullptr;
    const int warps = 4;
    // mixed: work items of at most 16 candidates (one warp each; smaller
    // items balance the persistent warps' tails), fewer when the batch would
    // not give every resident warp of the GPU one item
    int item = (int)std::min<int64_t>(16, std::max<int64_t>(1, (total + sm_count(ctx) * 16 - 1) / (sm_count(ctx) * 16)));
    if (ctx->tune_item > 0) item = std::min(ctx->tune_item, 32);
    if (dT) item = std::min(item, 16);   // the T-channel kernel's items hold at most 16 candidates
    int tile = tile_size(ctx, total, warps);
    if (ctx->tune_tile64 > 0) tile = std::min(ctx->tune_tile64, 32 * warps);
    rc = get_plan(ctx, prec, win, n_win, prec == GB_MIXED ? item : tile, &plan);
    if (rc != GB_OK) return rc;
    if (prec == GB_FP64)
        return launch_loglik_fp64(ctx, *plan, dA, dE, wA, wE, theta, logL, dh, hh, dh_im, dT, wT,
                                  (cudaStream_t)stream);
    return launch_loglik_mixed(ctx, *plan, dA, dE, wA, wE, theta, logL, dh, hh, dh_im, dT, wT, (cudaStream_t)stream);
}

}  // namespace

extern "C" {

int gb_loglik(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
              const double* dE, const double* wA, const double* wE, int64_t n_bins, const double* theta,
              int64_t n_rows, double* logL, double* dh, double* hh, void* stream) {
    return loglik_impl(ctx, "gb_loglik", prec, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, dh, nullptr,
                       hh, stream);
}

int gb_loglik_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                  const double* dE, const double* dT, const double* wA, const double* wE, const double* wT,
                  int64_t n_bins, const double* theta, int64_t n_rows, double* logL, double* dh, double* hh,
                  void* stream) {
    if (ctx && (!dT || !wT)) return set_error(ctx, GB_EINVAL, "gb_loglik_aet: dT and wT are required");
    return loglik_impl(ctx, "gb_loglik_aet", prec, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, dh,
                       nullptr, hh, stream, dT, wT);
}

int gb_loglik_phase(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                    const double* dE, const double* wA, const double* wE, int64_t n_bins, const double* theta,
                    int64_t n_rows, double* logL, double* dh, double* dh_im, double* hh, void* stream) {
    if (ctx && !dh_im) return set_error(ctx, GB_EINVAL, "gb_loglik_phase: dh_im is null");
    return loglik_impl(ctx, "gb_loglik_phase", prec, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, dh,
                       dh_im, hh, stream);
}

int gb_loglik_grad_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                       const double* dE, const double* dT, const double* wA, const double* wE, const double* wT,
                       int64_t n_bins, const double* theta, int64_t n_rows, double* logL, double* grad,
                       void* stream);

int gb_loglik_grad(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                   const double* dE, const double* wA, const double* wE, int64_t n_bins, const double* theta,
                   int64_t n_rows, double* logL, double* grad, void* stream) {
    return gb_loglik_grad_aet(ctx, prec, win, n_win, dA, dE, nullptr, wA, wE, nullptr, n_bins, theta, n_rows, logL,
                              grad, stream);
}

int gb_loglik_phase_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                        const double* dE, const double* dT, const double* wA, const double* wE, const double* wT,
                        int64_t n_bins, const double* theta, int64_t n_rows, double* logL, double* dh,
                        double* dh_im, double* hh, void* stream) {
    if (ctx && !dh_im) return set_error(ctx, GB_EINVAL, "gb_loglik_phase_aet: dh_im is null");
    if (ctx && (!dT || !wT)) return set_error(ctx, GB_EINVAL, "gb_loglik_phase_aet: dT and wT are required");
    return loglik_impl(ctx, "gb_loglik_phase_aet", prec, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, dh,
                       dh_im, hh, stream, dT, wT);
}

int gb_loglik_grad_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                       const double* dE, const double* dT, const double* wA, const double* wE, const double* wT,
                       int64_t n_bins, const double* theta, int64_t n_rows, double* logL, double* grad,
                       void* stream) {
    if (!ctx) return GB_EINVAL;
    if ((dT == nullptr) != (wT == nullptr)) return set_error(ctx, GB_EINVAL, "gb_loglik_grad_aet: dT and wT together");
    if (prec != GB_FP64 && prec != GB_MIXED) return set_error(ctx, GB_EINVAL, "gb_loglik_grad: unknown precision");
    int64_t total = 0;
    int rc = check_windows(ctx, "gb_loglik_grad", win, n_win, n_bins, n_rows, &total);
    if (rc != GB_OK) return rc;
    if (total == 0) return GB_OK;
    if (!dA || !dE || !wA || !wE || !theta || !grad) return set_error(ctx, GB_EINVAL, "gb_loglik_grad: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_loglik_grad: cudaSetDevice");
    const Plan* plan = nullptr;
    // distinct plan keys for the gradient kernels; FP64: CTAs of two warps;
    // mixed: warp work items of at most 32 candidates
    int item = (int)std::min<int64_t>(32, std::max<int64_t>(1, (total + sm_count(ctx) * 8 - 1) / (sm_count(ctx) * 8)));
    rc = get_plan(ctx, prec + 16, win, n_win, prec == GB_MIXED ? item : tile_size(ctx, total, 2), &plan);
    if (rc != GB_OK) return rc;
    if (prec == GB_FP64)
        return launch_grad_fp64(ctx, *plan, dA, dE, wA, wE, theta, logL, grad, dT, wT, (cudaStream_t)stream);
    return launch_grad_mixed(ctx, *plan, dA, dE, wA, wE, theta, logL, grad, dT, wT, (cudaStream_t)stream);
}

int gb_autotune(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win, const double* dA,
                const double* dE, const double* wA, const double* wE, int64_t n_bins, const double* theta,
                int64_t n_rows, double* logL, int32_t reps, gb_tuning_t* chosen, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (prec != GB_FP64 && prec != GB_MIXED) return set_error(ctx, GB_EINVAL, "gb_autotune: unknown precision");
    int64_t total = 0;
    int rc = check_windows(ctx, "gb_autotune", win, n_win, n_bins, n_rows, &total);
    if (rc != GB_OK) return rc;
    if (!dA || !dE || !wA || !wE || !theta || !logL) return set_error(ctx, GB_EINVAL, "gb_autotune: null pointer");
    if (reps < 1) reps = 3;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_autotune: cudaSetDevice");
    struct Cfg {
        int item, bpsm, tile;
    };
    std::vector<Cfg> cfgs;
    cfgs.push_back({0, 0, 0});   // built-in heuristics first
    if (prec == GB_MIXED) {
        for (int item : {2, 4, 8, 16, 32})
            for (int bpsm : {0, 1, 2, 3}) cfgs.push_back({item, bpsm, 0});
    } else {
        for (int tile : {16, 32, 64, 128}) cfgs.push_back({0, 0, tile});
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_autotune: events");
    double best = 1e300, first = 0.0;
    Cfg pick = cfgs[0];
    for (size_t i = 0; i < cfgs.size() && rc == GB_OK; ++i) {
        ctx->tune_item = cfgs[i].item;
        ctx->tune_bpsm = cfgs[i].bpsm;
        ctx->tune_tile64 = cfgs[i].tile;
        rc = gb_loglik(ctx, prec, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, nullptr, nullptr, stream);
        if (rc != GB_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && rc == GB_OK; ++r)
            rc = gb_loglik(ctx, prec, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, nullptr, nullptr,
                           stream);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_error(ctx, e, "gb_autotune: timing");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / reps;
        if (i == 0) first = per;
        if (per < best) {
            best = per;
            pick = cfgs[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune_item = pick.item;
    ctx->tune_bpsm = pick.bpsm;
    ctx->tune_tile64 = pick.tile;
    if (rc != GB_OK) return rc;
    if (chosen) {
        chosen->item = pick.item;
        chosen->blocks_per_sm = pick.bpsm;
        chosen->tile = pick.tile;
        chosen->reserved = 0;
        chosen->ms = best;
        chosen->ms_default = first;
    }
    return GB_OK;
}

int gb_waveform_aet(gb_ctx_t* ctx, int prec, const double* theta, int64_t B, int32_t N, double* hA, double* hE,
                    double* hT, int64_t* q, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (prec != GB_FP64 && prec != GB_MIXED) return set_error(ctx, GB_EINVAL, "gb_waveform_aet: unknown precision");
    if (B < 0) return set_error(ctx, GB_EINVAL, "gb_waveform_aet: B < 0");
    if (!valid_size(N)) return set_error(ctx, GB_EINVAL, "gb_waveform_aet: N must be a power of two in [32, 1024]");
    if (B == 0) return GB_OK;
    if (!theta || !hA || !hE || !hT || !q) return set_error(ctx, GB_EINVAL, "gb_waveform_aet: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_waveform_aet: cudaSetDevice");
    if (prec == GB_FP64) return launch_waveform_fp64(ctx, theta, B, N, hA, hE, hT, q, (cudaStream_t)stream);
    return launch_waveform_mixed(ctx, theta, B, N, hA, hE, hT, q, (cudaStream_t)stream);
}

int gb_waveform(gb_ctx_t* ctx, int prec, const double* theta, int64_t B, int32_t N, double* hA, double* hE,
                int64_t* q, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (prec != GB_FP64 && prec != GB_MIXED) return set_error(ctx, GB_EINVAL, "gb_waveform: unknown precision");
    if (B < 0) return set_error(ctx, GB_EINVAL, "gb_waveform: B < 0");
    if (!valid_size(N)) return set_error(ctx, GB_EINVAL, "gb_waveform: N must be a power of two in [32, 1024]");
    if (B == 0) return GB_OK;
    if (!theta || !hA || !hE || !q) return set_error(ctx, GB_EINVAL, "gb_waveform: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_waveform: cudaSetDevice");
    if (prec == GB_FP64) return launch_waveform_fp64(ctx, theta, B, N, hA, hE, nullptr, q, (cudaStream_t)stream);
    return launch_waveform_mixed(ctx, theta, B, N, hA, hE, nullptr, q, (cudaStream_t)stream);
}

int gb_loglik_rows(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win, const double* dA, const double* dE,
                   const double* wA, const double* wE, int64_t n_bins, const double* theta, int64_t n_rows,
                   const int32_t* rows, const int32_t* row_lo, const int32_t* row_hi, double* logL, double* dh,
                   double* hh, void* stream) {
    if (!ctx) return GB_EINVAL;
    int64_t total = 0;
    int rc = check_windows(ctx, "gb_loglik_rows", win, n_win, n_bins, n_rows, &total);
    if (rc != GB_OK) return rc;
    if (total == 0) return GB_OK;
    if (n_rows > (int64_t)INT32_MAX) return set_error(ctx, GB_EINVAL, "gb_loglik_rows: more than 2^31 - 1 rows");
    if (!dA || !dE || !wA || !wE || !theta || !rows || !row_lo || !row_hi || !logL)
        return set_error(ctx, GB_EINVAL, "gb_loglik_rows: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_loglik_rows: cudaSetDevice");
    const Plan* plan = nullptr;
    rc = get_plan(ctx, GB_FP64, win, n_win, tile_size(ctx, total, 4), &plan);
    if (rc != GB_OK) return rc;
    int nc_max = 0;
    for (int i = 0; i < n_win; ++i) nc_max = std::max(nc_max, win[i].n_cand);
    // CTAs per window: enough for every listed row of the largest window to
    // get its own warp, at most about two waves of the GPU in all
    const int ctas = (int)std::max<int64_t>(
        1, std::min<int64_t>((nc_max + 127) / 128, (2 * (int64_t)sm_count(ctx) + n_win - 1) / n_win));
    return launch_loglik_rows64(ctx, plan->d_win, n_win, plan->n_max, ctas, dA, dE, wA, wE, theta, rows, row_lo,
                                row_hi, logL, dh, hh, nullptr, (cudaStream_t)stream);
}

int gb_mh_certified(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win, const double* dA, const double* dE,
                    const double* wA, const double* wE, int64_t n_bins, const double* theta, const double* log_g,
                    const double* log_u, const double* temperature, int32_t literal, double eps, int32_t max_iter,
                    double* logL, double* dh, double* hh, int32_t* chain_idx, int32_t* n_accept, int32_t* n_exact,
                    int32_t* pending, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_win < 0) return set_error(ctx, GB_EINVAL, "gb_mh_certified: n_win < 0");
    if (n_win == 0) return GB_OK;
    if (!win) return set_error(ctx, GB_EINVAL, "gb_mh_certified: null window array");
    const int32_t n = win[0].n_cand;
    for (int i = 0; i < n_win; ++i)
        if (win[i].n_cand != n || win[i].cand_off != (int64_t)i * n)
            return set_error(ctx, GB_EINVAL, "gb_mh_certified: window w must hold rows [w n, (w + 1) n) (one chain "
                                             "of n proposals per window)");
    const int64_t n_rows = (int64_t)n_win * n;
    if (n_rows > (int64_t)INT32_MAX) return set_error(ctx, GB_EINVAL, "gb_mh_certified: more than 2^31 - 1 rows");
    int64_t total = 0;
    int rc = check_windows(ctx, "gb_mh_certified", win, n_win, n_bins, n_rows, &total);
    if (rc != GB_OK) return rc;
    if (n == 0) {
        // empty chains: nothing to certify, so nothing is pending and no row was re-evaluated
        if (!pending) return set_error(ctx, GB_EINVAL, "gb_mh_certified: null pointer");
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e == cudaSuccess) e = cudaMemsetAsync(pending, 0, sizeof(int32_t), (cudaStream_t)stream);
        if (e == cudaSuccess && n_exact) e = cudaMemsetAsync(n_exact, 0, sizeof(int32_t) * (size_t)n_win, (cudaStream_t)stream);
        return e == cudaSuccess ? GB_OK : cuda_error(ctx, e, "gb_mh_certified: outputs");
    }
    if (!(eps > 0.0) || !(eps < 1e-2)) return set_error(ctx, GB_EINVAL, "gb_mh_certified: eps must be in (0, 1e-2)");
    if (max_iter < 1 || max_iter > 64) return set_error(ctx, GB_EINVAL, "gb_mh_certified: max_iter must be in [1, 64]");
    if (literal != 0 && literal != 1) return set_error(ctx, GB_EINVAL, "gb_mh_certified: literal must be 0 or 1");
    if (!dA || !dE || !wA || !wE || !theta || !log_g || !log_u || !temperature || !logL || !dh || !hh ||
        !chain_idx || !n_accept || !pending)
        return set_error(ctx, GB_EINVAL, "gb_mh_certified: null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_certified: cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    // scratch (CertScratch): per row the bound, queue and step entries, then
    // per chain the queue range, then the counters that start at zero each
    // call: per row the mark, per pass and chain the rows, steps and finished
    // CTAs, per pass the rows and flips
    const size_t a = 256;
    auto up = [a](size_t x) { return (x + a - 1) / a * a; };
    const size_t passes = (size_t)max_iter + 1, R = (size_t)n_rows, Wn = (size_t)n_win;
    const size_t off_q = up(sizeof(float) * R);
    const size_t off_s = off_q + up(sizeof(int32_t) * R);
    const size_t off_lo = off_s + up(sizeof(int32_t) * R);
    const size_t off_hi = off_lo + up(sizeof(int32_t) * Wn);
    const size_t off_zero = off_hi + up(sizeof(int32_t) * Wn);
    const size_t zero_bytes = sizeof(int32_t) * (R + 3 * passes * Wn + 2 * passes);
    const size_t bytes = off_zero + up(zero_bytes);
    if (bytes > ctx->cert_bytes) {
        if (ctx->d_cert) cudaFree(ctx->d_cert);
        ctx->d_cert = nullptr;
        ctx->cert_bytes = 0;
        e = cudaMalloc(&ctx->d_cert, bytes);
        if (e != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? set_error(ctx, GB_ENOMEM, "gb_mh_certified: scratch")
                                                  : cuda_error(ctx, e, "gb_mh_certified: scratch");
        ctx->cert_bytes = bytes;
    }
    unsigned char* b = (unsigned char*)ctx->d_cert;
    CertScratch cs;
    cs.err = (float*)b;
    cs.queue = (int32_t*)(b + off_q);
    cs.steps = (int32_t*)(b + off_s);
    cs.q_lo = (int32_t*)(b + off_lo);
    cs.q_hi = (int32_t*)(b + off_hi);
    cs.mark = (int32_t*)(b + off_zero);
    cs.cnt = cs.mark + R;
    cs.scnt = cs.cnt + passes * Wn;
    cs.done = cs.scnt + passes * Wn;
    cs.n_new = cs.done + passes * Wn;
    cs.n_flip = cs.n_new + passes;
    // the FP64 plan of this layout holds the device copy of the windows
    const Plan* plan64 = nullptr;
    rc = get_plan(ctx, GB_FP64, win, n_win, tile_size(ctx, total, 4), &plan64);
    if (rc != GB_OK) return rc;
    const gb_window_t* d_win = plan64->d_win;
    const int n_max = plan64->n_max;
    // every proposal in mixed precision, with <d|h>, <h|h> for the bounds
    rc = loglik_impl(ctx, "gb_mh_certified", GB_MIXED, win, n_win, dA, dE, wA, wE, n_bins, theta, n_rows, logL, dh,
                     nullptr, hh, stream);
    if (rc != GB_OK) return rc;
    e = cudaMemsetAsync(cs.mark, 0, zero_bytes, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_certified: reset");
    const int ctas = (int)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)n + 127) / 128, (2 * (int64_t)sm_count(ctx) + n_win - 1) / n_win));
    // pass 0 on the mixed values; then per iteration: the rows the last pass
    // queued in FP64 (over their mixed values), the flips of its unsettled
    // steps, and only when one flipped the chains and a pass again
    rc = launch_mh(ctx, n_win, n, logL, log_g, log_u, temperature, literal, chain_idx, n_accept, nullptr, s);
    if (rc == GB_OK)
        rc = launch_mh_certify(ctx, cs, n_win, n, logL, dh, hh, log_g, log_u, temperature, literal, eps, chain_idx, 0,
                               nullptr, s);
    for (int it = 1; it <= max_iter && rc == GB_OK; ++it) {
        rc = launch_loglik_rows64(ctx, d_win, n_win, n_max, ctas, dA, dE, wA, wE, theta, cs.queue, cs.q_lo, cs.q_hi,
                                  logL, nullptr, nullptr, cs.n_new + it - 1, s);
        if (rc == GB_OK)
            rc = launch_mh_flip(ctx, cs, n_win, n, logL, log_g, log_u, temperature, literal, chain_idx, it - 1, s);
        if (rc == GB_OK)
            rc = launch_mh(ctx, n_win, n, logL, log_g, log_u, temperature, literal, chain_idx, n_accept,
                           cs.n_flip + it - 1, s);
        if (rc == GB_OK)
            rc = launch_mh_certify(ctx, cs, n_win, n, logL, dh, hh, log_g, log_u, temperature, literal, eps,
                                   chain_idx, it, cs.n_flip + it - 1, s);
    }
    if (rc != GB_OK) return rc;
    int* n_new = cs.n_new;
    int* cnt = cs.cnt;
    e = cudaMemcpyAsync(pending, n_new + max_iter, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && n_exact) {
        // rows re-evaluated per chain: the queues of the passes before the last
        rc = launch_sum_rows(ctx, cnt, n_win, max_iter, n_exact, s);
        if (rc != GB_OK) return rc;
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_certified: outputs");
    return GB_OK;
}

int gb_snr_multi(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win, const double* dA, const double* dE,
                 const double* wA, const double* wE, int64_t n_bins, const double* theta, int64_t n_rows, int32_t kmax,
                 double* gram, double* dh, double* rho, void* stream) {
    if (!ctx) return GB_EINVAL;
    int64_t total = 0;
    int rc = check_windows(ctx, "gb_snr_multi", win, n_win, n_bins, n_rows, &total);
    if (rc != GB_OK) return rc;
    if (kmax < 1 || kmax > 64) return set_error(ctx, GB_EINVAL, "gb_snr_multi: kmax must be in [1, 64]");
    for (int i = 0; i < n_win; ++i)
        if (win[i].n_cand > kmax) return set_error(ctx, GB_EINVAL, "gb_snr_multi: a window holds more than kmax sources");
    if (n_win == 0) return GB_OK;
    if (!wA || !wE || !gram || (total > 0 && !theta)) return set_error(ctx, GB_EINVAL, "gb_snr_multi: null pointer");
    if ((dh || rho) && (!dA || !dE)) return set_error(ctx, GB_EINVAL, "gb_snr_multi: dh and rho need dA and dE");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_snr_multi: cudaSetDevice");
    const Plan* plan = nullptr;
    rc = get_plan(ctx, GB_FP64, win, n_win, tile_size(ctx, std::max<int64_t>(total, 1), 4), &plan);
    if (rc != GB_OK) return rc;
    return launch_multi_gram(ctx, plan->d_win, n_win, plan->n_max, (dh || rho) ? dA : nullptr, dE, wA, wE, theta,
                             kmax, gram, dh, rho, (cudaStream_t)stream);
}

}  // extern "C"
