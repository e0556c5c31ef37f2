// ctx.cu -- context, geometry and twiddle tables, launch plans, error state.
#include <cstdio>
#include <cstring>
#include <algorithm>

#include "gb_internal.cuh"

namespace gb {

int set_error(gb_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_error(gb_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(ctx, e == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA, m);
}

// ---------------------------------------------------------------------------
// geometry tables: rigid equal-arm triangle on the first-order orbit
//   x_i = AU cos a + AU e/2 (cos(2a - b_i) - 3 cos b_i)
//   y_i = AU sin a + AU e/2 (sin(2a - b_i) - 3 sin b_i)
//   z_i = -sqrt3 AU e cos(a - b_i),   e = L / (2 sqrt3 AU), a = 2 pi t / yr
// sampled at t_n = n T/N.
// ---------------------------------------------------------------------------
__global__ void build_tables_kernel(int N, double T, double L, double* tab64, float* tab32) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double ecc = L / (2.0 * sqrt(3.0) * kAU);
    const double t = (double)n * (T / (double)N);
    const double a = 2.0 * kPi * t / kYear;
    double sa, ca;
    sincos(a, &sa, &ca);
    double x[3][3];
    for (int i = 0; i < 3; ++i) {
        const double b = 2.0 * kPi * i / 3.0;
        x[i][0] = kAU * ca + 0.5 * kAU * ecc * (cos(2.0 * a - b) - 3.0 * cos(b));
        x[i][1] = kAU * sa + 0.5 * kAU * ecc * (sin(2.0 * a - b) - 3.0 * sin(b));
        x[i][2] = -sqrt(3.0) * kAU * ecc * cos(a - b);
    }
    double* X64 = tab64;
    double* A64 = tab64 + 9 * N;
    const double centre[3] = {kAU * ca, kAU * sa, 0.0};
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) X64[(i * 3 + c) * N + n] = x[i][c];
    const int em[3] = {0, 1, 2}, rc[3] = {1, 2, 0};
    double arm[3][3];
    for (int a_ = 0; a_ < 3; ++a_) {
        double d[3], nn = 0.0;
        for (int c = 0; c < 3; ++c) {
            d[c] = x[rc[a_]][c] - x[em[a_]][c];
            nn += d[c] * d[c];
        }
        nn = sqrt(nn);
        for (int c = 0; c < 3; ++c) {
            arm[a_][c] = d[c] / nn;
            A64[(a_ * 3 + c) * N + n] = arm[a_][c];
        }
    }
    // float tables, lane-permuted: sample n sits at p = (n mod R)*32 + brev5(n / R)
    const int R = N / 32;
    const int p = (n % R) * 32 + brev5(n / R);
    float rho[2][3];
    for (int i = 0; i < 2; ++i)
        for (int c = 0; c < 3; ++c) rho[i][c] = (float)((x[i][c] - centre[c]) / kC);
    const float chi = (float)ca, shi = (float)sa;
    const float4 g0 = make_float4(rho[0][0], rho[0][1], rho[0][2], rho[1][0]);
    const float4 g1 = make_float4(rho[1][1], rho[1][2], (float)arm[0][0], (float)arm[0][1]);
    const float4 g2 = make_float4((float)arm[0][2], (float)arm[1][0], (float)arm[1][1], (float)arm[1][2]);
    const float4 g3 = make_float4(chi, (float)(ca - (double)chi), shi, (float)(sa - (double)shi));
    float4* G4 = (float4*)tab32;
    G4[p] = g0;
    G4[N + p] = g1;
    G4[2 * N + p] = g2;
    G4[3 * N + p] = g3;
    // the same in natural order (sample n at n), after the lane twiddles
    float4* G4n = (float4*)(tab32 + 18 * N);
    G4n[n] = g0;
    G4n[N + n] = g1;
    G4n[2 * N + n] = g2;
    G4n[3 * N + n] = g3;
    // the same as component pairs of the sample pair (n, n + 32) that lane
    // n mod 32 takes in one step (N >= 64): float4 f of pair step h holds
    // components 2f and 2f + 1 of both samples, (c_2f(n), c_2f(n+32),
    // c_2f+1(n), c_2f+1(n+32)), at f N/2 + 32 h + lane
    const int r = n / 32, l = n % 32;
    // cos a, sin a in Q1.31 for the fixed-point carrier phase: natural order
    // (every N) and, below, in the paired layout
    auto q31i = [](double x) { return (int)fmin(fmax(rint(x * 2147483648.0), -2147483647.0), 2147483647.0); };
    auto q31 = [&](double x) { return __int_as_float(q31i(x)); };
    ((int2*)(tab32 + 54 * N))[n] = make_int2(q31i(ca), q31i(sa));
    if (N >= 64) {
        // components 12..15: cos a, sin a (float), then cos a, sin a in Q1.31
        // (int bits) for the fixed-point carrier phase of the paired slow part
        const float comp[16] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w,
                                g2.x, g2.y, g2.z, g2.w, chi, shi, q31(ca), q31(sa)};
        float* GP = tab32 + 34 * N;
        const int odd = r & 1;
        for (int f = 0; f < 8; ++f) {
            float* e = GP + 4 * ((size_t)f * (N / 2) + 32 * (r / 2) + l);
            e[odd] = comp[2 * f];
            e[2 + odd] = comp[2 * f + 1];
        }
    }
    // lane twiddle exp(-2 pi i r l / N) at entry n = r*32 + l
    float* LT = tab32 + 16 * N;
    double s, co;
    sincospi(2.0 * (double)(r * l) / (double)N, &s, &co);
    LT[2 * n] = (float)co;
    LT[2 * n + 1] = (float)(-s);
    ((float4*)(tab32 + 50 * N))[n] = make_float4((float)co, (float)co, (float)(-s), (float)(-s));
}

__global__ void build_twiddles_kernel(double* tw64, float* tw32) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kTwiddles) return;
    double s, c;
    sincospi((double)k / 512.0, &s, &c);   // exp(-2 pi i k / 1024)
    tw64[2 * k] = c;
    tw64[2 * k + 1] = -s;
    tw32[2 * k] = (float)c;
    tw32[2 * k + 1] = (float)(-s);
}

// Build the geometry tables of every size and the twiddles into memory the
// caller provides (laid out like a context's), asynchronously on `s`.
cudaError_t build_tables_into(double T, double L, double* const tab64[kNumSizes], float* const tab32[kNumSizes],
                              double* tw64, float* tw32, cudaStream_t s) {
    for (int i = 0; i < kNumSizes; ++i) {
        const int N = 32 << i;
        build_tables_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, T, L, tab64[i], tab32[i]);
    }
    build_twiddles_kernel<<<(kTwiddles + 127) / 128, 128, 0, s>>>(tw64, tw32);
    return cudaGetLastError();
}


OrbitTables64 tables64(const gb_ctx* ctx, int N) {
    const double* t = ctx->d_tab64[size_index(N)];
    return OrbitTables64{t, t + 9 * N};
}

OrbitTables32 tables32(const gb_ctx* ctx, int N) {
    const float* t = ctx->d_tab32[size_index(N)];
    return OrbitTables32{(const float4*)t, (const float2*)(t + 16 * N), (const float4*)(t + 18 * N),
                         (const float4*)(t + 34 * N), (const float4*)(t + 50 * N), (const int2*)(t + 54 * N)};
}

TabSet64 tabset64(const gb_ctx* ctx) {
    TabSet64 s;
    for (int i = 0; i < kNumSizes; ++i) s.t[i] = tables64(ctx, 32 << i);
    return s;
}

TabSet32 tabset32(const gb_ctx* ctx) {
    TabSet32 s;
    for (int i = 0; i < kNumSizes; ++i) s.t[i] = tables32(ctx, 32 << i);
    return s;
}

// ---------------------------------------------------------------------------
// launch plans
// ---------------------------------------------------------------------------
static uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

static void free_plan(Plan& p) {
    if (p.d_win) cudaFree(p.d_win);
    if (p.d_tiles) cudaFree(p.d_tiles);
    if (p.d_meta) cudaFree(p.d_meta);
    if (p.d_prep) cudaFree(p.d_prep);
    if (p.d_head) cudaFree(p.d_head);
    p.d_win = nullptr;
    p.d_tiles = nullptr;
    p.d_meta = nullptr;
    p.d_prep = nullptr;
    p.d_head = nullptr;
}

// scratch of the mixed-precision kernels: per-window meta (with the offsets
// of each window's float copy), the float copies, the work-queue head
static cudaError_t alloc_mixed_scratch(Plan& p, const gb_window_t* win, int n_win) {
    std::vector<WinMeta> meta(n_win > 0 ? n_win : 1);
    long long off = 0;
    for (int w = 0; w < n_win; ++w) {
        meta[w].dd = 0.0;
        meta[w].sig = 1.0;
        meta[w].prep_off = off;
        meta[w].use_t = 0;
        meta[w].pad = 0;
        off += win[w].W;
    }
    p.n_prep = off;
    cudaError_t e = cudaMalloc(&p.d_meta, sizeof(WinMeta) * meta.size());
    if (e == cudaSuccess) e = cudaMemcpy(p.d_meta, meta.data(), sizeof(WinMeta) * meta.size(), cudaMemcpyHostToDevice);
    // float window copies: A and E, then T (filled only when the T channel is given)
    if (e == cudaSuccess) e = cudaMalloc(&p.d_prep, 2 * sizeof(Win32) * (size_t)(off > 0 ? off : 1));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_head, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p.d_head, 0, 2 * sizeof(int));
    return e;
}

int get_plan(gb_ctx* ctx, int prec, const gb_window_t* win, int32_t n_win, int tile_cands,
             const Plan** out) {
    uint64_t key = 1469598103934665603ull;
    key = fnv1a(&prec, sizeof prec, key);
    key = fnv1a(&tile_cands, sizeof tile_cands, key);
    key = fnv1a(&n_win, sizeof n_win, key);
    key = fnv1a(win, sizeof(gb_window_t) * (size_t)n_win, key);
    ctx->clock++;
    for (auto& p : ctx->plans)
        if (p.key == key && p.prec == prec && p.n_win == n_win && p.tile_cands == tile_cands &&
            (n_win == 0 || std::memcmp(p.win.data(), win, sizeof(gb_window_t) * (size_t)n_win) == 0)) {
            p.last_use = ctx->clock;
            *out = &p;
            return GB_OK;
        }
    // build the tile list: every window split into chunks of tile_cands,
    // most expensive tiles first so that the tail of the grid is short
    std::vector<Tile> tiles;
    std::vector<double> cost;
    int n_max = 0, w_max = 0;
    for (int w = 0; w < n_win; ++w) {
        const gb_window_t& g = win[w];
        n_max = std::max(n_max, g.N);
        w_max = std::max(w_max, g.W);
        for (int64_t c = 0; c < g.n_cand; c += tile_cands) {
            Tile t;
            t.win = w;
            t.pad = 0;
            t.c_begin = g.cand_off + c;
            t.c_end = g.cand_off + std::min<int64_t>(g.n_cand, c + tile_cands);
            tiles.push_back(t);
            cost.push_back((double)(t.c_end - t.c_begin) * g.N * (log2_size(g.N) + 12));
        }
    }
    std::vector<int> order(tiles.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // mixed plans: items of windows with N >= 512 first (their own kernel)
    int n_large = 0;
    if ((prec & 15) == GB_MIXED) {
        std::stable_partition(order.begin(), order.end(), [&](int a) { return win[tiles[a].win].N >= 512; });
        for (const Tile& t : tiles) n_large += win[t.win].N >= 512 ? 1 : 0;
    }
    std::vector<Tile> sorted(tiles.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = tiles[order[i]];
    if ((prec == GB_MIXED || prec == GB_MIXED + 16) && tile_cands >= 4) {
        // The persistent warps take the items in this order, so the last ones
        // set the tail.  With R warps resident (likelihood: 16 per SM for
        // N <= 256, 8 for N >= 512; gradient: 8 and 4), the last R/2 items of
        // each range are split into halves
        // and the last R/4 of those halves into halves again: the last round
        // is shared out in smaller items, while the extra per-item set-ups
        // stay few (a list-scheduling model of the queue with the measured
        // set-up cost puts this near the best split; splitting the last 2R
        // items costs more in set-ups than it saves).
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms <= 0)
            sms = 152;
        auto split_last = [](std::vector<Tile>& v, size_t k) {
            k = std::min(k, v.size());
            std::vector<Tile> out(v.begin(), v.end() - k);
            for (size_t i = v.size() - k; i < v.size(); ++i) {
                const Tile t = v[i];
                const int64_t len = t.c_end - t.c_begin;
                if (len >= 2) {
                    Tile a = t, b = t;
                    a.c_end = b.c_begin = t.c_begin + len / 2;
                    out.push_back(a);
                    out.push_back(b);
                } else {
                    out.push_back(t);
                }
            }
            v.swap(out);
        };
        std::vector<Tile> large(sorted.begin(), sorted.begin() + n_large), small(sorted.begin() + n_large, sorted.end());
        const size_t per_sm = prec == GB_MIXED ? 16 : 8;
        const size_t r_large = (size_t)sms * per_sm / 2, r_small = (size_t)sms * per_sm;
        split_last(large, r_large / 2);
        split_last(large, r_large / 4);
        split_last(small, r_small / 2);
        split_last(small, r_small / 4);
        n_large = (int)large.size();
        sorted = large;
        sorted.insert(sorted.end(), small.begin(), small.end());
    }

    Plan p;
    p.key = key;
    p.prec = prec;
    p.n_win = n_win;
    p.n_tiles = (int)sorted.size();
    p.n_max = n_max;
    p.w_max = w_max;
    p.n_large = n_large;
    p.tile_cands = tile_cands;
    p.win.assign(win, win + n_win);
    p.last_use = ctx->clock;
    cudaError_t e;
    if (n_win > 0) {
        e = cudaMalloc(&p.d_win, sizeof(gb_window_t) * n_win);
        if (e != cudaSuccess) return cuda_error(ctx, e, "plan: cudaMalloc windows");
        e = cudaMemcpy(p.d_win, win, sizeof(gb_window_t) * n_win, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_plan(p);
            return cuda_error(ctx, e, "plan: copy windows");
        }
    }
    if (!sorted.empty()) {
        e = cudaMalloc(&p.d_tiles, sizeof(Tile) * sorted.size());
        if (e != cudaSuccess) {
            free_plan(p);
            return cuda_error(ctx, e, "plan: cudaMalloc tiles");
        }
        e = cudaMemcpy(p.d_tiles, sorted.data(), sizeof(Tile) * sorted.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_plan(p);
            return cuda_error(ctx, e, "plan: copy tiles");
        }
    }
    if ((prec & 15) == GB_MIXED) {
        e = alloc_mixed_scratch(p, win, n_win);
        if (e != cudaSuccess) {
            free_plan(p);
            return cuda_error(ctx, e, "plan: mixed-precision scratch");
        }
    }
    const size_t kMaxPlans = 16;
    if (ctx->plans.size() >= kMaxPlans) {
        auto lru = std::min_element(ctx->plans.begin(), ctx->plans.end(),
                                    [](const Plan& a, const Plan& b) { return a.last_use < b.last_use; });
        // a kernel still running may read the evicted plan: wait for the device
        cudaDeviceSynchronize();
        free_plan(*lru);
        ctx->plans.erase(lru);
    }
    ctx->plans.push_back(p);
    *out = &ctx->plans.back();
    return GB_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

int gb_ctx_create(gb_ctx_t** out, const gb_obs_t* obs, int device) {
    if (!out) return GB_EINVAL;
    *out = nullptr;
    if (!obs || !(obs->T_obs > 0.0) || !(obs->arm_L > 0.0) || obs->orbit_model != 0) return GB_EINVAL;
    gb_ctx* ctx = new gb_ctx();
    ctx->device = device;
    ctx->obs = *obs;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return GB_ECUDA;
    }
    e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_tw64, sizeof(double) * 2 * kTwiddles);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_tw32, sizeof(float) * 2 * kTwiddles);
    for (int i = 0; i < kNumSizes && e == cudaSuccess; ++i) {
        const int N = 32 << i;
        e = cudaMalloc(&ctx->d_tab64[i], sizeof(double) * kTab64PerN * N);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_tab32[i], sizeof(float) * kTab32PerN * N);
        if (e == cudaSuccess) {
            build_tables_kernel<<<(N + 127) / 128, 128>>>(N, obs->T_obs, obs->arm_L, ctx->d_tab64[i],
                                                         ctx->d_tab32[i]);
            ++ctx->launches;
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        build_twiddles_kernel<<<(kTwiddles + 127) / 128, 128>>>(ctx->d_tw64, ctx->d_tw32);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    // MH scratch for 262,144 proposals in 1,024 chunks, so that common chain
    // sizes never allocate inside a call (or a stream capture)
    if (e == cudaSuccess) {
        const size_t b = mh_scratch_bytes(1024, 262144);
        e = cudaMalloc(&ctx->d_mh, b);
        if (e == cudaSuccess) ctx->mh_bytes = b;
    }
    if (e != cudaSuccess) {
        gb_ctx_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA;
    }
    *out = ctx;
    return GB_OK;
}

int gb_ctx_destroy(gb_ctx_t* ctx) {
    if (!ctx) return GB_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& p : ctx->plans) free_plan(p);
    for (int i = 0; i < kNumSizes; ++i) {
        if (ctx->d_tab64[i]) cudaFree(ctx->d_tab64[i]);
        if (ctx->d_tab32[i]) cudaFree(ctx->d_tab32[i]);
    }
    if (ctx->d_tw64) cudaFree(ctx->d_tw64);
    if (ctx->d_tw32) cudaFree(ctx->d_tw32);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_mh) cudaFree(ctx->d_mh);
    if (ctx->d_cert) cudaFree(ctx->d_cert);
    delete ctx;
    return GB_OK;
}

const char* gb_last_error(const gb_ctx_t* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t gb_launch_count(const gb_ctx_t* ctx) { return ctx ? ctx->launches : 0; }

int gb_ctx_check(gb_ctx_t* ctx) {
    if (!ctx) return GB_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_ctx_check");
    if (status & kStatusBudget)
        return set_error(ctx, GB_ETIMEOUT,
                         std::string("a persistent kernel stopped at the context's time budget; rows of the items "
                                     "it did not take were not written") +
                             (status & kStatusNonFinite ? "; a kernel also met a non-finite parameter" : ""));
    if (status != 0) return set_error(ctx, GB_EINVAL, "a kernel met a non-finite parameter");
    return GB_OK;
}

int gb_ctx_set_time_budget(gb_ctx_t* ctx, double seconds) {
    if (!ctx) return GB_EINVAL;
    if (!(seconds >= 0.0) || seconds > 1.0e9)
        return set_error(ctx, GB_EINVAL, "gb_ctx_set_time_budget: seconds must be in [0, 1e9]");
    ctx->budget_ns = (unsigned long long)(seconds * 1.0e9);
    if (seconds > 0.0 && ctx->budget_ns == 0ULL) ctx->budget_ns = 1ULL;
    return GB_OK;
}

int gb_ctx_set_kernel_events(gb_ctx_t* ctx, void* start, void* end) {
    if (!ctx) return GB_EINVAL;
    if ((start == nullptr) != (end == nullptr))
        return set_error(ctx, GB_EINVAL, "gb_ctx_set_kernel_events: give both events or neither");
    ctx->kev_start = (cudaEvent_t)start;
    ctx->kev_end = (cudaEvent_t)end;
    return GB_OK;
}

}  // extern "C"
