// mh.cu -- independence Metropolis-Hastings chains from precomputed values
// (Sec. III.G, Alg. 4, Eq. 13).
//
// The proposal does not depend on the chain state, so all log-likelihoods are
// computed first and each chain is a scan over its proposals.  The scan is
// made parallel across chunks of proposals without changing a single decision.
//
// Acceptance of proposal j depends on the current state c only through its
// weight w_c (w = logL/T - log g, or logL - log g for the literal form), and it
// is monotone in w_c: the IEEE difference fl(w_j - w_c) does not increase when
// w_c does, and neither does its quotient by a positive T.  So the set of
// current weights that accept j is {w_c <= tau_j} for one double tau_j (or
// empty), found exactly from a first guess w_j - log u_j and a few evaluations
// of the double test (a bisection over the ordered doubles when the guess is
// more than three steps away).  Mapping doubles to order-preserving integers
// ("keys") turns the scan into integer comparisons:
//     state key s (key of w_c);  proposal j is accepted iff s <= K_j.
//
// Launches:
//   summary  one CTA per (chain, chunk).  The first accepted proposal of the
//            chunk, for an unknown incoming state, is one of the prefix
//            records of K (positions where K exceeds every earlier K); for
//            each record the CTA follows the chain from there to the chunk's
//            end and stores the exit state and acceptance count.  K and the
//            state keys go to global memory for the write launch.
//   combine  a sequential pass over the chunk summaries (the first record
//            with s <= K_r gives the exit) that yields the incoming state of
//            every chunk and the acceptance count: inside each write CTA for
//            chains of at most 32 chunks, else one CTA per chain beforehand.
//   write    one CTA per (chain, chunk): from its incoming state, follows the
//            chain through the chunk and writes the state after every step.
// A chunk with more than 32 records, and every chunk of a literal-form chain
// whose T is not a positive finite number (where the test is not monotone),
// is scanned with the double test itself in the combine and write launches.
// Every decision equals the one a one-at-a-time double-precision scan takes.
#include <cfloat>
#include <climits>
#include <cmath>

#include <math_constants.h>

#include "gb_internal.cuh"

#ifndef GB_MH_CHUNK
#define GB_MH_CHUNK 512
#endif

namespace gb {
namespace {

constexpr int kMhThreads = 256;
constexpr int kMhWarps = kMhThreads / 32;
constexpr int kMhChunk = GB_MH_CHUNK;   // proposals per chunk
constexpr int kMhRec = 32;              // records summarised per chunk
constexpr int kCombineBatch = 32;       // chunk summaries staged in shared memory at a time

static_assert(kMhChunk % 32 == 0 && kMhChunk >= 32 && kMhChunk <= 2048, "chunk size");

struct MhSummary {          // one per (chain, chunk)
    long long K[kMhRec];    // threshold keys of the records, increasing
    long long s[kMhRec];    // exit state key when the chunk is entered through record r
    int32_t c[kMhRec];      // exit state index
    int32_t n[kMhRec];      // acceptances on that path, the record included
    int32_t count;          // records, or -1: scan this chunk with the double test
    int32_t pad[3];
};
struct MhEntry {            // incoming state of a chunk
    long long s;
    int32_t c;
    int32_t pad;
};

constexpr long long kSignMask = 0x7FFFFFFFFFFFFFFFLL;
constexpr long long kEmpty = LLONG_MIN;      // threshold of a proposal no state accepts
constexpr long long kNaNState = LLONG_MAX;   // key of a NaN weight: accepts nothing
constexpr long long kKeyNegInf = -0x7FF0000000000000LL;
constexpr long long kKeyPosInf = 0x7FF0000000000000LL;

__device__ __forceinline__ bool is_nan(double x) {
    return (__double_as_longlong(x) & kSignMask) > kKeyPosInf;
}
// order key of a non-NaN double: x < y  <=>  key(x) < key(y); -0 and +0 share key 0
__device__ __forceinline__ long long dkey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : -(b & kSignMask);
}
__device__ __forceinline__ double from_key(long long k) {
    return k >= 0 ? __longlong_as_double(k) : __longlong_as_double((-k) | LLONG_MIN);
}
__device__ __forceinline__ long long state_key(double w) { return is_nan(w) ? kNaNState : dkey(w); }

// The three forms of the test, fixed at compile time so that no division is
// issued where the rule has none:
//   kPlain    w = logL - log g,      Delta = w_i - w_c   (either form at T = 1)
//   kTempered w = logL/T - log g,    Delta = w_i - w_c   (default form)
//   kDivide   v = logL - log g,      Delta = (v_i - v_c)/T   (literal form)
enum { kPlain = 0, kTempered = 1, kDivide = 2 };

__device__ __forceinline__ int rule_of(double T, int literal) {
    return T == 1.0 ? kPlain : (literal ? kDivide : kTempered);
}
// the threshold form holds unless the literal rule divides by a T that is not positive and finite
__device__ __forceinline__ bool keys_valid(int rule, double T) { return rule != kDivide || (T > 0.0 && T <= DBL_MAX); }

// weight of one proposal, in the oracle's rounding order
template <int RULE>
__device__ __forceinline__ double weight(double l, double g, double T) {
    if (RULE == kTempered) return __dadd_rn(__ddiv_rn(l, T), -g);
    return __dadd_rn(l, -g);
}

// Eq. 13: accept iff log u < min(0, Delta); a NaN Delta (or NaN log u) rejects
template <int RULE>
__device__ __forceinline__ bool accept(double wj, double uj, double wc, double T) {
    double d = __dadd_rn(wj, -wc);
    if (RULE == kDivide) d = __ddiv_rn(d, T);
    if (is_nan(d) || is_nan(uj)) return false;
    const long long ku = dkey(uj);
    return ku < 0 && ku < dkey(d);
}

// Largest key k with accept(w, u, from_key(k)), or kEmpty.  Needs the test to
// be monotone (plain and tempered rules, or T positive and finite).  For u < 0
// the set is empty exactly when w is NaN or -inf (Delta is then NaN or -inf
// for every state); otherwise accept(.., -inf) holds, and accept(.., +inf)
// never does.
template <int RULE>
__device__ long long threshold(double w, double u, double T) {
    if (is_nan(u) || dkey(u) >= 0 || is_nan(w) || dkey(w) == kKeyNegInf) return kEmpty;
    long long lo = kKeyNegInf, hi = kKeyPosInf;   // accept(lo) holds, accept(hi) does not
    const double g = RULE == kDivide ? __dadd_rn(w, -__dmul_rn(u, T)) : __dadd_rn(w, -u);
    if (!is_nan(g)) {
        long long k = min(max(dkey(g), kKeyNegInf), kKeyPosInf);
        if (accept<RULE>(w, u, from_key(k), T)) {
            lo = k;
            for (int it = 0; it < 3 && lo + 1 < hi; ++it) {
                if (!accept<RULE>(w, u, from_key(lo + 1), T)) return lo;
                ++lo;
            }
        } else {
            hi = k;
            for (int it = 0; it < 3 && hi - 1 > lo; ++it) {
                if (accept<RULE>(w, u, from_key(hi - 1), T)) return hi - 1;
                --hi;
            }
        }
    }
    while ((unsigned long long)hi - (unsigned long long)lo > 1ULL) {
        const long long mid = lo + (long long)(((unsigned long long)hi - (unsigned long long)lo) >> 1);
        if (accept<RULE>(w, u, from_key(mid), T)) lo = mid;
        else hi = mid;
    }
    return lo;
}

// thresholds and state keys of the proposals [p0, p0 + len) into shared memory
template <int RULE>
__device__ void chunk_keys(const double* L, const double* G, const double* U, double T, int p0, int len,
                           long long* K, long long* S) {
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
        const double w = weight<RULE>(L[p0 + j], G[p0 + j], T);
        S[j] = state_key(w);
        K[j] = threshold<RULE>(w, U[p0 + j], T);
    }
}

// first local position >= p (below len) whose proposal a state of key s accepts, else len
__device__ __forceinline__ int next_accept(const long long* K, int p, int len, long long s, int lane) {
    for (int b = p; b < len; b += 32) {
        const int j = b + lane;
        const unsigned ball = __ballot_sync(0xffffffffu, j < len && s <= K[j]);
        if (ball) return b + __ffs(ball) - 1;
    }
    return len;
}

// One warp scans proposals [a, b) with the double test from state c (weight
// wc); writes the state after every step into out when out is not null.
template <int RULE>
__device__ void scan_exact(const double* L, const double* G, const double* U, double T, int a, int b, int& c,
                           double& wc, int& n_acc, int32_t* out, int lane) {
    int p = a;
    while (p < b) {
        int hit = -1;
        for (int base = p; base < b; base += 32) {
            const int j = base + lane;
            double wj = 0.0;
            bool ok = false;
            if (j < b) {
                wj = weight<RULE>(L[j], G[j], T);
                ok = accept<RULE>(wj, U[j], wc, T);
            }
            const unsigned ball = __ballot_sync(0xffffffffu, ok);
            const int stop = ball ? base + __ffs(ball) - 1 : min(b, base + 32);
            if (out && j < stop) out[j] = c;
            if (ball) {
                hit = stop;
                wc = __shfl_sync(0xffffffffu, wj, __ffs(ball) - 1);
                break;
            }
        }
        if (hit < 0) break;
        c = hit;
        if (out && lane == 0) out[c] = c;
        ++n_acc;
        p = hit + 1;
    }
}

// run-time dispatch on the chain's rule (uniform within a CTA)
__device__ __forceinline__ double weight_rt(int rule, double l, double g, double T) {
    return rule == kTempered ? weight<kTempered>(l, g, T) : weight<kPlain>(l, g, T);
}
__device__ __forceinline__ void chunk_keys_rt(int rule, const double* L, const double* G, const double* U, double T,
                                              int p0, int len, long long* K, long long* S) {
    if (rule == kPlain) chunk_keys<kPlain>(L, G, U, T, p0, len, K, S);
    else if (rule == kTempered) chunk_keys<kTempered>(L, G, U, T, p0, len, K, S);
    else chunk_keys<kDivide>(L, G, U, T, p0, len, K, S);
}
__device__ __forceinline__ void scan_exact_rt(int rule, const double* L, const double* G, const double* U, double T,
                                              int a, int b, int& c, double& wc, int& n_acc, int32_t* out, int lane) {
    if (rule == kPlain) scan_exact<kPlain>(L, G, U, T, a, b, c, wc, n_acc, out, lane);
    else if (rule == kTempered) scan_exact<kTempered>(L, G, U, T, a, b, c, wc, n_acc, out, lane);
    else scan_exact<kDivide>(L, G, U, T, a, b, c, wc, n_acc, out, lane);
}

// chunk k of a chain covers proposals [1 + k C, min(n, 1 + (k+1) C))
__device__ __forceinline__ int chunk_start(int k) { return 1 + k * kMhChunk; }

constexpr int kSegWin = kMhChunk / kMhThreads > 0 ? kMhChunk / kMhThreads : 1;   // 32-wide windows per warp

// Summary of one (chain, chunk): thresholds and state keys (kept in global
// memory for the write launch), prefix records of the thresholds, and for
// each record the exit state of the chain entered there.
__global__ void __launch_bounds__(kMhThreads) mh_summary_kernel(int n, int n_chunks, const double* __restrict__ logL,
                                                                const double* __restrict__ log_g,
                                                                const double* __restrict__ log_u,
                                                                const double* __restrict__ temperature, int literal,
                                                                MhSummary* __restrict__ sum, long long* __restrict__ gK,
                                                                long long* __restrict__ gS, const int* __restrict__ gate) {
    if (gate && *gate == 0) return;   // inputs unchanged since the last chains: keep them
    __shared__ long long K[kMhChunk], S[kMhChunk];
    __shared__ signed char rec_id[kMhChunk];
    __shared__ int rec_pos[kMhRec], rec_link[kMhRec], rec_c[kMhRec], rec_n[kMhRec];
    __shared__ long long rec_s[kMhRec], seg_max[kMhWarps];
    __shared__ int seg_cnt[kMhWarps];
    const int r = blockIdx.x / n_chunks, k = blockIdx.x - r * n_chunks;
    MhSummary& out = sum[(size_t)r * n_chunks + k];
    const double T = temperature[r];
    const int rule = rule_of(T, literal);
    if (!keys_valid(rule, T)) {
        if (threadIdx.x == 0) out.count = -1;
        return;
    }
    const size_t base = (size_t)r * (size_t)n;
    const int p0 = chunk_start(k), len = min(kMhChunk, n - p0);
    chunk_keys_rt(rule, logL + base, log_g + base, log_u + base, T, p0, len, K, S);
    for (int j = threadIdx.x; j < len; j += blockDim.x) rec_id[j] = -1;
    __syncthreads();
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
        gK[base + p0 + j] = K[j];
        gS[base + p0 + j] = S[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // prefix records of K: each warp takes kSegWin consecutive windows
    long long v[kSegWin], exc[kSegWin];
    long long run = kEmpty;
#pragma unroll
    for (int q = 0; q < kSegWin; ++q) {
        const int j = (warp * kSegWin + q) * 32 + lane;
        v[q] = j < len ? K[j] : kEmpty;
        long long inc = v[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, t);
        }
        const long long e = __shfl_up_sync(0xffffffffu, inc, 1);
        exc[q] = lane == 0 ? run : max(run, e);
        run = max(run, __shfl_sync(0xffffffffu, inc, 31));
    }
    if (lane == 0) seg_max[warp] = run;
    __syncthreads();
    long long before = kEmpty;
    for (int w = 0; w < warp; ++w) before = max(before, seg_max[w]);
    unsigned balls[kSegWin];
    int mine = 0;
#pragma unroll
    for (int q = 0; q < kSegWin; ++q) {
        const int j = (warp * kSegWin + q) * 32 + lane;
        balls[q] = __ballot_sync(0xffffffffu, j < len && v[q] > max(before, exc[q]));
        mine += __popc(balls[q]);
    }
    if (lane == 0) seg_cnt[warp] = mine;
    __syncthreads();
    int off = 0, cnt = 0;
    for (int w = 0; w < kMhWarps; ++w) {
        if (w < warp) off += seg_cnt[w];
        cnt += seg_cnt[w];
    }
    if (cnt > kMhRec) {
        if (threadIdx.x == 0) out.count = -1;
        return;
    }
#pragma unroll
    for (int q = 0; q < kSegWin; ++q) {
        if (balls[q] >> lane & 1u) {
            const int j = (warp * kSegWin + q) * 32 + lane;
            const int id = off + __popc(balls[q] & ((1u << lane) - 1u));
            rec_pos[id] = j;
            rec_id[j] = (signed char)id;
        }
        off += __popc(balls[q]);
    }
    __syncthreads();
    // follow the chain from each record until the chunk ends or it reaches a later record
    for (int m = warp; m < cnt; m += kMhWarps) {
        int c = rec_pos[m], acc = 1, link = -1;
        long long s = S[c];
        for (;;) {
            const int j = next_accept(K, c + 1, len, s, lane);
            if (j >= len) break;
            if (rec_id[j] >= 0) {
                link = rec_id[j];
                break;
            }
            c = j;
            s = S[j];
            ++acc;
        }
        if (lane == 0) {
            rec_link[m] = link;
            rec_c[m] = c;
            rec_s[m] = s;
            rec_n[m] = acc;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // a path that reaches record m' continues as m' does: resolve the links
        // (they point to later records) by pointer jumping
        int link = -1, c = 0, acc = 0;
        long long s = 0;
        if (lane < cnt) {
            link = rec_link[lane];
            c = rec_c[lane];
            s = rec_s[lane];
            acc = rec_n[lane];
        }
        for (int step = 0; step < 5; ++step) {
            const int src = link >= 0 ? link : lane;
            const int link2 = __shfl_sync(0xffffffffu, link, src);
            const int c2 = __shfl_sync(0xffffffffu, c, src);
            const long long s2 = __shfl_sync(0xffffffffu, s, src);
            const int acc2 = __shfl_sync(0xffffffffu, acc, src);
            if (link >= 0) {
                acc += acc2;
                c = c2;
                s = s2;
                link = link2;
            }
        }
        if (lane < cnt) {
            out.K[lane] = K[rec_pos[lane]];
            out.s[lane] = s;
            out.c[lane] = p0 + c;
            out.n[lane] = acc;
        }
        if (lane == 0) out.count = cnt;
    }
}

// Chunk summaries [0, nb) staged in shared memory, applied in order by one
// warp to the state (c, s); a chunk without a summary is scanned with the
// double test.  Returns through c, s, acc.
struct StagedSummaries {
    long long K[kCombineBatch][kMhRec], s[kCombineBatch][kMhRec];
    int c[kCombineBatch][kMhRec], n[kCombineBatch][kMhRec], count[kCombineBatch];
};

__device__ void stage_summaries(StagedSummaries& st, const MhSummary* sm, int nb) {
    for (int i = threadIdx.x; i < nb * kMhRec; i += blockDim.x) {
        const int b = i / kMhRec, l = i - b * kMhRec;
        const MhSummary& t = sm[b];
        if (l == 0) st.count[b] = t.count;
        st.K[b][l] = t.K[l];
        st.s[b][l] = t.s[l];
        st.c[b][l] = t.c[l];
        st.n[b][l] = t.n[l];
    }
}

__device__ void apply_summaries(const StagedSummaries& st, int k0, int nb, int n, int rule, double T,
                                const double* L, const double* G, const double* U, MhEntry* en, int& c,
                                long long& s, int& acc, int lane) {
    for (int b = 0; b < nb; ++b) {
        const int k = k0 + b;
        if (en && lane == 0) {
            en[k].s = s;
            en[k].c = c;
        }
        const int cnt = st.count[b];
        if (cnt >= 0) {
            const unsigned ball = __ballot_sync(0xffffffffu, lane < cnt && s <= st.K[b][lane]);
            if (ball) {
                const int f = __ffs(ball) - 1;
                c = st.c[b][f];
                s = st.s[b][f];
                acc += st.n[b][f];
            }
        } else {
            const int p0 = chunk_start(k);
            double wc = weight_rt(rule, L[c], G[c], T);
            scan_exact_rt(rule, L, G, U, T, p0, min(n, p0 + kMhChunk), c, wc, acc, nullptr, lane);
            s = state_key(wc);
        }
    }
}

// Incoming state of every chunk and the acceptance count, for chains of more
// than kCombineBatch chunks (shorter chains combine inside the write launch).
__global__ void __launch_bounds__(kMhThreads) mh_combine_kernel(int n, int n_chunks, const double* __restrict__ logL,
                                                                const double* __restrict__ log_g,
                                                                const double* __restrict__ log_u,
                                                                const double* __restrict__ temperature, int literal,
                                                                const MhSummary* __restrict__ sum,
                                                                MhEntry* __restrict__ entry, int32_t* __restrict__ chain,
                                                                int32_t* __restrict__ n_accept,
                                                                const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ StagedSummaries st;
    const int r = blockIdx.x;
    const size_t base = (size_t)r * (size_t)n;
    const double* L = logL + base;
    const double* G = log_g + base;
    const double* U = log_u + base;
    const double T = temperature[r];
    const int rule = rule_of(T, literal);
    const MhSummary* sm = sum + (size_t)r * n_chunks;
    MhEntry* en = entry + (size_t)r * n_chunks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int c = 0, acc = 0;
    long long s = state_key(weight_rt(rule, L[0], G[0], T));
    if (threadIdx.x == 0) chain[base] = 0;
    for (int k0 = 0; k0 < n_chunks; k0 += kCombineBatch) {
        const int nb = min(kCombineBatch, n_chunks - k0);
        __syncthreads();
        stage_summaries(st, sm + k0, nb);
        __syncthreads();
        if (warp == 0) apply_summaries(st, k0, nb, n, rule, T, L, G, U, en, c, s, acc, lane);
    }
    if (threadIdx.x == 0 && n_accept) n_accept[r] = acc;
}

// Writes the chain through one chunk from its incoming state: read from
// `entry` when given, else combined here from the summaries of the earlier
// chunks (at most kCombineBatch of them).  The last chunk of a chain also
// writes the acceptance count in that case, the first one chain[0].
__global__ void __launch_bounds__(kMhThreads) mh_write_kernel(int n, int n_chunks, const double* __restrict__ logL,
                                                              const double* __restrict__ log_g,
                                                              const double* __restrict__ log_u,
                                                              const double* __restrict__ temperature, int literal,
                                                              const MhSummary* __restrict__ sum,
                                                              const MhEntry* __restrict__ entry,
                                                              const long long* __restrict__ gK,
                                                              const long long* __restrict__ gS,
                                                              int32_t* __restrict__ chain, int32_t* __restrict__ n_accept,
                                                              const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ long long K[kMhChunk], S[kMhChunk];
    __shared__ StagedSummaries st;
    __shared__ int in_c, in_acc;
    __shared__ long long in_s;
    const int r = blockIdx.x / n_chunks, k = blockIdx.x - r * n_chunks;
    const size_t base = (size_t)r * (size_t)n;
    const double* L = logL + base;
    const double* G = log_g + base;
    const double* U = log_u + base;
    int32_t* out = chain + base;
    const double T = temperature[r];
    const int rule = rule_of(T, literal);
    const size_t slot = (size_t)r * n_chunks + k;
    const int p0 = chunk_start(k), len = min(kMhChunk, n - p0);
    const bool keyed = sum[slot].count >= 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (keyed)
        for (int j = threadIdx.x; j < len; j += blockDim.x) {
            K[j] = gK[base + p0 + j];
            S[j] = gS[base + p0 + j];
        }
    if (entry) {
        if (threadIdx.x == 0) {
            in_c = entry[slot].c;
            in_s = entry[slot].s;
            in_acc = 0;
        }
    } else {
        stage_summaries(st, sum + (size_t)r * n_chunks, k);
        __syncthreads();
        if (warp == 0) {
            int c = 0, acc = 0;
            long long s = state_key(weight_rt(rule, L[0], G[0], T));
            apply_summaries(st, 0, k, n, rule, T, L, G, U, nullptr, c, s, acc, lane);
            if (lane == 0) {
                in_c = c;
                in_s = s;
                in_acc = acc;
            }
        }
        if (k == 0 && threadIdx.x == 0) out[0] = 0;
    }
    __syncthreads();
    if (warp != 0) return;
    int c = in_c, acc = in_acc;
    long long s = in_s;
    if (!keyed) {
        double wc = weight_rt(rule, L[c], G[c], T);
        scan_exact_rt(rule, L, G, U, T, p0, p0 + len, c, wc, acc, out, lane);
    } else {
        int p = 0;
        while (p < len) {
            int hit = -1;
            for (int b = p; b < len; b += 32) {
                const int j = b + lane;
                const unsigned ball = __ballot_sync(0xffffffffu, j < len && s <= K[j]);
                const int stop = ball ? b + __ffs(ball) - 1 : min(len, b + 32);
                if (j < stop) out[p0 + j] = c;
                if (ball) {
                    hit = stop;
                    break;
                }
            }
            if (hit < 0) break;
            c = p0 + hit;
            s = S[hit];
            if (lane == 0) out[c] = c;
            ++acc;
            p = hit + 1;
        }
    }
    if (!entry && k == n_chunks - 1 && lane == 0 && n_accept) n_accept[r] = acc;
}

constexpr int kCertChunk = kMhThreads;   // steps per certification CTA
// bound on the float rounding of the mixed path's data, weights and sums,
// relative to |h| (|d| + |h|): a float copy of the data and of the weights
// and a compensated sum each contribute about 6e-8
constexpr float kMixedRoundingBound = 1e-6f;

// Error bound of one proposal's mixed value on the chain's decision scale.
// The mixed path returns logL~ = <d|h~> - <h~|h~>/2 - <d|d>/2 with the
// template h~ = h + dh, so
//     logL~ - logL = <d - h|dh> - <dh|dh>/2 + (float rounding of the data,
//                    the weights and the compensated sums),
// and with |dh| <= eps |h| (weighted norm over the window) and the rounding at
// most cf |h| (|d| + |h|):
//     |logL~ - logL| <= eps |h| |d - h| + eps^2 |h|^2/2 + cf |h| (|d| + |h|),
//     |d - h| <= |d - h~| + eps |h|,  |d - h~|^2 = -2 logL~,  |d|^2 = <d|d>,
// every norm taken from the outputs (in float, with 3e-7 of the magnitudes
// added for their own rounding), plus 1e-12 of the magnitudes for the double
// epilogue.  Divided by the chain's T, with 1e-15 of the magnitudes of
// logL/T, log g and w added for the rounding of w = logL/T - log g (or
// (logL - log g)/T), two rows' bounds add up to the uncertainty of
// Delta = w_i - w_c.  Rounded up; +inf when a value is not finite.
__device__ __forceinline__ float mixed_bound_f(float lf, float d1, float h2, float gf, float invT, float eps,
                                               float cf) {
    const float mag = fabsf(d1) + fabsf(h2) + fabsf(lf);
    const float dd = fabsf(2.0f * (d1 - 0.5f * h2 - lf)) + 3e-7f * mag;
    const float nh = sqrtf(fmaxf(h2, 0.0f)), nd = sqrtf(dd);
    const float nr = sqrtf(fmaxf(-2.0f * lf, 0.0f) + 3e-7f * mag) + eps * nh;
    float b = (eps * nh * nr + 0.5f * eps * eps * fmaxf(h2, 0.0f) + cf * nh * (nd + nh) + 1e-12f * (mag + dd)) * invT +
              1e-15f * (fabsf(lf) * invT + fabsf(gf) * fmaxf(1.0f, invT) + fabsf(lf * invT - gf));
    b *= 1.0001f;
    return (isfinite(b) && isfinite(lf) && isfinite(gf) && invT > 0.0f) ? b : CUDART_INF_F;
}

// logL, log g of one row in float (the bound's own inputs)
struct RowF {
    float l, g;
};

__device__ __forceinline__ bool accept_rt(int rule, double wj, double uj, double wc, double T) {
    if (rule == kPlain) return accept<kPlain>(wj, uj, wc, T);
    if (rule == kTempered) return accept<kTempered>(wj, uj, wc, T);
    return accept<kDivide>(wj, uj, wc, T);
}

// Certification of chains built from values of which some carry an error
// bound (one CTA per chain and chunk of kCertChunk steps).  Pass 0 computes
// the bounds (mixed_bound_f) and stores them in err; later passes read them
// (0 once a row is re-evaluated).  Step i (i >= 1)
// compares proposal i with the state c = chain[i - 1] before it; its double
// decision log u_i < Delta is the one exact values give unless
// |log u_i - Delta| <= err_i + err_c (err = 0 for exact values; the bounds do
// not change during a pass).  Every step it cannot settle is recorded in the
// chain's step list, and the rows of i and c that are not exact and not
// queued yet (mark) are appended to the chain's queue (rows r n + i), to be
// re-evaluated in FP64.  Pass p's entries of chain r follow those of the
// earlier passes; the chain's last CTA of the pass writes their range
// [q_lo[r], q_hi[r]).  A step whose log u is NaN or >= 0 rejects under any
// value.  When the gate is zero the launch does nothing.
__global__ void __launch_bounds__(kMhThreads) mh_certify_kernel(
    int n, int n_chunks, int pass, int n_chains, const double* __restrict__ logL, const double* __restrict__ dh,
    const double* __restrict__ hh, float eps, float cf, const double* __restrict__ log_g,
    const double* __restrict__ log_u, const double* __restrict__ temperature, int literal,
    const int32_t* __restrict__ chain, float* __restrict__ err, int32_t* __restrict__ mark,
    int32_t* __restrict__ queue, int32_t* __restrict__ steps, int* __restrict__ cnt, int* __restrict__ scnt,
    int* __restrict__ done, int32_t* __restrict__ q_lo, int32_t* __restrict__ q_hi, const int* __restrict__ gate,
    int* __restrict__ n_new) {
    if (gate && *gate == 0) return;
    __shared__ int local, nstep, off, soff, last, s_rule;
    __shared__ float s_invT;
    __shared__ int32_t rows[2 * kCertChunk], stp[kCertChunk];
    const int r = blockIdx.x / n_chunks, k = blockIdx.x - r * n_chunks;
    const size_t base = (size_t)r * (size_t)n;
    if (threadIdx.x == 0) {
        local = nstep = 0;
        // the chain's rule and 1/T, formed once (a double division per thread
        // would load the FP64 pipe as much as the rest of the pass)
        const double T = temperature[r];
        s_rule = rule_of(T, literal);
        s_invT = (T > 0.0 && T <= DBL_MAX) ? (float)(1.0 / T) : 0.0f;
    }
    __syncthreads();
    const int rule = s_rule;
    const float invT = s_invT;
    const int i = 1 + k * kCertChunk + (int)threadIdx.x;
    if (i < n) {
        const int c = chain[base + i - 1];
        const RowF fi{(float)logL[base + i], (float)log_g[base + i]};
        const RowF fc{(float)logL[base + c], (float)log_g[base + c]};
        float ei, ec;
        if (pass == 0) {
            ei = mixed_bound_f(fi.l, (float)dh[base + i], (float)hh[base + i], fi.g, invT, eps, cf);
            ec = mixed_bound_f(fc.l, (float)dh[base + c], (float)hh[base + c], fc.g, invT, eps, cf);
            err[base + i] = ei;
            if (i == 1)
                err[base] = mixed_bound_f((float)logL[base], (float)dh[base], (float)hh[base], (float)log_g[base], invT,
                                          eps, cf);
        } else {
            ei = err[base + i];
            ec = err[base + c];
        }
        const double u = log_u[base + i];
        const long long ku = __double_as_longlong(u);
        // a NaN log u, or one that is not below zero, rejects under any value
        bool settled = (ei == 0.0f && ec == 0.0f) || is_nan(u) || !(ku < 0 && ku != LLONG_MIN);
        if (!settled) {
            // float test first: Delta and log u in float, with a margin of
            // 1e-6 of the magnitudes that covers the conversions and the
            // float operations, so that it settles only steps the double
            // test below settles too
            float li = fi.l, lc = fc.l;
            if (rule == kTempered) {
                li *= invT;
                lc *= invT;
            }
            float df = (li - fi.g) - (lc - fc.g);
            float S = fabsf(li) + fabsf(fi.g) + fabsf(lc) + fabsf(fc.g);
            if (rule == kDivide) {
                df *= invT;
                S *= invT;
            }
            const float uf = (float)u;
            const float thr = (ei + ec) * 1.000001f + 1e-6f * (S + fabsf(uf));
            settled = isfinite(df) && isfinite(thr) && fabsf(uf - df) > thr;
        }
        if (!settled) {
            const double T = temperature[r];
            const double wi = weight_rt(rule, logL[base + i], log_g[base + i], T);
            const double wc = weight_rt(rule, logL[base + c], log_g[base + c], T);
            double d = __dadd_rn(wi, -wc);
            if (rule == kDivide) d = __ddiv_rn(d, T);
            const double m = (double)ei + (double)ec;
            settled = isfinite(d) && isfinite(m) && fabs(u - d) > m;
        }
        if (!settled) {
            stp[atomicAdd(&nstep, 1)] = i;
            if (ei > 0.0f && atomicExch(&mark[base + i], 1) == 0) rows[atomicAdd(&local, 1)] = (int32_t)(base + i);
            if (ec > 0.0f && atomicExch(&mark[base + c], 1) == 0) rows[atomicAdd(&local, 1)] = (int32_t)(base + c);
        }
    }
    __syncthreads();
    int* cr = cnt + (size_t)pass * n_chains + r;
    if (threadIdx.x == 0) {
        off = local ? atomicAdd(cr, local) : 0;
        soff = nstep ? atomicAdd(scnt + (size_t)pass * n_chains + r, nstep) : 0;
        if (local) atomicAdd(n_new, local);
    }
    __syncthreads();
    int lo = 0;
    for (int q = 0; q < pass; ++q) lo += cnt[(size_t)q * n_chains + r];
    for (int j = threadIdx.x; j < local; j += blockDim.x) queue[base + lo + off + j] = rows[j];
    for (int j = threadIdx.x; j < nstep; j += blockDim.x) steps[base + soff + j] = stp[j];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done + (size_t)pass * n_chains + r, 1) == n_chunks - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        q_lo[r] = lo;
        q_hi[r] = lo + atomicAdd(cr, 0);
    }
}

// After the FP64 re-evaluation of pass p's rows (one CTA per chain): their
// bounds become 0, and every step the pass could not settle is decided again
// from the exact values; n_flip counts the steps whose decision differs from
// the chain's (chain[i] == i iff step i accepted).  Without a flip the chain
// is the exact one: every other step was settled within bounds that hold.
__global__ void __launch_bounds__(kMhThreads) mh_flip_kernel(
    int n, int pass, int n_chains, const double* __restrict__ logL, const double* __restrict__ log_g,
    const double* __restrict__ log_u, const double* __restrict__ temperature, int literal,
    const int32_t* __restrict__ chain, float* __restrict__ err, const int32_t* __restrict__ queue,
    const int32_t* __restrict__ steps, const int* __restrict__ scnt, const int32_t* __restrict__ q_lo,
    const int32_t* __restrict__ q_hi, const int* __restrict__ gate, int* __restrict__ n_flip) {
    if (gate && *gate == 0) return;
    const int r = blockIdx.x;
    const size_t base = (size_t)r * (size_t)n;
    for (int j = q_lo[r] + (int)threadIdx.x; j < q_hi[r]; j += blockDim.x) err[queue[base + j]] = 0.0f;
    const double T = temperature[r];
    const int rule = rule_of(T, literal);
    const int ns = scnt[(size_t)pass * n_chains + r];
    int flips = 0;
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        const int i = steps[base + k];
        const int c = chain[base + i - 1];
        const double wi = weight_rt(rule, logL[base + i], log_g[base + i], T);
        const double wc = weight_rt(rule, logL[base + c], log_g[base + c], T);
        flips += accept_rt(rule, wi, log_u[base + i], wc, T) != (chain[base + i] == i);
    }
    if (flips) atomicAdd(n_flip, flips);
}

// out[r] = sum over passes p < n_pass of cnt[p][r] (one thread per chain)
__global__ void sum_rows_kernel(const int* __restrict__ cnt, int n_chains, int n_pass, int32_t* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_chains) return;
    int s = 0;
    for (int p = 0; p < n_pass; ++p) s += cnt[(size_t)p * n_chains + r];
    out[r] = s;
}

}  // namespace

int ensure_mh_scratch(gb_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->mh_bytes) return GB_OK;
    if (ctx->d_mh) cudaFree(ctx->d_mh);
    ctx->d_mh = nullptr;
    ctx->mh_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->d_mh, bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(ctx, GB_ENOMEM, "MH scratch")
                                                                 : cuda_error(ctx, e, "MH scratch");
    ctx->mh_bytes = bytes;
    return GB_OK;
}

// summaries and incoming states per (chain, chunk), then two int64 keys per proposal
size_t mh_scratch_bytes(size_t chunk_slots, size_t proposals) {
    return chunk_slots * (sizeof(MhSummary) + sizeof(MhEntry)) + proposals * 2 * sizeof(long long);
}

}  // namespace gb

using namespace gb;

namespace gb {

int launch_mh(gb_ctx* ctx, int32_t n_chains, int32_t n, const double* logL, const double* log_g, const double* log_u,
              const double* temperature, int32_t literal, int32_t* chain_idx, int32_t* n_accept, const int* gate,
              cudaStream_t st) {
    const int n_chunks = (n - 1 + kMhChunk - 1) / kMhChunk;
    const size_t slots = (size_t)n_chains * (size_t)n_chunks;
    if (slots > (size_t)INT_MAX) return set_error(ctx, GB_EINVAL, "gb_mh_independence: too many chunks");
    const size_t props = (size_t)n_chains * (size_t)n;
    int rc = ensure_mh_scratch(ctx, mh_scratch_bytes(slots > 0 ? slots : 1, props));
    if (rc != GB_OK) return rc;
    MhSummary* sum = (MhSummary*)ctx->d_mh;
    MhEntry* entry = (MhEntry*)(sum + slots);
    long long* gK = (long long*)(entry + slots);
    long long* gS = gK + props;
    const bool fused = n_chunks > 0 && n_chunks <= kCombineBatch;
    if (n_chunks > 0)
        mh_summary_kernel<<<(unsigned)slots, kMhThreads, 0, st>>>(n, n_chunks, logL, log_g, log_u, temperature,
                                                                  literal, sum, gK, gS, gate);
    if (n_chunks > 0) ++ctx->launches;
    if (!fused)
        mh_combine_kernel<<<n_chains, kMhThreads, 0, st>>>(n, n_chunks, logL, log_g, log_u, temperature, literal,
                                                           sum, entry, chain_idx, n_accept, gate);
    if (!fused) ++ctx->launches;
    if (n_chunks > 0)
        mh_write_kernel<<<(unsigned)slots, kMhThreads, 0, st>>>(n, n_chunks, logL, log_g, log_u, temperature,
                                                                literal, sum, fused ? nullptr : entry, gK, gS,
                                                                chain_idx, n_accept, gate);
    if (n_chunks > 0) ++ctx->launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_independence launch");
    return GB_OK;
}

int launch_mh_certify(gb_ctx* ctx, const CertScratch& cs, int32_t n_chains, int32_t n, const double* logL,
                      const double* dh, const double* hh, const double* log_g, const double* log_u,
                      const double* temperature, int32_t literal, double eps, const int32_t* chain_idx, int pass,
                      const int* gate, cudaStream_t st) {
    const int n_chunks = (n - 1 + kCertChunk - 1) / kCertChunk;
    if (n_chunks > 0) {
        mh_certify_kernel<<<(unsigned)((size_t)n_chains * n_chunks), kMhThreads, 0, st>>>(
            n, n_chunks, pass, n_chains, logL, dh, hh, (float)eps, kMixedRoundingBound, log_g, log_u, temperature,
            literal, chain_idx, cs.err, cs.mark, cs.queue, cs.steps, cs.cnt, cs.scnt, cs.done, cs.q_lo, cs.q_hi, gate,
            cs.n_new + pass);
        ++ctx->launches;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "mh_certify launch");
    return GB_OK;
}

int launch_mh_flip(gb_ctx* ctx, const CertScratch& cs, int32_t n_chains, int32_t n, const double* logL,
                   const double* log_g, const double* log_u, const double* temperature, int32_t literal,
                   const int32_t* chain_idx, int pass, cudaStream_t st) {
    mh_flip_kernel<<<n_chains, kMhThreads, 0, st>>>(n, pass, n_chains, logL, log_g, log_u, temperature, literal,
                                                    chain_idx, cs.err, cs.queue, cs.steps, cs.scnt, cs.q_lo, cs.q_hi,
                                                    cs.n_new + pass, cs.n_flip + pass);
    ++ctx->launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "mh_flip launch");
    return GB_OK;
}

int launch_sum_rows(gb_ctx* ctx, const int* cnt, int32_t n_chains, int n_pass, int32_t* out, cudaStream_t st) {
    sum_rows_kernel<<<(n_chains + 127) / 128, 128, 0, st>>>(cnt, n_chains, n_pass, out);
    ++ctx->launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "sum_rows launch");
    return GB_OK;
}

}  // namespace gb

extern "C" int gb_mh_independence(gb_ctx_t* ctx, int32_t n_chains, int32_t n, const double* logL,
                                  const double* log_g, const double* log_u, const double* temperature,
                                  int32_t literal, int32_t* chain_idx, int32_t* n_accept, void* stream) {
    if (!ctx) return GB_EINVAL;
    if (n_chains < 0 || n < 0) return set_error(ctx, GB_EINVAL, "gb_mh_independence: negative size");
    if (n_chains == 0 || n == 0) return GB_OK;
    if (!logL || !log_g || !log_u || !temperature || !chain_idx)
        return set_error(ctx, GB_EINVAL, "gb_mh_independence: null pointer");
    if (literal != 0 && literal != 1) return set_error(ctx, GB_EINVAL, "gb_mh_independence: literal must be 0 or 1");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gb_mh_independence: cudaSetDevice");
    return launch_mh(ctx, n_chains, n, logL, log_g, log_u, temperature, literal, chain_idx, n_accept, nullptr,
                     (cudaStream_t)stream);
}
