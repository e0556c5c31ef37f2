/*
 * gb.h -- C ABI of libgb, the GB300-native batched Galactic-binary likelihood.
 *
 * The library evaluates, for batches of 8-parameter Galactic-binary candidates
 * grouped by frequency window, the TDI A/E template by the fast/slow
 * decomposition and the noise-weighted inner products of Strub et al.,
 * "Accelerating global parameter estimation of gravitational waves from
 * Galactic binaries using a genetic algorithm and GPUs" (arXiv:2307.03763):
 *
 *   log-likelihood       log p(d|theta) = -1/2 <d - s|d - s>        (Eq. 2)
 *   inner product        <x|y> = 4 Re int x~ y~* / S df             (Eq. 3)
 *   channel sum, A and E sum over {A, E}; A = (Z-X)/sqrt2,
 *                        E = (X-2Y+Z)/sqrt6                          (Eqs. 4-5)
 *   SNR, best amplitude  rho = <d|s>/sqrt<s|s>, A_max = <d|s'>/<s'|s'> (Eqs. 6-7)
 *   MH acceptance        min(1, [L_p/L_c g_c/g_p]^(1/T))            (Eq. 13, Alg. 4)
 *
 * Conventions the paper leaves open (it cites the waveform model) are fixed
 * as follows and are the same in every entry point:
 *   theta (8 doubles per candidate, this order):
 *       f0 [Hz], fdot [Hz/s], beta [rad, ecliptic latitude],
 *       lambda [rad, ecliptic longitude], A [strain amplitude],
 *       iota [rad], psi [rad], phi0 [rad]
 *   carrier bin  q = floor(f0 T + fdot T^2/2 + 1/2), one IEEE rounding per
 *       operation in the order ((f0*T) + ((0.5*fdot)*T)*T) + 0.5
 *   slow part sampled at t_n = n T/N, N-point DFT, template on bins
 *       q - N/2 .. q + N/2 - 1 with h~(f_{q+m}) = (T/2N) S_m
 *   inner product over window bins k0 .. k0+W-1:
 *       <x|y> = (4/T) Re sum_k w_k x_k y_k*,  w_k = 1/S(f_k)
 *   template bins outside the window are dropped.
 *   Orbit: rigid equal-arm triangle (arm L) on the first-order heliocentric
 *   orbit; first-generation equal-arm TDI.
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller unless
 * stated otherwise; complex arrays are interleaved (re, im) doubles.  The
 * library owns only the context (orbit tables, twiddles, cached launch plans,
 * a device status word).  All compute calls are asynchronous on `stream`
 * (a cudaStream_t passed as void*; NULL = legacy default stream).
 *
 * Errors: every call returns GB_OK (0) or a negative code; gb_last_error()
 * gives the message of the last failing call on that context.  Argument
 * errors are detected on the host before anything is launched.  A candidate
 * with a non-finite parameter gets NaN outputs and sets GB_EINVAL in the
 * context's device status word, which gb_ctx_check() reads (synchronising).
 */
#ifndef GB_H
#define GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_OK        0
#define GB_EINVAL   -1   /* bad argument (host check) or non-finite theta (device) */
#define GB_ECUDA    -2   /* a CUDA runtime call failed */
#define GB_ETIMEOUT -3   /* a persistent kernel stopped at the context's time budget */
#define GB_ENOMEM   -4   /* device allocation failed */

#define GB_FP64   0      /* every step in IEEE double */
#define GB_MIXED  1      /* carrier phase modulo one cycle in 64-bit fixed point
                            (double-word float arithmetic for candidates outside
                            its ranges), per-candidate set-up and carrier offset
                            in double; response, FFT and inner products in float
                            with compensated sums; inputs and outputs stay double */

#define GB_N_MIN  32
#define GB_N_MAX  1024

typedef struct gb_ctx gb_ctx_t;

/* Observation: T_obs [s], arm length L [m]; orbit_model 0 = rigid equal-arm
 * first-order orbit (the only model). */
typedef struct {
    double  T_obs;
    double  arm_L;
    int32_t orbit_model;
    int32_t reserved;
} gb_obs_t;

/* One frequency window (Sec. III.A-D: the data are analysed per segment and
 * the inner-product integral is limited to it).
 *   k0        first frequency bin of the window (f = k / T_obs)
 *   data_off  index of the window's first bin in dA, dE, wA, wE
 *   cand_off  first candidate row of the window in theta and the outputs
 *   W         bins in the window (>= 0)
 *   N         template samples, a power of two in [GB_N_MIN, GB_N_MAX]
 *   n_cand    candidates of the window (>= 0)
 * Windows may share data; candidate ranges must not overlap. */
typedef struct {
    int64_t k0;
    int64_t data_off;
    int64_t cand_off;
    int32_t W;
    int32_t N;
    int32_t n_cand;
    int32_t reserved;
} gb_window_t;

/* Create a context on CUDA device `device` and build its orbit and twiddle
 * tables (allocates device memory; synchronous).  *ctx is NULL on failure.
 * T_obs > 0, arm_L > 0, orbit_model == 0. */
int gb_ctx_create(gb_ctx_t** ctx, const gb_obs_t* obs, int device);

/* Free the context and everything it owns.  NULL is accepted. */
int gb_ctx_destroy(gb_ctx_t* ctx);

/* Message of the last failing call on `ctx` (never NULL; "" if none). */
const char* gb_last_error(const gb_ctx_t* ctx);

/* Work budget of the persistent mixed-precision kernels (gb_loglik and
 * gb_loglik_grad with GB_MIXED), in seconds; 0 (the default) means none.
 * Each warp of such a launch stops taking work items once `seconds` have
 * passed since it started, by the GPU's global timer, and flags the stop in
 * the status word, so the next gb_ctx_check returns GB_ETIMEOUT.  The rows of
 * the items not taken are not written.  The FP64 kernels and the other entry
 * points ignore the budget.  A bounded launch time for batches whose cost the
 * caller cannot predict (the paper has no counterpart).  GB_EINVAL unless
 * 0 <= seconds <= 1e9. */
int gb_ctx_set_time_budget(gb_ctx_t* ctx, double seconds);

/* Events around the next mixed-precision likelihood launch (instrumentation
 * for benchmarks; the paper has no counterpart).  `start` and `end` are
 * cudaEvent_t handles the caller created and owns (with timing enabled, for
 * cudaEventElapsedTime).  The next call on this context that launches the
 * mixed-precision likelihood kernels (gb_loglik, gb_loglik_aet,
 * gb_loglik_phase, gb_loglik_phase_aet with GB_MIXED, or gb_mh_certified)
 * records `start` on its stream after the window preparation, just before
 * those kernels, and `end` just after them; the context then forgets both.
 * NULL for both clears them.  GB_EINVAL if exactly one is NULL. */
int gb_ctx_set_kernel_events(gb_ctx_t* ctx, void* start, void* end);

/* Number of kernels the context's calls have launched so far, counted on
 * the host at each launch (the paper has no counterpart: instrumentation for
 * benchmarks).  0 for a NULL context.  Not thread safe across concurrent
 * calls on one context, like the rest of the API. */
uint64_t gb_launch_count(const gb_ctx_t* ctx);

/* Synchronise the device, read and clear the context's status word.
 * Returns GB_OK; GB_ETIMEOUT if a persistent kernel stopped at the time
 * budget (gb_ctx_set_time_budget) since the last check; else GB_EINVAL if a
 * kernel met a non-finite parameter since the last check. */
int gb_ctx_check(gb_ctx_t* ctx);

/* Frequency-domain A/E templates (the signal model s(theta) of Sec. III,
 * first paragraph, with the response of Eqs. 4-5).
 *   theta  B x 8 doubles (device)
 *   B      number of templates (>= 0)
 *   N      template samples (power of two in [GB_N_MIN, GB_N_MAX])
 *   hA, hE B x N complex (device, written): entry [b][j] is bin q_b - N/2 + j
 *   q      B int64 carrier bins (device, written)
 * prec = GB_MIXED computes the unit-amplitude template in float and scales
 * it by A in double on output. */
int gb_waveform(gb_ctx_t* ctx, int prec, const double* theta, int64_t B, int32_t N,
                double* hA, double* hE, int64_t* q, void* stream);

/* gb_waveform with the T channel, hT laid out like hA (B x N complex,
 * device, written); either precision. */
int gb_waveform_aet(gb_ctx_t* ctx, int prec, const double* theta, int64_t B, int32_t N,
                    double* hA, double* hE, double* hT, int64_t* q, void* stream);

/* Batched log-likelihood over windows (Eq. 2 restricted to each window,
 * Sec. III.D):  logL = <d|h> - <h|h>/2 - <d|d>/2.
 *   win        n_win descriptors (HOST array, read during the call)
 *   dA, dE     complex data of all windows (device, interleaved)
 *   wA, wE     1/S per bin (device)
 *   n_bins     length of dA, dE (complex entries), wA, wE; every window must
 *              satisfy data_off + W <= n_bins (checked, else GB_EINVAL)
 *   theta      candidate rows (device, n_rows x 8)
 *   n_rows     rows of theta and of the outputs; every window must satisfy
 *              cand_off + n_cand <= n_rows (checked, else GB_EINVAL)
 *   logL       per candidate (device, written)
 *   dh, hh     <d|h>, <h|h> per candidate (device, written; may be NULL) --
 *              rho and A_max of Eqs. 6-7 follow from them
 * Rows not covered by any window are not written.  The first call with a
 * given window layout uploads a launch plan (synchronous allocation and
 * copy); later calls with the identical layout reuse it and only launch. */
int gb_loglik(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
              const double* dA, const double* dE, const double* wA, const double* wE,
              int64_t n_bins, const double* theta, int64_t n_rows,
              double* logL, double* dh, double* hh, void* stream);

/* gb_loglik with the T channel T = (X + Y + Z)/sqrt3 (Eq. 5).  The paper
 * keeps T only above half the transfer frequency, f* / 2 = c/(4 pi L), where
 * its response is not suppressed (Sec. II): a window whose lowest frequency
 * k0/T_obs is at least f* / 2 sums A, E and T in every inner product
 * (including <d|d>); the others use A and E only.  dT (complex, interleaved)
 * and wT (1/S_T) are laid out like dA and wA (device, n_bins entries, not
 * NULL).  Everything else as gb_loglik.  The mixed path transforms T as
 * one channel pair of T's even and odd samples (an N/2-point transform),
 * then takes the radix-2 step to T's N bins. */
int gb_loglik_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
                  const double* dA, const double* dE, const double* dT, const double* wA, const double* wE,
                  const double* wT, int64_t n_bins, const double* theta, int64_t n_rows,
                  double* logL, double* dh, double* hh, void* stream);

/* gb_loglik plus the imaginary part of the data-template product,
 *   dh_im = (4/T) Im sum_k w_k d_k h_k*    (device, n_rows, written; not NULL)
 * per candidate.  The template depends on phi0 only through the common
 * factor exp(i phi0) of Sec. III's signal model, so
 *   <d|h(phi0 + delta)> = cos(delta) dh + sin(delta) dh_im,
 * dh_im is <d|h> at phi0 + pi/2, and the phase-maximised <d|h> is
 * sqrt(dh^2 + dh_im^2) at delta = atan2(dh_im, dh).  Same inputs, outputs,
 * layout rules and errors as gb_loglik; GB_EINVAL when dh_im is NULL. */
int gb_loglik_phase(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
                    const double* dA, const double* dE, const double* wA, const double* wE,
                    int64_t n_bins, const double* theta, int64_t n_rows,
                    double* logL, double* dh, double* dh_im, double* hh, void* stream);

/* Gradient of the log-likelihood, d logL / d theta, for every candidate, by
 * the adjoint (reverse-mode) method: the template is recomputed, never
 * stored.  Same inputs as gb_loglik; grad is n x 8 (device, written), in the
 * theta order.  q is held fixed (its derivative is zero almost everywhere).
 * logL (may be NULL) receives the log-likelihood. */
int gb_loglik_grad(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
                   const double* dA, const double* dE, const double* wA, const double* wE,
                   int64_t n_bins, const double* theta, int64_t n_rows,
                   double* logL, double* grad, void* stream);

/* gb_loglik_phase with the T channel in the windows above f* / 2 of Sec. II
 * (as gb_loglik_aet): dh_im sums over A, E and T alike, so it is the
 * three-channel <d|h> at phi0 + pi/2.  dT, wT as in gb_loglik_aet (not NULL);
 * dh_im not NULL; otherwise the inputs, outputs and errors of gb_loglik. */
int gb_loglik_phase_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
                        const double* dA, const double* dE, const double* dT, const double* wA,
                        const double* wE, const double* wT, int64_t n_bins, const double* theta,
                        int64_t n_rows, double* logL, double* dh, double* dh_im, double* hh, void* stream);

/* gb_loglik_grad of gb_loglik_aet's likelihood: the T channel in the windows
 * whose lowest frequency is at least f* / 2.  dT and wT as in
 * gb_loglik_aet (device, not NULL; both NULL gives gb_loglik_grad). */
int gb_loglik_grad_aet(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
                       const double* dA, const double* dE, const double* dT, const double* wA,
                       const double* wE, const double* wT, int64_t n_bins, const double* theta,
                       int64_t n_rows, double* logL, double* grad, void* stream);

/* Independence Metropolis-Hastings chains from precomputed values
 * (Sec. III.G, Alg. 4, Eq. 13).  Row r of each n_chains x n input is one
 * chain:  logL (log-likelihood of proposal i), log_g (log proposal density),
 * log_u (log of a U(0,1) variate), temperature (n_chains, > 0).
 * For i = 1..n-1 with current state c:
 *     Delta = (logL_i - logL_c)/T + (log_g_c - log_g_i)      (literal = 0)
 *     Delta = ((logL_i - logL_c) + (log_g_c - log_g_i))/T    (literal = 1)
 *     accept iff log_u_i < min(0, Delta)   (a NaN Delta rejects)
 * evaluated in IEEE double in this rounding order: w_i = logL_i/T - log_g_i,
 * Delta = w_i - w_c (literal = 0); v_i = logL_i - log_g_i,
 * Delta = (v_i - v_c)/T (literal = 1).
 * chain_idx (n_chains x n int32, device, written): chain[0] = 0 and
 * chain[i] = state after step i.  n_accept (n_chains int32, written). */
int gb_mh_independence(gb_ctx_t* ctx, int32_t n_chains, int32_t n,
                       const double* logL, const double* log_g, const double* log_u,
                       const double* temperature, int32_t literal,
                       int32_t* chain_idx, int32_t* n_accept, void* stream);

/* FP64 log-likelihood of listed rows (Eq. 2 over each window, as gb_loglik
 * with GB_FP64).  Window w's entries are the rows rows[cand_off + j] for j in
 * [row_lo[w], row_hi[w]) (clamped to [0, n_cand)); an entry outside the
 * window's rows [cand_off, cand_off + n_cand) is skipped.  Those rows of logL,
 * dh and hh (dh, hh may be NULL) are written with exactly the bits gb_loglik
 * (GB_FP64) gives them; every other row is left as it is.  The list lengths
 * live on the device, so a caller can enqueue this call behind a kernel that
 * fills the lists, without a host round trip (this is how gb_mh_certified
 * re-evaluates the proposals it cannot settle; the paper has no counterpart).
 *   rows    n_rows int32 (device), window w's entries from rows + cand_off
 *   row_lo, row_hi   n_win int32 each (device)
 * Windows, data and theta as gb_loglik; n_rows < 2^31. */
int gb_loglik_rows(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win,
                   const double* dA, const double* dE, const double* wA, const double* wE,
                   int64_t n_bins, const double* theta, int64_t n_rows,
                   const int32_t* rows, const int32_t* row_lo, const int32_t* row_hi,
                   double* logL, double* dh, double* hh, void* stream);

/* One posterior round of Alg. 4 (Sec. III.G, Eq. 13): the log-likelihood of
 * every proposal in mixed precision and independence MH chains equal, step for
 * step, to the chains built from GB_FP64 log-likelihoods (gb_loglik with
 * GB_FP64, then gb_mh_independence).
 *
 * Window w holds one chain: its proposals are rows [w n, (w + 1) n) of theta,
 * log_g, log_u and the outputs (n = n_cand, the same for every window,
 * cand_off = w n).  log_g, log_u, temperature, literal: as gb_mh_independence.
 *
 * Method.  With the mixed template h~ = h + dh, logL~ - logL =
 * <d - h|dh> - <dh|dh>/2 plus the float rounding of the data, weights and
 * sums, so a mixed value differs from the FP64 one by at most
 *     e = eps |h| |d - h| + eps^2 |h|^2/2 + 1e-6 |h| (|d| + |h|)
 * (plus 1e-12 of the magnitudes) when the template's error is at most
 * eps |h| in the window's weighted norm (Cauchy-Schwarz; |d|^2 = <d|d>,
 * |h|^2 = <h|h>, |d - h| <= (-2 logL~)^1/2 + eps |h|, all from the outputs).
 * The chain is built from the mixed values; a step whose decision
 * log u_i < Delta could change within the bounds of proposal i and of the state
 * before it has those two rows re-evaluated in FP64 (gb_loglik_rows, bit for
 * bit gb_loglik's) and is decided again from the exact values.  Every other
 * step was settled within bounds that hold, so unless one of those decisions
 * differs from the chain's, the chain is the FP64 one; if one does, the chain
 * is built again and certified anew, up to max_iter times.
 *
 *   eps        bound on the mixed template's relative error, in (0, 1e-2).
 *              Over every row of the posterior (160,000), population
 *              (262,144) and band (5.6 million; N = 32 ... 1024, 0.3 - 20 mHz,
 *              SNR up to 2,000) workloads the measured |logL_mixed -
 *              logL_fp64| is at most 0.134 of e at the binding's default
 *              eps = 1e-5 (a factor of 7.4; 29 on the band and population
 *              workloads).
 *   max_iter   re-evaluation passes, in [1, 64] (2 suffice in practice)
 *   logL       n_win n (device, written): mixed values, FP64 on re-evaluated rows
 *   dh, hh     n_win n (device, written): the mixed <d|h>, <h|h>
 *   chain_idx, n_accept   as gb_mh_independence (device, written)
 *   n_exact    n_win int32 (device, written; may be NULL): rows re-evaluated
 *   pending    one int32 (device, written): 0 when the chains are certified;
 *              else the rows the last pass still queued -- call again with a
 *              larger max_iter
 * Everything is enqueued on `stream` without a host synchronisation; the
 * context keeps the flags and queues (allocated on the first call with a
 * given size).  Errors as gb_loglik. */
int gb_mh_certified(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win,
                    const double* dA, const double* dE, const double* wA, const double* wE,
                    int64_t n_bins, const double* theta, const double* log_g, const double* log_u,
                    const double* temperature, int32_t literal, double eps, int32_t max_iter,
                    double* logL, double* dh, double* hh, int32_t* chain_idx, int32_t* n_accept,
                    int32_t* n_exact, int32_t* pending, void* stream);

/* Multi-signal SNR (Sec. III.D, Eq. 11) and the inner products it is made
 * of, in FP64.  Window w's sources are its candidate rows
 * theta[cand_off .. cand_off + n_cand) (K_w = n_cand <= kmax <= 64), each
 * with the template of gb_waveform (GB_FP64, N of the window) restricted to
 * the window's bins.  Writes
 *   gram  n_win x kmax x kmax (device): G_w[i][j] = <s_i|s_j> for i, j < K_w
 *         (the other entries are left as they are)
 *   dh    n_rows (device, may be NULL): <d|s_i> of every source row
 *   rho   n_win (device, may be NULL): sum_i <d|s_i> / sqrt(sum_ij G_w[i][j]),
 *         the SNR of the sum of the window's templates; NaN for K_w = 0
 * The scaled error and overlap of a recovered against an injected source
 * (Sec. IV, Eqs. 19-20) follow from the Gram matrix of the pair:
 * delta = (G_rr - 2 G_ri + G_ii)/G_rr, O = G_ri / sqrt(G_rr G_ii).
 * wA, wE are required; dA, dE only when dh or rho is requested.  A source
 * with a non-finite parameter gives NaN entries and sets the status word.
 * Windows as gb_loglik; one CTA per window, sum_w K_w (K_w + 1)/2 template
 * evaluations. */
int gb_snr_multi(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win,
                 const double* dA, const double* dE, const double* wA, const double* wE,
                 int64_t n_bins, const double* theta, int64_t n_rows, int32_t kmax,
                 double* gram, double* dh, double* rho, void* stream);

/* Launch shapes chosen by gb_autotune: candidates per work item and resident
 * CTAs per SM of the persistent mixed-precision kernels (0 = built-in
 * heuristic), candidates per CTA tile of the FP64 kernel, and the measured
 * milliseconds per call with the choice and with the heuristics. */
typedef struct {
    int32_t item;
    int32_t blocks_per_sm;
    int32_t tile;
    int32_t reserved;
    double ms;
    double ms_default;
} gb_tuning_t;

/* Launch-shape autotuner (the paper has no counterpart; it times the
 * batched evaluation of Sec. III.G on the caller's own batch).  Runs
 * gb_loglik with prec on the given inputs for a set of launch shapes (mixed:
 * 2, 4, 8, 16 or 32 candidates per work item x 1, 2, 3 or all resident CTAs
 * per SM; FP64: 16 to 128 candidates per CTA tile), reps timed calls each,
 * keeps the fastest in the context for later calls and reports it in chosen
 * (may be NULL).  logL (n_rows doubles, device) is overwritten.  Synchronous;
 * allocates launch plans for the trial shapes. */
int gb_autotune(gb_ctx_t* ctx, int prec, const gb_window_t* win, int32_t n_win,
                const double* dA, const double* dE, const double* wA, const double* wE,
                int64_t n_bins, const double* theta, int64_t n_rows, double* logL, int32_t reps,
                gb_tuning_t* chosen, void* stream);

/* Prior box of one window: lower and upper bounds of the eight parameters in
 * theta order (Table 1 of the paper gives its prior; the box is the
 * caller's). */
typedef struct {
    double lo[8];
    double hi[8];
} gb_box_t;

/* Genetic-search settings: tournament size (>= 1), probability of a blend
 * crossover, per-parameter mutation probability, mutation standard deviation
 * as a fraction of the box width. */
typedef struct {
    int32_t tournament;
    int32_t reserved;
    double p_cross;
    double p_mut;
    double mut_scale;
} gb_ga_params_t;

/* One generation of the genetic search of every window's population.  The
 * paper maximises the SNR of Eq. 6 over the parameters other than A with
 * differential evolution and sets A from Eq. 7 (Alg. 2, Sec. III.D); this is a
 * genetic algorithm with that objective.
 *   theta      n_win x pop x 8 population (device), pop individuals per window
 *              (pop <= 32768: the population's fitness is held in shared memory)
 *   dh, hh     <d|h>, <h|h> of every individual (device, from gb_loglik)
 *   dh_im      imaginary parts from gb_loglik_phase (device, may be NULL):
 *              in a window whose phi0 range spans 2 pi the fitness is then
 *              maximised over phi0, rho = sqrt(dh^2 + dh_im^2)/sqrt(hh), and
 *              the best individual is rotated to phi0 + atan2(dh_im, dh)
 *              (wrapped into the box) with A_max = A sqrt(dh^2 + dh_im^2)/hh
 *   box        n_win prior boxes (device)
 *   seed       key of the Philox-4x32-10 draws
 *   generation_in, generation_out   one uint64 each (device): the draws
 *              are counted by *generation_in; the call writes
 *              *generation_out = *generation_in + 1, so two alternating slots
 *              advance the search when the same launches are replayed
 *   params     settings (host)
 *   grad       n_win x 8 gradient of logL at each window's best individual of
 *              the previous call (device, may be NULL): slots 1..4 then take
 *              steps of radius 0.3, 0.1, 0.03, 0.01 along it in natural units
 *   theta_out  next population (device, must not alias theta): slot 0 is the
 *              best individual with A set to A_max = A <d|h>/<h|h> (Eq. 7),
 *              the rest are tournament children with blend crossover and
 *              Gaussian mutation, folded back into the box
 *   best       n_win x 8 best individuals (device, written; may be NULL) */
int gb_ga_step(gb_ctx_t* ctx, int32_t n_win, int32_t pop, const double* theta, const double* dh,
               const double* hh, const double* dh_im, const gb_box_t* box, uint64_t seed, const uint64_t* generation_in,
               uint64_t* generation_out, const gb_ga_params_t* params, const double* grad,
               double* theta_out, double* best, void* stream);

/* Gaussian proposals of the independence sampler (Alg. 4 draws n samples per
 * round from the current proposal distribution; Sec. III.G).  For window w
 * and proposal i, with counter-based Philox-4x32-10 draws keyed by seed and
 * counted by (*round_in, w, i, block):
 *   z_j  eight Box-Muller normals from the first two blocks
 *        (z_2m = r cos 2 pi v, z_2m+1 = r sin 2 pi v, r = sqrt(-2 log u),
 *         u, v = (x + 1/2) 2^-32 of consecutive 32-bit words)
 *   theta = mu_w + L_w z               (L_w lower triangular, row-major 8x8)
 *   log_g = -|z|^2/2 - sum_j log L_w,jj - 4 log(2 pi)
 *   log_u = log of a uniform from the first word of the third block
 * mu: n_win x 8, chol: n_win x 64 (device); theta n_win x n x 8, log_g and
 * log_u n_win x n (device, written).  round_in/round_out: one uint64 each
 * (device), *round_out = *round_in + 1, so replayed launches draw new
 * samples.  n_win <= 65535. */
int gb_draw_gaussian(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* mu, const double* chol,
                     uint64_t seed, const uint64_t* round_in, uint64_t* round_out, double* theta,
                     double* log_g, double* log_u, void* stream);

/* Gaussian refit of the independence proposal between the temperatures of
 * Alg. 4 (the paper refits paired 2-D kernel density estimates; this is the
 * Gaussian counterpart).  For window w, over the n states theta[w][chain[w][i]]
 * (device; chain as written by gb_mh_independence, so a state weighs the
 * steps spent in it), with u the number of accepted moves (i >= 1 with
 * chain[i] = i) and P = chol[w] chol[w]^T the current proposal:
 *   mean  mu_w = sample mean
 *   C     = ratio (g inflate S + (1 - g) P),  S the sample covariance
 *           (divisor n - 1), g = u / (u + kappa)
 *   M     = L0^-1 C L0^-T            (L0 = chol0[w], lower triangular)
 *   M_jk /= d_j d_k, d_j = max(1, sqrt(M_jj var_floor))   (variances <= 1/var_floor)
 *   M_jj += var_floor;  chol[w] = L0 chol(M)   (overwritten)
 * ratio is the next temperature over this one (the tempered target's
 * variance scales with T); kappa is a pseudo-count that keeps a round with
 * few acceptances close to the current proposal.  A non-finite M is replaced
 * by the identity.  theta n_win x n x 8, chain n_win x n int32, chol0 and
 * chol n_win x 64 (row-major, lower triangular; chol must not alias chol0),
 * mu n_win x 8 (device).  n >= 2, ratio > 0, inflate > 0, kappa >= 0,
 * 0 < var_floor < 1. */
int gb_gauss_refit(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* theta, const int32_t* chain,
                   const double* chol0, double ratio, double inflate, double kappa, double var_floor,
                   double* mu, double* chol, void* stream);

/* Paired two-dimensional kernel-density proposals of Alg. 4 (Sec. III.G: the
 * posterior obtained at one temperature, as a KDE over the parameter pairs
 * (f0, fdot), (lambda, beta), (A, iota), is the proposal of the next; psi and
 * phi0 stay uniform over their narrow reduced ranges).  Window w's reduced
 * box is box[w] = lo[8], hi[8] (device, n_win x 16, hi > lo).  Each pair's
 * estimate is a grid x grid table of cumulative cell probabilities,
 * cdf[w][p][c] for the flattened cell c = i grid + j (i the first
 * parameter's cell: (f0, fdot), (lambda, beta), (A, iota) for p = 0, 1, 2;
 * device, n_win x 3 x grid^2 doubles), over the extent
 * ext[w][p] = (x0, x1, y0, y1) (device, n_win x 3 x 4 doubles).  A table with
 * cdf[c] = (c + 1)/grid^2 over the box's extents is uniform over the box
 * (the first temperature).
 *
 * gb_kde_build: from the chain (n_win x n int32, as written by
 * gb_mh_independence) over theta (n_win x n x 8).  Per axis, with the n
 * entries theta[chain[i]] in [a, b], h = s (u + 1)^(-1/6) (s their standard
 * deviation, u the accepted moves) and c0 = (hi - lo)/grid, the extent is
 * [max(lo, a - 3h - c0), min(hi, b + 3h + c0)] (written to ext).  The
 * entries are counted per cell (floor((x - x0)/(x1 - x0) grid), clamped),
 * smoothed per axis by the Gaussian of width h (weights exp(-d^2/2 sigma^2),
 * sigma = h/cell, |d| <= min(ceil(3 sigma), grid - 1), normalised; mass past
 * the grid edge dropped), normalised, mixed with a uniform floor_mass (0..1)
 * and summed into cdf.
 *
 * gb_kde_draw: n proposals per window.  With Philox-4x32-10 words
 * w_0..w_11 from key seed and counters (*round_in, w, i, 0..2), u_k =
 * (w_k + 1/2) 2^-32: pair p takes the first cell c with cdf[c] > u_3p (the
 * last if none) and the point x0 + (cell + u_3p+1) (x1 - x0)/grid (y alike with
 * u_3p+2);
 * psi = lo + u_9 (hi - lo), phi0 with u_10;
 *   log_g = sum_p log((cdf[c] - cdf[c-1]) / cell area) - log(psi width)
 *           - log(phi0 width),   log_u = log u_11.
 * theta n_win x n x 8, log_g, log_u n_win x n (device, written);
 * *round_out = *round_in + 1.  grid in [2, 128], n_win <= 65535. */
/* Noise estimate within a frequency segment (Sec. III.C): for window w and
 * channel c (0 = A, 1 = E) the median over the window's W bins of the
 * periodogram 2 (Re d_k^2 + Im d_k^2) / T_obs (the data are continuous-FT
 * samples, so this is the paper's 2 |DFT|^2 / (N f_sample)); for even W the
 * mean of the two middle values.  debias != 0 divides by ln 2 (the median of
 * an exponential variate is ln 2 times its mean), else the median as printed.
 *   win        n_win descriptors (HOST array; W <= 4096, data_off + W <= n_bins)
 *   dA, dE     complex data (device, interleaved, n_bins entries)
 *   S          n_win x 2 estimates (device, written; NaN for W = 0)
 *   wA, wE     weights (device, may both be NULL): the window's bins are set
 *              to 1/S, the segment's constant noise weight; windows whose
 *              bins overlap must not ask for weights (each window writes all
 *              of its bins, so overlapping windows would race)
 * The estimate is re-run after signals are subtracted (the paper's dynamic
 * noise estimate). */
int gb_noise_median(gb_ctx_t* ctx, const gb_window_t* win, int32_t n_win, const double* dA, const double* dE,
                    int64_t n_bins, int32_t debias, double* S, double* wA, double* wE, void* stream);

int gb_kde_build(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* theta, const int32_t* chain,
                 const double* box, int32_t grid, double floor_mass, double* cdf, double* ext, void* stream);
int gb_kde_draw(gb_ctx_t* ctx, int32_t n_win, int32_t n, const double* box, int32_t grid, const double* cdf,
                const double* ext, uint64_t seed, const uint64_t* round_in, uint64_t* round_out, double* theta,
                double* log_g, double* log_u, void* stream);

/* n blocks of Philox-4x32-10 (Salmon et al., SC 2011) with key = seed and
 * counter (i, 0, 0, 0), i < n, written as 4 words per block (device).  The
 * generator the genetic search draws from; exported so that it can be
 * checked against its published definition. */
int gb_philox4x32(gb_ctx_t* ctx, uint64_t seed, uint32_t n, uint32_t* out, void* stream);

/* Allocation-free variant of gb_loglik with prec = GB_MIXED.
 *
 * The paper has no counterpart to this entry point.  It serves callers that
 * must not allocate device memory while they run: a plugin inside a host
 * application that hands out all device memory through its own pool, or a
 * latency-critical loop that cannot accept the device-wide synchronisation
 * that cudaMalloc and cudaFree imply.  It needs no context.
 *
 * Windows, data, candidates and outputs are those of gb_loglik (device
 * pointers, host window array), and so are the results.  All scratch memory
 * (geometry tables and twiddles, window descriptors and work items,
 * per-window values, float copies of the windows, work-queue heads, the
 * status word) lives in one static device array of about 8.7 MB, which every
 * GPU that loads the library holds until the process exits.  Limits:
 * n_win <= 4096, the windows' W add up to at most 262144 bins, at most 65536
 * work items (about two million candidates); beyond them the call returns
 * GB_EINVAL with a message.
 *
 * The call runs on the current CUDA device.  Each call takes the device
 * address of the static array (cudaGetSymbolAddress, which allocates
 * nothing); the first call on a device, a call in a new CUDA context (after a
 * device reset) and any call with a different T_obs or arm_L also build the
 * tables into it.  Make that first call before any stream capture.  The call
 * itself returns GB_EINVAL on a stream that is capturing a graph: it uploads
 * its work items from host staging that the next call overwrites.  Every call
 * shares the one array and leaves its contents behind; what must start at
 * zero (queue heads, status word) is reset by the call itself.  Calls that
 * overlap on the GPU (other streams, other host threads) race on the array:
 * the caller must serialise them.
 *   status   one int32 (device, may be NULL), written when the call's kernels
 *            finish: 0, or 1 when a candidate had a non-finite parameter
 *            (its outputs are NaN); every call reports its own candidates only
 *   err      (may be NULL) receives a message of at most err_len bytes when
 *            the call fails on the host. */
int gb_loglik_mixed_noalloc(const gb_obs_t* obs, const gb_window_t* win, int32_t n_win,
                            const double* dA, const double* dE, const double* wA, const double* wE,
                            int64_t n_bins, const double* theta, int64_t n_rows,
                            double* logL, double* dh, double* hh, int32_t* status, void* stream,
                            char* err, int32_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* GB_H */
