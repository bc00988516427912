/*
 * tkdv.h - C ABI of the GB300 (sm_103a) rejection sampler for the
 * truncated-KdV (TKdV) Gibbs measure of Moore & Foerster, "In search of rogue
 * waves: a novel proposal distribution for parallelized rejection sampling of
 * the truncated KdV Gibbs measure" (arXiv 2411.16952).
 *
 * What one proposal does (Sec. IV.B of the paper):
 *   draw X ~ gamma_Sigma, the anisotropic Gaussian of Eqs. (24)-(26)
 *   (or X ~ gamma, Eq. 14, for the uniform proposal of Eq. 15);
 *   project X^ = X/|X| onto the energy sphere S^{2K-1};
 *   compute log f/(M g) by Eq. (40) with H2 (Eq. 20), H3 (Eq. 42 or the grid
 *   cubature of Eq. 2) and beta H (Eq. 43);
 *   accept with probability f/(M g); an accepted X^ is a wave field through
 *   Eq. (16).
 *
 * Conventions used throughout
 *   - K in [1, 128] complex modes; a state is the real vector
 *     xhat = [xhat_1..xhat_K | xhat_{K+1}..xhat_{2K}] (cosine half | sine
 *     half), u_k = sqrt(E0/2pi) (xhat_k - i xhat_{K+k}) (Eq. 16).
 *   - r is the ratio C3/C2 of Eq. (43).  Together with K, E0 and beta' it is
 *     the full parameter set of the method (Sec. IV.A).
 *   - Random stream (the paper names none): Philox4x32-10 with key
 *     (seed_lo, seed_hi) and counter (block j, idx_lo, idx_hi, point_id).
 *     Mode k takes the Box-Muller pair in words 2h, 2h+1 of block
 *     j = (k-1)/2, h = (k-1) % 2 (cosine -> X_k, sine -> X_{K+k}).  The accept
 *     uniform is word 0 of block ceil(K/2).  A word w maps to
 *     (2 floor(w/512) + 1) 2^-24, except that a radius or accept word in the
 *     lowest bucket (w < 512) is refined by word 0 of the blocks with counter
 *     (2^31 + L 2^24 + g, idx_lo, idx_hi, point_id), g = 4 j + word, L = 1, 2:
 *     U = 2^-23 u(w_1) if w_1 >= 512, else 2^-46 u(w_2); so U stays uniform
 *     down to 2^-70 and a draw with log f/(M g) < ln 2^-24 can be accepted.
 *     Accept iff ln U < log f/(M g).
 *     Given (parameters, seed, point_id, log M) the accepted set of an index
 *     range is therefore a fixed set, whatever the launch shape.
 *   - Return values: 0 on success, a negative TKDV_ERR_* code otherwise;
 *     sampler_last_error() then holds a one-line message.  No entry point
 *     aborts the process or falls back to a CPU path.
 *   - Ownership: a sampler handle owns every device buffer it allocates
 *     (cudaMalloc at create time); the caller owns every host buffer it
 *     passes in.  All calls on one handle must come from one host thread at
 *     a time.
 */
#ifndef TKDV_H
#define TKDV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define TKDV_OK 0
#define TKDV_ERR_INVALID_ARG (-1) /* parameter out of range (message says which) */
#define TKDV_ERR_NO_ALPHA (-2)    /* paper proposal with beta' >= K^2 sum 1/k^2: Eq. (29) has no root */
#define TKDV_ERR_CUDA (-3)        /* a CUDA runtime call failed (message has the CUDA error string) */
#define TKDV_ERR_OOM (-4)         /* cudaMalloc / cudaMallocHost failed */
#define TKDV_ERR_TIMEOUT (-5)     /* a device wait hit its iteration limit; results of that run are void */
#define TKDV_ERR_UNSUPPORTED (-6) /* requested form not available on this device */
#define TKDV_ERR_ENVELOPE (-7)    /* envelope search failed (non-finite log M) */
#define TKDV_ERR_TOO_LARGE (-8)   /* sampler_run_static: more proposals than its fixed scratch holds */

/* tkdv_check_radius_error: diagnostic (the paper has no counterpart).  The
   one-thread fast path (K <= 64) computes the Box-Muller radius rho = -2 ln u
   of the uniform map's 2^23 values with the hardware base-2 logarithm; its
   accept guard band assumes |rho_f32 - rho| <= 2^-21 + 2^-21 rho.  This runs
   all 2^23 values on the current device against an FP64 logarithm and returns
   the largest ratio of the error to that bound (at most 1 if the assumption
   holds) and a word that attains it (worst_word may be NULL).  Allocates 8
   bytes of device memory for the call.  Errors: INVALID_ARG (max_ratio NULL),
   OOM, CUDA. */
int tkdv_check_radius_error(double *max_ratio, uint32_t *worst_word);

/* tkdv_check_radius_error_log: the same check for the warp form (K > 64),
   whose radius is -2 logf(u) with the full-precision logarithm; its guard band
   assumes the purely relative bound |rho_f32 - rho| <= 2^-22 rho. */
int tkdv_check_radius_error_log(double *max_ratio, uint32_t *worst_word);

/* ---- proposal kinds (Sec. III) ------------------------------------------ */
#define TKDV_PROPOSAL_UNIFORM 0 /* uniform measure mu0 on the sphere (Eq. 15); the naive baseline */
#define TKDV_PROPOSAL_PAPER 1   /* projected anisotropic Gaussian, sigma_k^2 of Eq. (25) at alpha* */
#define TKDV_PROPOSAL_LEARNED 2 /* paper sigma_k^2 times exp(c_k), c_k given per point (see tkdv_point) */

/* ---- H3 forms ------------------------------------------------------------ */
#define TKDV_H3_TRIAD_F32 0   /* double sum of Eq. (42) on FP32 CUDA cores */
#define TKDV_H3_GRID_BF16X3 1 /* grid cubature of Eq. (2) as a tensor-core contraction, BF16 hi/lo x3 */
#define TKDV_H3_AUTO 2        /* the library chooses: the grid form where it exists (sm_10x device, K <= 64,
                                 not SIR), else the triad form; sampler_autotune then times both forms
                                 and all their launch shapes and keeps the fastest; sampler_h3_form
                                 tells which */

#define TKDV_MAX_POINTS 64
#define TKDV_HIST_BINS 256
#define TKDV_N_EXCEED 25
#define TKDV_KMAX 128

/* One parameter point (Sec. IV.A: K, E0, beta', C3/C2 are the only parameters). */
typedef struct {
    double beta_p;  /* normalised inverse temperature beta' (Eq. 21), >= 0 */
    double E0;      /* energy (Eq. 5), > 0 */
    double r;       /* C3/C2 (Eq. 43), any real */
    int proposal;   /* TKDV_PROPOSAL_* */
    uint32_t point_id;  /* fourth Philox counter word for this point */
    int override_logM;  /* 1: use logM below instead of the library's envelope search */
    double logM;        /* log of the rejection constant M of Eq. (45) when overridden */
    /* TKDV_PROPOSAL_LEARNED only: host array of K per-mode log-variance
       corrections c_k (k = 1..K); sigma_k^2 = sigma_k^2(paper) * exp(c_k).
       Copied at create time; may be NULL for the other proposals. */
    const double *log_var_correction;
    /* SIR runs only (tkdv_options.sir): expected copies per unit of
       exp(log f/(Mg)); a proposal is kept n ~ Poisson(sir_c exp(log f/(Mg)))
       times.  > 0; ignored by rejection runs. */
    double sir_c;
} tkdv_point;

/* Options shared by all points of one handle. */
typedef struct {
    int K;                    /* modes, 1..128, common to all points of the handle; the triad form runs
                                 K <= 64 one proposal per thread and 65..128 one warp per four proposals
                                 (same stream, same decisions); the grid form and SIR need K <= 64 */
    int h3_mode;              /* TKDV_H3_* */
    int grid_N;               /* grid points of the grid form (TKDV_H3_GRID_BF16X3, or TKDV_H3_AUTO with
                                 K <= 64): multiple of 32, > 3K, <= 256; 0: the smallest such (128 for K = 32) */
    uint64_t sample_capacity; /* accepted records kept per handle (ring; excess is counted, not kept) */
    void *cuda_stream;        /* cudaStream_t to launch on; NULL: the handle makes its own */
    int use_graph;            /* 1: launch each run as one CUDA graph (default), 0: plain launches */
    int ctas_per_sm;          /* 0: occupancy maximum; else persistent CTAs per SM */
    int threads_per_cta;      /* 0: default (256); 128 or 256 */
    int sir;                  /* 0: rejection sampling (Sec. IV.B); 1: sampling-importance resampling with
                                 the same proposal (named in Sec. IV.B): every proposal carries the weight
                                 exp(log f/(Mg)) and is kept n ~ Poisson(sir_c exp(log f/(Mg))) times, n drawn
                                 by inversion of its accept uniform, n = #{k >= 1 : U < P(N >= k)}; given
                                 their total the copies are the multinomial SIR draw.  Triad form only.
                                 Every proposal that may get a copy is decided in the FP64 pass, which
                                 holds 4M proposals per run: keep sir_c sum exp(log f/(Mg)) per run well
                                 below that; proposals beyond it get no copy and are counted in
                                 n_fallback. */
} tkdv_options;

/* Statistics of one point, accumulated over runs until sampler_reset().
   u0 = u(xi = 0) of each accepted field (Eq. 8). */
typedef struct {
    uint64_t n_proposals;
    uint64_t n_accepted;
    uint64_t n_near_threshold;      /* |ln U - log f/(Mg)| < 1e-6 (decided in FP64) */
    uint64_t n_refined;             /* proposals decided on the FP64 path (guard band) */
    uint64_t n_envelope_violations; /* proposals with log f/(Mg) > 0: M was too small */
    uint64_t n_dropped;             /* accepted records that did not fit the ring */
    uint64_t n_fallback;            /* guard-band proposals decided in FP32 because the FP64
                                       queue was full (0 unless a run queued > 4M of them) */
    double max_delta;               /* largest log f/(Mg) seen (FP32 path) */
    double logM;                    /* envelope used */
    double alpha_star;              /* root of Eq. (29) (paper / learned proposals), else 1 */
    double sum_u0[4];               /* sum over accepted of u0^p, p = 1..4 */
    double mean, var, skew, kurt;   /* of u0 over accepted samples */
    uint64_t hist[TKDV_HIST_BINS];  /* u0 histogram on [hist_lo, hist_hi] */
    double hist_lo, hist_hi;        /* -/+ sqrt(2 K E0 / pi), the largest |u| on the sphere */
    uint64_t exceed[TKDV_N_EXCEED]; /* accepted with u0 > 0.25 i sqrt(E0/pi), i = 0..24 (Sec. V.D) */
    double spectrum[TKDV_KMAX];     /* sum over accepted of s_k = xhat_k^2 + xhat_{K+k}^2 = |u_k|^2 2pi/E0,
                                       k = 1..K (0 beyond K); spectrum / n_accepted is the mean power
                                       spectrum of Sec. V.A.  Each term is rounded to 2^-28. */
    /* SIR runs: n_accepted, the histogram, moments, exceedances and spectrum
       count every copy; n_kept counts the proposals with at least one copy.
       The importance-sampling sums run over all proposals, with w =
       exp(log f/(Mg)) from the FP32 path: E_f[phi] ~ sum w phi / sum w and
       the effective sample size is sir_sum_w^2 / sir_sum_w2 (FP64 sums of
       FP32 terms; their last bits depend on the launch shape). */
    uint64_t n_kept;
    double sir_sum_w, sir_sum_w2, sir_sum_wS; /* sum w, w^2, w S (S = H2/E0) */
    double sir_sum_w_u0[4];                   /* sum w u0^p, p = 1..4 */
} tkdv_stats;

/* Accepted-sample record, as stored in the device ring and returned by
   sampler_samples(): this 32-byte header followed by float xhat[2K], the
   projected state in [cosine | sine] order; records are
   tkdv_record_bytes(K) bytes apart (16-byte multiple). */
typedef struct {
    uint64_t idx;    /* proposal index within its point's stream */
    uint32_t point;  /* point number within the handle (0-based) */
    uint32_t flags;  /* bit 0: decided on the FP64 path; bit 1: near threshold;
                        bits 8..31: copies (SIR runs; 0 in rejection runs) */
    float H2, H3;    /* Eqs. (20) and (42) of the accepted state */
    float u0;        /* u(xi = 0) */
    float delta;     /* log f/(M g) */
} tkdv_record;

size_t tkdv_record_bytes(int K);

typedef struct tkdv_sampler tkdv_sampler;

/* sampler_create: one parameter point with default options (K given here,
   triad H3, 2^20-record ring, own stream).  Runs the per-point precompute of
   Sec. IV.B on the host: alpha* (Eq. 29), sigma_k (Eq. 25) and log M
   (Eq. 45), then allocates device buffers.  The 4th argument is C3/C2.
   Errors: INVALID_ARG (K outside 1..128, E0 <= 0, beta' < 0, unknown
   proposal), NO_ALPHA, OOM, CUDA.  *out is NULL on error. */
int sampler_create(int K, double beta_p, double E0, double r, int proposal, tkdv_sampler **out);

/* sampler_create_ex: n_points (1..64) points sharing opt->K and opt->h3_mode,
   run together by one persistent launch (batched form).  Errors as above,
   plus UNSUPPORTED for the grid form on a device without tcgen05.  The grid
   form keeps one copy of the mirror-pair basis per CTA (grid_N/2 rows x KA
   columns, KA = 2 x the mode bound 16, 32 or 64, BF16 hi and lo) and two to
   four warpgroups, each with its own 128-proposal A tile (128 x KA, hi and
   lo) and grid_N TMEM columns; a launch shape is offered only where its
   warpgroups x grid_N <= 512 TMEM columns and its tiles fit the shared
   memory. */
int sampler_create_ex(const tkdv_point *points, int n_points, const tkdv_options *opt,
                      tkdv_sampler **out);

/* sampler_run: n_proposals new proposals for every point, continuing each
   point's index where the previous run stopped.  Asynchronous on the
   handle's stream: returns after the launch; statistics accumulate on the
   device.  Errors: INVALID_ARG, CUDA, TIMEOUT (from an earlier run). */
int sampler_run(tkdv_sampler *h, uint64_t n_proposals, uint64_t seed);

/* sampler_run_budgets: budgets[p] proposals for point p (uneven budgets). */
int sampler_run_budgets(tkdv_sampler *h, const uint64_t *budgets, uint64_t seed);

/* sampler_run_ranges: proposals idx0[p] .. idx0[p] + count[p] - 1 of every
   point p; does not move the points' running index. */
int sampler_run_ranges(tkdv_sampler *h, const uint64_t *idx0, const uint64_t *count, uint64_t seed);

/* sampler_stats: waits for the handle's stream, then fills out[p] for
   p = 0..n_out-1 (n_out <= number of points).  Moments are reduced from
   exact 64-bit fixed-point sums (u0^p scaled by 2^28, 2^24, 2^20, 2^16). */
int sampler_stats(tkdv_sampler *h, tkdv_stats *out, int n_out);

/* sampler_samples: waits, then copies up to max_records accepted records
   (tkdv_record_bytes(K) bytes each, unordered) to dst, a host buffer if
   dst_on_device == 0, else a device buffer; *n_out = records copied. */
int sampler_samples(tkdv_sampler *h, void *dst, int dst_on_device, uint64_t max_records,
                    uint64_t *n_out);

/* sampler_field_maxima: the largest surface displacement of each of the
   first min(max_records, kept) records (in the order sampler_samples returns
   them) on the 2K-point grid xi_j = -pi + pi j / K of Sec. V.D:
   umax[i] = max_j u(xi_j), u from Eqs. (8), (16); jmax[i] = the maximising j
   (the smallest on ties; jmax may be NULL).  The field with the largest umax
   among m accepted fields is the "1-in-m event" of Figs. 8-11.  umax and jmax
   are host arrays of max_records entries; *n_out receives the count.  Runs
   one kernel on the handle's stream (synchronises); allocates 8 bytes per
   record of device memory for the call.  Errors: INVALID_ARG, OOM, CUDA. */
int sampler_field_maxima(tkdv_sampler *h, uint64_t max_records, double *umax, int32_t *jmax, uint64_t *n_out);

/* sampler_reset: zero statistics, the record ring and the running indices. */
int sampler_reset(tkdv_sampler *h);

/* sampler_sync: wait for all work queued on the handle's stream; returns
   TIMEOUT if a device wait of any earlier run gave up. */
int sampler_sync(tkdv_sampler *h);

/* sampler_set_deadline_ns: time budget of every persistent CTA in later
   runs (0 = none).  A CTA past its budget takes no further chunk; the run
   then ends early and sampler_sync / sampler_stats return TKDV_ERR_TIMEOUT
   once (the flag is cleared when reported).  Statistics hold the proposals
   that did run. */
int sampler_set_deadline_ns(tkdv_sampler *h, uint64_t ns);

/* sampler_set_trace: grid form only (tcgen05 contraction).  Later runs write,
   for each of point 0's first n proposals of the run (index idx0[0] + i),
   the pair (log f/(Mg), T) as two floats at dev_buf[2i], where
   H3 = 2 pi (E0/2pi)^{3/2} T (Eq. 42 in these units).  A proposal with a
   refined word (K radius words and the accept word: about K+1 in 2^23, see the stream rule above) is decided in
   the FP64 pass only and traced as two NaNs.  dev_buf is the
   caller's device buffer of 2n floats; n = 0 switches the trace off.
   Errors: INVALID_ARG, UNSUPPORTED (triad form). */
int sampler_set_trace(tkdv_sampler *h, void *dev_buf, uint64_t n);

/* sampler_point_info: alpha*, log M and the K proposal variances sigma_k^2
   (Eq. 25, or the learned ones) of point p; any output may be NULL. */
int sampler_point_info(tkdv_sampler *h, int p, double *alpha_star, double *logM, double *sigma2);

/* sampler_replay: per-proposal outputs of point p for the n host-listed
   indices (a test and debugging path that runs the same device code as the
   sampler).  out is a host array of n * (8 + 2K) doubles per proposal:
   [delta, lnU, accept, flags, H2, H3, u0, S, xhat_1..xhat_2K]. */
int sampler_replay(tkdv_sampler *h, int p, const uint64_t *idx, uint64_t n, uint64_t seed,
                   double *out);

/* sampler_autotune: time the persistent launch on `calib_proposals` per point
   for each candidate (CTAs per SM, threads per CTA and register budget, the
   triad form's two accept paths, and for TKDV_H3_AUTO both H3 forms; best of
   four timed runs each) and keep the fastest for later runs.  Resets
   statistics afterwards.  *best_us receives the best time (may be NULL). */
int sampler_autotune(tkdv_sampler *h, uint64_t calib_proposals, double *best_us);

/* sampler_h3_form: the H3 form the next run uses, TKDV_H3_TRIAD_F32 or
   TKDV_H3_GRID_BF16X3 (for a TKDV_H3_AUTO handle: the library's choice).
   Errors: INVALID_ARG (h NULL). */
int sampler_h3_form(const tkdv_sampler *h);

/* sampler_batch_run: one call for a batch of points: sampler_create_ex with
   (points, n_points, opt), budgets[p] proposals of point p from index 0 with
   `seed`, the statistics of every point into out (n_points entries, host,
   caller-owned), then sampler_destroy.  Errors as sampler_create_ex,
   sampler_run_budgets and sampler_stats; the message is in
   sampler_last_error(NULL). */
int sampler_batch_run(const tkdv_point *points, int n_points, const tkdv_options *opt, const uint64_t *budgets,
                      uint64_t seed, tkdv_stats *out);

/* sampler_set_launch: pin the launch shape of later runs instead of the
   default or autotuned one.  variant: triad form 0 = 128 threads, 1 = 256
   threads, 2 = 256 threads held to 128 registers (two CTAs per SM), 3..5 the
   same with the per-lane accept path (for K > 64: 0..2 of the warp form; SIR
   runs: 1; grid form, by mode bound: K <= 16: 0 = four warpgroups per CTA,
   1 = two; 16 < K <= 32: 0 = four, 1 = three, 2 = two; 32 < K <= 64: 0 = two;
   each offered where it fits, see sampler_create_ex).  ctas_per_sm: 1 .. the
   occupancy maximum of that variant, 0 for the maximum.  Results do not depend on the launch shape.
   Errors: INVALID_ARG (no such variant for the handle's form, ctas_per_sm
   above the maximum), CUDA. */
int sampler_set_launch(tkdv_sampler *h, int variant, int ctas_per_sm);

/* sampler_launch_config: the launch shape of the next run. */
int sampler_launch_config(tkdv_sampler *h, int *ctas, int *threads_per_cta, uint32_t *chunk);

/* ---- one run without any allocation --------------------------------------
   sampler_run_static: the paper has no counterpart; this is a service for
   callers that cannot allocate device memory: code whose device memory is
   owned by another allocator (a framework that reserved the whole pool up
   front), latency-critical loops where cudaMalloc/cudaFree would synchronise
   the device, and plugin hosts that forbid device allocation.

   It runs proposals idx0 .. idx0 + n_proposals - 1 of one point with the same
   kernels as sampler_run_ranges() and calls no cudaMalloc, cudaFree or other
   allocating routine.  Its scratch (the point table, statistics, counters and
   the FP64 guard-band queue, about 4 MiB) is a fixed array inside this
   library that every GPU which loads the library holds until the process
   exits.  The first call on a device looks up that array's device address
   (cudaGetSymbolAddress, once per device); make that first call before any
   stream capture.  Every call shares the array: each call clears it first,
   and calls whose work overlaps on the GPU (other host threads, other
   streams) race on it and must not be issued.
     K           modes, 1..128
     point       host struct; override_logM must be 1 with the envelope in
                 logM (tkdv_log_M computes it), else TKDV_ERR_INVALID_ARG
     n_proposals at most TKDV_STATIC_MAX_PROPOSALS, else TKDV_ERR_TOO_LARGE
                 (split larger ranges over several calls with advancing idx0)
     records     caller's DEVICE buffer on the current device, holding at
                 least capacity * tkdv_record_bytes(K) bytes (may be NULL
                 with capacity 0); the kernels write up to capacity records
                 into it, so a smaller buffer is overrun (the library cannot
                 check the size of a raw pointer)
     n_records   host; records written (<= capacity), may be NULL
     stats       host; statistics of this call alone, may be NULL
     cuda_stream stream to run on (NULL: the legacy default stream)
   The call returns after the run has finished.  Errors: INVALID_ARG,
   NO_ALPHA, TOO_LARGE, CUDA, TIMEOUT. */
#define TKDV_STATIC_MAX_PROPOSALS 262144
int sampler_run_static(int K, const tkdv_point *point, uint64_t idx0, uint64_t n_proposals, uint64_t seed,
                       void *records, uint64_t capacity, uint64_t *n_records, tkdv_stats *stats,
                       void *cuda_stream);

const char *sampler_last_error(const tkdv_sampler *h);
void sampler_destroy(tkdv_sampler *h);

/* ---- learned proposal ------------------------------------------------------
   Not in the paper.  A 4 -> 64 -> 64 -> 64 MLP (tanh hidden layers, linear
   output) maps the features of a parameter point (tkdv_mlp_features) to
   per-mode log-variance corrections c_k of the paper's proposal:
   sigma_k'^2 = sigma_k^2 (Eq. 25) * e^{c_k}, c gauge-fixed to mean zero over
   k = 1..K (the proposal density is unchanged by a common factor).  The
   proposal stays a projected centred Gaussian, so its density keeps the closed
   form of Eqs. (33)-(38) and the accept test stays exact (pass c as
   tkdv_point.log_var_correction; the envelope is recomputed for it).
   Training minimises, per point over accepted samples i (draws from f),
     J_tau = tau log mean_i exp((z_i + ell_i)/tau),  ell_i = -log g(xh_i)
           = K ln Q_i - sum_k ln w'_k,  z_i = -beta H_i;
   tau <= 0 means the plain mean (KL(f || g) up to a constant).  Parameters:
   FP32 masters updated by Adam, used as BF16 copies; FP32 accumulation.
   Parameter layout (TKDV_MLP_NPARAM floats): W1[64][4], b1[64], W2[64][64],
   b2[64], W3[64][64], b3[64] (row = output unit).  All calls synchronise. */
#define TKDV_MLP_NPARAM 8640
typedef struct tkdv_mlp tkdv_mlp;
/* hidden layers seeded normal, output layer zero (c = 0: the paper proposal) */
int tkdv_mlp_create(uint64_t seed, tkdv_mlp **out);
void tkdv_mlp_destroy(tkdv_mlp *m);
const char *tkdv_mlp_last_error(const tkdv_mlp *m);
/* out4 = [ln beta'/ln 100, ln E0, ln(1 + beta' C3/C2 / 100)/ln 100, K/64] */
int tkdv_mlp_features(int K, double beta_p, double E0, double r, double *out4);
/* FP32 masters and/or the BF16 values in use (as floats), host arrays of NPARAM */
int tkdv_mlp_get_params(tkdv_mlp *m, float *master, float *bf16_values);
/* replaces the masters (BF16 copies refreshed), resets Adam */
int tkdv_mlp_set_params(tkdv_mlp *m, const float *master);
/* c_out (P x 64, host): gauge-fixed corrections for P feature rows (P x 4) */
int tkdv_mlp_infer(tkdv_mlp *m, int P, const double *feats, const int *K, double *c_out);
/* training set from host arrays: per point K, features (P x 4), paper weights
   w_k = 1/sigma_k^2 (P x 64), counts[p] rows; s_rows holds sum(counts) rows of
   round_up(max K, 4) floats (s_k = xh_k^2 + xh_{K+k}^2, zero padded), point
   after point; z (sum(counts) floats, may be NULL: zeros) = -beta H */
int tkdv_mlp_set_data(tkdv_mlp *m, int P, const int *K, const double *feats, const double *w_paper,
                      const uint64_t *counts, const float *s_rows, const float *z);
/* training set from a DEVICE buffer of n_records sampler records
   (tkdv_record layout, K_records modes): record point p -> training point p,
   at most max_per_point rows each; zcoef[2p] = beta'/(E0 K^2), zcoef[2p+1] = C3/C2 */
int tkdv_mlp_set_data_records(tkdv_mlp *m, int P, const int *K, const double *feats, const double *w_paper,
                              const double *zcoef, const void *records_dev, uint64_t n_records, int K_records,
                              uint64_t max_per_point);
/* rows per point of the current training set */
int tkdv_mlp_rows(tkdv_mlp *m, uint64_t *counts);
/* one pass: forward, loss, backward (grad_out: NPARAM floats, may be NULL),
   and an Adam update with learning rate lr when update != 0; *loss = sum over
   points of J (before the update) */
int tkdv_mlp_step(tkdv_mlp *m, float lr, float tau, int update, double *loss, float *grad_out);

/* ---- host precompute, exported for tests --------------------------------- */
/* alpha* = root of F(alpha) = 1 - (alpha/K) sum_k 1/(1 + alpha beta' k^2/K^3)
   (Eq. 29).  Errors: INVALID_ARG, NO_ALPHA. */
int tkdv_alpha_star(int K, double beta_p, double *out);

/* log M = max over the sphere of log f/g (Eq. 45), searched from the
   Dirichlet kernel of Eq. (46) and other starts.  sigma2 (K values) gives the
   pair variances for the Gaussian proposals; NULL for the uniform proposal. */
int tkdv_log_M(int K, double beta_p, double E0, double r, const double *sigma2, double *out);

#ifdef __cplusplus
}
#endif
#endif /* TKDV_H */
