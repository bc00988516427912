/*
 * oracle.h - plain FP64 CPU oracle for rejection sampling of the truncated-KdV
 * (TKdV) Gibbs measure (Moore & Foerster, "In search of rogue waves", arXiv
 * 2411.16952).
 *
 * TEST INFRASTRUCTURE ONLY.  tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference leg of bench.py are the only code allowed to load or
 * call this library.  It shares no code, header, table or constant generator
 * with the CUDA library; the two meet only through their inputs (parameters,
 * seeds, proposal indices).
 *
 * All arithmetic is IEEE FP64 with no reordering beyond what the paper's
 * formulas state.  Every function cites the passage of the paper it follows.
 */
#ifndef TKDV_ORACLE_H
#define TKDV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_KMAX 128
#define ORC_HIST_BINS 256
#define ORC_EXCEED 25

/* proposal kinds */
#define ORC_PROPOSAL_UNIFORM 0 /* uniform measure mu0 on the sphere, Eq. (15) */
#define ORC_PROPOSAL_PAPER 1   /* anisotropic Gaussian, Eqs. (24)-(25) with alpha* */
#define ORC_PROPOSAL_DIAG 2    /* any diagonal Gaussian with pair variances sigma2[k] */

typedef struct {
    int K;          /* Galerkin cutoff, 1..128 (Eq. 8) */
    int proposal;   /* ORC_PROPOSAL_* */
    double E0;      /* energy, Eq. (5) */
    double beta_p;  /* normalised inverse temperature beta', Eq. (21) */
    double r;       /* nonlinearity-to-dispersion ratio C3/C2, Eq. (43) */
    double alpha;   /* alpha* (root of Eq. 29) for the paper proposal */
    double sigma2[ORC_KMAX]; /* pair variances sigma_k^2, k = 1..K */
    double logM;    /* log of the rejection constant M, Eq. (45) */
} orc_point;

typedef struct {
    uint64_t idx;
    double lnU;     /* log of the accept uniform */
    double logfg;   /* log f/g of Eq. (40) (up to the constant dropped there) */
    double delta;   /* logfg - logM = log of the acceptance probability */
    double H2, H3;  /* Eqs. (20) and (42) */
    double S;       /* sum_k k^2 (xh_k^2 + xh_{K+k}^2) */
    double u0;      /* u(xi = 0), Eq. (8) */
    int accept;     /* lnU < delta */
    int near;       /* |lnU - delta| < 1e-6 */
    double xhat[2 * ORC_KMAX];
} orc_rec;

typedef struct {
    uint64_t n_prop, n_acc, n_near, n_viol;
    double max_delta;
    double u_cap;                    /* sqrt(2 K E0 / pi) */
    double sum_u0[4];                /* sum of u0^p, p = 1..4, accepted only */
    double sum_grid[4];              /* sum of u(xi_j)^p over the 2K-point grid */
    double spectrum[ORC_KMAX];       /* sum of |u_k|^2 / (E0/2pi) = s_k */
    uint64_t hist[ORC_HIST_BINS];    /* histogram of u0 on [-u_cap, u_cap] */
    uint64_t exceed[ORC_EXCEED];     /* #accepted with u0 > 0.25*i*sqrt(E0/pi) */
} orc_stats;

/* Philox4x32-10 block (Salmon, Moraes, Dror & Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform in (0,1) from one 32-bit word: (2*floor(w/512) + 1) / 2^24. */
double orc_uniform(uint32_t w);
/* The uniform of word w at stream position g of proposal idx, its lowest
 * bucket (w < 512) refined from further Philox blocks down to 2^-70. */
double orc_uniform_ext(uint32_t w, uint32_t g, const uint32_t key[2], uint64_t idx, uint32_t point_id);
/* Box-Muller pair from two uniforms. */
void orc_box_muller(double u1, double u2, double *z_cos, double *z_sin);
/* The 2K standard normals and the accept uniform of proposal idx (stream layout). */
void orc_stream(int K, uint64_t seed, uint32_t point_id, uint64_t idx, double *z, double *u_acc);
/* Indices in [idx0, idx0+n) whose stream has a word in the lowest bucket of
 * the uniform map: which = 1 radius words, 2 the accept word, 3 either.
 * Writes the first `cap` to out; returns how many there are. */
uint64_t orc_tail_scan(int K, uint64_t seed, uint32_t point_id, uint64_t idx0, uint64_t n, int which,
                       uint64_t *out, uint64_t cap);

double orc_H2(int K, double E0, const double *xh);
double orc_H3_double(int K, double E0, const double *xh);
double orc_H3_triple(int K, double E0, const double *xh);
double orc_H3_grid(int K, double E0, const double *xh, int N);
double orc_u_at(int K, double E0, const double *xh, double xi);

double orc_F_alpha(int K, double beta_p, double alpha);
double orc_alpha_star(int K, double beta_p);
/* fills alpha and sigma2 for ORC_PROPOSAL_PAPER / UNIFORM; returns 0 or -1 (no root) */
int orc_point_init(orc_point *pt, int K, double E0, double beta_p, double r, int proposal);

double orc_log_fg(const orc_point *pt, const double *xh);
/* log M by Nelder-Mead from the Dirichlet kernel plus extra starts; writes argmax */
double orc_log_M(const orc_point *pt, int n_random_starts, uint64_t seed, double *xh_best);
/* Nelder-Mead maximisation of log f/g from one start (restarted until stable) */
double orc_nelder_mead(const orc_point *pt, const double *xh0, double *xh_out, long max_evals);

/* Replay the proposals listed in idx[0..n) (any order); nthreads <= 0 means 1. */
int orc_replay(const orc_point *pt, uint64_t seed, uint32_t point_id, const uint64_t *idx,
               uint64_t n, int nthreads, orc_rec *out);
/* Run proposals idx0 .. idx0+n-1 and reduce them into statistics. */
int orc_run_stats(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx0,
                  uint64_t n, int nthreads, orc_stats *out);
/* Same, but collect accepted records (first `cap`) instead of statistics. */
uint64_t orc_run_accepted(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx0,
                          uint64_t n, int nthreads, orc_rec *out, uint64_t cap);

/* Sampling-importance resampling with the same proposal (see oracle.c). */
typedef struct {
    uint64_t n_prop;     /* proposals */
    uint64_t n_kept;     /* proposals with at least one copy */
    uint64_t n_copies;   /* resampled fields, counted with multiplicity */
    double sum_w, sum_w2;          /* sum of the weights exp(Delta) and of their squares */
    double sum_wS, sum_w_u0[4];    /* weighted sums of S and of u0^p (importance sampling) */
    double sum_nS, sum_n_u0[4];    /* the same over the resampled fields */
    double spectrum[ORC_KMAX];     /* sum over resampled fields of s_k */
} orc_sir_stats;

/* P(N >= k) for N ~ Poisson(lambda), k >= 1. */
double orc_poisson_tail(double lambda, int k);
/* #{k >= 1 : u < P(N >= k)}: a Poisson(lambda) count by inversion of u. */
int orc_poisson_count(double lambda, double u);
/* SIR over proposals idx0 .. idx0+n-1 with c copies per unit exp(Delta):
 * statistics, and the kept proposals (records and copy counts, first cap, in
 * index order); returns the number of kept proposals. */
uint64_t orc_run_sir(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx0, uint64_t n, double c,
                     int nthreads, orc_sir_stats *out, orc_rec *kept, uint32_t *kept_n, uint64_t cap);

#ifdef __cplusplus
}
#endif
#endif
