/*
 * oracle.c - plain FP64 CPU oracle for rejection sampling of the truncated-KdV
 * Gibbs measure (Moore & Foerster, arXiv 2411.16952).
 *
 * TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference leg of bench.py are the only callers.  The product
 * (the CUDA library and its binding) never loads this file and shares no code
 * with it.
 *
 * The oracle follows the algorithm of Sec. IV.B in the paper's order: draw X
 * from the anisotropic Gaussian (Eqs. 24-26), project X^ = X/|X|, evaluate
 * f/g by Eq. (40) with H2 from Eq. (20), H3 from the double sum Eq. (42) and
 * beta*H from Eq. (43), and accept with probability f/(M g).  It is slow on
 * purpose: every proposal is evaluated from scratch in FP64.
 *
 * Readings where the paper is silent (it names no random stream and no accept
 * rule) are stated at the code that takes them:
 *   - random stream: Philox4x32-10 (Salmon et al., SC'11), key = (seed_lo,
 *     seed_hi), counter = (block j, idx_lo, idx_hi, point_id);
 *   - mode k (1-based) takes the Box-Muller pair from words 2h, 2h+1 of block
 *     j = (k-1)/2, h = (k-1) % 2: cosine part -> X_k, sine part -> X_{K+k};
 *   - the accept uniform is word 0 of block ceil(K/2);
 *   - a word w maps to the uniform (2*floor(w/512) + 1) * 2^-24 in (0,1);
 *   - accept iff ln U < ln(f/(M g)) (strict).
 */
#include "oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------
 * Philox4x32-10, written from the description in Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two
 * 32x32->64 multiplications whose high halves are xored with the other two
 * counter words and the round key; the key is bumped by the Weyl constants
 * between rounds.
 * ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* (2 m + 1) / 2^24 with m = floor(w / 512): never 0 or 1, exact in FP32 too. */
double orc_uniform(uint32_t w)
{
    return (2.0 * (double)(w >> 9) + 1.0) * 0x1p-24;
}

/* The uniform of the word at position g (4 * block + word) of proposal idx,
 * with its lowest bucket refined.  orc_uniform alone puts every u < 2^-23 at
 * 2^-24; that caps the Box-Muller radius (-2 ln u <= 33.3) and the accept
 * test (ln U >= -16.6), so a draw whose log ratio is below -16.6 could never
 * be accepted although Sec. IV.B accepts it with probability e^Delta.  A word
 * in the lowest bucket (w < 512) is therefore followed, level by level, by
 * word 0 of the Philox block with counter (2^31 + L 2^24 + g, idx_lo, idx_hi,
 * point_id), L = 1, 2: U = 2^-23 u(w_1) if w_1 >= 512, else 2^-46 u(w_2).
 * U is then uniform on (0, 1) with 23 bits of relative resolution down to
 * 2^-70. */
double orc_uniform_ext(uint32_t w, uint32_t g, const uint32_t key[2], uint64_t idx, uint32_t point_id)
{
    if (w >= 512u)
        return orc_uniform(w);
    double scale = 1.0;
    for (uint32_t level = 1; level <= 2; ++level) {
        uint32_t ctr[4] = {0x80000000u + (level << 24) + g, (uint32_t)idx, (uint32_t)(idx >> 32), point_id};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        scale *= 0x1p-23;
        if (out[0] >= 512u || level == 2)
            return scale * orc_uniform(out[0]);
    }
    return 0.0; /* not reached */
}

/* Box-Muller: two independent standard normals from two uniforms; these are
 * the draws from the standard normal d(gamma) of Eq. (14). */
void orc_box_muller(double u1, double u2, double *z_cos, double *z_sin)
{
    double rad = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    *z_cos = rad * cos(ang);
    *z_sin = rad * sin(ang);
}

void orc_stream(int K, uint64_t seed, uint32_t point_id, uint64_t idx, double *z, double *u_acc)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4], w[4];
    for (int k = 1; k <= K; ++k) {
        int j = (k - 1) / 2, h = (k - 1) % 2;
        ctr[0] = (uint32_t)j;
        ctr[1] = (uint32_t)idx;
        ctr[2] = (uint32_t)(idx >> 32);
        ctr[3] = point_id;
        orc_philox4x32_10(ctr, key, w);
        double u1 = orc_uniform_ext(w[2 * h], (uint32_t)(4 * j + 2 * h), key, idx, point_id);
        orc_box_muller(u1, orc_uniform(w[2 * h + 1]), &z[k - 1], &z[K + k - 1]);
    }
    ctr[0] = (uint32_t)((K + 1) / 2);
    ctr[1] = (uint32_t)idx;
    ctr[2] = (uint32_t)(idx >> 32);
    ctr[3] = point_id;
    orc_philox4x32_10(ctr, key, w);
    *u_acc = orc_uniform_ext(w[0], (uint32_t)(4 * ((K + 1) / 2)), key, idx, point_id);
}

uint64_t orc_tail_scan(int K, uint64_t seed, uint32_t point_id, uint64_t idx0, uint64_t n, int which,
                       uint64_t *out, uint64_t cap)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t found = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t idx = idx0 + i;
        uint32_t ctr[4] = {0, (uint32_t)idx, (uint32_t)(idx >> 32), point_id}, w[4];
        int hit = 0;
        if (which & 1) {
            for (int j = 0; j < (K + 1) / 2 && !hit; ++j) {
                ctr[0] = (uint32_t)j;
                orc_philox4x32_10(ctr, key, w);
                /* the radius words of block j: word 0 (mode 2j+1) and word 2 (mode 2j+2) */
                if (w[0] < 512u || (2 * j + 2 <= K && w[2] < 512u))
                    hit = 1;
            }
        }
        if ((which & 2) && !hit) {
            ctr[0] = (uint32_t)((K + 1) / 2);
            orc_philox4x32_10(ctr, key, w);
            if (w[0] < 512u)
                hit = 1;
        }
        if (hit) {
            if (found < cap)
                out[found] = idx;
            ++found;
        }
    }
    return found;
}

/* ---------------------------------------------------------------------------
 * Hamiltonian pieces on the sphere.  xh is the real spectral vector
 * [xh_1..xh_K | xh_{K+1}..xh_{2K}] of Sec. II.C, and the microstate is
 * u_k = sqrt(E0/2pi) (xh_k - i xh_{K+k}) (Eq. 16).
 * ------------------------------------------------------------------------- */

/* Eq. (20): H2 = E0 sum_k k^2 (xh_k^2 + xh_{K+k}^2). */
double orc_H2(int K, double E0, const double *xh)
{
    double s = 0.0;
    for (int k = 1; k <= K; ++k)
        s += (double)k * (double)k * (xh[k - 1] * xh[k - 1] + xh[K + k - 1] * xh[K + k - 1]);
    return E0 * s;
}

static void orc_microstate(int K, double E0, const double *xh, double complex *u)
{
    double c = sqrt(E0 / (2.0 * M_PI));
    u[0] = 0.0; /* u_0 = 0: zero momentum, Eq. (5) */
    for (int k = 1; k <= K; ++k) u[k] = c * (xh[k - 1] - I * xh[K + k - 1]);
}

/* Eq. (42): H3 = 2 pi sum_{n=1}^K Re( conj(u_n) sum_{k=1}^{n-1} u_k u_{n-k} ). */
double orc_H3_double(int K, double E0, const double *xh)
{
    double complex u[ORC_KMAX + 1];
    orc_microstate(K, E0, xh, u);
    double h = 0.0;
    for (int n = 1; n <= K; ++n) {
        double complex t = 0.0;
        for (int k = 1; k <= n - 1; ++k) t += u[k] * u[n - k];
        h += creal(conj(u[n]) * t);
    }
    return 2.0 * M_PI * h;
}

/* Eq. (41): H3 = (pi/3) sum over k1+k2+k3 = 0, |k_i| <= K of u_k1 u_k2 u_k3,
 * with u_{-k} = conj(u_k) and u_0 = 0 (Sec. II.B). */
double orc_H3_triple(int K, double E0, const double *xh)
{
    double complex u[ORC_KMAX + 1];
    orc_microstate(K, E0, xh, u);
    double complex s = 0.0;
    for (int k1 = -K; k1 <= K; ++k1) {
        for (int k2 = -K; k2 <= K; ++k2) {
            int k3 = -k1 - k2;
            if (k3 < -K || k3 > K) continue;
            double complex a = k1 >= 0 ? u[k1] : conj(u[-k1]);
            double complex b = k2 >= 0 ? u[k2] : conj(u[-k2]);
            double complex c = k3 >= 0 ? u[k3] : conj(u[-k3]);
            s += a * b * c;
        }
    }
    return (M_PI / 3.0) * creal(s);
}

/* Eq. (8): u(xi) = sum_k a_k cos(k xi) + b_k sin(k xi), with
 * a_k = 2 Re u_k = 2 sqrt(E0/2pi) xh_k and b_k = -2 Im u_k = 2 sqrt(E0/2pi) xh_{K+k}
 * (Eq. 7 and Eq. 16). */
double orc_u_at(int K, double E0, const double *xh, double xi)
{
    double c2 = 2.0 * sqrt(E0 / (2.0 * M_PI));
    double s = 0.0;
    for (int k = 1; k <= K; ++k)
        s += c2 * xh[k - 1] * cos(k * xi) + c2 * xh[K + k - 1] * sin(k * xi);
    return s;
}

/* Eq. (2): H3 = (1/6) int_{-pi}^{pi} u^3 dxi, here by the N-point rectangle rule
 * on xi_j = -pi + 2 pi j / N; exact when N > 3K because u^3 is a trigonometric
 * polynomial of degree 3K. */
double orc_H3_grid(int K, double E0, const double *xh, int N)
{
    double s = 0.0;
    for (int j = 0; j < N; ++j) {
        double xi = -M_PI + 2.0 * M_PI * (double)j / (double)N;
        double u = orc_u_at(K, E0, xh, xi);
        s += u * u * u;
    }
    return (1.0 / 6.0) * (2.0 * M_PI / (double)N) * s;
}

/* ---------------------------------------------------------------------------
 * Proposal distribution (Sec. III).
 * ------------------------------------------------------------------------- */

/* Eq. (29): F(alpha) = 1 - (alpha/K) sum_k 1 / (1 + alpha beta' k^2 / K^3). */
double orc_F_alpha(int K, double beta_p, double alpha)
{
    double K3 = (double)K * (double)K * (double)K;
    double s = 0.0;
    for (int k = 1; k <= K; ++k) s += 1.0 / (1.0 + alpha * beta_p * (double)k * (double)k / K3);
    return 1.0 - alpha / (double)K * s;
}

/* alpha* = root of F (Sec. III.A, "numerical root-finder"): F(0) = 1 and F
 * decreases, so bracket [0, hi] by doubling and bisect to full precision.
 * Returns NaN when F stays positive (no root). */
double orc_alpha_star(int K, double beta_p)
{
    double lo = 0.0, hi = 1.0;
    while (orc_F_alpha(K, beta_p, hi) > 0.0) {
        lo = hi;
        hi *= 2.0;
        if (hi > 1e300) return NAN;
    }
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_F_alpha(K, beta_p, mid) > 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

int orc_point_init(orc_point *pt, int K, double E0, double beta_p, double r, int proposal)
{
    memset(pt, 0, sizeof(*pt));
    pt->K = K;
    pt->E0 = E0;
    pt->beta_p = beta_p;
    pt->r = r;
    pt->proposal = proposal;
    pt->alpha = 1.0;
    for (int k = 1; k <= K; ++k) pt->sigma2[k - 1] = 1.0;
    if (proposal == ORC_PROPOSAL_PAPER) {
        double a = orc_alpha_star(K, beta_p);
        if (isnan(a)) return -1;
        pt->alpha = a;
        double K3 = (double)K * (double)K * (double)K;
        /* Eq. (25): sigma_k^2 = 1 / (1 + alpha* beta' k^2 / K^3) */
        for (int k = 1; k <= K; ++k)
            pt->sigma2[k - 1] = 1.0 / (1.0 + a * beta_p * (double)k * (double)k / K3);
    }
    return 0;
}

/* log f/g up to an additive constant:
 *   Eq. (43)  beta H = beta' / (E0 K^2) (H2 - (C3/C2) H3)
 *   Eq. (40)  f/g = exp(-beta H) (1 + alpha* beta' S / K^3)^K   (paper proposal)
 *   uniform proposal: g is constant (Eq. 15), f/g = exp(-beta H)
 *   general diagonal Gaussian: g = Const a(xh)^-K with a(xh) from Eq. (33)
 *   (Eq. 37), so f/g = exp(-beta H) (2 a(xh))^K. */
double orc_log_fg(const orc_point *pt, const double *xh)
{
    int K = pt->K;
    double H2 = orc_H2(K, pt->E0, xh);
    double H3 = orc_H3_double(K, pt->E0, xh);
    double bH = pt->beta_p / (pt->E0 * (double)K * (double)K) * (H2 - pt->r * H3);
    if (pt->proposal == ORC_PROPOSAL_UNIFORM) return -bH;
    if (pt->proposal == ORC_PROPOSAL_PAPER) {
        double S = H2 / pt->E0;
        double K3 = (double)K * (double)K * (double)K;
        return -bH + (double)K * log(1.0 + pt->alpha * pt->beta_p * S / K3);
    }
    double a2 = 0.0;
    for (int k = 1; k <= K; ++k)
        a2 += (xh[k - 1] * xh[k - 1] + xh[K + k - 1] * xh[K + k - 1]) / pt->sigma2[k - 1];
    return -bH + (double)K * log(a2);
}

/* ---------------------------------------------------------------------------
 * Rejection constant M = sup f/g (Eq. 45) by Nelder-Mead (Sec. IV.A).  The
 * search runs over y in R^{2K} with xh = y/|y|, which covers the sphere.
 * Standard coefficients (reflection 1, expansion 2, contraction 1/2, shrink
 * 1/2, as in Lagarias et al.).
 * ------------------------------------------------------------------------- */
static double orc_nm_value(const orc_point *pt, const double *y, double *tmp)
{
    int n = 2 * pt->K;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += y[i] * y[i];
    if (!(s > 0.0)) return -INFINITY;
    s = sqrt(s);
    for (int i = 0; i < n; ++i) tmp[i] = y[i] / s;
    return orc_log_fg(pt, tmp);
}

/* One Nelder-Mead run maximising log f/g from the simplex {x0, x0 + step e_i}. */
static double orc_nm_once(const orc_point *pt, double *x, double step, long max_evals, long *evals)
{
    int n = 2 * pt->K;
    int m = n + 1;
    double *P = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double *F = (double *)malloc(sizeof(double) * (size_t)m);
    double *cen = (double *)malloc(sizeof(double) * (size_t)n);
    double *xr = (double *)malloc(sizeof(double) * (size_t)n);
    double *xe = (double *)malloc(sizeof(double) * (size_t)n);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < m; ++i) {
        for (int d = 0; d < n; ++d) P[i * n + d] = x[d];
        if (i > 0) P[i * n + (i - 1)] += step;
        F[i] = orc_nm_value(pt, &P[i * n], tmp);
        ++*evals;
    }
    for (;;) {
        /* sort vertices so F is descending (best = largest first) */
        for (int i = 1; i < m; ++i) {
            for (int j = i; j > 0 && F[j] > F[j - 1]; --j) {
                double t = F[j];
                F[j] = F[j - 1];
                F[j - 1] = t;
                for (int d = 0; d < n; ++d) {
                    double q = P[j * n + d];
                    P[j * n + d] = P[(j - 1) * n + d];
                    P[(j - 1) * n + d] = q;
                }
            }
        }
        double spread = F[0] - F[m - 1];
        double diam = 0.0;
        for (int i = 1; i < m; ++i)
            for (int d = 0; d < n; ++d) {
                double q = fabs(P[i * n + d] - P[d]);
                if (q > diam) diam = q;
            }
        if (*evals >= max_evals || (spread <= 1e-15 * (1.0 + fabs(F[0])) && diam <= 1e-9)) break;
        for (int d = 0; d < n; ++d) {
            double s = 0.0;
            for (int i = 0; i < m - 1; ++i) s += P[i * n + d];
            cen[d] = s / (double)(m - 1);
        }
        double *worst = &P[(m - 1) * n];
        for (int d = 0; d < n; ++d) xr[d] = cen[d] + (cen[d] - worst[d]);
        double fr = orc_nm_value(pt, xr, tmp);
        ++*evals;
        if (fr > F[0]) {
            for (int d = 0; d < n; ++d) xe[d] = cen[d] + 2.0 * (xr[d] - cen[d]);
            double fe = orc_nm_value(pt, xe, tmp);
            ++*evals;
            if (fe > fr) {
                memcpy(worst, xe, sizeof(double) * (size_t)n);
                F[m - 1] = fe;
            } else {
                memcpy(worst, xr, sizeof(double) * (size_t)n);
                F[m - 1] = fr;
            }
            continue;
        }
        if (fr > F[m - 2]) {
            memcpy(worst, xr, sizeof(double) * (size_t)n);
            F[m - 1] = fr;
            continue;
        }
        int shrink = 0;
        if (fr > F[m - 1]) { /* outside contraction */
            for (int d = 0; d < n; ++d) xe[d] = cen[d] + 0.5 * (xr[d] - cen[d]);
            double fc = orc_nm_value(pt, xe, tmp);
            ++*evals;
            if (fc >= fr) {
                memcpy(worst, xe, sizeof(double) * (size_t)n);
                F[m - 1] = fc;
            } else {
                shrink = 1;
            }
        } else { /* inside contraction */
            for (int d = 0; d < n; ++d) xe[d] = cen[d] + 0.5 * (worst[d] - cen[d]);
            double fc = orc_nm_value(pt, xe, tmp);
            ++*evals;
            if (fc > F[m - 1]) {
                memcpy(worst, xe, sizeof(double) * (size_t)n);
                F[m - 1] = fc;
            } else {
                shrink = 1;
            }
        }
        if (shrink) {
            for (int i = 1; i < m; ++i) {
                for (int d = 0; d < n; ++d) P[i * n + d] = P[d] + 0.5 * (P[i * n + d] - P[d]);
                F[i] = orc_nm_value(pt, &P[i * n], tmp);
                ++*evals;
            }
        }
    }
    /* best vertex after the final sort */
    int b = 0;
    for (int i = 1; i < m; ++i)
        if (F[i] > F[b]) b = i;
    double best = F[b];
    double s = 0.0;
    for (int d = 0; d < n; ++d) s += P[b * n + d] * P[b * n + d];
    s = sqrt(s);
    for (int d = 0; d < n; ++d) x[d] = P[b * n + d] / s;
    free(P);
    free(F);
    free(cen);
    free(xr);
    free(xe);
    free(tmp);
    return best;
}

/* Nelder-Mead from xh0, restarted from its own best point with a fresh simplex
 * until a restart no longer improves the maximum. */
double orc_nelder_mead(const orc_point *pt, const double *xh0, double *xh_out, long max_evals)
{
    int n = 2 * pt->K;
    double x[2 * ORC_KMAX];
    memcpy(x, xh0, sizeof(double) * (size_t)n);
    long evals = 0;
    double best = -INFINITY;
    double step = 0.1;
    for (int restart = 0; restart < 60 && evals < max_evals; ++restart) {
        double v = orc_nm_once(pt, x, step, max_evals, &evals);
        if (v <= best + 1e-14 * (1.0 + fabs(best)) && restart > 0) {
            if (v > best) best = v;
            if (step < 1e-6) break;
            step *= 0.1;
            continue;
        }
        best = v;
    }
    if (xh_out) memcpy(xh_out, x, sizeof(double) * (size_t)n);
    return best;
}

/* log M (Eq. 45).  The paper starts Nelder-Mead from the zero-mean Dirichlet
 * kernel u_k = sqrt(E0/(2 pi K)) for all k (Eq. 46), i.e. xh_k = 1/sqrt(K) on
 * the cosine half.  Because Nelder-Mead is a local method, the oracle also
 * starts from every single-mode state and from n_random_starts seeded random
 * directions and keeps the largest maximum.  The starts run on separate
 * threads; the result does not depend on the thread count. */
typedef struct {
    const orc_point *pt;
    double x0[2 * ORC_KMAX], xo[2 * ORC_KMAX];
    double v;
} orc_nm_job;

static void *orc_nm_worker(void *arg)
{
    orc_nm_job *jb = (orc_nm_job *)arg;
    jb->v = orc_nelder_mead(jb->pt, jb->x0, jb->xo, 400000);
    return NULL;
}

double orc_log_M(const orc_point *pt, int n_random_starts, uint64_t seed, double *xh_best)
{
    int K = pt->K, n = 2 * K;
    int ns = 1 + K + (n_random_starts > 0 ? n_random_starts : 0);
    orc_nm_job *jobs = (orc_nm_job *)calloc((size_t)ns, sizeof(orc_nm_job));
    pthread_t *th = (pthread_t *)calloc((size_t)ns, sizeof(pthread_t));
    for (int s = 0; s < ns; ++s) {
        jobs[s].pt = pt;
        if (s == 0) {
            for (int k = 1; k <= K; ++k) jobs[s].x0[k - 1] = 1.0 / sqrt((double)K);
        } else if (s <= K) {
            jobs[s].x0[s - 1] = 1.0;
        } else {
            double u;
            orc_stream(K, seed, 0xFFFFFFFFu, (uint64_t)(s - K - 1), jobs[s].x0, &u);
        }
    }
    for (int s = 0; s < ns; ++s) pthread_create(&th[s], NULL, orc_nm_worker, &jobs[s]);
    for (int s = 0; s < ns; ++s) pthread_join(th[s], NULL);
    int b = 0;
    for (int s = 1; s < ns; ++s)
        if (jobs[s].v > jobs[b].v) b = s;
    double best = jobs[b].v;
    if (xh_best) memcpy(xh_best, jobs[b].xo, sizeof(double) * (size_t)n);
    free(jobs);
    free(th);
    return best;
}

/* ---------------------------------------------------------------------------
 * The rejection algorithm (Sec. IV.B), one proposal at a time.
 * ------------------------------------------------------------------------- */
static void orc_one(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx, orc_rec *rc)
{
    int K = pt->K, n = 2 * K;
    double z[2 * ORC_KMAX], u_acc;
    orc_stream(K, seed, point_id, idx, z, &u_acc);
    /* draw X from d(gamma_Sigma), Eq. (26): the pair (X_k, X_{K+k}) has variance sigma_k^2 */
    double X[2 * ORC_KMAX];
    for (int k = 1; k <= K; ++k) {
        double sd = pt->proposal == ORC_PROPOSAL_UNIFORM ? 1.0 : sqrt(pt->sigma2[k - 1]);
        X[k - 1] = sd * z[k - 1];
        X[K + k - 1] = sd * z[K + k - 1];
    }
    /* project onto the sphere: X^ = X / |X| */
    double nn = 0.0;
    for (int i = 0; i < n; ++i) nn += X[i] * X[i];
    nn = sqrt(nn);
    memset(rc, 0, sizeof(*rc));
    for (int i = 0; i < n; ++i) rc->xhat[i] = X[i] / nn;
    /* acceptance probability f/(M g) via Eq. (40) */
    rc->idx = idx;
    rc->H2 = orc_H2(K, pt->E0, rc->xhat);
    rc->H3 = orc_H3_double(K, pt->E0, rc->xhat);
    rc->S = rc->H2 / pt->E0;
    rc->logfg = orc_log_fg(pt, rc->xhat);
    rc->delta = rc->logfg - pt->logM;
    rc->lnU = log(u_acc);
    rc->accept = rc->lnU < rc->delta;
    rc->near = fabs(rc->lnU - rc->delta) < 1e-6;
    rc->u0 = orc_u_at(K, pt->E0, rc->xhat, 0.0);
}

static void orc_stats_zero(orc_stats *st, const orc_point *pt)
{
    memset(st, 0, sizeof(*st));
    st->max_delta = -INFINITY;
    st->u_cap = sqrt(2.0 * (double)pt->K * pt->E0 / M_PI);
}

static void orc_stats_add(orc_stats *st, const orc_point *pt, const orc_rec *rc)
{
    int K = pt->K;
    st->n_prop += 1;
    if (rc->delta > st->max_delta) st->max_delta = rc->delta;
    if (rc->delta > 0.0) st->n_viol += 1;
    if (rc->near) st->n_near += 1;
    if (!rc->accept) return;
    st->n_acc += 1;
    double p = 1.0;
    for (int q = 0; q < 4; ++q) {
        p *= rc->u0;
        st->sum_u0[q] += p;
    }
    /* the 2K surface-displacement values of a field (Sec. V.D) */
    for (int j = 0; j < 2 * K; ++j) {
        double xi = -M_PI + 2.0 * M_PI * (double)j / (double)(2 * K);
        double u = orc_u_at(K, pt->E0, rc->xhat, xi), pu = 1.0;
        for (int q = 0; q < 4; ++q) {
            pu *= u;
            st->sum_grid[q] += pu;
        }
    }
    for (int k = 1; k <= K; ++k)
        st->spectrum[k - 1] += rc->xhat[k - 1] * rc->xhat[k - 1] + rc->xhat[K + k - 1] * rc->xhat[K + k - 1];
    double f = (rc->u0 + st->u_cap) / (2.0 * st->u_cap) * (double)ORC_HIST_BINS;
    int b = (int)floor(f);
    if (b < 0) b = 0;
    if (b > ORC_HIST_BINS - 1) b = ORC_HIST_BINS - 1;
    st->hist[b] += 1;
    double sigma0 = sqrt(pt->E0 / M_PI); /* sigma = sqrt(E0/pi), Sec. V.D */
    for (int i = 0; i < ORC_EXCEED; ++i)
        if (rc->u0 > 0.25 * (double)i * sigma0) st->exceed[i] += 1;
}

static void orc_stats_merge(orc_stats *a, const orc_stats *b)
{
    a->n_prop += b->n_prop;
    a->n_acc += b->n_acc;
    a->n_near += b->n_near;
    a->n_viol += b->n_viol;
    if (b->max_delta > a->max_delta) a->max_delta = b->max_delta;
    for (int q = 0; q < 4; ++q) {
        a->sum_u0[q] += b->sum_u0[q];
        a->sum_grid[q] += b->sum_grid[q];
    }
    for (int k = 0; k < ORC_KMAX; ++k) a->spectrum[k] += b->spectrum[k];
    for (int i = 0; i < ORC_HIST_BINS; ++i) a->hist[i] += b->hist[i];
    for (int i = 0; i < ORC_EXCEED; ++i) a->exceed[i] += b->exceed[i];
}

/* ---- threading: contiguous slices of the work, merged in slice order ---- */
typedef struct {
    const orc_point *pt;
    uint64_t seed;
    uint32_t point_id;
    const uint64_t *idx_list; /* replay: explicit indices */
    uint64_t idx0, begin, end;
    orc_rec *recs;
    orc_stats st;
    orc_rec *acc_out;
    uint64_t acc_cap, acc_n, acc_room;
    int mode;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    orc_rec rc;
    for (uint64_t i = jb->begin; i < jb->end; ++i) {
        if (jb->mode == 0) {
            orc_one(jb->pt, jb->seed, jb->point_id, jb->idx_list[i], &jb->recs[i]);
        } else if (jb->mode == 1) {
            orc_one(jb->pt, jb->seed, jb->point_id, jb->idx0 + i, &rc);
            orc_stats_add(&jb->st, jb->pt, &rc);
        } else {
            orc_one(jb->pt, jb->seed, jb->point_id, jb->idx0 + i, &rc);
            if (rc.accept) {
                if (jb->acc_n < jb->acc_cap) {
                    if (jb->acc_n == jb->acc_room) {
                        jb->acc_room = jb->acc_room ? 2 * jb->acc_room : 64;
                        jb->acc_out = (orc_rec *)realloc(jb->acc_out, sizeof(orc_rec) * (size_t)jb->acc_room);
                    }
                    jb->acc_out[jb->acc_n] = rc;
                }
                jb->acc_n += 1;
            }
        }
    }
    return NULL;
}

static int orc_parallel(orc_job *proto, uint64_t n, int nthreads, orc_job **jobs_out)
{
    if (nthreads <= 0) nthreads = 1;
    if ((uint64_t)nthreads > n && n > 0) nthreads = (int)n;
    if (n == 0) nthreads = 1;
    orc_job *jobs = (orc_job *)calloc((size_t)nthreads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].begin = n * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    orc_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    *jobs_out = jobs;
    return nthreads;
}

int orc_replay(const orc_point *pt, uint64_t seed, uint32_t point_id, const uint64_t *idx,
               uint64_t n, int nthreads, orc_rec *out)
{
    orc_job proto;
    memset(&proto, 0, sizeof(proto));
    proto.pt = pt;
    proto.seed = seed;
    proto.point_id = point_id;
    proto.idx_list = idx;
    proto.recs = out;
    proto.mode = 0;
    orc_job *jobs;
    orc_parallel(&proto, n, nthreads, &jobs);
    free(jobs);
    return 0;
}

int orc_run_stats(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx0,
                  uint64_t n, int nthreads, orc_stats *out)
{
    orc_job proto;
    memset(&proto, 0, sizeof(proto));
    proto.pt = pt;
    proto.seed = seed;
    proto.point_id = point_id;
    proto.idx0 = idx0;
    proto.mode = 1;
    orc_stats_zero(&proto.st, pt);
    orc_job *jobs;
    int nt = orc_parallel(&proto, n, nthreads, &jobs);
    orc_stats_zero(out, pt);
    for (int t = 0; t < nt; ++t) orc_stats_merge(out, &jobs[t].st);
    free(jobs);
    return 0;
}

uint64_t orc_run_accepted(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx0,
                          uint64_t n, int nthreads, orc_rec *out, uint64_t cap)
{
    /* each thread keeps its accepted records (grown on demand, at most cap),
       then the slices are packed in thread order, i.e. in index order */
    orc_job proto;
    memset(&proto, 0, sizeof(proto));
    proto.pt = pt;
    proto.seed = seed;
    proto.point_id = point_id;
    proto.idx0 = idx0;
    proto.mode = 2;
    proto.acc_cap = cap;
    orc_job *jobs;
    int nt = orc_parallel(&proto, n, nthreads, &jobs);
    uint64_t total = 0, w = 0;
    for (int t = 0; t < nt; ++t) {
        uint64_t got = jobs[t].acc_n < cap ? jobs[t].acc_n : cap;
        for (uint64_t i = 0; i < got && w < cap; ++i) out[w++] = jobs[t].acc_out[i];
        total += jobs[t].acc_n;
        free(jobs[t].acc_out);
    }
    free(jobs);
    return total;
}

/* ---------------------------------------------------------------------------
 * Sampling-importance resampling (SIR) with the same proposal.  Sec. IV.B
 * names SIR with g as the alternative use of the proposal: every draw
 * carries the importance weight f/g, proportional to exp(Delta), Delta =
 * log f/(Mg) the quantity of the rejection test (log M only shifts it), and
 * the resampled set keeps each draw in proportion to its weight.  Here draw
 * i gets an independent Poisson number of copies n_i ~ Poisson(c exp(Delta_i)),
 * drawn by inversion of the draw's accept uniform U_i:
 * n_i = #{k >= 1 : U_i < P(N >= k)}.  Conditioned on their total the n_i are
 * multinomial with probabilities exp(Delta_i) / sum_j exp(Delta_j), the
 * classical SIR draw; c sets the expected total.
 * ------------------------------------------------------------------------- */

/* P(N >= k) for N ~ Poisson(lambda), k >= 1: the tail series
 * e^-l l^k/k! sum_i l^i k!/(k+i)! for lambda <= k + 1 (no cancellation),
 * else 1 - e^-l sum_{j<k} l^j/j!. */
double orc_poisson_tail(double lambda, int k)
{
    if (lambda <= 0.0)
        return 0.0;
    if (lambda <= k + 1.0) {
        double lead = exp(-lambda + k * log(lambda) - lgamma(k + 1.0));
        double term = 1.0, sum = 1.0;
        for (int i = 1; i < 200; ++i) {
            term *= lambda / (k + i);
            sum += term;
            if (term < 1e-18 * sum)
                break;
        }
        return lead * sum;
    }
    double p = exp(-lambda), s = p;
    for (int j = 1; j < k; ++j) {
        p *= lambda / j;
        s += p;
    }
    return 1.0 - s;
}

/* n = #{k >= 1 : u < P(N >= k)} for N ~ Poisson(lambda). */
int orc_poisson_count(double lambda, double u)
{
    int n = 0;
    while (n < 100000 && u < orc_poisson_tail(lambda, n + 1))
        ++n;
    return n;
}

/* One proposal of the SIR run: its weight terms and its number of copies. */
static void orc_sir_add(orc_sir_stats *st, const orc_point *pt, const orc_rec *rc, double c, orc_rec *kept,
                        uint32_t *kept_n, uint64_t cap, uint64_t *n_kept)
{
    st->n_prop += 1;
    double w = exp(rc->delta);
    st->sum_w += w;
    st->sum_w2 += w * w;
    st->sum_wS += w * rc->S;
    double p = w;
    for (int q = 0; q < 4; ++q) {
        p *= rc->u0;
        st->sum_w_u0[q] += p;
    }
    int n = orc_poisson_count(c * w, exp(rc->lnU));
    if (n == 0) return;
    if (*n_kept < cap) {
        kept[*n_kept] = *rc;
        kept_n[*n_kept] = (uint32_t)n;
    }
    *n_kept += 1;
    st->n_kept += 1;
    st->n_copies += (uint64_t)n;
    st->sum_nS += n * rc->S;
    p = (double)n;
    for (int q = 0; q < 4; ++q) {
        p *= rc->u0;
        st->sum_n_u0[q] += p;
    }
    for (int k = 1; k <= pt->K; ++k)
        st->spectrum[k - 1] += n * (rc->xhat[k - 1] * rc->xhat[k - 1] + rc->xhat[pt->K + k - 1] * rc->xhat[pt->K + k - 1]);
}

typedef struct {
    const orc_point *pt;
    uint64_t seed, idx0, begin, end, cap, n_kept;
    uint32_t point_id;
    double c;
    orc_sir_stats st;
    orc_rec *kept;
    uint32_t *kept_n;
} orc_sir_job;

static void *orc_sir_worker(void *arg)
{
    orc_sir_job *jb = (orc_sir_job *)arg;
    orc_rec rc;
    for (uint64_t i = jb->begin; i < jb->end; ++i) {
        orc_one(jb->pt, jb->seed, jb->point_id, jb->idx0 + i, &rc);
        orc_sir_add(&jb->st, jb->pt, &rc, jb->c, jb->kept, jb->kept_n, jb->cap, &jb->n_kept);
    }
    return NULL;
}

uint64_t orc_run_sir(const orc_point *pt, uint64_t seed, uint32_t point_id, uint64_t idx0, uint64_t n, double c,
                     int nthreads, orc_sir_stats *out, orc_rec *kept, uint32_t *kept_n, uint64_t cap)
{
    if (nthreads <= 0) nthreads = 1;
    if ((uint64_t)nthreads > n && n > 0) nthreads = (int)n;
    if (n == 0) nthreads = 1;
    orc_sir_job *jobs = (orc_sir_job *)calloc((size_t)nthreads, sizeof(orc_sir_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        orc_sir_job *jb = &jobs[t];
        jb->pt = pt;
        jb->seed = seed;
        jb->point_id = point_id;
        jb->idx0 = idx0;
        jb->c = c;
        jb->begin = n * (uint64_t)t / (uint64_t)nthreads;
        jb->end = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
        jb->cap = cap;
        jb->kept = (orc_rec *)malloc(sizeof(orc_rec) * (size_t)(cap ? cap : 1));
        jb->kept_n = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(cap ? cap : 1));
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_sir_worker, &jobs[t]);
    orc_sir_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    memset(out, 0, sizeof(*out));
    uint64_t total = 0, w = 0;
    for (int t = 0; t < nthreads; ++t) {
        orc_sir_stats *s = &jobs[t].st;
        out->n_prop += s->n_prop;
        out->n_kept += s->n_kept;
        out->n_copies += s->n_copies;
        out->sum_w += s->sum_w;
        out->sum_w2 += s->sum_w2;
        out->sum_wS += s->sum_wS;
        out->sum_nS += s->sum_nS;
        for (int q = 0; q < 4; ++q) {
            out->sum_w_u0[q] += s->sum_w_u0[q];
            out->sum_n_u0[q] += s->sum_n_u0[q];
        }
        for (int k = 0; k < ORC_KMAX; ++k) out->spectrum[k] += s->spectrum[k];
        uint64_t got = jobs[t].n_kept < cap ? jobs[t].n_kept : cap;
        for (uint64_t i = 0; i < got && w < cap; ++i) {
            kept[w] = jobs[t].kept[i];
            kept_n[w] = jobs[t].kept_n[i];
            ++w;
        }
        total += jobs[t].n_kept;
        free(jobs[t].kept);
        free(jobs[t].kept_n);
    }
    free(jobs);
    free(th);
    return total;
}
