// Per-point constants of the sampler (host side), shared by the handle API
// and the allocation-free entry point: the proposal variances of Eq. (25)
// (optionally corrected by the learned log-variances) and the table the
// kernels read: coefficients of log f/(Mg) (Eqs. 40, 43), output scales and
// the FP32 decision guard.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/tkdv.h"
#include "tkdv_internal.h"

namespace tkdv {

int proposal_variances(int K, const tkdv_point &q, double *alpha, double *s2) {
    *alpha = 1.0;
    for (int k = 0; k < K; ++k) s2[k] = 1.0;
    if (q.proposal == TKDV_PROPOSAL_UNIFORM) return TKDV_OK;
    int rc = tkdv_alpha_star(K, q.beta_p, alpha);
    if (rc != TKDV_OK) return rc;
    const double K3 = (double)K * K * K;
    for (int k = 1; k <= K; ++k) {
        s2[k - 1] = 1.0 / (1.0 + *alpha * q.beta_p * (double)k * k / K3);  // Eq. (25)
        if (q.proposal == TKDV_PROPOSAL_LEARNED) {
            const double c = q.log_var_correction[k - 1];
            if (!std::isfinite(c)) return TKDV_ERR_INVALID_ARG;
            s2[k - 1] *= std::exp(c);
        }
    }
    return TKDV_OK;
}

void fill_point_const(int K, const tkdv_point &q, const double *s2, double logM, bool grid, PointConst &c) {
    std::memset(&c, 0, sizeof(c));
    for (int k = 0; k < kKMax; ++k) {
        const bool on = k < K;
        c.sigma[k] = on ? (float)std::sqrt(s2[k]) : 0.f;
        c.sigma_d[k] = on ? std::sqrt(s2[k]) : 0.0;
        c.act[k] = on ? 1.f : 0.f;
    }
    const double K2 = (double)K * K;
    const double cc = std::sqrt(q.E0 / (2.0 * M_PI));
    const double h3s = 2.0 * M_PI * cc * cc * cc;
    c.cS_d = -q.beta_p / K2;                                          // Eq. (43), H2 = E0 S
    c.cH_d = q.beta_p * q.r / (q.E0 * K2) * h3s;                      // Eq. (43), H3 = h3s T
    c.cQ_d = q.proposal == TKDV_PROPOSAL_UNIFORM ? 0.0 : (double)K;  // Eq. (40) / (37)
    c.logM = logM;
    c.cS = (float)c.cS_d;
    c.cH = (float)c.cH_d;
    c.cQ = (float)c.cQ_d;
    c.logM_f = (float)logM;
    c.u0s = (float)(2.0 * cc);
    c.h3s = (float)h3s;
    c.E0 = (float)q.E0;
    const double ucap = std::sqrt(2.0 * K * q.E0 / M_PI);
    c.hist_a = (float)(kHistBins / (2.0 * ucap));
    c.hist_b = (float)(kHistBins / 2);
    c.exc_a = (float)(1.0 / (0.25 * std::sqrt(q.E0 / M_PI)));
    // Guard band of the FP32 decision; proposals inside it are decided in
    // FP64.  (1) Rounding: the FP32 value of log f/(Mg) carries the rounding
    // of ~2K+16 chained operations on each term; T additionally sums O(K)
    // products per mode with |T| <= sqrt(K) on the sphere.  The band is eight
    // times that bound.  (2) The relative part of the radius error: e in every
    // rho moves each component by e/2, hence S and Q by at most 2e and T by at
    // most 3e relative; 4 kRhoRelErr covers both.  (3) Its absolute part
    // eps = kRhoAbsErr moves the amplitude a_m = sigma_m sqrt(rho_m) by
    // sigma_m |rho' - rho| / (sqrt(rho') + sqrt(rho)) <= eps sigma_m / sqrt(rho'),
    // rho' the computed radius (also where the floor of rho_fast applies), so
    // by E = eps sum_m sigma_m / sqrt(rho'_m) in total, computed per draw; a
    // factor 2 covers the rounding of that sum.  With n = |x|^2: S moves by at
    // most 4 K^2 E / sqrt(n), T by 6 sqrt(K) E / sqrt(n) (its cubic form has
    // derivative below 3n per mode on the sphere, and |T| <= sqrt(K)), ln Q by
    // 2E/sqrt(n) through n and by K eps (1 + max sigma^2) / n through the raw
    // normals.
    //
    // The warp form (K > 64, sampler_k128.cu) sums differently: a mode sum
    // (|x|^2, S|x|^2, Q|x|^2) passes each term through at most 12 roundings
    // (its own 3, 4 per lane, 5 in the warp tree), a triad term through at most
    // 50 (8 on its anti-diagonal, 31 in its tile, 3 over rounds, 5 in the warp
    // tree, 3 in the scaling), so chains of 32 and 64 replace 2K + 16; the
    // hardware sine and cosine add at most 2^-21.4 = 6.1 ulp per component,
    // well inside the factor eight.  Its radius -2 logf(u) has no absolute
    // error and a relative one below kRhoLogRelErr, so the per-draw terms (3)
    // vanish.
    const bool warp = K > 64;
    const double eps = std::ldexp(1.0, -24);
    const double rel = warp ? kRhoLogRelErr : kRhoRelErr, abs_err = warp ? 0.0 : kRhoAbsErr;
    const double gam = 8.0 * (warp ? 32.0 : 2.0 * K + 16.0) * eps + 4.0 * rel;
    const double gam_t = 8.0 * (warp ? 64.0 : 2.0 * K + 16.0) * eps + 4.0 * rel;
    c.guard_abs = (float)(1e-6 + gam * std::fabs(c.cQ_d));
    c.guard_rel = (float)gam;
    c.guard_h = (float)(gam_t * std::fabs(c.cH_d) * std::sqrt((double)K));
    double smax = 0.0;
    for (int k = 0; k < K; ++k) smax = std::max(smax, s2[k]);
    c.guard_e = (float)(2.0 * abs_err *
                        (4.0 * K2 * std::fabs(c.cS_d) + 6.0 * std::sqrt((double)K) * std::fabs(c.cH_d) +
                         2.0 * std::fabs(c.cQ_d)));
    c.guard_q = (float)(std::fabs(c.cQ_d) * K * abs_err * (1.0 + smax));
    if (grid) {
        // BF16 hi/lo x3: |dU_j| <= 2^-15.4 sqrt(2K) |x| per grid value, so with
        // sum_j U_j^2 = (N/2)|x|^2 the error of T is below 2^-14.4 sqrt(2K)
        c.guard_h += (float)(std::ldexp(1.0, -14) * std::sqrt(2.0 * K) * std::fabs(c.cH_d));
    }
    c.sir_c = q.sir_c > 0 ? q.sir_c : 1.0;
    c.sir_lnc = (float)std::log(c.sir_c);
    c.point_id = q.point_id;
    c.K = K;
}

}  // namespace tkdv
